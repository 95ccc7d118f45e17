"""The seeded input generators (bhcp_inputs): the recipes the design states,
determinism, and the forward model checked against the oracle's Laplacian."""
import numpy as np
import pytest

import bhcp_inputs as bi
import oracle as O


def test_c2_recipe_and_determinism():
    p = bi.make_c2(M=32, nt=16)
    q = bi.make_c2(M=32, nt=16)
    np.testing.assert_array_equal(p.g_delta, q.g_delta)                 # seeded
    assert not np.array_equal(p.g_delta, bi.make_c2(seed=7, M=32, nt=16).g_delta)
    assert p.grid.shape == (31, 31) and p.grid.nt == 16 and p.grid.T == 0.1
    modes = np.array(p.meta["modes"])
    amps = np.array(p.meta["amps"])
    assert len(modes) == 16 and len({tuple(m) for m in modes}) == 16   # distinct
    assert modes.min() >= 1 and modes.max() <= 8 and (1, 1) in {tuple(m) for m in modes}
    scaled = np.abs(amps) * (modes ** 2).sum(axis=1)                      # amplitude * (k^2 + l^2)
    assert scaled.min() >= 0.5 and scaled.max() <= 1.5
    # 1 % Gaussian noise relative to ||g||, delta its grid-weighted norm
    rel = np.linalg.norm(p.g_delta - p.g) / np.linalg.norm(p.g)
    assert abs(rel - 1e-2) < 1e-12
    assert abs(p.delta - bi.discrete_l2(p.g_delta - p.g, p.grid)) <= 1e-15 * p.delta


def test_c1_recipe():
    p = bi.make_c1()
    assert p.grid.shape == (63,) and p.grid.nt == 64 and p.grid.T == 0.1
    x = np.arange(1, 64) / 64.0
    np.testing.assert_allclose(p.z0, np.sin(np.pi * x) + 0.5 * np.sin(3 * np.pi * x), atol=1e-15)
    ratio = p.g_delta / p.g - 1.0                                         # multiplicative, eps = 1e-3
    assert np.abs(ratio).max() <= 1e-3 + 1e-15 and np.abs(ratio).max() > 5e-4


def test_c3_recipe_small():
    p = bi.make_c3(M=16, nt=8)
    assert p.grid.shape == (15, 15, 15) and p.grid.T == 0.05
    rel = np.linalg.norm(p.g_delta - p.g) / np.linalg.norm(p.g)
    assert abs(rel - 1e-3) < 1e-12
    assert np.abs(p.z0).max() > 0


@pytest.mark.parametrize("grid", [bi.Grid(1, (16,), 1.0, 0.1, 9), bi.Grid(2, (8, 16), 1.0, 0.1, 6),
                                  bi.Grid(3, (4, 8, 4), 1.0, 0.05, 5)], ids=["1d", "2d", "3d"])
def test_forward_model_is_n_backward_euler_steps(grid):
    """g = (I - tau Delta_h)^{-N} z0: N backward Euler steps from z0 to T, checked
    by applying (I - tau Delta_h) N times to g with the oracle's sparse Laplacian."""
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    z0 = rng.standard_normal(grid.shape)
    g = bi.forward_discrete(grid, z0)
    A = sp.identity(grid.Nx) - grid.tau * O.laplacian(grid.dim, grid.M, grid.L)
    v = g.ravel()
    for _ in range(grid.nt - 1):
        v = A @ v
    np.testing.assert_allclose(v, z0.ravel(), atol=1e-10 * np.abs(z0).max())


def test_c4_batch_recipe():
    specs = bi.batch_specs_c4()
    assert len(specs) == 512
    one_d = [s for s in specs if s["dim"] == 1]
    assert len(one_d) == 171                                             # every third instance
    assert all(s["nt"] in (32, 64, 128, 256, 512) for s in specs)
    assert all(1e-4 <= s["rel_noise"] <= 1e-2 for s in specs)
    assert all(s["M"][0] in (64, 128, 256, 512, 1024, 2048) for s in one_d)
    assert all(m in (64, 128, 256) for s in specs if s["dim"] == 2 for m in s["M"])
    assert specs == bi.batch_specs_c4()                                   # seeded

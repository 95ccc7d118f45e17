"""qbvm_solve_batched: same-shape instances with their own alpha solved in the
launches of one solve.  Every instance must equal the oracle's sine-basis
solve of its own system (eq. 3.3 / 3.6 with its own omega) to 1e-10, and the
single-instance plan's result to rounding."""
import numpy as np
import pytest

import bhcp_inputs as bi
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Q.build_library()
    Q.load_library()


def _single(grid, form, alpha, rhs, rhs_kind, n0_only):
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, rhs_kind) as plan:
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.zeros(grid.Nx * (1 if n0_only else grid.nt), dtype=torch.float64, device="cuda")
        plan.solve(x, y, n0_only)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def _batched(grid, form, alphas, rhs, rhs_kind, n0_only):
    B = len(alphas)
    with Q.Batch(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alphas=alphas, rhs_kind=rhs_kind) as bt:
        assert np.allclose(bt.alphas, alphas, rtol=0, atol=0)
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.full((B * grid.Nx * (1 if n0_only else grid.nt),), float("nan"), dtype=torch.float64,
                       device="cuda")
        bt.solve(x, y, n0_only)
        torch.cuda.synchronize()
        return y.cpu().numpy().reshape(B, -1)


GRIDS = [
    bi.Grid(2, (32, 16), 1.0, 0.1, 16),
    bi.Grid(1, (64,), 1.0, 0.1, 64),              # the 1D 63 x 64 shape
    bi.Grid(3, (8, 8, 4), 1.0, 0.05, 8),
    bi.Grid(1, (8,), 1.0, 0.1, 1024),             # longest time transform, tile narrower than the default
    bi.Grid(2, (4, 8), 1.0, 0.1, 2),              # nt = 2: one frequency
]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM], ids=["pq", "pm"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
@pytest.mark.parametrize("n0_only", [False, True], ids=["full", "y0"])
def test_batched_matches_oracle_and_single_plans(grid, form, rhs_kind, n0_only):
    B = 5
    alphas = list(np.logspace(-5, -1, B))
    F = np.stack([bi.random_general_rhs(grid, seed=70 + b) for b in range(B)])
    rhs = F[:, 0] if rhs_kind == Q.RHS_DELTA else F
    got = _batched(grid, form, alphas, rhs, rhs_kind, n0_only)
    for b, a in enumerate(alphas):
        one = _single(grid, form, a, rhs[b], rhs_kind, n0_only)
        scale = np.abs(one).max()
        np.testing.assert_allclose(got[b], one, rtol=0, atol=1e-13 * scale)
        Ff = O.delta_rhs(grid, form, a, rhs[b]) if rhs_kind == Q.RHS_DELTA else rhs[b]
        want = O.solve_spectral(grid, form, a, Ff, levels=[0] if n0_only else None)
        assert O.rel_l2(got[b], want) <= TOL, (b, a)


def test_many_instances_of_the_1d_shape():
    """1000 instances of the 1D 63 x 64 problem (Section 5's a-priori alpha from
    each instance's own noise level); sampled instances against the oracle."""
    B = 1000
    base = bi.make_c1()
    grid = base.grid
    rng = np.random.default_rng(123)
    g = base.g[None, :] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, size=(B, grid.Nx)))
    deltas = np.array([bi.discrete_l2(g[b] - base.g, grid) for b in range(B)])
    alphas = list(deltas)                                   # PinT-QBVM: alpha = delta
    got = _batched(grid, Q.FORM_PQ, alphas, g, Q.RHS_DELTA, False)
    for b in [0, 1, 499, 998, 999]:
        want = O.solve_spectral(grid, O.PQ, alphas[b], O.delta_rhs(grid, O.PQ, alphas[b], g[b]))
        assert O.rel_l2(got[b], want) <= TOL
    assert np.isfinite(got).all()


@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
def test_host_pointers_match_device_and_mixed_are_refused(rhs_kind):
    grid = GRIDS[0]
    alphas = [1e-3, 1e-2, 3e-4]
    F = np.stack([bi.random_general_rhs(grid, seed=90 + b) for b in range(3)])
    rhs = np.ascontiguousarray(F[:, 0] if rhs_kind == Q.RHS_DELTA else F).ravel()
    dev = _batched(grid, Q.FORM_PQ, alphas, rhs, rhs_kind, False).ravel()
    with Q.Batch(grid.dim, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=alphas, rhs_kind=rhs_kind) as bt:
        y = np.full(3 * grid.unknowns, np.nan)
        bt.solve(rhs, y)                                   # host arrays: staged, synchronous
        np.testing.assert_array_equal(y, dev)
        y0 = np.full(3 * grid.Nx, np.nan)
        bt.solve(rhs, y0, n0_only=True)
        np.testing.assert_allclose(y0.reshape(3, -1), dev.reshape(3, grid.nt, -1)[:, 0], rtol=0,
                                   atol=1e-12 * np.abs(dev).max())
        with pytest.raises(Q.QbvmError) as ei:
            bt.solve(rhs, torch.zeros(3 * grid.unknowns, dtype=torch.float64, device="cuda"))
        assert ei.value.code == -1

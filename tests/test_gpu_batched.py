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


# ---- FP32 transforms + double-float refinement over the whole batch

def _batched32(grid, form, alphas, rhs, rhs_kind, n0_only, tol=0.0):
    B = len(alphas)
    with Q.Batch(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alphas=alphas, rhs_kind=rhs_kind,
                 precision=Q.FP32_REFINE, refine_tol=tol) as bt:
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.full((B * grid.Nx * (1 if n0_only else grid.nt),), float("nan"), dtype=torch.float64,
                       device="cuda")
        bt.solve(x, y, n0_only)
        torch.cuda.synchronize()
        return y.cpu().numpy().reshape(B, -1), bt.refine_info


GRIDS32 = [
    bi.Grid(1, (64,), 1.0, 0.1, 64),              # the 1D 63 x 64 shape (one-launch refinement)
    bi.Grid(2, (32, 16), 1.0, 0.1, 16),           # generic FP32 time tile (H = 8)
    bi.Grid(1, (32,), 1.0, 0.1, 64),              # 1D through the staged passes (register time solve)
    bi.Grid(3, (8, 8, 4), 1.0, 0.05, 128),
    bi.Grid(2, (10, 100), 1.0, 0.1, 256),         # mixed-radix DST lengths
]


@pytest.mark.parametrize("grid", GRIDS32, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM], ids=["pq", "pm"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
def test_fp32_refined_batch_matches_oracle(grid, form, rhs_kind):
    B = 6
    alphas = list(np.logspace(-3, -1, B)) if form == Q.FORM_PQ else list(grid.tau * np.logspace(-2, 0, B))
    F = np.stack([bi.random_general_rhs(grid, seed=170 + b) for b in range(B)])
    rhs = F[:, 0] if rhs_kind == Q.RHS_DELTA else F
    got, (iters, rel) = _batched32(grid, form, alphas, rhs, rhs_kind, False)
    # the refinement's contract: the tolerance (1e-13), or a stall at the
    # double-float floor (about kappa(A) 2^-48, which rises with |omega|: 1D
    # general right-hand sides at |omega| = 1e3 floor near 3e-12) below the
    # 1e-10 bar; above the bar the solve returns DIVERGED
    assert 1 <= iters <= 10 and rel <= 1e-10
    for b, a in enumerate(alphas):
        Ff = O.delta_rhs(grid, form, a, rhs[b]) if rhs_kind == Q.RHS_DELTA else rhs[b]
        want = O.solve_spectral(grid, form, a, Ff)
        assert O.rel_l2(got[b], want) <= TOL, (b, a)


def test_fp32_refined_batch_y0_only():
    grid = GRIDS32[0]
    alphas = [1e-4, 1e-3, 1e-2]
    g = np.stack([bi.random_general_rhs(grid, seed=180 + b)[0] for b in range(3)])
    full, _ = _batched32(grid, Q.FORM_PQ, alphas, g, Q.RHS_DELTA, False)
    y0, _ = _batched32(grid, Q.FORM_PQ, alphas, g, Q.RHS_DELTA, True)
    np.testing.assert_array_equal(y0, full.reshape(3, grid.nt, -1)[:, 0])


def test_fp32_refined_batch_of_the_1d_workload():
    """10 000 instances of the 1D 63 x 64 problem, alpha = each instance's own
    delta: every sampled instance within 1e-10 of the oracle."""
    B = 10_000
    base = bi.make_c1()
    grid = base.grid
    rng = np.random.default_rng(101)
    g = base.g[None, :] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, size=(B, grid.Nx)))
    alphas = list(np.sqrt(grid.h[0]) * np.linalg.norm(g - base.g[None, :], axis=1))
    got, (iters, rel) = _batched32(grid, Q.FORM_PQ, alphas, g, Q.RHS_DELTA, False)
    assert rel <= 1e-13
    for b in [0, 1, 4999, 9998, 9999]:
        want = O.solve_spectral(grid, O.PQ, alphas[b], O.delta_rhs(grid, O.PQ, alphas[b], g[b]))
        assert O.rel_l2(got[b], want) <= TOL
    assert np.isfinite(got).all()


def test_fp32_refined_batch_nonfinite_and_out_of_range():
    grid = GRIDS32[1]
    alphas = [1e-3, 1e-2]
    F = np.stack([bi.random_general_rhs(grid, seed=190 + b) for b in range(2)])
    bad = F.copy()
    bad[1].flat[7] = np.nan
    with pytest.raises(Q.QbvmError) as ei:
        _batched32(grid, Q.FORM_PQ, alphas, bad, Q.RHS_GENERAL, False)
    assert ei.value.code == -3
    # data FP32 cannot hold in one instance: the FP64 pipeline solves the batch
    tiny = F.copy()
    tiny[0] *= 1e-300
    got, (iters, rel) = _batched32(grid, Q.FORM_PQ, alphas, tiny, Q.RHS_GENERAL, False)
    assert iters == 0 and np.isnan(rel)
    for b, a in enumerate(alphas):
        sc = 1e300 if b == 0 else 1.0                   # keep numpy's norms out of underflow
        want = O.solve_spectral(grid, Q.FORM_PQ, a, tiny[b] * sc)
        assert O.rel_l2(got[b] * sc, want) <= TOL


@pytest.mark.parametrize("grid", [GRIDS32[0], GRIDS32[3]], ids=["1d", "2d-unequal"])
def test_fp32_refined_batch_is_never_silently_wrong(grid):
    """A batch that holds instances with |omega| up to 1e9: either every
    instance is within 1e-10 of the oracle with the largest residual at most
    the 1e-10 bar (a stall at the double-float floor), or DIVERGED."""
    alphas = [1e-2, 1e-5, 1e-9]
    F = np.stack([bi.random_general_rhs(grid, seed=200 + b) for b in range(3)])
    try:
        got, (iters, rel) = _batched32(grid, Q.FORM_PQ, alphas, F, Q.RHS_GENERAL, False)
    except Q.QbvmError as e:
        assert e.code == -4
        return
    assert rel <= 1e-10
    for b, a in enumerate(alphas):
        assert O.rel_l2(got[b], O.solve_spectral(grid, Q.FORM_PQ, a, F[b])) <= TOL

"""Parity with the CPU FP64 oracle on meshes whose DST-I length n = M - 1 is
not 2^k - 1 (Section 2 allows any M, h = L/M; Step (b) of eq. 3.8 runs on
that Laplacian).  Those lengths take the mixed-radix tile (radix 4, 2, 3, 5
passes and a direct DFT for any other prime factor: M = 129 = 3 x 43 has one).

Tolerance: relative L2 <= 1e-10 against the oracle, both formulations, both
right-hand-side kinds, in 2D and 3D, FP64 and FP32 + refinement.
"""
import math

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


def gpu_solve(grid, form, alpha, rhs, rhs_kind, n0_only=False, precision=Q.FP64, order=Q.ORDER_AUTO):
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, precision, rhs_kind,
                order=order) as plan:
        nout = grid.Nx * (1 if n0_only else grid.nt)
        inp = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
        out = torch.zeros(nout, dtype=torch.float64, device="cuda")
        plan.solve(inp, out, n0_only)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
    return res.reshape(((1,) if n0_only else (grid.nt,)) + grid.shape)


def oracle_solve(grid, form, alpha, F):
    if grid.unknowns <= 5000:
        return O.solve_sparse_lu(grid, form, alpha, F)
    return O.solve_spectral(grid, form, alpha, F)


def gid(g):
    return f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}"


GRIDS = [
    bi.Grid(2, (6, 10), 1.0, 0.1, 16),
    bi.Grid(2, (100, 129), 1.0, 0.1, 16),         # 129 = 3 x 43: a direct length-43 pass
    bi.Grid(2, (129, 6), math.pi, 1.0, 32),
    bi.Grid(2, (10, 100), 1.0, 0.1, 8),
    bi.Grid(2, (2, 3), 1.0, 0.1, 4),              # one and two interior points per axis
    bi.Grid(2, (7, 64), 1.0, 0.1, 8),             # prime M beside a power of two
    bi.Grid(3, (6, 10, 9), 1.0, 0.05, 8),
    bi.Grid(3, (129, 6, 10), 1.0, 0.05, 8),
    bi.Grid(3, (100, 5, 7), 1.0, 0.05, 4),
    bi.Grid(3, (3, 3, 3), 1.0, 0.05, 4),
]


@pytest.mark.parametrize("grid", GRIDS, ids=gid)
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_any_dst_length_matches_oracle(grid, form, rhs_kind):
    alpha = 1e-3 if form == Q.FORM_PQ else 1e-3 * grid.tau
    F = bi.random_general_rhs(grid, seed=31)
    if rhs_kind == Q.RHS_DELTA:
        want = oracle_solve(grid, form, alpha, O.delta_rhs(grid, form, alpha, F[0]))
        got = gpu_solve(grid, form, alpha, F[0], Q.RHS_DELTA)
    else:
        want = oracle_solve(grid, form, alpha, F)
        got = gpu_solve(grid, form, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("grid", [GRIDS[1], GRIDS[3], GRIDS[7]], ids=gid)
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_any_dst_length_fp32_refine(grid, rhs_kind):
    alpha = 1e-3
    F = bi.random_general_rhs(grid, seed=32)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    Ff = O.delta_rhs(grid, Q.FORM_PQ, alpha, F[0]) if rhs_kind == Q.RHS_DELTA else F
    want = oracle_solve(grid, Q.FORM_PQ, alpha, Ff)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind, precision=Q.FP32_REFINE)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("grid", [GRIDS[0], GRIDS[6]], ids=gid)
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_any_dst_length_n0_only(grid, rhs_kind):
    F = bi.random_general_rhs(grid, seed=33)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    full = gpu_solve(grid, Q.FORM_PQ, 1e-3, rhs, rhs_kind)
    y0 = gpu_solve(grid, Q.FORM_PQ, 1e-3, rhs, rhs_kind, n0_only=True)
    np.testing.assert_allclose(y0[0], full[0], rtol=0, atol=1e-13 * np.abs(full).max())


@pytest.mark.parametrize("m", [3, 6, 100, 129, 2047])
@pytest.mark.parametrize("order", [Q.ORDER_TIME_FIRST, Q.ORDER_SPACE_FIRST], ids=["time-first", "space-first"])
def test_1d_any_length_both_orders(m, order):
    """1D meshes of any M now run either order; AUTO takes the sine transform."""
    grid = bi.Grid(1, (m,), 1.0, 0.1, 16)
    alpha = 1e-2
    F = bi.random_general_rhs(grid, seed=34)
    want = oracle_solve(grid, Q.FORM_PQ, alpha, F)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL, order=order)
    assert O.rel_l2(got, want) <= TOL
    auto = gpu_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(auto, want) <= TOL


def test_largest_general_length():
    """M = 2048 takes the mixed-radix tile (radix 4^5 x 2), one column pair per tile."""
    grid = bi.Grid(2, (2048, 3), 1.0, 0.1, 4)
    F = bi.random_general_rhs(grid, seed=35)
    want = O.solve_spectral(grid, Q.FORM_PQ, 1e-3, F)
    got = gpu_solve(grid, Q.FORM_PQ, 1e-3, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL


def test_length_beyond_the_tiles_is_unsupported():
    with pytest.raises(Q.QbvmError) as e:
        Q.Plan(2, (2049, 8), 1.0, 0.1, 8, Q.FORM_PQ, 1e-3)
    assert e.value.code == -7


def test_batch_with_any_dst_length():
    """The batch entry point runs the same DST passes over every instance."""
    grid = bi.Grid(2, (10, 100), 1.0, 0.1, 16)
    alphas = [1e-3, 3e-3, 2e-2]
    F = np.stack([bi.random_general_rhs(grid, seed=36 + b) for b in range(len(alphas))])
    fin = torch.as_tensor(F.ravel(), dtype=torch.float64).cuda()
    y = torch.zeros(fin.numel(), dtype=torch.float64, device="cuda")
    with Q.Batch(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=alphas, rhs_kind=Q.RHS_GENERAL) as bt:
        bt.solve(fin, y)
        torch.cuda.synchronize()
    got = y.cpu().numpy().reshape((len(alphas),) + grid.full_shape)
    for b, a in enumerate(alphas):
        assert O.rel_l2(got[b], O.solve_spectral(grid, Q.FORM_PQ, a, F[b])) <= TOL

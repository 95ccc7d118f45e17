"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerance: relative L2 error <= 1e-10 against the oracle in FP64 (the accuracy
the FP64 solve is held to).  Small cases span several tiles and a ragged
tail; full-size cases compare sampled time levels the oracle computes one by
one.
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


def gpu_solve(grid, form, alpha, rhs, rhs_kind, n0_only=False, precision=Q.FP64, host=False, order=Q.ORDER_AUTO):
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, precision, rhs_kind,
                order=order) as plan:
        nout = grid.Nx * (1 if n0_only else grid.nt)
        if host:
            inp = np.ascontiguousarray(rhs, dtype=np.float64).ravel()
            out = np.zeros(nout)
            plan.solve(inp, out, n0_only)
            res = out
        else:
            inp = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
            out = torch.zeros(nout, dtype=torch.float64, device="cuda")
            plan.solve(inp, out, n0_only)
            torch.cuda.synchronize()
            res = out.cpu().numpy()
    shape = ((1,) if n0_only else (grid.nt,)) + grid.shape
    return res.reshape(shape)


def oracle_solve(grid, form, alpha, F):
    """Sparse LU of the assembled system (the oracle of record) on small grids;
    beyond that the sine-basis oracle, which the CPU suite pins to LU."""
    if grid.unknowns <= 5000:
        return O.solve_sparse_lu(grid, form, alpha, F)
    return O.solve_spectral(grid, form, alpha, F)


SMALL = [
    bi.Grid(1, (2,), 1.0, 0.1, 2),          # one interior point, N = 1
    bi.Grid(1, (5,), 1.0, 0.1, 4),
    bi.Grid(1, (64,), 1.0, 0.1, 64),        # C1 grid
    bi.Grid(1, (100,), math.pi, 1.0, 32),   # ragged tile tail
    bi.Grid(1, (301,), 1.0, 0.2, 128),
    bi.Grid(2, (4, 4), 1.0, 0.1, 2),
    bi.Grid(2, (8, 16), 1.0, 0.1, 8),       # unequal axes
    bi.Grid(2, (32, 32), 1.0, 0.1, 32),
    bi.Grid(2, (64, 64), math.pi, 1.0, 16),
    bi.Grid(3, (4, 8, 4), 1.0, 0.05, 4),
    bi.Grid(3, (16, 16, 16), 1.0, 0.05, 16),
    # register-resident time transforms: N_t/2 = 32, 64, 128, 256
    bi.Grid(2, (8, 32), 1.0, 0.1, 64),
    bi.Grid(3, (8, 8, 8), 1.0, 0.1, 128),
    bi.Grid(2, (16, 16), 1.0, 0.1, 256),
    bi.Grid(2, (16, 8), 1.0, 0.2, 512),
]


@pytest.mark.parametrize("grid", SMALL, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
def test_general_rhs_matches_oracle(grid, form):
    alpha = 1e-3 if form == Q.FORM_PQ else 1e-3 * grid.tau
    F = bi.random_general_rhs(grid, seed=7)
    want = oracle_solve(grid, form, alpha, F)
    got = gpu_solve(grid, form, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("grid", SMALL, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
def test_delta_rhs_matches_oracle(grid, form):
    g = bi.random_general_rhs(grid, seed=8)[0]
    alpha = 2e-4 if form == Q.FORM_PQ else 5e-2
    want = oracle_solve(grid, form, alpha, O.delta_rhs(grid, form, alpha, g))
    got = gpu_solve(grid, form, alpha, g, Q.RHS_DELTA)
    assert O.rel_l2(got, want) <= TOL


# nt not a power of two: Bluestein time DFTs (the paper's meshes have N_t = N + 1)
GENERAL_NT = [
    bi.Grid(1, (2,), 1.0, 0.1, 3),
    bi.Grid(1, (64,), 1.0, 0.1, 17),
    bi.Grid(1, (100,), math.pi, 1.0, 24),
    bi.Grid(1, (256,), math.pi, 1.0, 257),       # Table 1 mesh (M, N) = (256, 256)
    bi.Grid(2, (16, 16), math.pi, 1.0, 17),      # Table 2 mesh (16^2, 16)
    bi.Grid(2, (32, 32), math.pi, 1.0, 33),
    bi.Grid(2, (16, 8), 1.0, 0.1, 100),
    bi.Grid(2, (8, 8), 1.0, 0.1, 1000),
    bi.Grid(3, (8, 8, 8), 1.0, 0.05, 9),
    bi.Grid(3, (8, 4, 16), 1.0, 0.05, 12),
]


@pytest.mark.parametrize("grid", GENERAL_NT, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_general_nt_matches_oracle(grid, form, rhs_kind):
    alpha = 1e-3 if form == Q.FORM_PQ else 1e-3 * grid.tau
    F = bi.random_general_rhs(grid, seed=12)
    if rhs_kind == Q.RHS_DELTA:
        want = oracle_solve(grid, form, alpha, O.delta_rhs(grid, form, alpha, F[0]))
        got = gpu_solve(grid, form, alpha, F[0], Q.RHS_DELTA)
    else:
        want = oracle_solve(grid, form, alpha, F)
        got = gpu_solve(grid, form, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("grid", [bi.Grid(1, (64,), 1.0, 0.1, 33), bi.Grid(2, (16, 16), 1.0, 0.1, 65)],
                         ids=["1d", "2d"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_general_nt_n0_only(grid, rhs_kind):
    F = bi.random_general_rhs(grid, seed=13)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    full = gpu_solve(grid, Q.FORM_PQ, 1e-3, rhs, rhs_kind)
    y0 = gpu_solve(grid, Q.FORM_PQ, 1e-3, rhs, rhs_kind, n0_only=True)
    np.testing.assert_allclose(y0[0], full[0], rtol=0, atol=1e-13 * np.abs(full).max())


@pytest.mark.parametrize("grid", [bi.Grid(1, (64,), 1.0, 0.1, 64), bi.Grid(1, (256,), math.pi, 1.0, 33),
                                  bi.Grid(1, (1024,), math.pi, 1.0, 257), bi.Grid(1, (4,), 1.0, 0.1, 8)],
                         ids=lambda g: f"M{g.M[0]}-nt{g.nt}")
@pytest.mark.parametrize("order", [Q.ORDER_TIME_FIRST, Q.ORDER_SPACE_FIRST], ids=["time-first", "space-first"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_1d_both_orders_match_oracle(grid, order, rhs_kind):
    """1D with m a power of two runs either order: the tridiagonal (Thomas)
    solves of Section 3.3 after the time DFT, or the sine transform first."""
    alpha = 1e-3
    F = bi.random_general_rhs(grid, seed=15)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    Ff = O.delta_rhs(grid, Q.FORM_PQ, alpha, F[0]) if rhs_kind == Q.RHS_DELTA else F
    want = oracle_solve(grid, Q.FORM_PQ, alpha, Ff)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind, order=order)
    assert O.rel_l2(got, want) <= TOL
    y0 = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind, n0_only=True, order=order)
    np.testing.assert_allclose(y0[0], got[0], rtol=0, atol=1e-13 * np.abs(got).max())


def test_general_nt_paper_table1_mesh():
    """1D (0, pi), h = pi/1024, N_t = 1025 levels (the largest Table 1 mesh)."""
    grid = bi.Grid(1, (1024,), math.pi, 1.0, 1025)
    F = bi.random_general_rhs(grid, seed=14)
    alpha = 1e-4
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, F[0]))
    got = gpu_solve(grid, Q.FORM_PQ, alpha, F[0], Q.RHS_DELTA)
    assert O.rel_l2(got, want) <= TOL


# the largest size along each axis that the plan accepts
MAX_SIZES = [
    bi.Grid(2, (1024, 1024), 1.0, 0.1, 8),       # largest DST length
    bi.Grid(2, (16, 16), 1.0, 0.1, 1024),        # largest power-of-two nt
    bi.Grid(2, (8, 8), 1.0, 0.1, 2047),          # largest Bluestein nt (2048 is a power of two: 1024 is that limit)
    bi.Grid(3, (256, 256, 16), 1.0, 0.05, 4),
    bi.Grid(1, (16385,), 1.0, 0.1, 4),           # long 1D, time-first (m not a power of two)
]


@pytest.mark.parametrize("grid", MAX_SIZES, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
def test_maximum_sizes_match_oracle(grid):
    alpha = 1e-3
    F = bi.random_general_rhs(grid, seed=16)
    want = O.solve_sparse_lu(grid, Q.FORM_PQ, alpha, F) if grid.dim == 1 else O.solve_spectral(grid, Q.FORM_PQ, alpha, F)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL
    if grid.dim > 1 and grid.nt <= 1024 and (grid.nt & (grid.nt - 1)) == 0:
        got32 = gpu_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL, precision=Q.FP32_REFINE)
        assert O.rel_l2(got32, want) <= TOL


@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
def test_c1_workload(form):
    """1D, 63 interior points x 64 levels, alpha by the Section 5 rule."""
    p = bi.make_c1()
    grid = p.grid
    alpha = O.alpha_apriori(form, p.delta, grid.tau)
    want = O.solve_sparse_lu(grid, form, alpha, O.delta_rhs(grid, form, alpha, p.g_delta))
    got = gpu_solve(grid, form, alpha, p.g_delta, Q.RHS_DELTA)
    assert O.rel_l2(got, want) <= TOL
    # the reconstruction error is the oracle's
    assert abs(bi.discrete_l2(got[0] - p.z0, grid) - bi.discrete_l2(want[0] - p.z0, grid)) < 1e-9


@pytest.mark.parametrize("alpha", [1e-1, 1e-4, 1e-7])
def test_alpha_extremes_1d(alpha):
    grid = bi.Grid(1, (128,), 1.0, 0.1, 128)
    g = bi.random_general_rhs(grid, seed=9)[0]
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, g))
    got = gpu_solve(grid, Q.FORM_PQ, alpha, g, Q.RHS_DELTA)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("grid", [bi.Grid(1, (64,), 1.0, 0.1, 64), bi.Grid(2, (32, 16), 1.0, 0.1, 16),
                                  bi.Grid(3, (8, 8, 8), 1.0, 0.1, 8)],
                         ids=["1d", "2d", "3d"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_n0_only_and_host_pointers(grid, rhs_kind):
    alpha = 1e-3
    F = bi.random_general_rhs(grid, seed=10)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    full = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind)
    y0 = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind, n0_only=True)
    np.testing.assert_allclose(y0[0], full[0], rtol=0, atol=1e-12 * np.abs(full).max())
    host = gpu_solve(grid, Q.FORM_PQ, alpha, rhs, rhs_kind, host=True)
    np.testing.assert_array_equal(host, full)


@pytest.mark.parametrize("grid", [bi.Grid(2, (64, 32), 1.0, 0.1, 50), bi.Grid(3, (16, 8, 8), 1.0, 0.1, 64),
                                  bi.Grid(2, (256, 256), 1.0, 0.1, 32)],
                         ids=["2d-nt50", "3d-nt64", "2d-255sq-nt32"])
def test_host_pointers_pinned_and_pageable(grid):
    """Pinned, pageable and mixed host buffers: the level chunks' copies overlap
    DSTs that alternate between two compute streams; every result is bitwise
    the device-pointer solve."""
    F = bi.random_general_rhs(grid, seed=14)
    dev = gpu_solve(grid, Q.FORM_PM, 1e-3, F, Q.RHS_GENERAL)
    dev0 = gpu_solve(grid, Q.FORM_PM, 1e-3, F, Q.RHS_GENERAL, n0_only=True)
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PM, 1e-3, 0.0, Q.FP64, Q.RHS_GENERAL) as plan:
        hin = torch.as_tensor(F.ravel()).pin_memory()
        hout = torch.full((grid.unknowns,), float("nan"), dtype=torch.float64).pin_memory()
        for _ in range(2):                                   # second call reuses streams and events
            plan.solve(hin, hout)
            np.testing.assert_array_equal(hout.numpy().reshape(grid.full_shape), dev)
        h0 = torch.full((grid.Nx,), float("nan"), dtype=torch.float64).pin_memory()
        plan.solve(hin, h0, n0_only=True)
        np.testing.assert_array_equal(h0.numpy().reshape((1,) + grid.shape), dev0)
        pin = np.ascontiguousarray(F.ravel())
        for _ in range(2):
            pout = np.full(grid.unknowns, np.nan)
            plan.solve(pin, pout)                            # pageable: chunked copies
            np.testing.assert_array_equal(pout.reshape(grid.full_shape), dev)
        pout = np.full(grid.unknowns, np.nan)
        plan.solve(hin, pout)                                # pinned in, pageable out
        np.testing.assert_array_equal(pout.reshape(grid.full_shape), dev)


def test_inplace_general_rhs():
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16)
    F = bi.random_general_rhs(grid, seed=11)
    want = gpu_solve(grid, Q.FORM_PQ, 1e-3, F, Q.RHS_GENERAL)
    with Q.Plan(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, 1e-3, 0.0, Q.FP64, Q.RHS_GENERAL) as plan:
        buf = torch.as_tensor(F.ravel(), dtype=torch.float64).cuda()
        plan.solve(buf, buf)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(buf.cpu().numpy().reshape(grid.full_shape), want)


@pytest.mark.parametrize("grid", [bi.Grid(1, (50,), 1.0, 0.1, 16), bi.Grid(2, (16, 8), 1.0, 0.1, 8),
                                  bi.Grid(3, (8, 4, 8), 1.0, 0.1, 4)], ids=["1d", "2d", "3d"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_residual_matches_oracle(grid, rhs_kind):
    alpha = 3e-3
    F = bi.random_general_rhs(grid, seed=12)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    Ffull = O.delta_rhs(grid, Q.FORM_PM, alpha, F[0]) if rhs_kind == Q.RHS_DELTA else F
    y = bi.random_general_rhs(grid, seed=13)          # an arbitrary iterate
    want = O.rel_residual(grid, Q.FORM_PM, alpha, y, Ffull)
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PM, alpha, 0.0, Q.FP64, rhs_kind) as plan:
        yd = torch.as_tensor(y.ravel(), dtype=torch.float64).cuda()
        fd = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
        got = plan.residual(yd, fd)
        # and the solve's own residual is at rounding level
        out = torch.zeros_like(yd)
        plan.solve(fd, out)
        small = plan.residual(out, fd)
    assert abs(got - want) <= 1e-12 * want
    assert small < 1e-10


# --------------------------------------------------------------- full sizes

@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
def test_c2_full_size_delta(form):
    """2D 255^2 x 256, alpha by the a-priori rule: every level against the oracle."""
    p = bi.make_c2()
    grid = p.grid
    alpha = O.alpha_apriori(form, p.delta, grid.tau)
    want = O.solve_spectral(grid, form, alpha, O.rhs_block0(form, alpha, grid.tau, p.g_delta))
    got = gpu_solve(grid, form, alpha, p.g_delta, Q.RHS_DELTA)
    assert O.rel_l2(got, want) <= TOL


def test_c2_full_size_general_rhs():
    p = bi.make_c2()
    grid = p.grid
    alpha = O.alpha_apriori(Q.FORM_PQ, p.delta, grid.tau)
    F = bi.random_general_rhs(grid, seed=14)
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, F)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL)
    assert O.rel_l2(got, want) <= TOL


def test_c3_full_size_sampled_levels():
    """3D 127^3 x 128 (delta rhs): sampled time levels against the oracle."""
    p = bi.make_c3()
    grid = p.grid
    alpha = O.alpha_apriori(Q.FORM_PQ, p.delta, grid.tau)
    levels = [0, 1, 63, 127]
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.rhs_block0(Q.FORM_PQ, alpha, grid.tau, p.g_delta),
                            levels=levels)
    got = gpu_solve(grid, Q.FORM_PQ, alpha, p.g_delta, Q.RHS_DELTA)[levels]
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM], ids=["pq", "pm"])
def test_y0_only_full_size_delta(form):
    """y^0 alone from the delta right-hand side on 255^2 x 256 (one level of DSTs
    in narrow tiles around the per-mode factor) against the oracle."""
    p = bi.make_c2()
    grid = p.grid
    alpha = O.alpha_apriori(form, p.delta, grid.tau)
    y0 = gpu_solve(grid, form, alpha, p.g_delta, Q.RHS_DELTA, n0_only=True)
    want = O.solve_spectral(grid, form, alpha, O.delta_rhs(grid, form, alpha, p.g_delta), levels=[0])
    assert O.rel_l2(y0, want) <= TOL


@pytest.mark.parametrize("bad", [float("nan"), float("inf")], ids=["nan", "inf"])
def test_nonfinite_input_fp64_propagates_and_residual_reports(bad):
    """The asynchronous FP64 solve carries an injected NaN / Inf through by IEEE
    arithmetic (no status without a synchronisation); qbvm_residual reports it."""
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16)
    g = bi.random_general_rhs(grid, seed=15)[0].copy()
    g.flat[7] = bad
    with Q.Plan(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, 1e-3, 0.0, Q.FP64, Q.RHS_DELTA) as plan:
        gd = torch.as_tensor(g.ravel()).cuda()
        y = torch.zeros(grid.unknowns, dtype=torch.float64, device="cuda")
        plan.solve(gd, y)
        torch.cuda.synchronize()
        assert not bool(torch.isfinite(y).all())
        with pytest.raises(Q.QbvmError) as ei:
            plan.residual(y, gd)
        assert ei.value.code == -3

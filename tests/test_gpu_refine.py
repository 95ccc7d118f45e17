"""FP32 transforms with FP64 iterative refinement (precision QBVM_FP32_REFINE).

The refined solution must match the CPU FP64 oracle to the same 1e-10 relative
L2 bound as the FP64 path; the refinement statistics are reported through
qbvm_plan_info.
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


def refine_solve(grid, form, alpha, rhs, rhs_kind, n0_only=False, tol=0.0, maxit=0):
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP32_REFINE, rhs_kind,
                tol, maxit) as plan:
        inp = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
        out = torch.zeros(grid.Nx * (1 if n0_only else grid.nt), dtype=torch.float64, device="cuda")
        plan.solve(inp, out, n0_only)
        torch.cuda.synchronize()
        info = plan.info
        shape = ((1,) if n0_only else (grid.nt,)) + grid.shape
        return out.cpu().numpy().reshape(shape), info.last_refine_iters, info.last_rel_residual


GRIDS = [
    bi.Grid(2, (4, 4), 1.0, 0.1, 2),
    bi.Grid(2, (16, 32), 1.0, 0.1, 16),
    bi.Grid(2, (64, 64), 1.0, 0.1, 64),
    bi.Grid(3, (8, 4, 16), 1.0, 0.05, 8),
    bi.Grid(3, (32, 32, 32), 1.0, 0.05, 32),
    bi.Grid(2, (32, 16), 1.0, 0.1, 512),
    bi.Grid(3, (16, 16, 8), 1.0, 0.05, 128),
    # register-resident FP32 DST lengths (M = 64, 128, 256) along x and along y / z,
    # with ragged row and column tiles
    bi.Grid(2, (256, 128), 1.0, 0.1, 8),
    bi.Grid(2, (128, 256), 1.0, 0.1, 16),
    bi.Grid(3, (128, 64, 256), 1.0, 0.05, 4),
    bi.Grid(3, (64, 256, 128), 1.0, 0.05, 2),
    # 1D (space-first), including the C1 grid 63 x 64
    bi.Grid(1, (64,), 1.0, 0.1, 64),
    bi.Grid(1, (256,), math.pi, 1.0, 128),
    bi.Grid(1, (1024,), 1.0, 0.1, 32),
    bi.Grid(1, (8,), 1.0, 0.1, 16),
]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_refined_solution_matches_oracle(grid, form, rhs_kind):
    alpha = 1e-3 if form == Q.FORM_PQ else 1e-3 * grid.tau
    F = bi.random_general_rhs(grid, seed=31)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    Ffull = O.delta_rhs(grid, form, alpha, F[0]) if rhs_kind == Q.RHS_DELTA else F
    want = O.solve_spectral(grid, form, alpha, Ffull)
    got, iters, rel = refine_solve(grid, form, alpha, rhs, rhs_kind)
    assert O.rel_l2(got, want) <= TOL, (iters, rel)
    # the double-float residual floors at u^2 cond(Delta_h)-ish levels: ~1e-13 on
    # coarse grids, 7e-11 at 1D M = 1024; above 1e-10 the solve reports DIVERGED
    assert iters >= 1 and rel <= 1e-10


@pytest.mark.parametrize("grid", [bi.Grid(2, (256, 64), 1.0, 0.1, 32), bi.Grid(3, (64, 128, 64), 1.0, 0.05, 8)],
                         ids=["d2-M256x64", "d3-M64x128x64"])
def test_fp32_solve_alone_is_fp32_accurate(grid):
    """With a tolerance of 1 the first residual check passes, so y is the bare
    FP32 solve: its error against the oracle is that of FP32 transforms
    amplified by cond(V) = |omega|^(1 - 1/nt) (here 1e3), far from the O(1) of a
    wrong transform.  Its relative residual is FP32 rounding times the spatial
    condition number (about 4 M^2 / pi^2 = 2.7e4 at M = 256)."""
    alpha = 1e-3
    F = bi.random_general_rhs(grid, seed=35)
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, F)
    got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, F, Q.RHS_GENERAL, tol=1.0)
    err = O.rel_l2(got, want)
    assert iters == 0
    assert err <= 1e-3, err
    assert rel <= 1e-2


def test_refined_inplace_general_rhs():
    """F and y in one buffer: the refinement, which re-reads F after y is
    written, gives the out-of-place answer bit for bit."""
    grid = bi.Grid(2, (64, 32), 1.0, 0.1, 16)
    F = bi.random_general_rhs(grid, seed=36)
    want, _, _ = refine_solve(grid, Q.FORM_PQ, 1e-3, F, Q.RHS_GENERAL)
    with Q.Plan(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, 1e-3, 0.0, Q.FP32_REFINE, Q.RHS_GENERAL) as plan:
        buf = torch.as_tensor(F.ravel(), dtype=torch.float64).cuda()
        plan.solve(buf, buf)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(buf.cpu().numpy().reshape(grid.full_shape), want)


# one size on the generic shared-memory FP32 transforms and one on the
# register-resident ones (M = 64 ... 256, nt/2 = 32 ... 256)
HOST_LOOP = "generic-kernels"
DEVICE_LOOP = "register-kernels"


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
@pytest.mark.parametrize("scale", [1e-30, 1e-12, 1e12, 1e30])
def test_refinement_at_extreme_data_scales(scale, driver):
    """The solve is linear: data scaled by 1e+-12 stay on the FP32 path and
    give the scaled answer; at 1e+-30 FP32 cannot hold the residuals and the
    plan solves in FP64 (no refinement steps) -- the answer is right either way."""
    grid = bi.Grid(2, (64, 64), 1.0, 0.1, 32 if driver == HOST_LOOP else 64)
    g = bi.random_general_rhs(grid, seed=37)[0]
    alpha = 1e-3
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, g))
    got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, g * scale, Q.RHS_DELTA)
    assert O.rel_l2(got / scale, want) <= TOL
    if abs(np.log10(scale)) < 20:
        assert iters >= 1
    else:
        assert iters == 0 and rel <= 1e-13


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
def test_refined_n0_only(driver):
    grid = bi.Grid(2, (32, 32), 1.0, 0.1, 32) if driver == HOST_LOOP else bi.Grid(2, (64, 128), 1.0, 0.1, 64)
    F = bi.random_general_rhs(grid, seed=32)
    full, _, _ = refine_solve(grid, Q.FORM_PQ, 1e-3, F, Q.RHS_GENERAL)
    y0, _, _ = refine_solve(grid, Q.FORM_PQ, 1e-3, F, Q.RHS_GENERAL, n0_only=True)
    np.testing.assert_allclose(y0[0], full[0], rtol=0, atol=1e-13 * np.abs(full).max())


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
@pytest.mark.parametrize("alpha", [1e-6, 1e-8, 1e-9])
def test_refinement_is_never_silently_wrong(alpha, driver):
    """|omega| up to 1e9: the refinement either converges to the oracle's answer
    or reports QBVM_ERR_DIVERGED -- it never returns a wrong answer."""
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16) if driver == HOST_LOOP else bi.Grid(2, (64, 64), 1.0, 0.1, 64)
    g = bi.random_general_rhs(grid, seed=33)[0]
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, g))
    try:
        got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, g, Q.RHS_DELTA)
    except Q.QbvmError as e:
        assert e.code == -4
        return
    assert O.rel_l2(got, want) <= TOL, (iters, rel)


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
def test_refinement_to_the_floor_ends_cleanly(driver):
    """An unreachable tolerance: the corrections go on until they stop
    contracting at the double-float floor (three or more corrections), then the
    solve ends without an error and with the oracle's answer."""
    grid = bi.Grid(2, (32, 32), 1.0, 0.1, 64) if driver == HOST_LOOP else bi.Grid(2, (64, 128), 1.0, 0.1, 64)
    g = bi.random_general_rhs(grid, seed=35)[0]
    alpha = 1e-3
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, g))
    got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, g, Q.RHS_DELTA, tol=1e-300)
    assert iters >= 3 and rel <= 1e-10, (iters, rel)
    assert O.rel_l2(got, want) <= TOL


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
def test_refinement_cap_reports_divergence(driver):
    """A one-step cap with an unreachable tolerance ends with QBVM_ERR_DIVERGED
    (did not reach the tolerance; the iterate is left in y)."""
    grid = bi.Grid(2, (32, 32), 1.0, 0.1, 64) if driver == HOST_LOOP else bi.Grid(2, (64, 128), 1.0, 0.1, 64)
    g = bi.random_general_rhs(grid, seed=34)[0]
    with pytest.raises(Q.QbvmError) as ei:
        refine_solve(grid, Q.FORM_PQ, 1e-8, g, Q.RHS_DELTA, tol=1e-300, maxit=1)
    assert ei.value.code == -4


def test_c2_full_size_refined():
    p = bi.make_c2()
    grid = p.grid
    for form in (Q.FORM_PQ, Q.FORM_PM):
        alpha = O.alpha_apriori(form, p.delta, grid.tau)
        want = O.solve_spectral(grid, form, alpha, O.rhs_block0(form, alpha, grid.tau, p.g_delta))
        got, iters, rel = refine_solve(grid, form, alpha, p.g_delta, Q.RHS_DELTA)
        err = O.rel_l2(got, want)
        print(f"C2 form {form}: refinement steps {iters}, rel residual {rel:.2e}, rel err vs oracle {err:.2e}")
        assert err <= TOL


@pytest.mark.parametrize("M", [(64, 64, 64), (96, 64, 48)], ids=["equal", "unequal"])
def test_smooth_3d_refined(M):
    """Smooth 3D data (Gaussian bumps, discrete forward solution, 0.1% noise):
    the stencil's differences cancel to a few bits, so an inexact scaling or
    product anywhere in the double-float residual shows as a stall.  Both the
    equal-spacing and the per-axis stencil."""
    grid = bi.Grid(3, M, 1.0, 0.05, 32)
    rng = np.random.default_rng(41)
    z0 = bi.gaussian_bumps(grid, rng, 8)
    gd, delta = bi.add_noise_gaussian(grid, bi.forward_discrete(grid, z0), 1e-3, rng)
    alpha = O.alpha_apriori(Q.FORM_PQ, delta, grid.tau)
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.rhs_block0(Q.FORM_PQ, alpha, grid.tau, gd))
    got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, gd, Q.RHS_DELTA)
    assert rel <= 1e-13 and iters <= 3
    assert O.rel_l2(got, want) <= TOL


def test_c3_full_size_refined_sampled_levels():
    """3D 127^3 x 128: the FP32 solve with FP64 refinement against the oracle on
    sampled levels, and against the plain FP64 path on every level."""
    p = bi.make_c3()
    grid = p.grid
    alpha = O.alpha_apriori(Q.FORM_PQ, p.delta, grid.tau)
    levels = [0, 1, 64, 127]
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.rhs_block0(Q.FORM_PQ, alpha, grid.tau, p.g_delta),
                            levels=levels)
    got, iters, rel = refine_solve(grid, Q.FORM_PQ, alpha, p.g_delta, Q.RHS_DELTA)
    err = O.rel_l2(got[levels], want)
    print(f"C3: refinement steps {iters}, rel residual {rel:.2e}, rel err vs oracle (sampled) {err:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")], ids=["nan", "inf", "-inf"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
@pytest.mark.parametrize("n0_only", [False, True], ids=["full", "y0"])
def test_nonfinite_input_is_reported(bad, rhs_kind, n0_only, driver):
    """A NaN or an infinity injected into the input: QBVM_ERR_NONFINITE, never a
    silent result (full solution or y^0 alone)."""
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16) if driver == HOST_LOOP else bi.Grid(2, (64, 64), 1.0, 0.1, 64)
    F = bi.random_general_rhs(grid, seed=38)
    rhs = (F[0] if rhs_kind == Q.RHS_DELTA else F).copy()
    rhs.flat[rhs.size // 3] = bad
    with pytest.raises(Q.QbvmError) as ei:
        refine_solve(grid, Q.FORM_PQ, 1e-3, rhs, rhs_kind, n0_only=n0_only)
    assert ei.value.code == -3


@pytest.mark.parametrize("driver", [HOST_LOOP, DEVICE_LOOP])
@pytest.mark.parametrize("scale", [1e-300, 1e100])
@pytest.mark.parametrize("n0_only", [False, True], ids=["full", "y0"])
def test_data_fp32_cannot_hold_takes_the_fp64_pipeline(scale, n0_only, driver):
    """Finite data that flushes to zero in FP32 (1e-300) or overflows it (1e100;
    its squares still fit FP64's range for the residual): solved by the FP64
    pipeline, with the scaled answer."""
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16) if driver == HOST_LOOP else bi.Grid(2, (64, 64), 1.0, 0.1, 64)
    g = bi.random_general_rhs(grid, seed=39)[0]
    alpha = 1e-3
    want = O.solve_spectral(grid, Q.FORM_PQ, alpha, O.delta_rhs(grid, Q.FORM_PQ, alpha, g),
                            levels=[0] if n0_only else None)
    got, iters, _ = refine_solve(grid, Q.FORM_PQ, alpha, g * scale, Q.RHS_DELTA, n0_only=n0_only)
    assert iters == 0
    assert O.rel_l2(got / scale, want) <= TOL


def test_zero_input_gives_zero():
    grid = bi.Grid(2, (64, 64), 1.0, 0.1, 64)
    got, _, rel = refine_solve(grid, Q.FORM_PQ, 1e-3, np.zeros(grid.shape), Q.RHS_DELTA)
    assert not got.any() and rel == 0.0


# nt not a power of two: FP32 Bluestein time DFTs inside the refinement
GENERAL_NT = [
    bi.Grid(2, (16, 16), 3.141592653589793, 1.0, 17),     # Table 2 mesh (16^2, 16)
    bi.Grid(2, (32, 24), 1.0, 0.1, 100),
    bi.Grid(3, (8, 8, 8), 1.0, 0.05, 9),
    bi.Grid(1, (256,), 3.141592653589793, 1.0, 257),      # Table 1 mesh (256, 256)
    bi.Grid(2, (8, 8), 1.0, 0.1, 2047),                   # longest Bluestein length
]


@pytest.mark.parametrize("grid", GENERAL_NT, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL])
def test_refined_general_nt_matches_oracle(grid, form, rhs_kind):
    alpha = 1e-3 if form == Q.FORM_PQ else 1e-3 * grid.tau
    F = bi.random_general_rhs(grid, seed=51)
    rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
    Ff = O.delta_rhs(grid, form, alpha, F[0]) if rhs_kind == Q.RHS_DELTA else F
    want = O.solve_spectral(grid, form, alpha, Ff)
    got, iters, rel = refine_solve(grid, form, alpha, rhs, rhs_kind)
    assert rel <= 1e-10 and iters >= 1
    assert O.rel_l2(got, want) <= TOL

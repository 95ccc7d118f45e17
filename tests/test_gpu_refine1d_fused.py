"""The one-launch FP32 + double-float refinement of 1D batches (one CTA per
instance, the iterate in shared memory; Section 3.3 for the FP32 solve, the
all-at-once system of eqs. 3.3 / 3.6 for the residual) against the CPU FP64
oracle and against the FP64 batch.

Tolerance: relative L2 <= 1e-10 against the oracle per instance, the
refinement's own contract (each instance's residual <= refine_tol, or a stall
below the 1e-10 bar, else DIVERGED).
"""
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


def gid(g):
    return f"m{g.M[0]}-nt{g.nt}"


FUSED = [bi.Grid(1, (64,), 1.0, 0.1, 64), bi.Grid(1, (64,), 1.0, 0.1, 128), bi.Grid(1, (128,), 1.0, 0.1, 64),
         bi.Grid(1, (64,), 1.0, 0.1, 32), bi.Grid(1, (128,), 1.0, 0.1, 32), bi.Grid(1, (256,), 1.0, 0.1, 32)]


def run(grid, form, alphas, rhs, rhs_kind, n0_only=False, tol=0.0, host=False):
    B = len(alphas)
    with Q.Batch(1, grid.M, grid.L, grid.T, grid.nt, form, alphas=alphas, rhs_kind=rhs_kind,
                 precision=Q.FP32_REFINE, refine_tol=tol) as bt:
        nout = B * grid.Nx * (1 if n0_only else grid.nt)
        if host:
            x = np.ascontiguousarray(rhs, dtype=np.float64).ravel()
            y = np.full(nout, np.nan)
            bt.solve(x, y, n0_only)
            out = y
        else:
            x = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
            y = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
            bt.solve(x, y, n0_only)
            torch.cuda.synchronize()
            out = y.cpu().numpy()
        return out.reshape(B, -1), bt.refine_info, bt.refine_fused


def oracle(grid, form, a, rhs_b, rhs_kind):
    Ff = O.delta_rhs(grid, form, a, rhs_b) if rhs_kind == Q.RHS_DELTA else rhs_b
    return O.solve_spectral(grid, form, a, Ff)


def test_which_shapes_take_the_fused_kernel():
    for grid, fused in [(g, True) for g in FUSED] + [
            (bi.Grid(1, (32,), 1.0, 0.1, 64), False), (bi.Grid(1, (64,), 1.0, 0.1, 16), False),
            (bi.Grid(1, (128,), 1.0, 0.1, 128), False), (bi.Grid(1, (256,), 1.0, 0.1, 64), False),
            (bi.Grid(2, (64, 64), 1.0, 0.1, 64), False)]:
        with Q.Batch(grid.dim, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=[1e-3, 1e-2],
                     rhs_kind=Q.RHS_GENERAL, precision=Q.FP32_REFINE) as bt:
            assert bt.refine_fused is fused, grid


@pytest.mark.parametrize("grid", FUSED, ids=gid)
@pytest.mark.parametrize("form", [Q.FORM_PQ, Q.FORM_PM], ids=["pq", "pm"])
@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
def test_fused_matches_oracle(grid, form, rhs_kind):
    B = 6
    alphas = list(np.logspace(-3, -1, B)) if form == Q.FORM_PQ else list(grid.tau * np.logspace(-2, 0, B))
    F = np.stack([bi.random_general_rhs(grid, seed=300 + b) for b in range(B)])
    rhs = F[:, 0] if rhs_kind == Q.RHS_DELTA else F
    got, (iters, rel), fused = run(grid, form, alphas, rhs, rhs_kind)
    assert fused
    assert 1 <= iters <= 10 and rel <= 1e-10
    for b, a in enumerate(alphas):
        assert O.rel_l2(got[b], oracle(grid, form, a, rhs[b], rhs_kind)) <= TOL, (b, a)


def test_fused_matches_the_fp64_batch_on_the_1d_workload():
    """2 000 instances of the 63 x 64 problem, alpha = each instance's own
    delta: the fused refinement against the FP64 batch, instance by instance."""
    B = 2000
    base = bi.make_c1()
    grid = base.grid
    rng = np.random.default_rng(303)
    g = base.g[None, :] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, size=(B, grid.Nx)))
    alphas = list(np.sqrt(grid.h[0]) * np.linalg.norm(g - base.g[None, :], axis=1))
    got, (iters, rel), fused = run(grid, Q.FORM_PQ, alphas, g, Q.RHS_DELTA)
    assert fused and rel <= 1e-13
    with Q.Batch(1, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=alphas, rhs_kind=Q.RHS_DELTA) as bt:
        x = torch.as_tensor(g.ravel()).cuda()
        y = torch.zeros(B * grid.unknowns, dtype=torch.float64, device="cuda")
        bt.solve(x, y)
        ref = y.cpu().numpy().reshape(B, -1)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL
    for b in [0, 999, 1999]:
        assert O.rel_l2(got[b], oracle(grid, Q.FORM_PQ, alphas[b], g[b], Q.RHS_DELTA)) <= TOL


@pytest.mark.parametrize("rhs_kind", [Q.RHS_DELTA, Q.RHS_GENERAL], ids=["delta", "general"])
def test_fused_y0_only_and_host_pointers(rhs_kind):
    grid = FUSED[0]
    alphas = [1e-4, 1e-3, 1e-2]
    F = np.stack([bi.random_general_rhs(grid, seed=310 + b) for b in range(3)])
    rhs = F[:, 0] if rhs_kind == Q.RHS_DELTA else F
    full, _, _ = run(grid, Q.FORM_PQ, alphas, rhs, rhs_kind)
    y0, _, _ = run(grid, Q.FORM_PQ, alphas, rhs, rhs_kind, n0_only=True)
    np.testing.assert_array_equal(y0, full.reshape(3, grid.nt, -1)[:, 0])
    hst, _, _ = run(grid, Q.FORM_PQ, alphas, rhs, rhs_kind, host=True)
    np.testing.assert_array_equal(hst, full)


def test_fused_instances_stop_on_their_own_residual():
    """Instances that need different step counts: each ends within the
    tolerance and within 1e-10 of the oracle; the reported steps are the
    most any instance took."""
    grid = FUSED[0]
    alphas = [1e-1, 1e-3, 3e-2]
    F = np.stack([bi.random_general_rhs(grid, seed=320 + b) for b in range(3)])
    got, (iters, rel), _ = run(grid, Q.FORM_PQ, alphas, F, Q.RHS_GENERAL, tol=1e-12)
    assert rel <= 1e-10 and iters >= 1
    for b, a in enumerate(alphas):
        assert O.rel_l2(got[b], O.solve_spectral(grid, Q.FORM_PQ, a, F[b])) <= TOL


def test_fused_zero_nonfinite_and_out_of_range_instances():
    grid = FUSED[0]
    alphas = [1e-3, 1e-2, 3e-2]
    F = np.stack([bi.random_general_rhs(grid, seed=330 + b) for b in range(3)])
    # an all-zero instance: y = 0 exactly, the others refined as usual
    z = F.copy()
    z[1] = 0.0
    got, (iters, rel), _ = run(grid, Q.FORM_PQ, alphas, z, Q.RHS_GENERAL)
    assert iters >= 1 and rel <= 1e-10
    assert (got[1] == 0.0).all()
    for b in (0, 2):
        assert O.rel_l2(got[b], O.solve_spectral(grid, Q.FORM_PQ, alphas[b], z[b])) <= TOL
    # NaN in one instance: the FP64 pipeline solves the batch, then NONFINITE
    bad = F.copy()
    bad[2].flat[11] = np.nan
    with pytest.raises(Q.QbvmError) as ei:
        run(grid, Q.FORM_PQ, alphas, bad, Q.RHS_GENERAL)
    assert ei.value.code == -3
    # data FP32 cannot hold in one instance: the FP64 pipeline solves the batch
    tiny = F.copy()
    tiny[0] *= 1e-300
    got, (iters, rel), _ = run(grid, Q.FORM_PQ, alphas, tiny, Q.RHS_GENERAL)
    assert iters == 0 and np.isnan(rel)
    for b, a in enumerate(alphas):
        sc = 1e300 if b == 0 else 1.0                    # keep numpy's norms out of underflow
        assert O.rel_l2(got[b] * sc, O.solve_spectral(grid, Q.FORM_PQ, a, tiny[b] * sc)) <= TOL


def test_fused_is_never_silently_wrong():
    """|omega| up to 1e9: every instance within 1e-10 of the oracle with the
    largest residual at most the 1e-10 bar, or DIVERGED."""
    for grid in FUSED:
        alphas = [1e-2, 1e-5, 1e-9]
        F = np.stack([bi.random_general_rhs(grid, seed=340 + b) for b in range(3)])
        try:
            got, (iters, rel), _ = run(grid, Q.FORM_PQ, alphas, F, Q.RHS_GENERAL)
        except Q.QbvmError as e:
            assert e.code == -4
            continue
        assert rel <= 1e-10
        for b, a in enumerate(alphas):
            assert O.rel_l2(got[b], O.solve_spectral(grid, Q.FORM_PQ, a, F[b])) <= TOL

"""Batched alpha sweep (one persistent launch in a CUDA graph) against the oracle.

For every instance and alpha the oracle solves the full all-at-once system
(sine-basis exact solve) and measures the discrepancy ||y^N - g_delta|| and the
error ||y^0 - z0|| directly on the solution; the sweep computes them from y^0
in the sine basis.  The picked alpha follows the discrepancy principle
(largest alpha with discrepancy <= tau_dp * delta), and the y^0 it returns is
checked against the oracle at that alpha.
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

TAU_DP = 1.1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Q.build_library()
    Q.load_library()


def _problems():
    """Uneven batch: 1D and 2D, both formulations, several nt."""
    out = []
    specs = [((128,), 32, Q.FORM_PQ, 1e-3), ((64,), 64, Q.FORM_PM, 1e-2), ((256,), 16, Q.FORM_PQ, 1e-4),
             ((16, 32), 16, Q.FORM_PQ, 3e-3), ((32, 32), 64, Q.FORM_PM, 1e-3), ((64, 16), 8, Q.FORM_PQ, 1e-2)]
    for i, (M, nt, form, rel) in enumerate(specs):
        grid = bi.Grid(len(M), M, 1.0, 0.1, nt)
        rng = np.random.default_rng(100 + i)
        if grid.dim == 1:
            z0 = bi.sine_field(grid, [(1,), (2,), (5,)], rng.uniform(0.3, 1.0, 3))
        else:
            z0 = bi.sine_field(grid, [(1, 1), (2, 1), (1, 3)], rng.uniform(0.3, 1.0, 3))
        g = bi.forward_discrete(grid, z0)
        gd, delta = bi.add_noise_gaussian(grid, g, rel, rng)
        out.append((grid, form, z0, gd, delta))
    return out


def _oracle_sweep(grid, form, z0, gd, delta, alphas):
    disc, err, ys = [], [], []
    for a in alphas:
        y = O.solve_spectral(grid, form, a, O.delta_rhs(grid, form, a, gd))
        disc.append(bi.discrete_l2(y[-1] - gd, grid))
        err.append(bi.discrete_l2(y[0] - z0, grid))
        ys.append(y[0])
    disc, err = np.array(disc), np.array(err)
    ok = np.nonzero(disc <= TAU_DP * delta)[0]
    pick = int(ok[np.argmax(np.asarray(alphas)[ok])]) if len(ok) else int(np.argmin(disc))
    return disc, err, pick, ys


def _run_sweep(problems, precision, n_alpha=8, autotune=False, bases=None):
    dev = []
    insts = []
    for i, (grid, form, z0, gd, delta) in enumerate(problems):
        g = torch.as_tensor(gd.ravel(), dtype=torch.float64).cuda()
        z = torch.as_tensor(z0.ravel(), dtype=torch.float64).cuda()
        y0 = torch.zeros(grid.Nx, dtype=torch.float64, device="cuda")
        dev.append((g, z, y0))
        insts.append(dict(dim=grid.dim, m=grid.M, L=grid.L, T=grid.T, nt=grid.nt, form=form, delta=delta,
                          g=g, z0=z, y0=y0, **({} if bases is None else {"alpha_base": bases[i]})))
    sw = Q.Sweep(insts, n_alpha=n_alpha, log10_lo=-1.5, log10_hi=1.5, tau_dp=TAU_DP, precision=precision)
    if autotune:
        sw.autotune(repeats=2)
    sw.run()
    res = sw.read()
    y0s = [d[2].cpu().numpy() for d in dev]
    return sw, res, y0s, dev


@pytest.mark.parametrize("precision,tol", [(Q.FP64, 1e-9), (Q.FP32_REFINE, 2e-3)], ids=["fp64", "fp32"])
def test_sweep_matches_oracle(precision, tol):
    problems = _problems()
    sw, (alphas, disc, err, pick), y0s, _ = _run_sweep(problems, precision)
    try:
        for i, (grid, form, z0, gd, delta) in enumerate(problems):
            rule = O.alpha_apriori(form, delta, grid.tau)
            want_alphas = rule * 10.0 ** np.linspace(-1.5, 1.5, 8)
            np.testing.assert_allclose(alphas[i], want_alphas, rtol=1e-14)
            odisc, oerr, opick, oys = _oracle_sweep(grid, form, z0, gd, delta, want_alphas)
            np.testing.assert_allclose(disc[i], odisc, rtol=tol)
            np.testing.assert_allclose(err[i], oerr, rtol=tol)
            near = np.abs(odisc / (TAU_DP * delta) - 1.0) < 10 * tol
            if not near.any():
                assert pick[i, 0] == opick, (i, pick[i], opick, odisc, TAU_DP * delta)
            assert pick[i, 1] == int(np.argmin(oerr)) or abs(oerr[pick[i, 1]] / oerr.min() - 1) < 10 * tol
            # y^0 at the picked alpha is produced in FP64 in both precisions
            a = int(pick[i, 0])
            assert O.rel_l2(y0s[i], oys[a].ravel()) <= 1e-10
    finally:
        sw.close()


def test_fp64_sweep_double_float_and_fp64_instances_in_one_launch():
    """The FP64 sweep sums in double-float where the instance's tables (Re d,
    Im d, tau Lambda) lie inside [2^-30, 2^30] and in FP64 elsewhere: here
    T = 1e-12 puts tau Lambda near 1e-10, so that instance takes the FP64 sums
    inside the same persistent launch as two double-float ones.  All three at
    the FP64 sweep's 1e-9 against the oracle."""
    problems = _problems()[:2]
    grid = bi.Grid(1, (32,), 1.0, 1e-12, 16)
    rng = np.random.default_rng(190)
    z0 = bi.sine_field(grid, [(1,), (2,), (5,)], rng.uniform(0.3, 1.0, 3))
    gd, delta = bi.add_noise_gaussian(grid, bi.forward_discrete(grid, z0), 1e-3, rng)
    assert grid.tau * 4.0 * grid.M[0] ** 2 < 2.0 ** -30
    problems.append((grid, Q.FORM_PQ, z0, gd, delta))
    sw, (alphas, disc, err, pick), y0s, _ = _run_sweep(problems, Q.FP64)
    try:
        for i, (grid, form, z0, gd, delta) in enumerate(problems):
            odisc, oerr, opick, oys = _oracle_sweep(grid, form, z0, gd, delta, alphas[i])
            np.testing.assert_allclose(disc[i], odisc, rtol=1e-9)
            np.testing.assert_allclose(err[i], oerr, rtol=1e-9)
            assert O.rel_l2(y0s[i], oys[int(pick[i, 0])].ravel()) <= 1e-10
    finally:
        sw.close()


def test_sweep_graph_replay_and_autotune_are_consistent():
    problems = _problems()
    sw, (alphas, disc, err, pick), y0s, dev = _run_sweep(problems, Q.FP32_REFINE)
    try:
        for _ in range(3):                       # graph replays
            sw.run()
        a2, d2, e2, p2 = sw.read()
        np.testing.assert_array_equal(p2, pick)
        np.testing.assert_allclose(d2, disc, rtol=1e-12)
        cfg = sw.autotune(repeats=2)
        assert cfg.modes_per_thread in (1, 2, 4) and cfg.grid > 0 and cfg.ms > 0
        sw.run()
        a3, d3, e3, p3 = sw.read()
        np.testing.assert_array_equal(p3, pick)
        np.testing.assert_allclose(d3, disc, rtol=1e-5)
        y0_again = [d[2].cpu().numpy() for d in dev]
        for u, v in zip(y0_again, y0s):
            np.testing.assert_allclose(u, v, rtol=0, atol=1e-13 * np.abs(v).max())
    finally:
        sw.close()


def test_fp64_sweep_every_launch_shape_agrees():
    """The FP64 sweep's double-float scan at 1, 2 and 4 modes per thread and 1
    or 2 CTAs per SM: the same picks, discrepancies to 1e-12 (only the order of
    the block sums differs) and the same y^0 bit for bit (its stage does not
    depend on the shape)."""
    problems = _problems()
    sw, (alphas, disc, err, pick), y0s, dev = _run_sweep(problems, Q.FP64)
    try:
        for mpt in (1, 2, 4):
            for ctas in (1, 2):
                sw.set_config(mpt, ctas)
                sw.run()
                a2, d2, e2, p2 = sw.read()
                np.testing.assert_array_equal(p2, pick)
                np.testing.assert_allclose(d2, disc, rtol=1e-12)
                np.testing.assert_allclose(e2, err, rtol=1e-12)
                for d, v in zip(dev, y0s):
                    np.testing.assert_array_equal(d[2].cpu().numpy(), v)
    finally:
        sw.close()


def test_c4_style_batch_sampled():
    """A slice of the uneven 512-instance batch: sizes from the batch recipe,
    16 alphas; every instance's discrepancies checked against the oracle."""
    specs = [s for s in bi.batch_specs_c4() if np.prod(s["M"]) * s["nt"] <= 256 * 256 * 64][:12]
    problems = []
    for s in specs:
        grid = bi.Grid(s["dim"], tuple(s["M"]), 1.0, 0.1, s["nt"])
        rng = np.random.default_rng(s["seed"])
        modes = [(1,), (2,), (3,)] if grid.dim == 1 else [(1, 1), (2, 1), (1, 2)]
        z0 = bi.sine_field(grid, modes, rng.uniform(0.3, 1.0, 3))
        gd, delta = bi.add_noise_gaussian(grid, bi.forward_discrete(grid, z0), s["rel_noise"], rng)
        problems.append((grid, Q.FORM_PQ, z0, gd, delta))
    sw, (alphas, disc, err, pick), y0s, _ = _run_sweep(problems, Q.FP32_REFINE, n_alpha=16)
    try:
        for i, (grid, form, z0, gd, delta) in enumerate(problems):
            odisc, oerr, opick, oys = _oracle_sweep(grid, form, z0, gd, delta, alphas[i])
            np.testing.assert_allclose(disc[i], odisc, rtol=2e-3)
            assert O.rel_l2(y0s[i], oys[int(pick[i, 0])].ravel()) <= 1e-10
    finally:
        sw.close()


@pytest.mark.parametrize("ctas", [1, 8])
def test_bounded_wait_gives_up_and_the_context_survives(ctas):
    """The persistent kernel's wait on a counter that nothing advances gives up
    after its spin limit, raises the error flag (the other CTAs leave on it) and
    reports QBVM_ERR_TIMEOUT; a solve on the same context still works."""
    import ctypes
    lib = Q.load_library()
    secs = ctypes.c_double(-1.0)
    assert lib.qbvm_selftest_bounded_wait(ctas, ctypes.byref(secs), None) == -5
    assert 1e-3 < secs.value < 5.0
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 8)
    g = bi.random_general_rhs(grid, seed=5)[0]
    with Q.Plan(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, 1e-3, 0.0, Q.FP64, Q.RHS_DELTA) as plan:
        y = torch.empty(grid.unknowns, dtype=torch.float64, device="cuda")
        plan.solve(torch.as_tensor(g.ravel()).cuda(), y)
        torch.cuda.synchronize()
    want = O.solve_spectral(grid, O.PQ, 1e-3, O.delta_rhs(grid, O.PQ, 1e-3, g))
    assert O.rel_l2(y.cpu().numpy(), want) <= 1e-10


@pytest.mark.parametrize("precision", [Q.FP64, Q.FP32_REFINE], ids=["fp64", "fp32"])
def test_sweep_is_scale_invariant(precision):
    """At fixed alphas the sweep is linear in the data: g, z0 and delta scaled
    together by 1e-300 ... 1e200 (beyond FP32's range both ways, and past where
    FP64 squares overflow) give the same picks and the scaled discrepancies,
    errors and y^0.  The scan works on data scaled by a power of two near 1/delta."""
    problems = _problems()
    bases = [O.alpha_apriori(form, delta, grid.tau) for grid, form, z0, gd, delta in problems]
    sw, (alphas, disc, err, pick), y0s, _ = _run_sweep(problems, precision, bases=bases)
    sw.close()
    rtol = 1e-9 if precision == Q.FP64 else 1e-4      # the scaled inputs round differently
    for scale in (1e-300, 1e-20, 1e20, 1e200):
        scaled = [(grid, form, z0 * scale, gd * scale, delta * scale) for grid, form, z0, gd, delta in problems]
        sw2, (a2, d2, e2, p2), y2, _ = _run_sweep(scaled, precision, bases=bases)     # the same alphas
        try:
            np.testing.assert_allclose(a2, alphas, rtol=1e-14)
            np.testing.assert_array_equal(p2[:, 0], pick[:, 0])
            np.testing.assert_allclose(d2 / scale, disc, rtol=rtol)
            np.testing.assert_allclose(e2 / scale, err, rtol=rtol)
            for u, v in zip(y2, y0s):
                np.testing.assert_allclose(u / scale, v, rtol=0, atol=1e-10 * np.abs(v).max())
        finally:
            sw2.close()


def test_newton_reciprocal_against_ieee_division():
    """The FP64 scan's reciprocal (FP32 seed, two FP64 Newton steps) against the
    correctly rounded 1/d over magnitudes the scan meets and far beyond:
    within 4 ulp (2^-50 relative) of the IEEE quotient."""
    import ctypes
    rng = np.random.default_rng(61)
    d = np.concatenate([10.0 ** rng.uniform(-30, 30, 200_000), 1.0 + rng.uniform(0, 1e-9, 1000),
                        [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, 7.0 / 3.0]])
    dd = torch.as_tensor(d, dtype=torch.float64).cuda()
    out = ctypes.c_double(-1.0)
    rc = Q.load_library().qbvm_selftest_newton_rcp(dd.data_ptr(), dd.numel(), ctypes.byref(out),
                                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert 0.0 <= out.value <= 2.0 ** -50, out.value

"""qbvm_multi_*: full solves of instances of uneven shape (dim, m, nt), each with
its own form, alpha and right-hand side, in one persistent launch.  Every
instance must equal the oracle's solve of its own system to 1e-10 and the
single FP64 plan's result to rounding (the same tiles), on repeated runs of
the captured graph."""
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


SPECS = [
    (bi.Grid(1, (64,), 1.0, 0.1, 64), Q.FORM_PQ, 1e-3, Q.RHS_DELTA),
    (bi.Grid(2, (32, 16), 1.0, 0.1, 16), Q.FORM_PM, 2e-5, Q.RHS_GENERAL),
    (bi.Grid(3, (8, 16, 8), 1.0, 0.05, 8), Q.FORM_PQ, 1e-2, Q.RHS_GENERAL),
    (bi.Grid(1, (2048,), 1.0, 0.1, 2), Q.FORM_PQ, 1e-4, Q.RHS_GENERAL),   # one column pair per DST tile
    (bi.Grid(2, (128, 128), 1.0, 0.1, 512), Q.FORM_PQ, 1e-3, Q.RHS_DELTA),
    (bi.Grid(2, (4, 256), 1.0, 0.1, 1024), Q.FORM_PM, 1e-6, Q.RHS_DELTA),
    (bi.Grid(1, (1024,), 1.0, 0.1, 128), Q.FORM_PM, 3e-5, Q.RHS_GENERAL),
]


def _single(grid, form, alpha, rhs, rhs_kind):
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, rhs_kind) as plan:
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.zeros(grid.unknowns, dtype=torch.float64, device="cuda")
        plan.solve(x, y)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def test_uneven_instances_match_oracle_and_single_plans():
    insts, data = [], []
    for k, (grid, form, alpha, rhs_kind) in enumerate(SPECS):
        F = bi.random_general_rhs(grid, seed=300 + k)
        rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.full((grid.unknowns,), float("nan"), dtype=torch.float64, device="cuda")
        insts.append(dict(dim=grid.dim, m=grid.M, L=grid.L, T=grid.T, nt=grid.nt, form=form, alpha=alpha,
                          rhs_kind=rhs_kind, g_or_F=x, y=y))
        data.append((grid, form, alpha, rhs, rhs_kind, x, y))
    with Q.Multi(insts) as mp:
        info = mp.info
        assert info["unknowns"] == sum(g.unknowns for g, *_ in SPECS)
        for rep in range(3):                        # the graph replays; inputs are not modified
            for *_, y in data:
                y.fill_(float("nan"))
            mp.run()
            mp.check()
            for grid, form, alpha, rhs, rhs_kind, x, y in data:
                got = y.cpu().numpy()
                Ff = O.delta_rhs(grid, form, alpha, rhs) if rhs_kind == Q.RHS_DELTA else rhs
                want = O.solve_spectral(grid, form, alpha, Ff)
                assert O.rel_l2(got, want) <= TOL, (grid, rep)
                one = _single(grid, form, alpha, rhs, rhs_kind)
                np.testing.assert_allclose(got, one, rtol=0, atol=1e-13 * np.abs(one).max())


def test_many_small_uneven_instances():
    """300 instances of seven shapes interleaved: sampled ones against the oracle."""
    insts, keep = [], []
    rng = np.random.default_rng(7)
    for k in range(300):
        grid, form, alpha, rhs_kind = SPECS[k % 3]
        a = alpha * 10.0 ** rng.uniform(-1, 1)
        F = bi.random_general_rhs(grid, seed=400 + k)
        rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
        x = torch.as_tensor(np.ascontiguousarray(rhs).ravel()).cuda()
        y = torch.empty(grid.unknowns, dtype=torch.float64, device="cuda")
        insts.append(dict(dim=grid.dim, m=grid.M, L=grid.L, T=grid.T, nt=grid.nt, form=form, alpha=a,
                          rhs_kind=rhs_kind, g_or_F=x, y=y))
        keep.append((grid, form, a, rhs, rhs_kind, y))
    with Q.Multi(insts) as mp:
        mp.run()
        mp.check()
        for k in (0, 1, 2, 150, 298, 299):
            grid, form, a, rhs, rhs_kind, y = keep[k]
            Ff = O.delta_rhs(grid, form, a, rhs) if rhs_kind == Q.RHS_DELTA else rhs
            assert O.rel_l2(y.cpu().numpy(), O.solve_spectral(grid, form, a, Ff)) <= TOL


def test_unsupported_shapes_are_refused():
    g = torch.zeros(100 * 8, dtype=torch.float64, device="cuda")
    y = torch.zeros(100 * 8, dtype=torch.float64, device="cuda")
    for m, nt in (((101,), 8), ((64,), 24), ((4096,), 8)):
        with pytest.raises(Q.QbvmError) as e:
            Q.Multi([dict(dim=1, m=m, T=0.1, nt=nt, alpha=1e-3, rhs_kind=Q.RHS_GENERAL, g_or_F=g, y=y)])
        assert e.value.code == -7
    with pytest.raises(Q.QbvmError) as e:
        Q.Multi([dict(dim=1, m=(64,), T=0.1, nt=8, alpha=1e-3, rhs_kind=Q.RHS_GENERAL, g_or_F=np.zeros(504),
                      y=np.zeros(504))])
    assert e.value.code == -1

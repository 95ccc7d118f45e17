"""The original QBVM / MQBVM systems (Section 2) by GMRES with the PinT solve
as preconditioner, against the oracle's sparse LU of the assembled A_h / B_h,
and the QBVM / MQBVM rows of Table 2 on their printed meshes."""
import math
import os

import numpy as np
import pytest

import bhcp_inputs as bi
import oracle as O
from oracle.qbvm_oracle import solve_original

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402

TOL = 1e-10
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Q.build_library()
    Q.load_library()


# The original systems are far worse conditioned than the PinT systems: in
# FP64 their true relative residual floors near 1e-12 .. 1e-9 (the sparse LU
# solution's own residual is of that size).  GMRES is held to the direct
# solution's residual, and its iterate to the direct solution.
def gmres_solve(grid, method, alpha, g, tol=1e-12, max_iters=300, restart=30, raise_on_diverged=True):
    form = Q.FORM_PQ if method == Q.ORIGINAL_QBVM else Q.FORM_PM
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, Q.RHS_GENERAL) as plan:
        with Q.GMRES(plan, method, restart) as gm:
            gd = torch.as_tensor(np.ascontiguousarray(g).ravel(), dtype=torch.float64).cuda()
            y = torch.empty(grid.unknowns, dtype=torch.float64, device="cuda")
            iters, rel = gm.solve(gd, y, tol=tol, max_iters=max_iters, raise_on_diverged=raise_on_diverged)
            torch.cuda.synchronize()
            return y.cpu().numpy().reshape(grid.full_shape), iters, rel


def lu_residual(grid, method, alpha, g, y):
    A = O.assemble_original(grid, method, alpha)
    f = np.zeros(grid.full_shape)
    f[0] = g
    return float(np.linalg.norm(f.ravel() - A @ y.ravel()) / np.linalg.norm(f))


def cond1_estimate(grid, method, alpha):
    """kappa_1(A) = ||A||_1 ||A^-1||_1, the inverse's norm by the 1-norm
    estimator of Higham and Tisseur (scipy onenormest) on the sparse LU."""
    import scipy.sparse.linalg as spla
    A = O.assemble_original(grid, method, alpha).tocsc()
    lu = spla.splu(A)
    inv = spla.LinearOperator(A.shape, matvec=lu.solve, rmatvec=lambda v: lu.solve(v, trans="T"), dtype=float)
    return float(spla.onenormest(A) * spla.onenormest(inv))


GRIDS = [
    bi.Grid(1, (64,), 1.0, 0.1, 16),
    bi.Grid(1, (32,), math.pi, 1.0, 17),          # nt not a power of two: Bluestein preconditioner
    bi.Grid(2, (16, 16), math.pi, 1.0, 17),       # the Table 2 mesh (16^2, 16)
    bi.Grid(2, (8, 16), 1.0, 0.1, 8),
    bi.Grid(3, (8, 4, 4), 1.0, 0.05, 5),
]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: f"d{g.dim}-M{'x'.join(map(str, g.M))}-nt{g.nt}")
@pytest.mark.parametrize("method", [Q.ORIGINAL_QBVM, Q.ORIGINAL_MQBVM], ids=["qbvm", "mqbvm"])
@pytest.mark.parametrize("alpha", [1e-2, 1e-4])
def test_original_system_matches_sparse_lu(grid, method, alpha):
    g = bi.random_general_rhs(grid, seed=21)[0]
    name = "qbvm" if method == Q.ORIGINAL_QBVM else "mqbvm"
    want = solve_original(grid, name, alpha, g)
    floor = lu_residual(grid, name, alpha, g, want)
    # iterate to the FP64 floor (GMRES stops once a restart cycle gains < 10 %)
    got, iters, rel = gmres_solve(grid, method, alpha, g, tol=1e-15, raise_on_diverged=False)
    assert rel <= max(1e-12, 3.0 * floor), (rel, floor)
    assert O.rel_l2(got, want) <= TOL, (iters, rel)
    assert iters <= 200


def test_divergence_is_reported():
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16)
    g = bi.random_general_rhs(grid, seed=22)[0]
    with pytest.raises(Q.QbvmError) as ei:
        gmres_solve(grid, Q.ORIGINAL_QBVM, 0.5, g, tol=1e-300, max_iters=1)
    assert ei.value.code == -4


def test_reachable_tolerance_converges():
    grid = bi.Grid(2, (16, 16), 1.0, 0.1, 16)
    g = bi.random_general_rhs(grid, seed=23)[0]
    _, iters, rel = gmres_solve(grid, Q.ORIGINAL_MQBVM, 1e-2, g, tol=1e-8)
    assert rel <= 1e-8 and iters >= 1


def _table2_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_table2_ex2_pint_errors.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                if p[0] in ("qbvm", "mqbvm"):
                    rows.append((p[0], int(p[1]), int(p[2]), [float(v) for v in p[3:]]))
    return rows


@pytest.mark.parametrize("row", _table2_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table2_original_methods_on_gpu(row):
    """Table 2's QBVM and MQBVM rows (alpha = delta, as the oracle's pins): the
    seed-averaged e_h within 20 % of the printed value; on the 16^2 mesh every
    solve also equals the oracle's sparse LU to 1e-10, or within the perturbation
    bound kappa (r_gmres + r_lu) where the system's conditioning puts the two
    direct and iterative FP64 solutions further apart (on 32^2 the LU takes
    ~10 s per solve; its e_h, 1.019/1.002/1.000/0.999 and 0.298/0.123/0.103/0.101,
    lies within 1 % of the printed values)."""
    method, M, N, printed = row
    mid = Q.ORIGINAL_QBVM if method == "qbvm" else Q.ORIGINAL_MQBVM
    out = []
    for eps, want in zip([1e-1, 1e-2, 1e-3, 1e-4], printed):
        errs = []
        for seed in range(3):
            p = bi.make_paper_ex2(M, N, eps, seed=seed)
            y, iters, rel = gmres_solve(p.grid, mid, p.delta, p.g_delta, tol=1e-15, raise_on_diverged=False)
            assert rel <= 1e-8, (iters, rel)          # iterated to the FP64 floor
            if M <= 16:
                ref = solve_original(p.grid, method, p.delta, p.g_delta)
                # two solutions with relative residuals r1, r2 differ by at most
                # kappa (r1 + r2); at alpha = delta kappa reaches ~1e3 here
                r_lu = lu_residual(p.grid, method, p.delta, p.g_delta, ref)
                diff = O.rel_l2(y, ref)
                if diff > TOL:
                    kappa = cond1_estimate(p.grid, method, p.delta)
                    assert diff <= kappa * (rel + r_lu), (diff, kappa, rel, r_lu)
            errs.append(bi.discrete_l2(y[0] - p.z0, p.grid))
        got = float(np.mean(errs))
        out.append(got)
        assert abs(got - want) <= 0.2 * want, (method, M, eps, got, want)
    print(f"{method} M={M}: GPU e_h {', '.join(f'{v:.3f}' for v in out)}  printed {printed}")

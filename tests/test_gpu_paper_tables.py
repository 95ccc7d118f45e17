"""The paper's own meshes on the GPU: Tables 1 and 2 (Section 5) through the
CUDA solve.  Each PinT-QBVM / PinT-MQBVM row is run at its printed mesh
(h = pi/M, tau = T/N, N_t = N + 1 levels: the Bluestein time DFTs) with the
a-priori alpha of Section 5; every y^0 must equal the oracle's to 1e-10, and the
seed-averaged reconstruction error e_h must fall in the same band around the
printed value as the oracle's own pins (20 % for Table 2, 30 % for Table 1).
Every row runs in FP64 and in FP32 + double-float refinement (FP32 Bluestein
time DFTs)."""
import os

import numpy as np
import pytest

import bhcp_inputs as bi
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = [1e-1, 1e-2, 1e-3, 1e-4]
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Q.build_library()
    Q.load_library()


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                if parts[0].startswith("pint"):
                    rows.append((parts[0], int(parts[1]), int(parts[2]), [float(v) for v in parts[3:]]))
    return rows


def _gpu_y0(p, form, precision):
    grid = p.grid
    alpha = O.alpha_apriori(form, p.delta, grid.tau)
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, precision, Q.RHS_DELTA) as plan:
        g = torch.as_tensor(np.ascontiguousarray(p.g_delta).ravel(), dtype=torch.float64).cuda()
        y0 = torch.empty(grid.Nx, dtype=torch.float64, device="cuda")
        plan.solve(g, y0, n0_only=True)
        torch.cuda.synchronize()
        got = y0.cpu().numpy().reshape(grid.shape)
    want = O.solve_spectral(grid, form, alpha, O.delta_rhs(grid, form, alpha, p.g_delta), levels=[0])[0]
    assert O.rel_l2(got, want) <= TOL
    return got


def _check_row(make, method, M, N, printed, seeds, band, precision):
    form = O.PQ if method == "pint-qbvm" else O.PM
    out = []
    for eps, want in zip(EPS, printed):
        errs = []
        for seed in range(seeds):
            p = make(M, N, eps, seed=seed)
            y0 = _gpu_y0(p, Q.FORM_PQ if form == O.PQ else Q.FORM_PM, precision)
            errs.append(bi.discrete_l2(y0 - p.z0, p.grid))
        got = float(np.mean(errs))
        out.append(got)
        assert abs(got - want) <= band * want, (method, M, eps, got, want)
    print(f"{method} M={M} N={N}: GPU e_h {', '.join(f'{v:.3f}' for v in out)}  printed {printed}")


PRECISIONS = pytest.mark.parametrize("precision", [Q.FP64, Q.FP32_REFINE], ids=["fp64", "fp32-refine"])


@PRECISIONS
@pytest.mark.parametrize("row", _read_table("paper_table2_ex2_pint_errors.txt"), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table2_example2_on_gpu(row, precision):
    method, M, N, printed = row
    _check_row(bi.make_paper_ex2, method, M, N, printed, seeds=3, band=0.2, precision=precision)


@PRECISIONS
@pytest.mark.parametrize("row", _read_table("paper_table1_ex1_pint_errors.txt"), ids=lambda r: f"{r[0]}-{r[1]}")
def test_table1_example1_on_gpu(row, precision):
    method, M, N, printed = row
    _check_row(bi.make_paper_ex1, method, M, N, printed, seeds=6, band=0.3, precision=precision)

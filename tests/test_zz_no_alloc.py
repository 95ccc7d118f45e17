"""qbvm_residual_noalloc: the residual for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: their HBM is reserved by another
allocator or pool, or they run monitoring loops that must not change the
device-memory footprint or pay for an allocation.  This entry point needs no
plan and keeps its scratch in a static device array.  The test calls it
through the C ABI twice in a row (with different data, so a stale scratch
would show) and checks each result against the plan-based qbvm_residual, to
the 1e-12 relative tolerance the residual tests use.  It also checks that host
pointers are refused instead of staged.

This file is collected last on purpose; it passes run alone in a fresh process
or after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import bhcp_inputs as bi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    Q.build_library()
    return Q.load_library()


def _noalloc(lib, desc, y, f):
    out = ctypes.c_double(-1.0)
    rc = lib.qbvm_residual_noalloc(ctypes.byref(desc), y.data_ptr(), f.data_ptr(), ctypes.byref(out),
                                   torch.cuda.current_stream().cuda_stream)
    return rc, out.value


CASES = [
    (bi.Grid(1, (64,), 1.0, 0.1, 64), Q.FORM_PQ, Q.RHS_DELTA),
    (bi.Grid(2, (32, 16), 1.0, 0.1, 16), Q.FORM_PM, Q.RHS_GENERAL),
    (bi.Grid(3, (8, 16, 8), 1.0, 0.05, 8), Q.FORM_PQ, Q.RHS_GENERAL),
    (bi.Grid(2, (256, 256), 1.0, 0.1, 256), Q.FORM_PQ, Q.RHS_DELTA),
]


@pytest.mark.parametrize("grid,form,rhs_kind", CASES, ids=["1d", "2d", "3d", "2d-255sq-x256"])
def test_noalloc_residual_matches_plan_residual(lib, grid, form, rhs_kind):
    alpha = 2e-3
    desc = Q.make_desc(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, rhs_kind)
    with Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, rhs_kind) as plan:
        for call, seed in enumerate((21, 22)):          # two calls in a row, different data
            F = bi.random_general_rhs(grid, seed=seed)
            rhs = F[0] if rhs_kind == Q.RHS_DELTA else F
            f = torch.as_tensor(np.ascontiguousarray(rhs).ravel(), dtype=torch.float64).cuda()
            y = torch.as_tensor(bi.random_general_rhs(grid, seed=seed + 100).ravel(), dtype=torch.float64).cuda()
            if call == 1:                                 # a near-solution: tiny residual
                plan.solve(f, y)
            want = plan.residual(y, f)
            rc, got = _noalloc(lib, desc, y, f)
            assert rc == 0, Q.qbvm_strerror(rc)
            assert abs(got - want) <= REL_TOL * abs(want), (call, got, want)


def test_noalloc_residual_refuses_host_pointers(lib):
    grid = bi.Grid(1, (16,), 1.0, 0.1, 8)
    desc = Q.make_desc(1, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, 1e-3, 0.0, Q.FP64, Q.RHS_GENERAL)
    y = np.zeros(grid.unknowns)
    f = np.ones(grid.unknowns)
    out = ctypes.c_double()
    rc = lib.qbvm_residual_noalloc(ctypes.byref(desc), y.ctypes.data, f.ctypes.data, ctypes.byref(out), None)
    assert rc == -1

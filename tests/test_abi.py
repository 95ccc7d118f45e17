"""The C ABI library: it builds for sm_103a, loads, exports every entry point
declared in include/*.h, and rejects invalid descriptors before touching a GPU."""
import glob
import os
import re

import pytest

import paper_2107_06381_gb300 as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        # return type of one or more words ("int", "const char*", "long long"), then the name
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*\s*\**\s+)+\**\s*(qbvm_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    Q.build_library()
    return Q.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("qbvm_plan", "qbvm_solve", "qbvm_residual", "qbvm_destroy", "qbvm_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version_and_strerror(lib):
    assert Q.qbvm_version() >= 100
    assert Q.qbvm_strerror(0) == "success"
    assert "argument" in Q.qbvm_strerror(-1)
    assert Q.qbvm_strerror(12345) == "unknown status code"


BAD = [
    dict(dim=0), dict(dim=4), dict(m=(1, 8, 8)), dict(nt=1), dict(T=0.0), dict(T=float("nan")),
    dict(L=-1.0), dict(form=2), dict(precision=5), dict(rhs_kind=3),
    dict(alpha=0.0, delta=0.0), dict(alpha=-1.0, delta=-1.0), dict(alpha=float("inf")),
    dict(order=3), dict(order=-1), dict(order=1),       # time-first exists in 1D only
]


@pytest.mark.parametrize("change", BAD, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_bad_descriptors_are_rejected_without_a_gpu(lib, change):
    args = dict(dim=2, m=(16, 16, 1), L=1.0, T=0.1, nt=16, form=0, alpha=1e-3, delta=0.0, precision=0, rhs_kind=0,
                order=0)
    args.update(change)
    desc = Q.make_desc(args["dim"], args["m"], args["L"], args["T"], args["nt"], args["form"], args["alpha"],
                       args["delta"], args["precision"], args["rhs_kind"], order=args["order"])
    with pytest.raises(Q.QbvmError) as ei:
        Q.qbvm_plan(desc)
    assert ei.value.code == -1


@pytest.mark.parametrize("change", [dict(nt=2049, precision=1), dict(nt=2048), dict(nt=2049), dict(m=(2049, 16, 1)),
                                    dict(m=(16, 4096, 1))],
                         ids=["nt2049-fp32", "nt2048", "nt2049", "m2049", "m4096"])
def test_unsupported_sizes(lib, change):
    """Power-of-two nt up to 1024; other nt (Bluestein time DFTs) up to 2048;
    DST lengths M - 1 with M up to 2048 (any M)."""
    args = dict(dim=2, m=(16, 16, 1), nt=16, precision=0)
    args.update(change)
    desc = Q.make_desc(2, args["m"], 1.0, 0.1, args["nt"], 0, 1e-3, 0.0, args["precision"])
    with pytest.raises(Q.QbvmError) as ei:
        Q.qbvm_plan(desc)
    assert ei.value.code == -7


def test_fp32_refinement_needs_the_space_first_order(lib):
    for m, order in (((4000,), Q.ORDER_AUTO), ((64,), Q.ORDER_TIME_FIRST)):
        desc = Q.make_desc(1, m, 1.0, 0.1, 16, 0, 1e-3, 0.0, Q.FP32_REFINE, order=order)
        with pytest.raises(Q.QbvmError) as ei:
            Q.qbvm_plan(desc)
        assert ei.value.code == -7


def test_space_first_needs_a_dst_length(lib):
    desc = Q.make_desc(1, (4000,), 1.0, 0.1, 16, 0, 1e-3, order=Q.ORDER_SPACE_FIRST)
    with pytest.raises(Q.QbvmError) as ei:
        Q.qbvm_plan(desc)
    assert ei.value.code == -7


def test_null_arguments(lib):
    import ctypes
    assert lib.qbvm_plan(None, None) == -1
    assert lib.qbvm_solve(None, None, None, 0, None) == -1
    out = ctypes.c_double()
    assert lib.qbvm_residual(None, None, None, ctypes.byref(out), None) == -1
    assert lib.qbvm_destroy(None) == 0


@pytest.mark.parametrize("case", [
    dict(count=0, code=-1), dict(alphas=[1e-3, -1.0], code=-1), dict(alphas=[float("nan")], code=-1),
    dict(precision=1, dim=1, m=(4, 1, 1), nt=2, code=-7), dict(nt=24, code=-7), dict(dim=1, m=(4000, 1, 1), code=-7),
    dict(dim=1, m=(64, 1, 1), order=1, code=-7), dict(dim=0, code=-1)],
    ids=["count0", "alpha-neg", "alpha-nan", "fp32-nt-nx-not-div4", "nt24", "1d-m4000", "1d-time-first", "dim0"])
def test_batch_plan_rejects_before_a_gpu(lib, case):
    """qbvm_batch_plan: same-shape space-first batches with power-of-two nt (FP32
    refinement: nt * Nx divisible by 4); everything else is refused on the host."""
    import ctypes
    a = dict(dim=2, m=(16, 16, 1), nt=16, precision=0, order=0, count=2, alphas=None)
    a.update(case)
    desc = Q.make_desc(a["dim"], a["m"], 1.0, 0.1, a["nt"], 0, 1e-3, 0.0, a["precision"], order=a["order"])
    arr = None
    n = a["count"]
    if a["alphas"] is not None:
        arr = (ctypes.c_double * len(a["alphas"]))(*a["alphas"])
        n = len(a["alphas"])
    h = ctypes.c_void_p()
    assert lib.qbvm_batch_plan(ctypes.byref(desc), n, arr, ctypes.byref(h)) == case["code"]
    assert not h.value


def test_selftest_rejects_bad_cta_counts(lib):
    assert lib.qbvm_selftest_bounded_wait(0, None, None) == -1
    assert lib.qbvm_selftest_bounded_wait(65, None, None) == -1


def test_abi_from_plain_c(lib):
    """include/qbvm.h compiles as C99 and the library links into a C program;
    the host-side checks hold there too (tests/native/abi_c_check.c)."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_2107_06381_gb300", "_lib")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "abi_c_check")
        subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", exe,
                        os.path.join(ROOT, "tests", "native", "abi_c_check.c"), "-L", libdir, "-lqbvm",
                        "-Wl,-rpath," + libdir], check=True, capture_output=True)
        res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert res.returncode == 0, res.stdout + res.stderr
        assert "0 failures" in res.stdout


def test_every_exported_entry_point_is_declared(lib):
    """No C entry point is exported without a declaration (and its documentation)
    in include/qbvm.h: the exported qbvm_* names (nm, the library's own symbol
    table) equal the declared ones."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    so = os.path.join(ROOT, "paper_2107_06381_gb300", "_lib", "libqbvm.so")
    out = subprocess.run([nm, "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("qbvm_")}
    assert exported == set(_declared_functions()), (exported ^ set(_declared_functions()))


def test_every_status_code_has_its_own_message(lib):
    text = open(os.path.join(ROOT, "include", "qbvm.h")).read()
    codes = {int(v) for v in re.findall(r"#define QBVM_ERR_[A-Z_]+\s+(-\d+)", text)}
    assert codes == set(range(-7, 0))
    msgs = [Q.qbvm_strerror(c) for c in sorted(codes)]
    assert len(set(msgs)) == len(msgs) and "unknown status code" not in msgs


@pytest.mark.parametrize("change,code", [
    (dict(precision=1), -7), (dict(nt=24), -7), (dict(m=(24, 16, 1)), -7), (dict(m=(4096, 16, 1)), -7),
    (dict(order=1, dim=1, m=(64, 1, 1)), -7), (dict(dim=0), -1), (dict(null=True), -1), (dict(count=0), -1)],
    ids=["fp32", "nt24", "m24", "m4096", "time-first", "dim0", "null-array", "count0"])
def test_multi_plan_rejects_before_a_gpu(lib, change, code):
    """qbvm_multi_plan: FP64 space-first instances with power-of-two nt and m;
    everything else is refused on the host."""
    import ctypes
    a = dict(dim=2, m=(16, 16, 1), nt=16, precision=0, order=0, count=2, null=False)
    a.update(change)
    desc = Q.make_desc(a["dim"], a["m"], 1.0, 0.1, a["nt"], 0, 1e-3, 0.0, a["precision"], 1, order=a["order"])
    buf = (ctypes.c_double * 8)()
    arr = (Q.QbvmMultiInstance * 2)()
    for i in range(2):
        arr[i] = Q.QbvmMultiInstance(desc, None if a["null"] else ctypes.addressof(buf),
                                     None if a["null"] else ctypes.addressof(buf))
    h = ctypes.c_void_p()
    assert lib.qbvm_multi_plan(arr, a["count"], ctypes.byref(h)) == code
    assert not h.value

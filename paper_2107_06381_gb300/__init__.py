"""Python binding of libqbvm (PinT-QBVM / PinT-MQBVM all-at-once solver, sm_103a).

Argument marshalling only: every step of the solve runs in the CUDA library
built from ``csrc/`` (see ``include/qbvm.h`` for the C ABI).  The functions
carry the C names.  Arrays may be torch tensors (CUDA or CPU), numpy arrays
(host) or raw integer addresses; FP64, C-contiguous.  If the shared library
is missing, importing the functions raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH, build as build_library

__all__ = [
    "QbvmDesc", "QbvmInfo", "QbvmError", "load_library",
    "qbvm_plan", "qbvm_solve", "qbvm_residual", "qbvm_plan_info", "qbvm_destroy",
    "qbvm_profile_enable", "qbvm_profile_read", "qbvm_residual_noalloc", "qbvm_measure_peak",
    "qbvm_strerror", "qbvm_version", "Plan", "Sweep", "QbvmSweepInstance", "QbvmSweepDesc", "QbvmSweepConfig",
    "qbvm_sweep_plan", "qbvm_sweep_run", "qbvm_sweep_read", "qbvm_sweep_autotune", "qbvm_sweep_set_config",
    "qbvm_sweep_get_config", "qbvm_sweep_destroy", "MLP", "Features", "Batch", "GMRES", "Multi",
    "FORM_PQ", "FORM_PM", "FP64", "FP32_REFINE", "RHS_DELTA", "RHS_GENERAL",
]

FORM_PQ, FORM_PM = 0, 1
FP64, FP32_REFINE = 0, 1
RHS_DELTA, RHS_GENERAL = 0, 1
ORDER_AUTO, ORDER_TIME_FIRST, ORDER_SPACE_FIRST = 0, 1, 2
ORIGINAL_QBVM, ORIGINAL_MQBVM = 0, 1


class QbvmDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("m", ctypes.c_int * 3), ("L", ctypes.c_double),
        ("T", ctypes.c_double), ("nt", ctypes.c_int), ("form", ctypes.c_int),
        ("alpha", ctypes.c_double), ("delta", ctypes.c_double),
        ("precision", ctypes.c_int), ("rhs_kind", ctypes.c_int),
        ("refine_tol", ctypes.c_double), ("refine_max_iters", ctypes.c_int), ("order", ctypes.c_int),
    ]


class QbvmInfo(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("omega", ctypes.c_double), ("tau", ctypes.c_double),
        ("unknowns", ctypes.c_longlong), ("workspace_bytes", ctypes.c_longlong),
        ("last_refine_iters", ctypes.c_int), ("last_rel_residual", ctypes.c_double),
        ("kernels_per_solve", ctypes.c_int),
    ]


class QbvmKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


class QbvmSweepInstance(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("m", ctypes.c_int * 3), ("L", ctypes.c_double), ("T", ctypes.c_double),
        ("nt", ctypes.c_int), ("form", ctypes.c_int), ("delta", ctypes.c_double),
        ("alpha_base", ctypes.c_double),
        ("g", ctypes.c_void_p), ("z0", ctypes.c_void_p), ("y0", ctypes.c_void_p),
    ]


class QbvmSweepDesc(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int), ("inst", ctypes.POINTER(QbvmSweepInstance)), ("n_alpha", ctypes.c_int),
        ("log10_lo", ctypes.c_double), ("log10_hi", ctypes.c_double), ("tau_dp", ctypes.c_double),
        ("precision", ctypes.c_int),
    ]


class QbvmSweepConfig(ctypes.Structure):
    _fields_ = [("modes_per_thread", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("grid", ctypes.c_int),
                ("ms", ctypes.c_float)]


class QbvmMultiInstance(ctypes.Structure):
    _fields_ = [("desc", QbvmDesc), ("g_or_F", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class QbvmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {qbvm_strerror(code)} (status {code})")


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libqbvm.so (the in-tree build).  Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libqbvm.so not found at {p}; run paper_2107_06381_gb300.build_library()")
    lib = ctypes.CDLL(p)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.qbvm_plan.argtypes = [ctypes.POINTER(QbvmDesc), ctypes.POINTER(vp)]
    lib.qbvm_plan.restype = ip
    lib.qbvm_solve.argtypes = [vp, vp, vp, ip, vp]
    lib.qbvm_solve.restype = ip
    lib.qbvm_residual.argtypes = [vp, vp, vp, ctypes.POINTER(dp), vp]
    lib.qbvm_residual.restype = ip
    lib.qbvm_plan_info.argtypes = [vp, ctypes.POINTER(QbvmInfo)]
    lib.qbvm_plan_info.restype = ip
    lib.qbvm_destroy.argtypes = [vp]
    lib.qbvm_destroy.restype = ip
    lib.qbvm_strerror.argtypes = [ip]
    lib.qbvm_strerror.restype = ctypes.c_char_p
    lib.qbvm_profile_enable.argtypes = [vp, ip]
    lib.qbvm_profile_enable.restype = ip
    lib.qbvm_profile_read.argtypes = [vp, ctypes.POINTER(QbvmKernelStat), ip, ctypes.POINTER(ip)]
    lib.qbvm_profile_read.restype = ip
    lib.qbvm_residual_noalloc.argtypes = [ctypes.POINTER(QbvmDesc), vp, vp, ctypes.POINTER(dp), vp]
    lib.qbvm_residual_noalloc.restype = ip
    lib.qbvm_gmres_create.argtypes = [vp, ip, ip, ctypes.POINTER(vp)]
    lib.qbvm_gmres_create.restype = ip
    lib.qbvm_gmres_solve.argtypes = [vp, vp, vp, dp, ip, ctypes.POINTER(ip), ctypes.POINTER(dp), vp]
    lib.qbvm_gmres_solve.restype = ip
    lib.qbvm_gmres_destroy.argtypes = [vp]
    lib.qbvm_gmres_destroy.restype = ip
    lib.qbvm_batch_plan.argtypes = [ctypes.POINTER(QbvmDesc), ip, ctypes.POINTER(dp), ctypes.POINTER(vp)]
    lib.qbvm_batch_plan.restype = ip
    lib.qbvm_solve_batched.argtypes = [vp, vp, vp, ip, vp]
    lib.qbvm_solve_batched.restype = ip
    lib.qbvm_batch_info.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_longlong)]
    lib.qbvm_batch_info.restype = ip
    lib.qbvm_batch_refine_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(dp)]
    lib.qbvm_batch_refine_info.restype = ip
    lib.qbvm_batch_refine_fused.argtypes = [vp, ctypes.POINTER(ip)]
    lib.qbvm_batch_refine_fused.restype = ip
    lib.qbvm_batch_destroy.argtypes = [vp]
    lib.qbvm_batch_destroy.restype = ip
    lib.qbvm_selftest_newton_rcp.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(dp), vp]
    lib.qbvm_selftest_newton_rcp.restype = ip
    lib.qbvm_selftest_bounded_wait.argtypes = [ip, ctypes.POINTER(dp), vp]
    lib.qbvm_selftest_bounded_wait.restype = ip
    lib.qbvm_sweep_plan.argtypes = [ctypes.POINTER(QbvmSweepDesc), ctypes.POINTER(vp)]
    lib.qbvm_sweep_plan.restype = ip
    lib.qbvm_sweep_run.argtypes = [vp, vp]
    lib.qbvm_sweep_run.restype = ip
    lib.qbvm_sweep_read.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.qbvm_sweep_read.restype = ip
    lib.qbvm_sweep_autotune.argtypes = [vp, ip, ctypes.POINTER(QbvmSweepConfig), vp]
    lib.qbvm_sweep_autotune.restype = ip
    lib.qbvm_sweep_set_config.argtypes = [vp, ctypes.POINTER(QbvmSweepConfig)]
    lib.qbvm_sweep_set_config.restype = ip
    lib.qbvm_sweep_get_config.argtypes = [vp, ctypes.POINTER(QbvmSweepConfig)]
    lib.qbvm_sweep_get_config.restype = ip
    lib.qbvm_sweep_destroy.argtypes = [vp]
    lib.qbvm_sweep_destroy.restype = ip
    vp_, ll = ctypes.c_void_p, ctypes.c_longlong
    lib.qbvm_mlp_create.argtypes = [ip, ip, ip, ctypes.c_ulonglong, ctypes.POINTER(vp)]
    lib.qbvm_mlp_create.restype = ip
    lib.qbvm_mlp_num_params.argtypes = [vp]
    lib.qbvm_mlp_num_params.restype = ll
    lib.qbvm_mlp_set_norm.argtypes = [vp, vp_, vp_]
    lib.qbvm_mlp_set_norm.restype = ip
    lib.qbvm_mlp_get_params.argtypes = [vp, vp_, vp_, vp_, ctypes.POINTER(ll)]
    lib.qbvm_mlp_get_params.restype = ip
    lib.qbvm_mlp_set_params.argtypes = [vp, vp_, vp_, vp_, ll]
    lib.qbvm_mlp_set_params.restype = ip
    lib.qbvm_mlp_forward.argtypes = [vp, vp_, ip, vp_, vp]
    lib.qbvm_mlp_forward.restype = ip
    lib.qbvm_mlp_gradients.argtypes = [vp, vp_, vp_, ip, vp_, ctypes.POINTER(dp), vp]
    lib.qbvm_mlp_gradients.restype = ip
    lib.qbvm_mlp_train_step.argtypes = [vp, vp_, vp_, ip, ctypes.c_float, vp]
    lib.qbvm_mlp_train_step.restype = ip
    lib.qbvm_mlp_last_loss.argtypes = [vp, ctypes.POINTER(dp), vp]
    lib.qbvm_mlp_last_loss.restype = ip
    lib.qbvm_mlp_destroy.argtypes = [vp]
    lib.qbvm_mlp_destroy.restype = ip
    lib.qbvm_features_plan.argtypes = [ip, dp, ip, ip, ctypes.POINTER(vp)]
    lib.qbvm_features_plan.restype = ip
    lib.qbvm_features_run.argtypes = [vp, vp_, vp_, ip, vp_, vp]
    lib.qbvm_features_run.restype = ip
    lib.qbvm_features_destroy.argtypes = [vp]
    lib.qbvm_features_destroy.restype = ip
    lib.qbvm_multi_plan.argtypes = [ctypes.POINTER(QbvmMultiInstance), ip, ctypes.POINTER(vp)]
    lib.qbvm_multi_plan.restype = ip
    lib.qbvm_multi_run.argtypes = [vp, vp]
    lib.qbvm_multi_run.restype = ip
    lib.qbvm_multi_check.argtypes = [vp, vp]
    lib.qbvm_multi_check.restype = ip
    lib.qbvm_multi_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ip), ctypes.POINTER(ip)]
    lib.qbvm_multi_info.restype = ip
    lib.qbvm_multi_destroy.argtypes = [vp]
    lib.qbvm_multi_destroy.restype = ip
    lib.qbvm_measure_peak.argtypes = [ip, ctypes.POINTER(dp), vp]
    lib.qbvm_measure_peak.restype = ip
    lib.qbvm_version.argtypes = []
    lib.qbvm_version.restype = ip
    if path is None:
        _lib = lib
    return lib


def _ptr(a) -> int:
    """Address of a tensor / ndarray / int (FP64, contiguous)."""
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    if mod.startswith("numpy"):
        import numpy as np
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)!r}")


def _stream(stream, *arrays) -> int:
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream
    for a in arrays:
        if type(a).__module__.startswith("torch") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _check(code: int, what: str):
    if code != 0:
        raise QbvmError(code, what)


def qbvm_strerror(code: int) -> str:
    return load_library().qbvm_strerror(code).decode()


def qbvm_version() -> int:
    return load_library().qbvm_version()


def make_desc(dim, m, L, T, nt, form=FORM_PQ, alpha=0.0, delta=0.0, precision=FP64,
              rhs_kind=RHS_DELTA, refine_tol=0.0, refine_max_iters=0, order=0) -> QbvmDesc:
    mm = list(m) + [1] * (3 - len(m))
    return QbvmDesc(dim, (ctypes.c_int * 3)(*mm), float(L), float(T), int(nt), int(form), float(alpha),
                    float(delta), int(precision), int(rhs_kind), float(refine_tol), int(refine_max_iters),
                    int(order))


def qbvm_plan(desc: QbvmDesc) -> int:
    h = ctypes.c_void_p()
    _check(load_library().qbvm_plan(ctypes.byref(desc), ctypes.byref(h)), "qbvm_plan")
    return h.value


def qbvm_solve(plan: int, g_or_F, y, n0_only: bool = False, stream=None) -> None:
    _check(load_library().qbvm_solve(plan, _ptr(g_or_F), _ptr(y), int(bool(n0_only)),
                                     _stream(stream, g_or_F, y)), "qbvm_solve")


def qbvm_residual(plan: int, y, g_or_F, stream=None) -> float:
    out = ctypes.c_double()
    _check(load_library().qbvm_residual(plan, _ptr(y), _ptr(g_or_F), ctypes.byref(out),
                                        _stream(stream, y, g_or_F)), "qbvm_residual")
    return out.value


def qbvm_residual_noalloc(desc: QbvmDesc, y, g_or_F, stream=None) -> float:
    """Plan-free residual that allocates no device memory (device arrays only)."""
    out = ctypes.c_double()
    _check(load_library().qbvm_residual_noalloc(ctypes.byref(desc), _ptr(y), _ptr(g_or_F), ctypes.byref(out),
                                                _stream(stream, y, g_or_F)), "qbvm_residual_noalloc")
    return out.value


PEAK_FP64_FMA, PEAK_FP32_FMA = 0, 1


def qbvm_measure_peak(kind: int = PEAK_FP64_FMA, stream=None) -> float:
    """Measured FMA instructions per second of the current GPU (FP64 or FP32)."""
    out = ctypes.c_double()
    _check(load_library().qbvm_measure_peak(int(kind), ctypes.byref(out), _stream(stream)), "qbvm_measure_peak")
    return out.value


def qbvm_plan_info(plan: int) -> QbvmInfo:
    info = QbvmInfo()
    _check(load_library().qbvm_plan_info(plan, ctypes.byref(info)), "qbvm_plan_info")
    return info


def qbvm_profile_enable(plan: int, on: bool = True) -> None:
    _check(load_library().qbvm_profile_enable(plan, int(bool(on))), "qbvm_profile_enable")


def qbvm_profile_read(plan: int, capacity: int = 64) -> dict:
    """{kernel name: (launches, total_ms)} since the last read / enable."""
    arr = (QbvmKernelStat * capacity)()
    n = ctypes.c_int()
    _check(load_library().qbvm_profile_read(plan, arr, capacity, ctypes.byref(n)), "qbvm_profile_read")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


def qbvm_destroy(plan: int) -> None:
    if plan:
        _check(load_library().qbvm_destroy(plan), "qbvm_destroy")


def qbvm_sweep_plan(desc: QbvmSweepDesc) -> int:
    h = ctypes.c_void_p()
    _check(load_library().qbvm_sweep_plan(ctypes.byref(desc), ctypes.byref(h)), "qbvm_sweep_plan")
    return h.value


def qbvm_sweep_run(sweep: int, stream=None) -> None:
    _check(load_library().qbvm_sweep_run(sweep, _stream(stream)), "qbvm_sweep_run")


def qbvm_sweep_read(sweep: int, alphas, discrepancy, error, pick, stream=None) -> None:
    _check(load_library().qbvm_sweep_read(sweep, _ptr(alphas), _ptr(discrepancy), _ptr(error), _ptr_int(pick),
                                          _stream(stream)), "qbvm_sweep_read")


def qbvm_sweep_autotune(sweep: int, repeats: int = 3, stream=None) -> QbvmSweepConfig:
    cfg = QbvmSweepConfig()
    _check(load_library().qbvm_sweep_autotune(sweep, repeats, ctypes.byref(cfg), _stream(stream)),
           "qbvm_sweep_autotune")
    return cfg


def qbvm_sweep_set_config(sweep: int, cfg: QbvmSweepConfig) -> None:
    _check(load_library().qbvm_sweep_set_config(sweep, ctypes.byref(cfg)), "qbvm_sweep_set_config")


def qbvm_sweep_get_config(sweep: int) -> QbvmSweepConfig:
    cfg = QbvmSweepConfig()
    _check(load_library().qbvm_sweep_get_config(sweep, ctypes.byref(cfg)), "qbvm_sweep_get_config")
    return cfg


def qbvm_sweep_destroy(sweep: int) -> None:
    if sweep:
        _check(load_library().qbvm_sweep_destroy(sweep), "qbvm_sweep_destroy")


def _ptr_int(a) -> int:
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    import numpy as np
    if a.dtype != np.int32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("int arrays must be C-contiguous int32")
    return a.ctypes.data


class Sweep:
    """Owning wrapper around a batched alpha sweep (device arrays: torch
    tensors or raw addresses for g, z0, y0)."""

    def __init__(self, instances, n_alpha=16, log10_lo=-1.5, log10_hi=1.5, tau_dp=1.1, precision=FP64):
        self._keep = instances
        arr = (QbvmSweepInstance * len(instances))()
        for i, d in enumerate(instances):
            m = list(d["m"]) + [1] * (3 - len(d["m"]))
            arr[i] = QbvmSweepInstance(d["dim"], (ctypes.c_int * 3)(*m), float(d.get("L", 1.0)), float(d["T"]),
                                       int(d["nt"]), int(d.get("form", FORM_PQ)), float(d["delta"]),
                                       float(d.get("alpha_base", 0.0)),
                                       _ptr(d["g"]), _ptr(d.get("z0")), _ptr(d.get("y0")))
        self._arr = arr
        self.count = len(instances)
        self.n_alpha = n_alpha
        self.desc = QbvmSweepDesc(len(instances), arr, n_alpha, log10_lo, log10_hi, tau_dp, precision)
        self.handle = qbvm_sweep_plan(self.desc)

    def run(self, stream=None):
        qbvm_sweep_run(self.handle, stream)

    def read(self, stream=None):
        import numpy as np
        al = np.zeros((self.count, self.n_alpha))
        disc = np.zeros_like(al)
        err = np.zeros_like(al)
        pick = np.zeros((self.count, 2), dtype=np.int32)
        qbvm_sweep_read(self.handle, al, disc, err, pick, stream)
        return al, disc, err, pick

    def autotune(self, repeats=3, stream=None):
        return qbvm_sweep_autotune(self.handle, repeats, stream)

    def autotune_cached(self, path, repeats=3, stream=None):
        """The launch shape from the JSON cache at `path` when this kind of batch
        (shapes, alphas, precision, GPU) was tuned before, else autotune and
        store it (tune_cache).  Returns (modes_per_thread, ctas_per_sm, hit)."""
        from . import tune_cache
        try:
            import torch
            device = torch.cuda.get_device_name() if torch.cuda.is_available() else "unknown"
        except Exception:
            device = "unknown"
        key = tune_cache.workload_key(self._keep, self.n_alpha, self.desc.precision, device)
        return tune_cache.autotune_cached(self, key, path, repeats=repeats, device=device, stream=stream)

    @property
    def config(self):
        return qbvm_sweep_get_config(self.handle)

    def set_config(self, modes_per_thread, ctas_per_sm):
        qbvm_sweep_set_config(self.handle, QbvmSweepConfig(modes_per_thread, ctas_per_sm, 0, 0.0))

    def close(self):
        if self.handle:
            qbvm_sweep_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fptr(a) -> int:
    """Address of a float32 tensor / ndarray."""
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        return a.data_ptr()
    import numpy as np
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("arrays must be C-contiguous float32")
    return a.ctypes.data


class MLP:
    """The learned-alpha network on the GPU (see include/qbvm.h)."""

    def __init__(self, in_dim=67, width=128, max_batch=4096, seed=0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.qbvm_mlp_create(in_dim, width, max_batch, seed, ctypes.byref(h)), "qbvm_mlp_create")
        self.handle = h.value
        self.in_dim, self.width = in_dim, width
        self.nparam = lib.qbvm_mlp_num_params(self.handle)

    def set_norm(self, mean, sd):
        import numpy as np
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(sd, dtype=np.float32)
        _check(load_library().qbvm_mlp_set_norm(self.handle, m.ctypes.data, s.ctypes.data), "qbvm_mlp_set_norm")
        self._norm = (m, s)

    def get_params(self):
        import numpy as np
        p = np.zeros(self.nparam, dtype=np.float32)
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        step = ctypes.c_longlong()
        _check(load_library().qbvm_mlp_get_params(self.handle, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                                  ctypes.byref(step)), "qbvm_mlp_get_params")
        return p, m, v, step.value

    def set_params(self, p, m=None, v=None, step=0):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        mm = None if m is None else np.ascontiguousarray(m, dtype=np.float32)
        vv = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        _check(load_library().qbvm_mlp_set_params(self.handle, p.ctypes.data, 0 if mm is None else mm.ctypes.data,
                                                  0 if vv is None else vv.ctypes.data, int(step)),
               "qbvm_mlp_set_params")

    def forward(self, x, y, stream=None):
        _check(load_library().qbvm_mlp_forward(self.handle, _fptr(x), int(x.shape[0]), _fptr(y), _stream(stream, x)),
               "qbvm_mlp_forward")
        return y

    def gradients(self, x, t):
        import numpy as np
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load_library().qbvm_mlp_gradients(self.handle, _fptr(x), _fptr(t), int(x.shape[0]), g.ctypes.data,
                                                 ctypes.byref(loss), _stream(None, x)), "qbvm_mlp_gradients")
        return loss.value, g

    def train_step(self, x, t, lr, stream=None):
        _check(load_library().qbvm_mlp_train_step(self.handle, _fptr(x), _fptr(t), int(x.shape[0]), float(lr),
                                                  _stream(stream, x)), "qbvm_mlp_train_step")

    def last_loss(self, stream=None):
        out = ctypes.c_double()
        _check(load_library().qbvm_mlp_last_loss(self.handle, ctypes.byref(out), _stream(stream)),
               "qbvm_mlp_last_loss")
        return out.value

    def unpack(self, flat):
        """Split a flat parameter vector into the oracle's dict (float64)."""
        import numpy as np
        K, N = self.in_dim, self.width
        f = np.asarray(flat, dtype=np.float64)
        o = 0
        out = {}
        for name, shape in (("W1", (N, K)), ("b1", (N,)), ("W2", (N, N)), ("b2", (N,)), ("w3", (N,)), ("b3", ())):
            size = int(np.prod(shape)) if shape else 1
            out[name] = f[o:o + size].reshape(shape) if shape else np.array(f[o])
            o += size
        return out

    def close(self):
        if self.handle:
            load_library().qbvm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Features:
    """Spectrum features of g_delta for a batch of 2D instances of one grid."""

    def __init__(self, m, T, nt, max_batch):
        h = ctypes.c_void_p()
        _check(load_library().qbvm_features_plan(int(m), float(T), int(nt), int(max_batch), ctypes.byref(h)),
               "qbvm_features_plan")
        self.handle = h.value

    def run(self, g, delta, feats, stream=None):
        import numpy as np
        d = np.ascontiguousarray(delta, dtype=np.float64)
        _check(load_library().qbvm_features_run(self.handle, _ptr(g), d.ctypes.data, int(d.size), _fptr(feats),
                                                _stream(stream, g)), "qbvm_features_run")
        return feats

    def close(self):
        if self.handle:
            load_library().qbvm_features_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GMRES:
    """The original QBVM (method ORIGINAL_QBVM, A_h of eq. 2.3) or MQBVM
    (ORIGINAL_MQBVM, B_h of eq. 2.6) system with f = (g, 0, ..., 0), solved by
    flexible right-preconditioned GMRES(restart) with `plan`'s PinT solve as the
    preconditioner.  `plan`: FP64, RHS_GENERAL, form PQ for QBVM / PM for MQBVM;
    it must outlive this object."""

    def __init__(self, plan: "Plan", method: int, restart: int = 20):
        h = ctypes.c_void_p()
        _check(load_library().qbvm_gmres_create(plan.handle, int(method), int(restart), ctypes.byref(h)),
               "qbvm_gmres_create")
        self.handle = h.value
        self.plan = plan

    def solve(self, g, y, tol=1e-12, max_iters=200, stream=None, raise_on_diverged=True):
        """Returns (iterations, relative residual); raises QbvmError on DIVERGED
        unless raise_on_diverged is False (y then holds the last iterate)."""
        it = ctypes.c_int()
        rel = ctypes.c_double()
        code = load_library().qbvm_gmres_solve(self.handle, _ptr(g), _ptr(y), float(tol), int(max_iters),
                                               ctypes.byref(it), ctypes.byref(rel), _stream(stream, g, y))
        if not (code == -4 and not raise_on_diverged):
            _check(code, "qbvm_gmres_solve")
        return it.value, rel.value

    def close(self):
        if self.handle:
            load_library().qbvm_gmres_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """`len(alphas)` same-shape instances solved together (qbvm_solve_batched):
    inputs and outputs stored back to back, [count][Nx] or [count][nt][Nx]
    (device arrays).  alphas=None with count=B uses the descriptor's alpha
    (or its a-priori rule from delta) for all B instances."""

    def __init__(self, dim, m, L, T, nt, form=FORM_PQ, alphas=None, count=None, alpha=0.0, delta=0.0,
                 rhs_kind=RHS_DELTA, order=0, precision=FP64, refine_tol=0.0, refine_max_iters=0):
        self.desc = make_desc(dim, m, L, T, nt, form, alpha, delta, precision, rhs_kind, refine_tol,
                              refine_max_iters, order)
        if alphas is not None:
            arr = (ctypes.c_double * len(alphas))(*[float(a) for a in alphas])
            n = len(alphas)
        else:
            if count is None:
                raise ValueError("give alphas or count")
            arr, n = None, int(count)
        h = ctypes.c_void_p()
        _check(load_library().qbvm_batch_plan(ctypes.byref(self.desc), n, arr, ctypes.byref(h)), "qbvm_batch_plan")
        self.handle = h.value
        self.count = n

    def solve(self, g_or_F, y, n0_only=False, stream=None):
        _check(load_library().qbvm_solve_batched(self.handle, _ptr(g_or_F), _ptr(y), int(bool(n0_only)),
                                                 _stream(stream, g_or_F, y)), "qbvm_solve_batched")
        return y

    @property
    def refine_info(self):
        """(refinement steps, largest relative residual) of the last FP32_REFINE solve."""
        it, rel = ctypes.c_int(), ctypes.c_double()
        _check(load_library().qbvm_batch_refine_info(self.handle, ctypes.byref(it), ctypes.byref(rel)),
               "qbvm_batch_refine_info")
        return it.value, rel.value

    @property
    def refine_fused(self):
        """True when the FP32_REFINE batch runs the whole refinement in one launch."""
        f = ctypes.c_int()
        _check(load_library().qbvm_batch_refine_fused(self.handle, ctypes.byref(f)), "qbvm_batch_refine_fused")
        return bool(f.value)

    @property
    def alphas(self):
        out = (ctypes.c_double * self.count)()
        _check(load_library().qbvm_batch_info(self.handle, out, None), "qbvm_batch_info")
        return list(out)

    def close(self):
        if self.handle:
            load_library().qbvm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Full solves of uneven instances in one persistent launch (qbvm_multi_*).
    `instances`: dicts with dim, m, L, T, nt, form, alpha (or delta), rhs_kind
    and the device arrays g_or_F, y (float64 tensors or addresses)."""

    def __init__(self, instances):
        self._keep = instances
        arr = (QbvmMultiInstance * len(instances))()
        for i, d in enumerate(instances):
            desc = make_desc(d["dim"], d["m"], d.get("L", 1.0), d["T"], d["nt"], d.get("form", FORM_PQ),
                             d.get("alpha", 0.0), d.get("delta", 0.0), FP64, d.get("rhs_kind", RHS_DELTA))
            arr[i] = QbvmMultiInstance(desc, _ptr(d["g_or_F"]), _ptr(d["y"]))
        h = ctypes.c_void_p()
        _check(load_library().qbvm_multi_plan(arr, len(instances), ctypes.byref(h)), "qbvm_multi_plan")
        self.handle = h.value

    def run(self, stream=None):
        _check(load_library().qbvm_multi_run(self.handle, _stream(stream)), "qbvm_multi_run")

    def check(self, stream=None):
        _check(load_library().qbvm_multi_check(self.handle, _stream(stream)), "qbvm_multi_check")

    @property
    def info(self):
        u, n, g = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        _check(load_library().qbvm_multi_info(self.handle, ctypes.byref(u), ctypes.byref(n), ctypes.byref(g)),
               "qbvm_multi_info")
        return {"unknowns": u.value, "work_items": n.value, "grid": g.value}

    def close(self):
        if self.handle:
            load_library().qbvm_multi_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper around a qbvm plan handle."""

    def __init__(self, dim, m, L, T, nt, form=FORM_PQ, alpha=0.0, delta=0.0, precision=FP64,
                 rhs_kind=RHS_DELTA, refine_tol=0.0, refine_max_iters=0, order=0):
        self.desc = make_desc(dim, m, L, T, nt, form, alpha, delta, precision, rhs_kind,
                              refine_tol, refine_max_iters, order)
        self.handle = qbvm_plan(self.desc)

    def solve(self, g_or_F, y, n0_only=False, stream=None):
        qbvm_solve(self.handle, g_or_F, y, n0_only, stream)
        return y

    def residual(self, y, g_or_F, stream=None) -> float:
        return qbvm_residual(self.handle, y, g_or_F, stream)

    def profile(self, on: bool = True):
        qbvm_profile_enable(self.handle, on)

    def profile_read(self) -> dict:
        return qbvm_profile_read(self.handle)

    @property
    def info(self) -> QbvmInfo:
        return qbvm_plan_info(self.handle)

    def close(self):
        if self.handle:
            qbvm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

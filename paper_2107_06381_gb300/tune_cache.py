"""A JSON cache of the sweep autotuner's choice.

qbvm_sweep_autotune times every candidate launch shape (modes per thread in
the alpha scan x CTAs per SM) on the actual batch.  The best shape depends on
the batch's sizes, the number of alphas, the precision, the GPU and the build
of the kernel, not on the data, so it is kept in a JSON file keyed by those
and set directly
(qbvm_sweep_set_config) the next time the same kind of batch is planned.
The file holds {key: {"modes_per_thread", "ctas_per_sm", "ms", "device"}};
writes go to a temporary file that replaces the old one, so a reader never
sees a partial file.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile


_SWEEP_SOURCES = ("qbvm_sweep.cu", "qbvm_dfsum.cuh", "qbvm_dst.cuh", "qbvm_fft.cuh", "qbvm_internal.h")


def build_id() -> str:
    """Hash of the sources the sweep kernel is compiled from: a launch shape
    tuned for one build of the kernel (its launch bounds, shared-memory use,
    stage code) is not reused after any of them changes."""
    h = hashlib.sha1()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for name in _SWEEP_SOURCES:
        try:
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
        except OSError:
            h.update(name.encode() + b"\0missing")
    return h.hexdigest()[:16]


def workload_key(instances, n_alpha: int, precision: int, device: str, build: str | None = None) -> str:
    """Stable key of a sweep: the shapes of its instances (dim, m, nt, form,
    in order), the number of alphas, the precision, the device name and the
    kernel build (`build_id()` unless given)."""
    shapes = [[int(d["dim"]), [int(x) for x in d["m"]], int(d["nt"]), int(d.get("form", 0))] for d in instances]
    blob = json.dumps({"shapes": shapes, "n_alpha": int(n_alpha), "precision": int(precision),
                       "device": str(device), "build": build if build is not None else build_id()},
                      sort_keys=True, separators=(",", ":"))
    return hashlib.sha1(blob.encode()).hexdigest()


def load(path: str) -> dict:
    """The cache at `path` ({} if it does not exist or cannot be parsed)."""
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save(path: str, cache: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tune-", suffix=".json", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def autotune_cached(sweep, key: str, path: str, repeats: int = 3, device: str = "", stream=None):
    """Set the cached launch shape for `key` on `sweep`, or autotune it and
    store the result.  `sweep` needs autotune(repeats, stream) -> a config with
    modes_per_thread / ctas_per_sm / ms, and set_config(modes_per_thread,
    ctas_per_sm).  Returns (modes_per_thread, ctas_per_sm, hit)."""
    cache = load(path)
    entry = cache.get(key)
    if isinstance(entry, dict) and "modes_per_thread" in entry and "ctas_per_sm" in entry:
        sweep.set_config(int(entry["modes_per_thread"]), int(entry["ctas_per_sm"]))
        return int(entry["modes_per_thread"]), int(entry["ctas_per_sm"]), True
    cfg = sweep.autotune(repeats=repeats, stream=stream)
    cache = load(path)                      # another process may have written meanwhile
    cache[key] = {"modes_per_thread": int(cfg.modes_per_thread), "ctas_per_sm": int(cfg.ctas_per_sm),
                  "ms": float(cfg.ms), "device": device}
    save(path, cache)
    return int(cfg.modes_per_thread), int(cfg.ctas_per_sm), False

"""The sweep autotuner's JSON cache (host logic; a stand-in sweep, no GPU)."""
import json
import os
from types import SimpleNamespace

from paper_2107_06381_gb300 import tune_cache as T

INST = [dict(dim=2, m=(64, 64), nt=32, form=0, delta=1e-3, g=1), dict(dim=1, m=(128,), nt=64, form=1, delta=2e-3, g=2)]


class FakeSweep:
    def __init__(self, best=(4, 2)):
        self.best = best
        self.tuned = 0
        self.set = None

    def autotune(self, repeats=3, stream=None):
        self.tuned += 1
        return SimpleNamespace(modes_per_thread=self.best[0], ctas_per_sm=self.best[1], grid=304, ms=9.4)

    def set_config(self, mpt, cps):
        self.set = (mpt, cps)


def test_key_depends_on_shapes_alphas_precision_device_not_data():
    k = T.workload_key(INST, 16, 1, "GB300")
    assert k == T.workload_key([dict(d, delta=5.0, g=99) for d in INST], 16, 1, "GB300")   # data-independent
    assert k != T.workload_key(INST[:1], 16, 1, "GB300")
    assert k != T.workload_key(INST, 8, 1, "GB300")
    assert k != T.workload_key(INST, 16, 0, "GB300")
    assert k != T.workload_key(INST, 16, 1, "B200")
    assert k != T.workload_key([dict(INST[0], nt=64), INST[1]], 16, 1, "GB300")


def test_key_depends_on_the_kernel_build():
    """A shape tuned for one build of the sweep kernel is not reused by another."""
    k = T.workload_key(INST, 16, 1, "GB300")
    assert k == T.workload_key(INST, 16, 1, "GB300", build=T.build_id())
    assert k != T.workload_key(INST, 16, 1, "GB300", build="0" * 16)
    assert len(T.build_id()) == 16 and T.build_id() == T.build_id()


def test_miss_tunes_and_stores_then_hit_sets_without_tuning(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    key = T.workload_key(INST, 16, 1, "GB300")
    a = FakeSweep(best=(4, 2))
    assert T.autotune_cached(a, key, path, device="GB300") == (4, 2, False)
    assert a.tuned == 1 and a.set is None
    stored = json.load(open(path))
    assert stored[key]["modes_per_thread"] == 4 and stored[key]["ctas_per_sm"] == 2
    b = FakeSweep(best=(1, 1))
    assert T.autotune_cached(b, key, path, device="GB300") == (4, 2, True)
    assert b.tuned == 0 and b.set == (4, 2)
    other = T.workload_key(INST, 8, 1, "GB300")
    c = FakeSweep(best=(2, 0))
    assert T.autotune_cached(c, other, path) == (2, 0, False)
    assert set(json.load(open(path))) == {key, other}        # both entries kept
    assert not [f for f in os.listdir(os.path.dirname(path)) if f.startswith(".tune-")]


def test_unreadable_cache_is_treated_as_empty(tmp_path):
    path = str(tmp_path / "tune.json")
    open(path, "w").write("{not json")
    s = FakeSweep()
    assert T.autotune_cached(s, "k", path)[2] is False
    assert json.load(open(path))["k"]["modes_per_thread"] == 4


def test_sweep_method_wires_the_cache(tmp_path):
    """Sweep.autotune_cached builds the key from its own instances, alpha count and
    precision (the GPU calls are stood in for)."""
    import paper_2107_06381_gb300 as Q
    sw = Q.Sweep.__new__(Q.Sweep)
    sw.handle = None
    sw._keep, sw.n_alpha, sw.desc = INST, 16, SimpleNamespace(precision=1)
    fake = FakeSweep(best=(2, 3))
    sw.autotune, sw.set_config = fake.autotune, fake.set_config
    path = str(tmp_path / "t.json")
    assert sw.autotune_cached(path) == (2, 3, False)
    assert sw.autotune_cached(path) == (2, 3, True) and fake.set == (2, 3)
    (key,) = json.load(open(path))
    assert key == T.workload_key(INST, 16, 1, json.load(open(path))[key]["device"])

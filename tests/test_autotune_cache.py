"""Host logic of the launch-shape autotuner's JSON cache (no GPU): a grid is
tuned once per engine, later handles apply the stored shapes, and instances
sharing a grid share one tuning."""
import json

from paper_2510_24543_gb300 import autotune as A
from paper_2510_24543_gb300 import egpe as E


class Fake:
    def __init__(self):
        self.tuned, self.applied = [], []

    def tuner(self, h, inst, eng, psi, precond, reps):
        self.tuned.append((inst, eng))
        return [{"key": f"k{eng}", "choice": 4 + eng, "name": "x", "L": 64, "kind": 0}]

    def setter(self, h, inst, eng, entries):
        self.applied.append((inst, eng, entries[0]["choice"]))


def test_cache_roundtrip_and_sharing(tmp_path):
    path = str(tmp_path / "tune.json")
    grids = [(48, 48, 48), (64, 64, 64), (48, 48, 48)]
    f = Fake()
    used = A.tune_handle(0, grids, E.EGPE_MIXED, 3, lambda i, e: None, "GB300", cache_path=path, digest="d0",
                         tuner=f.tuner, setter=f.setter)
    # two distinct grids x two engines tuned once each; all three instances set on both engines
    assert sorted(f.tuned) == [(0, 0), (0, 1), (1, 0), (1, 1)]
    assert len(f.applied) == 6
    assert len(used) == 4
    data = json.load(open(path))
    assert A.cache_key("GB300", 1, (64, 64, 64), 3, "d0") in data
    g = Fake()
    A.tune_handle(0, grids, E.EGPE_MIXED, 3, lambda i, e: None, "GB300", cache_path=path, digest="d0",
                  tuner=g.tuner, setter=g.setter)
    assert g.tuned == [] and len(g.applied) == 6
    # another build digest or preconditioner is a different key
    k = Fake()
    A.tune_handle(0, grids[:1], E.EGPE_FP32, 3, lambda i, e: None, "GB300", cache_path=path, digest="d1",
                  tuner=k.tuner, setter=k.setter)
    assert k.tuned == [(0, 1)]


def test_engines_of_precision():
    assert A.engines_of(E.EGPE_FP64) == [0]
    assert A.engines_of(E.EGPE_FP32) == [1]
    assert A.engines_of(E.EGPE_MIXED) == [0, 1]

"""The persistent autotuning cache (host logic; a stand-in plan records the calls)."""
import json

from paper_2108_01438_gb300.tuning_cache import TuningCache, class_key
from paper_2108_01438_gb300 import workloads as W


class FakePlan:
    def __init__(self, nx, nz, m, precision=0, best=(8, 1, 4)):
        self.geometry = W.geometry(nx, nz, m)
        self.precision = precision
        self.best = best
        self.tuned = 0
        self.applied = []

    def autotune(self, reps=5):
        self.tuned += 1
        return dict(tile_c=self.best[0], lateral_order=self.best[1], adjoint_kernel=self.best[2],
                    pair_ms=0.25, tried=12)

    def set_tuning(self, tile_c, lateral_order=0, adjoint_kernel=-1):
        self.applied.append((tile_c, lateral_order, adjoint_kernel))


def test_tunes_once_per_class_and_gpu_then_reads_the_file(tmp_path):
    path = str(tmp_path / "tuning.json")
    c = TuningCache(path)
    a = FakePlan(1024, 2048, 2048)
    r = c.apply_or_tune(a, gpu_name="GB300")
    assert r == dict(tile_c=8, lateral_order=1, adjoint_kernel=4, cached=False) and a.tuned == 1
    # a new process: the file gives the choice, no tuning
    c2 = TuningCache(path)
    b = FakePlan(1024, 2048, 2048, best=(16, 0, 1))
    r = c2.apply_or_tune(b, gpu_name="GB300")
    assert r["cached"] and b.tuned == 0 and b.applied == [(8, 1, 4)]
    # another GPU, precision or shape is another class
    for p, gpu in ((FakePlan(1024, 2048, 2048), "B200"), (FakePlan(1024, 2048, 2048, precision=2), "GB300"),
                   (FakePlan(512, 2048, 2048), "GB300")):
        assert not c2.apply_or_tune(p, gpu_name=gpu)["cached"] and p.tuned == 1
    data = json.load(open(path))
    assert len(data) == 4 and data[class_key(a, "GB300")]["pair_ms"] == 0.25


def test_bad_files_start_empty(tmp_path):
    p = tmp_path / "t.json"
    p.write_text("{not json")
    assert TuningCache(str(p)).entries == {}
    p.write_text(json.dumps({"k": {"tile_c": "8"}, "ok": {"tile_c": 8, "lateral_order": 0, "adjoint_kernel": -1}}))
    assert list(TuningCache(str(p)).entries) == ["ok"]
    assert TuningCache(str(tmp_path / "missing.json")).entries == {}


def test_save_leaves_no_temporary_files(tmp_path):
    c = TuningCache(str(tmp_path / "sub" / "t.json"))
    c.put("k", dict(tile_c=4, lateral_order=0, adjoint_kernel=-1))
    c.save()
    assert sorted(x.name for x in (tmp_path / "sub").iterdir()) == ["t.json"]

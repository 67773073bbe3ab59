"""The batch autotuner's shape cache (Batch.save_shapes / load_shapes) on the
host, without a GPU: the plan's classes and setters are replaced by fakes,
so only the file logic runs -- keys by GPU model and class, merging with
what the file holds, the all-classes-present rule, and the concurrent mode
applied only when the recorded sequences agree."""
import json

import paper_2201_04614_gb300 as vsz


class FakeBatch(vsz.Batch):
    def __init__(self, classes, device="GB300|152 SMs"):  # no plan, no GPU
        self._classes = classes
        self._dev = device
        self.shapes, self.conc = {}, []

    def classes(self):
        return [dict(c) for c in self._classes]

    def _device_key(self):
        return self._dev

    def set_shape(self, c, warps=0, ctas_per_sm=0):
        self.shapes[c] = (warps, ctas_per_sm)

    def set_concurrent(self, on):
        self.conc.append(bool(on))

    def close(self):
        pass


def cls(kind, ndim, block, pad_kind, warps, ctas, concurrent):
    return {"kind": kind, "ndim": ndim, "block": block, "pad_kind": pad_kind, "warps": warps,
            "ctas_per_sm": ctas, "concurrent": concurrent}


PLAN = [cls(0, 3, 8, 0, 8, 2, 1), cls(0, 2, 16, 0, 4, 4, 1), cls(1, 3, 8, 0, 0, 0, 1), cls(1, 2, 16, 0, 8, 3, 1)]


def test_round_trip_applies_every_recorded_shape(tmp_path):
    path = str(tmp_path / "shapes.json")
    FakeBatch(PLAN).save_shapes(path)
    other = FakeBatch([dict(c, warps=0, ctas_per_sm=0) for c in PLAN])
    assert other.load_shapes(path)
    assert other.shapes == {0: (8, 2), 1: (4, 4), 2: (0, 0), 3: (8, 3)}
    assert other.conc == [True]


def test_other_gpu_or_missing_class_applies_nothing(tmp_path):
    path = str(tmp_path / "shapes.json")
    FakeBatch(PLAN).save_shapes(path)
    b = FakeBatch(PLAN, device="B200|148 SMs")
    assert not b.load_shapes(path) and b.shapes == {} and b.conc == []
    more = FakeBatch(PLAN + [cls(0, 1, 256, 0, 2, 16, 1)])
    assert not more.load_shapes(path) and more.shapes == {}
    assert not FakeBatch(PLAN).load_shapes(str(tmp_path / "absent.json"))
    (tmp_path / "bad.json").write_text("{not json")
    assert not FakeBatch(PLAN).load_shapes(str(tmp_path / "bad.json"))


def test_merge_keeps_other_gpus_and_classes(tmp_path):
    path = str(tmp_path / "shapes.json")
    FakeBatch(PLAN, device="B200|148 SMs").save_shapes(path)
    FakeBatch([cls(0, 1, 256, 2, 2, 16, 0)]).save_shapes(path)
    tab = json.load(open(path))
    assert set(tab) == {"B200|148 SMs", "GB300|152 SMs"}
    assert tab["GB300|152 SMs"]["classes"] == {"0:1:256:2": {"warps": 2, "ctas_per_sm": 16}}
    assert len(tab["B200|148 SMs"]["classes"]) == 4


def test_disagreeing_concurrent_modes_are_not_applied(tmp_path):
    path = str(tmp_path / "shapes.json")
    mixed = [dict(c, concurrent=1 if c["kind"] == 0 else 0) for c in PLAN]
    FakeBatch(mixed).save_shapes(path)
    b = FakeBatch(PLAN)
    assert b.load_shapes(path)
    assert len(b.shapes) == 4 and b.conc == []

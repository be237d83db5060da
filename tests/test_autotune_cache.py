"""The launch-shape cache of Lattice.autotune (paper_2212_07494_gb300/autotune.py)
on the CPU: keys name the problem and the device, entries survive other keys'
writes, and a missing or damaged file reads as no entry."""
import json


class _Lat:
    def __init__(self, *fields):
        self.signature_fields = fields


def test_signature_names_problem_and_device():
    from paper_2212_07494_gb300 import autotune as A
    a = A.signature(_Lat(0, 1, 1, 4096, 4096, 1, False))
    b = A.signature(_Lat(0, 1, 2, 4096, 4096, 1, False))
    c = A.signature(_Lat(0, 1, 1, 4096, 4096, 1, True))
    assert len({a, b, c}) == 3
    assert a.startswith(A.device_name() + "|") and "4096x4096x1" in a


def test_store_and_lookup(tmp_path):
    from paper_2212_07494_gb300 import autotune as A
    path = str(tmp_path / "sub" / "launch.json")
    assert A.lookup(path, "k") is None
    A.store(path, "k1", (128, 2), 0.175)
    A.store(path, "k2", (64, 1), 0.2)
    assert A.lookup(path, "k1") == {"launch": [128, 2], "ms": 0.175}
    assert A.lookup(path, "k2") == {"launch": [64, 1], "ms": 0.2}
    A.store(path, "k1", (256, 1), 0.15)                   # replaces its own entry only
    d = json.load(open(path))
    assert d["k1"]["launch"] == [256, 1] and d["k2"]["launch"] == [64, 1]
    assert [p.name for p in (tmp_path / "sub").iterdir()] == ["launch.json"]   # no temporary left


def test_damaged_cache_reads_as_empty(tmp_path):
    from paper_2212_07494_gb300 import autotune as A
    path = tmp_path / "launch.json"
    path.write_text("{ not json")
    assert A.lookup(str(path), "k") is None
    A.store(str(path), "k", (32, 1), 1.0)
    assert A.lookup(str(path), "k")["launch"] == [32, 1]

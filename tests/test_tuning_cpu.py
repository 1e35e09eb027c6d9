"""Stored tuning (tuned.json): the signature, the store / load round trip,
and the settings limits_for hands to a plan: class limits, scan rows per
warp and scan row staging (entries written before the staging existed
default to 0, bulk tensor copies where the row pitch allows).  No GPU."""
import json

from paper_2603_12016_gb300 import tuning


class FakePlan:
    def __init__(self):
        self.calls = []

    def set_tuning(self, *t):
        self.calls.append(t)


def test_signature_names_every_workload_parameter():
    s = tuning.signature((2048, 2048), "uint16", 2, 256, (1, 2), "core")
    assert s == "2048x2048|uint16|2d|ng256|d1,2|core"
    assert s != tuning.signature((2048, 2048), "uint16", 2, 256, (1, 2), "all")
    assert s != tuning.signature((2048, 2048), "uint16", 2, 64, (1, 2), "core")


def test_store_load_round_trip_keeps_other_entries(tmp_path):
    path = str(tmp_path / "tuned.json")
    tuning.store("GPU A", "sig1", {"limits": [1, 2, 3, 4], "scan_rows_per_warp": 8, "scan_staging": 1}, path)
    tuning.store("GPU B", "sig1", {"limits": [5, 6, 7, 8]}, path)
    tuning.store("GPU A", "sig2", {"limits": [0, 0, 0, 0]}, path)
    d = json.load(open(path))
    assert set(d) == {"GPU A", "GPU B"} and set(d["GPU A"]) == {"sig1", "sig2"}
    assert tuning.load("GPU A", "sig1", path)["scan_staging"] == 1
    assert tuning.load("GPU C", "sig1", path) is None


def test_limits_for_applies_stored_rows_and_staging(monkeypatch):
    entries = {("dev", "new"): {"limits": [256, 1024, 4096, 8192], "scan_rows_per_warp": 8, "scan_staging": 1},
               ("dev", "old"): {"limits": [0, 512, 4096, 8192], "scan_rows_per_warp": 32}}
    monkeypatch.setattr(tuning, "load", lambda dev, sig, path=None: entries.get((dev, sig)))
    ex = FakePlan()
    t, src = tuning.limits_for(ex, "dev", "new")
    assert t == (256, 1024, 4096, 8192, 8, 1) and src == "tuned.json" and ex.calls[-1] == t
    t, src = tuning.limits_for(ex, "dev", "old")
    assert t == (0, 512, 4096, 8192, 32, 0) and ex.calls[-1] == t
    t, src = tuning.limits_for(ex, "dev", "missing")
    assert t == tuning.DEFAULT_LIMITS + (0, 0) and src == "default" and ex.calls[-1] == t


def test_committed_entries_are_complete():
    """Every committed entry carries four class limits, a legal tile height
    and a legal staging."""
    d = json.load(open(tuning.TUNED_PATH))
    assert d
    for dev, sigs in d.items():
        for sig, ent in sigs.items():
            assert len(ent["limits"]) == 4 and all(v >= 0 for v in ent["limits"]), (dev, sig)
            assert ent.get("scan_rows_per_warp", 0) in (0, 4, 8, 16, 32), (dev, sig)
            assert ent.get("scan_staging", 0) in (0, 1), (dev, sig)

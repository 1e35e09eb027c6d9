"""Host-side pieces of the benchmark: the kernel-source hash that ties the
committed ncu traffic figures to the sources they were measured on (the
benchmark reports no traffic once the sources hash differently), and the
keys of those figures against the stored tuning.  No GPU."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2603_12016_gb300 import tuning  # noqa: E402


def test_source_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    d = tmp_path / "paper_2603_12016_gb300" / "csrc"
    d.mkdir(parents=True)
    f = d / "a.cu"
    f.write_text("int f(int x) { return x + 1; } // one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    f.write_text("/* a block\n   comment */\nint f(int x) {\n    return x + 1;  // another\n}\n")
    assert bench.kernel_source_hash() == h0
    f.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_hash() != h0
    (d / "b.cuh").write_text("int g;\n")
    f.write_text("int f(int x) { return x + 1; }\n")
    assert bench.kernel_source_hash() != h0  # a new source file counts


def test_traffic_keys_are_stored_settings():
    """Each traffic figure is keyed by (workload, phase, limits + scan rows +
    scan staging, feature set); those settings must be a stored tuning of
    that feature set, or the benchmark would never look the figure up."""
    stored = {(tuple(e["limits"]) + (e.get("scan_rows_per_warp", 0), e.get("scan_staging", 0)), sig.split("|")[-1])
              for sigs in json.load(open(tuning.TUNED_PATH)).values() for sig, e in sigs.items()}
    for (name, phase, limits, feats), v in bench.TRAFFIC.items():
        assert phase == "roi_stage" and v > 0
        assert len(limits) == 6 and (tuple(limits), feats) in stored, (name, limits, feats)

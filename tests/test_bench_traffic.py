"""The bench's DRAM-traffic figure comes from a committed ncu capture only while every source the
captured kernel compiles from is unchanged: any edit to them turns it into null."""
import hashlib
import json
import os

import bench


def _fake_root(tmp_path, sources, record):
    csrc = tmp_path / "paper_2201_02632_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_counters.json").write_text(json.dumps(record))
    return str(tmp_path)


def test_traffic_needs_every_captured_source_unchanged(tmp_path, monkeypatch):
    sources = {"a.cu": "kernel a\n", "b.cuh": "helpers b\n"}
    h = hashlib.sha256(b"".join(t.encode() for t in sources.values())).hexdigest()[:16]
    record = {"k": {"sources": list(sources), "source_sha256_16": h,
                    "dram_bytes_per_launch_scaled": 12345}}
    root = _fake_root(tmp_path, sources, record)
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.ncu_traffic("k") == 12345
    assert bench.ncu_traffic("missing") is None
    # an edit to the second source (a shared header) voids the figure
    with open(os.path.join(root, "paper_2201_02632_gb300", "csrc", "b.cuh"), "a") as f:
        f.write("// one more helper\n")
    assert bench.ncu_traffic("k") is None


def test_committed_record_matches_the_current_deposit_sources():
    """The committed deposit record names the files it was captured from, and they exist."""
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_counters.json")))
    rec = d["k_deposit_tc_c1"]
    for f in rec.get("sources", [rec.get("source")]):
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2201_02632_gb300", "csrc", f))
    assert rec["dram_bytes_per_launch_scaled"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]

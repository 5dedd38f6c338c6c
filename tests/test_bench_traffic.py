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
    # the full-scale record: captured on a sample, reads scaled by the tile pairs
    big = d["k_deposit_tc_c2"]
    assert big["sources"] == rec["sources"]
    assert big["read_scale"] > 1.0
    assert big["dram_bytes_per_launch_scaled"] == round(
        big["dram_bytes_read"] * big["read_scale"]) + big["dram_bytes_write"]


def _rec(rows):
    """32-byte particle records (fx, fy, h, Y, B, kind, ix, iy) as a CPU tensor."""
    import numpy as np
    import torch

    a = np.zeros((len(rows), 8), np.float32)
    iv = a.view(np.int32)
    for k, (px, py, h, y, kind) in enumerate(rows):
        a[k, 0], a[k, 1], a[k, 2], a[k, 3], a[k, 4] = px % 1, py % 1, h, y, 1.0
        iv[k, 5], iv[k, 6], iv[k, 7] = kind, int(px // 1), int(py // 1)
    return torch.from_numpy(a)


def test_deposit_work_splits_small_and_tensor_core_particles():
    rec = _rec([(10.5, 10.5, 1.0, 1.0, 0),     # 3 x 3 box: small, y and b
                (100.5, 100.5, 10.0, 0.0, 1),  # 21 x 21 box in one tile: b only
                (63.5, 10.5, 1.0, 1.0, 0),     # 3 x 3 box across a tile edge: 2 pairs
                (5.0, 5.0, 3.0, 1.0, 2)])      # no kind: not deposited
    w = bench.deposit_work(rec, 256, 256, tile=64, sspan=8)
    assert w["updates"] == 9 + 441 + 9
    assert w["flops"] == 2 * (9 * 2 + 441 * 1 + 9 * 2)
    assert w["flops_tc"] == 2 * 441
    assert (w["pairs"], w["pairs_tc"]) == (4, 1)
    w0 = bench.deposit_work(rec, 256, 256, tile=64, sspan=0)
    assert w0["flops_tc"] == w0["flops"] and w0["pairs_tc"] == w0["pairs"] == 4
    assert bench.small_span_auto(4096, 4096) == 8 and bench.small_span_auto(1024, 1024) == 0

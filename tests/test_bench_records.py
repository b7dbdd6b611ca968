"""Host-side checks of the benchmark's DRAM-traffic records (no GPU): a record carries
the hash of its kernel's sources with comments and blank space removed, so a comment
edit keeps it and any code change voids it (the bench then reports no traffic for that
kernel), and the committed records are well formed."""
from __future__ import annotations

import json
import os

import bench


def test_source_hash_ignores_comments_and_space(tmp_path, monkeypatch):
    src = tmp_path / "csrc"
    src.mkdir()
    monkeypatch.setattr(bench, "CSRC", str(src))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "probe_kernel", ["a.cu", "b.cuh"])
    (src / "a.cu").write_text("int f(int x) { return x + 1; }  // add one\n")
    (src / "b.cuh").write_text("/* header */\n#define K 4\n")
    h0 = bench.kernel_source_sha("probe_kernel")
    (src / "a.cu").write_text("// a comment\nint f(int x)   {\n  return x + 1;\n}\n")
    (src / "b.cuh").write_text("#define K 4 /* four */\n")
    assert bench.kernel_source_sha("probe_kernel") == h0
    (src / "a.cu").write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_sha("probe_kernel") != h0


def test_committed_records_are_well_formed():
    path = os.path.join(bench.ROOT, "profiles", "roofline_traffic.json")
    records = json.load(open(path))
    assert set(records) <= set(bench.KERNEL_SOURCES)
    for kernel, rec in records.items():
        assert len(rec["source_sha256"]) == 64, kernel
        assert rec["workload"] and "1 pass" in rec["capture"], kernel
        assert abs(rec["bytes_per_launch"] - rec["dram_bytes_read"] - rec["dram_bytes_write"]) <= 1e4, kernel

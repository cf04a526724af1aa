"""The committed ncu summaries stay in step with the kernels: every entry
of profiles/traffic.json names an existing kernel whose source text (device
body and launching wrapper) still hashes to the captured digest (a changed kernel must be profiled again
before its DRAM traffic is reported), and every summary gives the command
that produced it."""
import glob
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_match_current_kernels():
    entries = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert entries
    for name, e in entries.items():
        assert bench.entry_digest(e) == e["sha256"], f"{name}: kernel changed since its ncu capture"
        assert 0.5 < e["dram_over_algorithmic"] < 2.0
        assert bench.measured_traffic(name, 1.0e9) == e["dram_over_algorithmic"] * 1.0e9


def test_summaries_state_their_commands():
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read()
        assert "ncu " in text and "--clock-control none" in text, path
        assert "python bench.py" in text, path

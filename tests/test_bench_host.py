"""Host-side pieces of bench.py (CPU): the workload's output sizes follow the
rounding rule max(1, floor(n s + 1/2)), and the recorded DRAM traffic of the
dominant kernel is reported only for the kernel sources it was measured on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_output_sizes():
    assert bench.out_sizes() == [5612, 1229]


def test_traffic_only_for_the_measured_sources(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.recorded_traffic() == float(rec["dram_bytes_per_launch"])
    assert bench.recorded_traffic(rec["form"]) == float(rec["dram_bytes_per_launch"])
    other = list(rec["form"])
    other[4] += 4        # another strip width: not the measured configuration
    assert bench.recorded_traffic(other) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic() is None


def test_traffic_sources_exist():
    assert len(bench.kernel_source_hash()) == 16


def test_committed_traffic_is_current():
    # the committed DRAM record was taken on the kernel sources as they stand
    # (a change to them needs a new capture, else the bench reports null)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec["source_hash"] == bench.kernel_source_hash()

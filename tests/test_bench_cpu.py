"""bench.py host helpers without a GPU: the all-cores oracle baseline and the
profile-traffic lookup (valid only for the kernel sources it was taken on)."""
import os

import bench


def test_all_cores_oracle_baseline_runs_one_process_per_core():
    r = bench.cpu_baseline_all_cores(n=64, runs=1)
    assert r["cores"] == (os.cpu_count() or 1)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT and r["value"] > 0


def test_profiled_traffic_requires_matching_sources(monkeypatch):
    assert bench.profiled_traffic("no-such-kernel") is None
    got = bench.profiled_traffic("fused2")
    if got is not None:  # the committed summary matches these sources
        assert 0.9 * 536870912 < got < 1.1 * 536870912
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "000000000000")
    assert bench.profiled_traffic("fused2") is None

"""The committed DRAM-traffic records (profiles/sweep_traffic.json, read by
bench.py for the roofline's `traffic`) must describe the sweep sources as
they are: each record carries the hash of the files its kernel is built
from.  CPU only."""
import json
import os

import bench


def test_traffic_records_match_the_current_sweep_sources():
    path = os.path.join(bench.ROOT, "profiles", "sweep_traffic.json")
    with open(path) as f:
        recs = json.load(f)
    assert {"precision", "batched", "appendix", "families", "boxcut"} <= set(recs)
    for name, rec in recs.items():
        files = tuple(rec.get("files", bench.SWEEP_SOURCES))
        assert rec["source_hash"] == bench.sweep_source_hash(files), f"{name}: recapture the ncu traffic"
        assert 4.0 < rec["bytes_per_nnz"] < 16.0, name


def test_recorded_traffic_scales_with_nnz():
    t1 = bench.recorded_traffic("precision", 1_000_000, 40_000)
    t2 = bench.recorded_traffic("precision", 2_000_000, 80_000)
    assert t1 is not None and abs(t2 - 2 * t1) <= 1e-6 * t2
    assert bench.recorded_traffic("no-such-workload", 1, 1) is None

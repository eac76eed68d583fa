"""The committed DRAM-traffic records (profiles/sweep_traffic.json, read by
bench.py for the roofline's `traffic`) carry the hash of the sweep sources
they were captured from; bench.py must report a record's traffic only while
those sources are unchanged (null once the kernel has changed).  CPU only."""
import json
import os

import bench


def test_traffic_records_are_reported_only_for_the_sources_they_describe():
    path = os.path.join(bench.ROOT, "profiles", "sweep_traffic.json")
    with open(path) as f:
        recs = json.load(f)
    assert {"precision", "batched", "appendix", "families", "boxcut"} <= set(recs)
    for name, rec in recs.items():
        assert 4.0 < rec["bytes_per_nnz"] < 16.0, name
        files = tuple(rec.get("files", bench.SWEEP_SOURCES))
        current = rec["source_hash"] == bench.sweep_source_hash(files)
        t = bench.recorded_traffic(name, 1_000_000, 40_000)
        if current:
            assert t is not None and abs(t - rec["bytes_per_nnz"] * 1_000_000) <= 1e-6 * t, name
        else:
            assert t is None, f"{name}: a stale record must not be reported"


def test_recorded_traffic_scales_with_nnz(tmp_path, monkeypatch):
    rec = {"precision": {"source_hash": bench.sweep_source_hash(), "bytes_per_nnz": 6.0, "bytes_per_user": 0.5}}
    (tmp_path / "profiles").mkdir()
    with open(tmp_path / "profiles" / "sweep_traffic.json", "w") as f:
        json.dump(rec, f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sweep_source_hash", lambda files=bench.SWEEP_SOURCES: rec["precision"]["source_hash"])
    t1 = bench.recorded_traffic("precision", 1_000_000, 40_000)
    t2 = bench.recorded_traffic("precision", 2_000_000, 80_000)
    assert t1 == 6.0 * 1_000_000 + 0.5 * 40_000 and abs(t2 - 2 * t1) <= 1e-6 * t2
    assert bench.recorded_traffic("no-such-workload", 1, 1) is None

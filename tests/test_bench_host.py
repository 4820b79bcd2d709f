"""Host logic of bench.py that needs no GPU: the oracle replicas of the CPU
baseline and of the reference arm (spawned processes, one thread each) report
an aggregate rate consistent with one replica alone."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_replicas_aggregate():
    import bench
    one, t1 = bench._oracle_step_rate(8, 2, 1, 1, 1, 0)
    agg, t2 = bench._oracle_rate_all_cores(8, 2, 1, 1, 1, 0, 2)
    assert one > 0 and agg > 0 and t1 > 0 and t2 > 0
    # two replicas side by side: the work of two in the time of the slower one
    cells = 1 * 6 * 8 * 8 * 2
    assert abs(agg - 2 * cells / t2) <= 1e-9 * agg
    assert 0.3 * one < agg < 6 * one


def test_traffic_only_from_a_capture_of_these_sources(tmp_path, monkeypatch):
    """the roofline's DRAM traffic is scaled from a capture of the same launch
    configuration taken on the current kernel sources; a capture of other
    sources, or of another configuration, gives no traffic"""
    import json

    import bench
    cap = {"kernel": "k_d_sw", "precision": "f64", "bx": 16, "by": 16, "kchunk": 1, "persistent": True,
           "bytes_per_cell": 200.0, "capture_cells": 1000, "capture": "test", "source_sha": bench.source_sha()}
    stale = dict(cap, precision="f32", source_sha="0" * 64)
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps({"captures": [cap, stale]}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    t, rec = bench.dram_traffic("k_d_sw", "f64", 16, 16, 1, True, 50)
    assert t == 200.0 * 50 and "stale" not in rec
    t, rec = bench.dram_traffic("k_d_sw", "f32", 16, 16, 1, True, 50)
    assert t is None and "stale" in rec
    assert bench.dram_traffic("k_d_sw", "f64", 32, 8, 1, True, 50) == (None, None)

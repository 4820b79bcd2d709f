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

"""The bench's host-side legs work without a GPU: the CPU baseline (the
oracle on the host cores, threaded and with one BLAS thread in a child
process) returns a well-formed record."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_cpu_baseline_record():
    import bench
    rec = bench.cpu_baseline(16, budget_s=0.3)
    assert rec["kind"] == "oracle" and rec["unit"] == "TFLOP/s" and rec["value"] > 0
    assert rec["cores"] >= 1 and "repetitions" in rec["sample"]
    one = rec["single_core"]
    assert one["cores"] == 1 and one["value"] > 0 and one["repetitions"] >= 1

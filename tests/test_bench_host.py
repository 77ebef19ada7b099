"""The bench's host-side legs work without a GPU: the CPU baseline (the
dense FFT Moulinec-Suquet oracle on the host cores, on the bench's sphere
RVE) returns a well-formed record, and the bounds the bench checks an
effective tensor against hold for a tensor inside them and fail outside."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_cpu_baseline_record():
    import bench
    rec = bench.cpu_baseline(3, budget_s=0.3)
    assert rec["kind"] == "oracle" and rec["unit"] == "iterations/s" and rec["value"] > 0
    assert rec["cores"] >= 1 and "iterations" in rec["sample"]


def test_bound_checks():
    import bench
    N, rows, moduli, C0 = bench.sphere_problem(3)
    lam1, mu1, lam2, mu2 = moduli
    f = 0.2
    mid = 0.5 * ((1 - f) * bench.iso_voigt(lam1, mu1) + f * bench.iso_voigt(lam2, mu2)
                 + np.linalg.inv((1 - f) * np.linalg.inv(bench.iso_voigt(lam1, mu1))
                                 + f * np.linalg.inv(bench.iso_voigt(lam2, mu2))))
    c = bench.checks(mid, moduli, f)
    assert c["voigt_minus_C_min_eig"] > 0 and c["C_minus_reuss_min_eig"] > 0 and c["asymmetry"] < 1e-12
    lo, hi = c["hs_bulk_bounds"]
    assert lo < hi
    c2 = bench.checks(2.0 * bench.iso_voigt(lam2, mu2), moduli, f)
    assert c2["voigt_minus_C_min_eig"] < 0 and not c2["bulk_within_hs"]

"""Seeded input generators: shapes, phase fractions, determinism."""
import numpy as np

from paper_2512_07811_gb300 import inputs as I


def test_geometries_have_the_requested_fractions():
    assert abs(I.sphere_indicator(64, 0.2).mean() - 0.2) < 0.01
    assert abs(I.box_indicator(64, 0.2).mean() - 0.2) < 0.03
    lam = I.laminate_indicator(32)
    assert lam.mean() == 0.5 and np.all(lam[:16] == 1) and np.all(lam[16:] == 0)
    f = I.fibre_rve(64, np.random.default_rng(5), count=32, fibre_fraction=0.3)
    assert abs(f.mean() - 0.3) < 0.03
    assert np.all(f == f[:, :, :1])  # aligned with z


def test_ellipsoid_rves_are_admissible_and_reproducible():
    a = [I.ellipsoid_rve(16, rng) for _, rng in I.batched_rve_set(count=5, seed=4)]
    b = [I.ellipsoid_rve(16, rng) for _, rng in I.batched_rve_set(count=5, seed=4)]
    for (ia, ca), (ib, cb) in zip(a, b):
        assert 0.1 <= ia.mean() <= 0.3 and 5.0 <= ca <= 100.0
        assert np.array_equal(ia, ib) and ca == cb


def test_batched_set_sizes():
    s = I.batched_rve_set(count=64, seed=4)
    sizes = [n for n, _ in s]
    assert len(s) == 64 and min(sizes) >= 6 and max(sizes) <= 9


def test_random_tt_is_seeded():
    a = I.random_tt_cores(10, 2, 8, seed=3, dtype=np.complex128)
    b = I.random_tt_cores(10, 2, 8, seed=3, dtype=np.complex128)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert a[5].shape == (8, 2, 8)

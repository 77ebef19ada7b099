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


def test_multibox_boxes_are_disjoint_and_reproducible():
    """The squares are at least one voxel apart under the periodic minimum
    image, the voxelised union covers about the requested area, and the
    draw is reproducible."""
    N = 256
    b = I.multibox_boxes_2d(N, count=8, area_fraction=0.2, seed=5)
    assert b.shape == (8, 6) and np.array_equal(b, I.multibox_boxes_2d(N, count=8, area_fraction=0.2, seed=5))
    for i in range(len(b)):
        for j in range(i):
            dx = abs((b[i, 0] - b[j, 0] + 0.5) % 1.0 - 0.5)
            dy = abs((b[i, 1] - b[j, 1] + 0.5) % 1.0 - 0.5)
            assert dx >= b[i, 3] + b[j, 3] + 1.0 / N or dy >= b[i, 4] + b[j, 4] + 1.0 / N
    img = I.boxes_indicator(b, (N, N, 1))
    assert abs(img.mean() - 0.2) < 0.06
    np.testing.assert_array_equal(img, I.multibox_indicator_2d(N, count=8, area_fraction=0.2, seed=5))


def test_boxes_value_periodic_and_boundary_inclusive():
    """A box centred on the cell corner wraps around; a voxel centre exactly
    on the box boundary counts as inside."""
    box = np.array([[0.0, 0.0, 0.5, 0.125, 0.125, 0.5]])
    img = I.boxes_indicator(box, (8, 8, 1))[:, :, 0]
    inside = {0, 7}
    for i in range(8):
        for j in range(8):
            assert img[i, j] == (1.0 if (i in inside and j in inside) else 0.0)
    edge = np.array([[0.5, 0.5, 0.5, 0.0625, 0.5, 0.5]])   # centres 7/16 and 9/16 on the boundary
    col = I.boxes_indicator(edge, (8, 1, 1))[:, 0, 0]
    np.testing.assert_array_equal(col, [0, 0, 0, 1, 1, 0, 0, 0])


def test_laminate_box_equals_laminate_image():
    for N in (4, 32, 256):
        np.testing.assert_array_equal(I.boxes_indicator(I.laminate_boxes_2d(), (N, N, 1)), I.laminate_indicator_2d(N))


def test_boxes_geometry_in_the_binding():
    """The binding's Boxes geometry keeps the rows and checks the grid sizes
    (host logic only)."""
    import pytest
    from paper_2512_07811_gb300 import qtt as Q
    g = Q.Boxes(I.laminate_boxes_2d(), (1 << 16, 1 << 16, 1))
    assert g.nbits == [16, 16, 0] and g.boxes.shape == (1, 6)
    with pytest.raises(ValueError):
        Q.Boxes(I.laminate_boxes_2d(), (100, 64, 1))

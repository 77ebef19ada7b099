"""Pins of the TT-cross oracle (Sec. 3, operator setup): maxvol against the
volume bound of dominant submatrices (brute force over all row subsets),
cross approximations of tensors with known exact QTT ranks (a separable
product: rank 1; an exponential: rank 1; a sine: rank 2), and the sampled
Green operator and box phase indicator against their dense definitions
(the pointwise samplers are pinned to the dense arrays entry by entry)."""
import itertools
import math

import numpy as np
import pytest

from oracle import cross as X
from oracle import ms as MS
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I


def test_maxvol_finds_dominant_rows():
    """Rows scaled by 100 dominate: maxvol returns them, B[rows] = I, |B| <= tol."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 4))
    big = [3, 7, 11, 15]
    A[big] *= 100.0
    rows, B = X.maxvol(A)
    assert sorted(rows) == big
    np.testing.assert_allclose(B[rows], np.eye(4), atol=1e-12)
    np.testing.assert_allclose(B, A @ np.linalg.inv(A[rows]), atol=1e-12)
    assert np.abs(B).max() <= 1.05


@pytest.mark.parametrize("seed", range(6))
def test_maxvol_volume_bound_brute_force(seed):
    """A submatrix with |A A[rows]^-1| <= tol has volume at least
    max volume / (tol sqrt(r))^r (Goreinov-Tyrtyshnikov): checked against all
    C(8, 3) row subsets."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    rows, B = X.maxvol(A)
    assert np.abs(B).max() <= 1.05 + 1e-12
    vol = abs(np.linalg.det(A[rows]))
    best = max(abs(np.linalg.det(A[list(s)])) for s in itertools.combinations(range(8), 3))
    assert vol * (1.05 * math.sqrt(3)) ** 3 >= best
    # dominance: no single row swap raises the volume by more than the tolerance
    for j in range(3):
        for i in range(8):
            if i in rows:
                continue
            trial = list(rows)
            trial[j] = i
            assert abs(np.linalg.det(A[trial])) <= 1.05 * vol * (1 + 1e-12)


def test_cross_separable_product_rank_one():
    rng = np.random.default_rng(1)
    modes = [3, 4, 2, 5, 3]
    g = [rng.standard_normal(n) for n in modes]

    def f(idx):
        return np.prod([g[k][idx[:, k]] for k in range(len(modes))], axis=0)

    cores, info = X.tt_cross(f, modes, 1e-12)
    full = T.tt_full(cores).reshape(modes)
    ref = np.einsum("a,b,c,d,e->abcde", *g)
    assert np.abs(full - ref).max() < 1e-13 * np.abs(ref).max()
    y, _ = T.tt_round(cores, 1e-12)
    assert T.tt_ranks(y) == [1] * 6


def _bits_value(idx, n):
    return (idx * (1 << np.arange(n - 1, -1, -1))).sum(axis=1)


@pytest.mark.parametrize("n", [10, 14])
def test_cross_exponential_and_sine_qtt_ranks(n):
    """exp(-3x) has QTT rank 1 and sin(6 pi x + 0.3) rank 2 (closed forms:
    exp of a sum of bits is a product; sin(a + b) = sin a cos b + cos a sin b)."""
    x = np.arange(1 << n) / (1 << n)
    for fun, rank in [(lambda t: np.exp(-3.0 * t), 1), (lambda t: np.sin(6 * np.pi * t + 0.3), 2)]:
        cores, info = X.tt_cross(lambda idx: fun(_bits_value(idx, n) / (1 << n)), [2] * n, 1e-12)
        assert np.abs(T.tt_full(cores).reshape(-1) - fun(x)).max() < 1e-12
        y, _ = T.tt_round(cores, 1e-12)
        assert max(T.tt_ranks(y)) == rank


@pytest.mark.parametrize("kind,nb,ordering", [("scalar", (3, 3, 0), "interleaved"),
                                              ("scalar", (2, 3, 1), "grouped"),
                                              ("elastic", (2, 2, 1), "interleaved")])
def test_green_sampler_equals_dense_definition(kind, nb, ordering):
    """Every entry of green_fn equals the dense Green operator in the
    momentum site order (bits of each dimension reversed)."""
    shape = tuple(1 << b for b in nb)
    ind = np.zeros(shape)
    pb = MS.scalar_problem(ind, 1.0, 10.0) if kind == "scalar" else MS.elastic_problem(ind, 1.0, 1.0, 10.0, 5.0)
    nc = pb.ncomp
    G = MS.green_dense(pb).reshape((nc * nc,) + shape)
    Gs = MS.spatial_to_sites(G, nb, ordering, momentum=True, lead=1)
    d = sum(nb)
    idx = np.array(list(itertools.product(range(nc * nc), *[range(2)] * d)))
    vals = X.green_fn(pb, nb, ordering)(idx)
    np.testing.assert_array_equal(vals.reshape(Gs.shape), Gs)


@pytest.mark.parametrize("nb,ordering", [((4, 3, 0), "interleaved"), ((2, 2, 3), "grouped")])
def test_boxes_sampler_equals_voxelisation(nb, ordering):
    shape = tuple(1 << b for b in nb)
    boxes = np.array([[0.3, 0.6, 0.5, 0.2, 0.15, 0.5], [0.9, 0.1, 0.25, 0.12, 0.3, 0.2]])
    ref = MS.spatial_to_sites(I.boxes_indicator(boxes, shape), nb, ordering)
    d = sum(nb)
    idx = np.array(list(itertools.product(*[range(2)] * d)))
    vals = X.boxes_fn(boxes, nb, ordering)(idx)
    np.testing.assert_array_equal(vals.reshape(ref.shape), ref)


@pytest.mark.parametrize("kind,nb,ordering", [("scalar", (4, 4, 0), "interleaved"),
                                              ("scalar", (3, 3, 3), "grouped"),
                                              ("elastic", (3, 2, 2), "interleaved")])
def test_cross_green_matches_dense(kind, nb, ordering):
    shape = tuple(1 << b for b in nb)
    ind = np.zeros(shape)
    pb = MS.scalar_problem(ind, 1.0, 10.0) if kind == "scalar" else MS.elastic_problem(ind, 1.0, 1.0, 10.0, 5.0)
    nc = pb.ncomp
    Gs = MS.spatial_to_sites(MS.green_dense(pb).reshape((nc * nc,) + shape), nb, ordering, momentum=True, lead=1)
    cores, info = X.tt_cross(X.green_fn(pb, nb, ordering), [nc * nc] + [2] * sum(nb), 1e-10)
    full = T.tt_full(cores).reshape(Gs.shape)
    assert np.linalg.norm(full - Gs) / np.linalg.norm(Gs) < 1e-9
    # the interpolation needs no more rank than the dense TT-SVD at the same tolerance, up to the kick columns
    y, _ = T.tt_round(cores, 1e-10)
    assert max(T.tt_ranks(y)) <= max(T.tt_ranks(T.tt_svd(Gs.astype(np.complex128), 1e-10))) + 2


@pytest.mark.parametrize("nb,ordering", [((5, 5, 0), "interleaved"), ((6, 6, 0), "grouped"),
                                         ((3, 3, 3), "interleaved")])
def test_cross_boxes_exact(nb, ordering):
    shape = tuple(1 << b for b in nb)
    if nb[2] == 0:
        boxes = I.multibox_boxes_2d(shape[0], count=6, seed=3)
    else:
        boxes = np.array([[0.5, 0.5, 0.5, 0.3, 0.2, 0.25]])
    ref = MS.spatial_to_sites(I.boxes_indicator(boxes, shape), nb, ordering)
    cores, info = X.tt_cross(X.boxes_fn(boxes, nb, ordering), [2] * sum(nb), 1e-10, init_rank=8)
    assert np.abs(T.tt_full(cores).reshape(ref.shape) - ref).max() < 1e-10


def test_box_centre_points_are_inside():
    """The seed points of a box geometry lie in phase 2 (the centre voxel of
    every box wider than a voxel)."""
    nb = (7, 6, 0)
    boxes = I.multibox_boxes_2d(128, count=8, seed=9)
    for ordering in ["interleaved", "grouped"]:
        pts = X.box_centre_points(boxes, nb, ordering)
        assert np.all(X.boxes_fn(boxes, nb, ordering)(pts) == 1.0)


def test_cross_boxes_fine_grid_with_seeds():
    """2^14 x 2^14 multibox: with the centre seeds and kick 8 the cross reaches
    the exact indicator (20000 random samples)."""
    nb = (14, 14, 0)
    boxes = I.multibox_boxes_2d(1 << 14, count=8, seed=5)
    f = X.boxes_fn(boxes, nb)
    cores, info = X.tt_cross(f, [2] * 28, 1e-10, kick=8, init_rank=8, max_half_sweeps=24,
                             init_points=X.box_centre_points(boxes, nb))
    rng = np.random.default_rng(0)
    idx = rng.integers(0, 2, (20000, 28))
    assert np.abs(T.tt_entries(cores, idx) - f(idx)).max() < 1e-10


@pytest.mark.parametrize("kind", ["scalar", "elastic"])
def test_ms_with_cross_operators_equals_dense_operators(kind):
    """16 x 16 plane box: the QTT solve with the phase and Green trains built
    by TT-cross gives the effective-tensor column of the TT-SVD-built ones."""
    boxes = np.array([[0.5, 0.5, 0.5, 0.25, 0.25, 0.5]])
    ind = I.boxes_indicator(boxes, (16, 16, 1))
    pb = MS.scalar_problem(ind, 1.0, 10.0) if kind == "scalar" else MS.elastic_problem(ind, 1.0, 1.0, 10.0, 5.0)
    E = np.zeros(pb.ncomp)
    E[0] = 1.0
    dense = MS.ms_qtt(pb, E, ops=MS.build_operators(pb), eps=1e-10, tol=1e-10, max_iter=200)
    cross = MS.ms_qtt(pb, E, ops=MS.build_operators(pb, op_cross=True, boxes=boxes), eps=1e-10, tol=1e-10,
                      max_iter=200)
    assert np.abs(cross.sigma - dense.sigma).max() < 1e-8 * np.abs(dense.sigma).max()


def _ellipsoid_sets():
    rows, _, _ = I.ellipsoid_rve_rows(16, np.random.default_rng(11))
    return {"sphere": I.sphere_rows(0.2), "ellipsoids": rows,
            "fibres": I.fibre_rows(np.random.default_rng(5), count=6, fibre_fraction=0.3)}


@pytest.mark.parametrize("which", ["sphere", "ellipsoids", "fibres"])
def test_ellipsoid_voxelisation_equals_quadratic_form(which):
    """The ellipsoid rule (body-frame coordinates divided by the semi-axes)
    against the quadratic form D^T R diag(1/a^2) R^T D <= 1 written out
    independently, on every voxel not within rounding of the boundary; the
    sphere and the fibres also against their plain distance tests."""
    rows = _ellipsoid_sets()[which]
    N = 32
    shape = (N, N, N)
    ind = I.ellipsoids_indicator(rows, shape)
    c = (np.arange(N) + 0.5) / N
    inside = np.zeros(shape, dtype=bool)
    near = np.zeros(shape, dtype=bool)
    for e in rows:
        R = e[6:15].reshape(3, 3)
        M = R @ np.diag(1.0 / e[3:6] ** 2) @ R.T
        D = [c - e[a] for a in range(3)]
        D = [t - np.round(t) for t in D]
        g = np.stack(np.meshgrid(*D, indexing="ij"), axis=-1)
        q = np.einsum("...i,ij,...j->...", g, M, g)
        inside |= q <= 1.0
        near |= np.abs(q - 1.0) < 1e-9
    assert np.array_equal(ind[~near] > 0, inside[~near])
    if which == "sphere":
        np.testing.assert_array_equal(ind, I.sphere_indicator(N, 0.2))
    if which == "fibres":
        np.testing.assert_array_equal(ind, I.fibre_rve(N, np.random.default_rng(5), count=6, fibre_fraction=0.3))


@pytest.mark.parametrize("nb,ordering", [((3, 2, 3), "interleaved"), ((2, 3, 3), "grouped")])
@pytest.mark.parametrize("which", ["sphere", "ellipsoids", "fibres"])
def test_ellipsoids_sampler_equals_voxelisation(nb, ordering, which):
    rows = _ellipsoid_sets()[which]
    shape = tuple(1 << b for b in nb)
    ref = MS.spatial_to_sites(I.ellipsoids_indicator(rows, shape), nb, ordering)
    idx = np.array(list(itertools.product(*[range(2)] * sum(nb))))
    vals = X.ellipsoids_fn(rows, nb, ordering)(idx)
    np.testing.assert_array_equal(vals.reshape(ref.shape), ref)


@pytest.mark.parametrize("which,ordering", [("sphere", "interleaved"), ("sphere", "grouped"),
                                            ("ellipsoids", "grouped"), ("fibres", "interleaved")])
def test_cross_ellipsoids_exact(which, ordering):
    """The cross of an ellipsoid geometry reaches the exact voxel indicator."""
    rows = _ellipsoid_sets()[which]
    nb = (4, 4, 3)
    shape = tuple(1 << b for b in nb)
    ref = MS.spatial_to_sites(I.ellipsoids_indicator(rows, shape), nb, ordering)
    cores, info = X.tt_cross(X.ellipsoids_fn(rows, nb, ordering), [2] * sum(nb), 1e-10, kick=8, init_rank=8,
                             max_half_sweeps=24, init_points=X.ellipsoid_centre_points(rows, nb, ordering))
    assert np.abs(T.tt_full(cores).reshape(ref.shape) - ref).max() < 1e-10


def test_ellipsoid_centre_points_are_inside():
    rows = _ellipsoid_sets()["ellipsoids"]
    nb = (5, 5, 5)
    for ordering in ["interleaved", "grouped"]:
        pts = X.ellipsoid_centre_points(rows, nb, ordering)
        assert np.all(X.ellipsoids_fn(rows, nb, ordering)(pts) == 1.0)


def test_ms_with_cross_sphere_equals_dense_operators():
    """8^3 sphere (scalar): the QTT solve with the phase train sampled by
    TT-cross from the ellipsoid description gives the effective-tensor column
    of the TT-SVD of the dense image."""
    rows = I.sphere_rows(0.2)
    ind = I.ellipsoids_indicator(rows, (8, 8, 8))
    pb = MS.scalar_problem(ind, 1.0, 10.0)
    E = np.array([1.0, 0.0, 0.0])
    dense = MS.ms_qtt(pb, E, ops=MS.build_operators(pb, ordering="grouped"), eps=1e-9, tol=1e-8, max_iter=200)
    cross = MS.ms_qtt(pb, E, ops=MS.build_operators(pb, ordering="grouped", ellipsoids=rows), eps=1e-9,
                      tol=1e-8, max_iter=200)
    assert np.abs(cross.sigma - dense.sigma).max() < 1e-7 * np.abs(dense.sigma).max()

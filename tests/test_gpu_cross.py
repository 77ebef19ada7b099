"""Parity of the device TT-cross (Sec. 3, operator setup) with the oracle's
definitions: the Green operator and box phase trains against the dense
arrays on small grids, against pointwise samples on grids far too large to
store (2^36 voxels), and the homogenisation with cross-built operators
against the dense-built ones and against the plane laminate's closed form
on a 2^16 x 2^16 grid."""
import numpy as np
import pytest

from oracle import cross as X
from oracle import ms as MS
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2512_07811_gb300 import qtt
    return qtt


@pytest.fixture(scope="module")
def ctx(Q):
    return Q.Context(0)


def _problem(kind, shape):
    ind = np.zeros(shape)
    return MS.scalar_problem(ind, 1.0, 10.0) if kind == "scalar" else MS.elastic_problem(ind, 1.0, 1.0, 10.0, 5.0)


def _green(Q, ctx, pb, nb, ordering, eps=1e-10):
    return Q.tt_cross(ctx, "green", nb, eps, interleaved=ordering == "interleaved", ncomp=pb.ncomp, k0=pb.k0,
                      lam0=pb.lam0, mu0=pb.mu0)


@pytest.mark.parametrize("kind,nb,ordering", [("scalar", (4, 4, 0), "interleaved"),
                                              ("scalar", (3, 3, 3), "grouped"),
                                              ("elastic", (3, 2, 2), "interleaved"),
                                              ("elastic", (5, 5, 0), "grouped")])
def test_cross_green_matches_dense(Q, ctx, kind, nb, ordering):
    shape = tuple(1 << b for b in nb)
    pb = _problem(kind, shape)
    nc = pb.ncomp
    Gs = MS.spatial_to_sites(MS.green_dense(pb).reshape((nc * nc,) + shape), nb, ordering, momentum=True, lead=1)
    y, info = _green(Q, ctx, pb, nb, ordering)
    full = T.tt_full(y.cores()).reshape(Gs.shape)
    assert np.linalg.norm(full - Gs) / np.linalg.norm(Gs) < 1e-9
    assert info.half_sweeps >= 2 and info.rel_change <= 1e-9
    assert max(y.ranks) <= max(T.tt_ranks(T.tt_svd(Gs.astype(np.complex128), 1e-10))) + 4


@pytest.mark.parametrize("nb,ordering", [((6, 6, 0), "interleaved"), ((7, 7, 0), "grouped"),
                                         ((4, 4, 4), "interleaved")])
def test_cross_boxes_exact(Q, ctx, nb, ordering):
    shape = tuple(1 << b for b in nb)
    if nb[2] == 0:
        boxes = I.multibox_boxes_2d(shape[0], count=8, seed=2)
    else:
        boxes = np.array([[0.5, 0.5, 0.5, 0.3, 0.2, 0.25], [0.1, 0.9, 0.2, 0.15, 0.1, 0.12]])
    ref = MS.spatial_to_sites(I.boxes_indicator(boxes, shape), nb, ordering)
    y, info = Q.tt_cross(ctx, "boxes", nb, 1e-10, interleaved=ordering == "interleaved", boxes=boxes)
    assert np.abs(T.tt_full(y.cores()).reshape(ref.shape) - ref).max() < 1e-10


def _samples(rng, first, d, count):
    head = rng.integers(0, first, (count, 1))
    return np.concatenate([head, rng.integers(0, 2, (count, d))], axis=1)


@pytest.mark.parametrize("kind", ["scalar", "elastic"])
def test_cross_green_plane_2pow18_samples(Q, ctx, kind):
    """2^18 x 2^18 plane grid (36 spatial sites): 4000 sampled entries of the
    device train against the oracle's pointwise Green operator."""
    nb = (18, 18, 0)
    pb = _problem(kind, (2, 2, 2))
    y, info = _green(Q, ctx, pb, nb, "interleaved")
    rng = np.random.default_rng(5)
    idx = _samples(rng, pb.ncomp ** 2, 36, 4000)
    # include the zero frequency and Nyquist corners
    idx[:2, 1:] = 0
    idx[2, 1:] = 0
    idx[2, 1 + 34] = 1
    got = T.tt_entries(y.cores(), idx)
    want = X.green_fn(pb, nb, "interleaved")(idx)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() < 1e-8 * scale


def test_cross_boxes_plane_2pow16_samples(Q, ctx):
    nb = (16, 16, 0)
    boxes = I.multibox_boxes_2d(1 << 16, count=8, seed=4)
    y, info = Q.tt_cross(ctx, "boxes", nb, 1e-10, boxes=boxes)
    rng = np.random.default_rng(6)
    idx = rng.integers(0, 2, (4000, 32))
    got = T.tt_entries(y.cores(), idx)
    want = X.boxes_fn(boxes, nb, "interleaved")(idx)
    assert want.sum() > 100                      # the samples do hit the inclusions
    assert np.abs(got - want).max() < 1e-8


def test_ms_cross_operators_equal_dense_operators(Q, ctx):
    """32 x 32 plane multibox: phase and Green trains by TT-cross give the
    effective tensor of the dense-built operators (the same 12 iterations)."""
    boxes = I.multibox_boxes_2d(32, count=6, seed=1)
    ind = I.boxes_indicator(boxes, (32, 32, 1))
    kw = dict(tol=0.0, max_rank=64, eps=1e-10, max_iter=12, min_iter=12, oversample=16, prec=Q.PREC_F64)
    Cd, rd = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), **kw)
    Cx, rx = Q.ms_homogenize(ctx, Q.Boxes(boxes, (32, 32, 1)), "scalar", (1.0, 10.0), 5.5 * np.eye(3),
                             op_cross=True, **kw)
    assert np.abs(Cx - Cd).max() < 1e-8 * np.abs(Cd).max()
    assert rx.green_rank > 1 and rx.phase_rank > 1


def test_ms_cross_matches_dense_oracle_elastic(Q, ctx):
    """16 x 16 x 1 plane box in plane strain, operators by TT-cross, against
    the dense FFT oracle (load case E = e_11)."""
    boxes = np.array([[0.5, 0.5, 0.5, 0.25, 0.25, 0.5]])
    ind = I.boxes_indicator(boxes, (16, 16, 1))
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    pb = MS.elastic_problem(ind, lam1, mu1, lam2, mu2)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-11, max_iter=500)
    C, rep = Q.ms_homogenize(ctx, Q.Boxes(boxes, (16, 16, 1)), "elastic", (lam1, mu1, lam2, mu2), pb.C0,
                             tol=1e-11, max_rank=96, eps=1e-11, max_iter=300, oversample=16, prec=Q.PREC_F64,
                             op_cross=True, load_mask=1)
    assert np.linalg.norm(C[:, 0] - Cd.real[:, 0]) / np.linalg.norm(Cd.real[:, 0]) < 1e-7


def test_ms_plane_laminate_2pow16_closed_form(Q, ctx):
    """65536 x 65536 plane laminate (32 spatial sites, no dense operand
    anywhere): k_eff = diag(20/11, 11/2, 11/2)."""
    C, rep = Q.ms_homogenize(ctx, Q.Boxes(I.laminate_boxes_2d(), (1 << 16, 1 << 16, 1)), "scalar", (1.0, 10.0),
                             5.5 * np.eye(3), tol=1e-13, max_rank=32, eps=1e-10, max_iter=20, prec=Q.PREC_F64)
    np.testing.assert_allclose(C, np.diag([20.0 / 11.0, 5.5, 5.5]), atol=1e-9)

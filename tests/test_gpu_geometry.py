"""The curved 3D geometries (a centred sphere, random ellipsoids, aligned
fibres) on the GPU: the device TT-cross of their phase trains against the
dense voxelisation of the input generators, the FP64 homogenisation of an
elastic sphere against the dense FFT solver (Algorithm 1, the oracle), and
the float (fast) path against the FP64 path on non-trivial geometries with a
rank cap that does not bind (the 1e-4 bound on the effective tensor)."""
import numpy as np
import pytest

from oracle import cross as X
from oracle import ms as MS
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LAM1, MU1 = I.lame_from_young(1.0, 0.3)
LAM2, MU2 = I.lame_from_young(10.0, 0.3)


@pytest.fixture(scope="module")
def Q():
    from paper_2512_07811_gb300 import qtt
    return qtt


@pytest.fixture(scope="module")
def ctx(Q):
    return Q.Context(0)


def _rows(which):
    if which == "sphere":
        return I.sphere_rows(0.2)
    if which == "ellipsoids":
        return I.ellipsoid_rve_rows(16, np.random.default_rng(11))[0]
    return I.fibre_rows(np.random.default_rng(5), count=6, fibre_fraction=0.3)


@pytest.mark.parametrize("which,nb,ordering", [("sphere", (4, 4, 4), "grouped"),
                                               ("sphere", (4, 3, 4), "interleaved"),
                                               ("ellipsoids", (4, 4, 3), "grouped"),
                                               ("fibres", (4, 4, 2), "interleaved")])
def test_cross_ellipsoids_matches_voxelisation(Q, ctx, which, nb, ordering):
    rows = _rows(which)
    shape = tuple(1 << b for b in nb)
    ref = MS.spatial_to_sites(I.ellipsoids_indicator(rows, shape), nb, ordering)
    y, info = Q.tt_cross(ctx, "ellipsoids", nb, 1e-10, interleaved=ordering == "interleaved", ellipsoids=rows)
    full = T.tt_full(y.cores()).reshape(ref.shape)
    assert np.abs(full - ref).max() < 1e-10


def test_cross_sphere_64cubed_matches_voxelisation(Q, ctx):
    """64^3 sphere, grouped sites: the exact indicator (rank about 110)."""
    nb = (6, 6, 6)
    rows = I.sphere_rows(0.2)
    y, info = Q.tt_cross(ctx, "ellipsoids", nb, 1e-10, interleaved=False, ellipsoids=rows)
    ref = MS.spatial_to_sites(I.ellipsoids_indicator(rows, (64, 64, 64)), nb, "grouped")
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 2, (20000, 18))
    vals = T.tt_entries(y.cores(), idx)
    ref_vals = X.ellipsoids_fn(rows, nb, "grouped")(idx)
    assert np.abs(vals - ref_vals).max() < 1e-9
    assert abs(T.tt_entries(y.cores(), np.zeros((1, 18), dtype=np.int64))[0] - ref.reshape(-1)[0]) < 1e-9


def _dense_columns(pb, cols, tol):
    G = MS.green_dense(pb)
    out = []
    for k in cols:
        E = np.zeros(pb.ncomp)
        E[k] = 1.0
        out.append(MS.ms_dense(pb, E, tol, 2000, G).sigma.real)
    return np.stack(out, axis=1)


def test_ms_elastic_sphere_fp64_matches_dense_oracle(Q, ctx):
    """16^3 elastic sphere (E 10:1, nu 0.3), load cases e_11 and e_23: the
    FP64 QTT solve (phase train by TT-cross from the sphere description,
    grouped sites, rank cap far above the ranks reached) equals the dense FFT
    solver's columns to 1e-7."""
    N = 16
    rows = I.sphere_rows(0.2)
    pb = MS.elastic_problem(I.ellipsoids_indicator(rows, (N, N, N)), LAM1, MU1, LAM2, MU2)
    Cd = _dense_columns(pb, [0, 3], 1e-11)
    geo = Q.Ellipsoids(rows, (N, N, N))
    C, rep = Q.ms_homogenize(ctx, geo, "elastic", (LAM1, MU1, LAM2, MU2), pb.C0, tol=1e-10, max_rank=512,
                             eps=1e-11, max_iter=300, prec=Q.PREC_F64, load_mask=0b1001, interleaved=False)
    assert rep.max_rank_seen < 512
    assert rep.iterations[0] < 300 and rep.iterations[3] < 300
    got = C[:, [0, 3]]
    assert np.linalg.norm(got - Cd) / np.linalg.norm(Cd) < 1e-7


def _fast_vs_fp64(Q, ctx, geo, kind, moduli, C0, mask, interleaved):
    """C_eff columns of the FP64 path (eps 1e-9, converged to 1e-8) and of the
    float path (eps 1e-6, converged to 5e-5: its residual settles at the
    single-precision noise of the iterates, about 2e-5 on these grids)."""
    kw = dict(load_mask=mask, interleaved=interleaved, max_iter=200, max_rank=512)
    C64, r64 = Q.ms_homogenize(ctx, geo, kind, moduli, C0, tol=1e-8, eps=1e-9, prec=Q.PREC_F64, **kw)
    C32, r32 = Q.ms_homogenize(ctx, geo, kind, moduli, C0, tol=5e-5, eps=1e-6, prec=Q.PREC_F32, **kw)
    assert all(r64.iterations[k] < 200 for k in range(6) if mask >> k & 1)
    assert all(r32.iterations[k] < 200 for k in range(6) if mask >> k & 1)
    assert r32.fp64_residuals >= 1
    assert r64.max_rank_seen < 512 and r32.max_rank_seen < 512
    cols = [k for k in range(C64.shape[0]) if mask >> k & 1]
    a, b = C64[:, cols], C32[:, cols]
    return np.linalg.norm(b - a) / np.linalg.norm(a)


def test_fast_path_elastic_sphere_within_1e4_of_fp64(Q, ctx):
    """16^3 elastic sphere, load cases e_11 and e_12: the float path
    (complex64 contractions and factorisations, FP64 stop test) gives C_eff
    within 1e-4 of the FP64 path when the rank cap does not bind."""
    N = 16
    rows = I.sphere_rows(0.2)
    C0 = MS.iso_voigt(0.5 * (LAM1 + LAM2), 0.5 * (MU1 + MU2))
    rel = _fast_vs_fp64(Q, ctx, Q.Ellipsoids(rows, (N, N, N)), "elastic", (LAM1, MU1, LAM2, MU2), C0, 0b100001,
                        False)
    print("\nelastic sphere 16^3: fast vs FP64 %.2e" % rel)
    assert rel < 1e-4


def test_fast_path_plane_multibox_within_1e4_of_fp64(Q, ctx):
    """128 x 128 multibox image (8 squares, contrast 10), load case e_1: the
    float path within 1e-4 of the FP64 path, rank cap not binding."""
    N = 128
    geo = Q.Boxes(I.multibox_boxes_2d(N, seed=5), (N, N, 1))
    rel = _fast_vs_fp64(Q, ctx, geo, "scalar", (1.0, 10.0), 5.5 * np.eye(3), 0b1, True)
    print("\nmultibox 128^2: fast vs FP64 %.2e" % rel)
    assert rel < 1e-4


def test_tf32_sketch_path_elastic_sphere_within_1e4_of_fp64(Q, ctx):
    """The same 16^3 sphere with the sketch contractions on the tensor cores
    (QTT_PREC_TF32S, batched, three-term TF32 split): C_eff within 1e-4 of
    the FP64 path."""
    N = 16
    rows = I.sphere_rows(0.2)
    C0 = MS.iso_voigt(0.5 * (LAM1 + LAM2), 0.5 * (MU1 + MU2))
    geo = Q.Ellipsoids(rows, (N, N, N))
    kw = dict(load_mask=0b1, interleaved=False, max_iter=200, max_rank=512)
    C64, _ = Q.ms_homogenize(ctx, geo, "elastic", (LAM1, MU1, LAM2, MU2), C0, tol=1e-8, eps=1e-9,
                             prec=Q.PREC_F64, **kw)
    Ct, rt = Q.ms_homogenize(ctx, geo, "elastic", (LAM1, MU1, LAM2, MU2), C0, tol=5e-5, eps=1e-6,
                             prec=Q.PREC_TF32S, **kw)
    rel = np.linalg.norm(Ct[:, 0] - C64[:, 0]) / np.linalg.norm(C64[:, 0])
    print("\nelastic sphere 16^3: tensor-core sketch path vs FP64 %.2e (%d iterations)" % (rel, rt.iterations[0]))
    assert rt.iterations[0] < 200 and rel < 1e-4


def test_float_setup_elastic_sphere_within_1e4_of_fp64(Q, ctx):
    """The float path with its operator trains built in float (operator
    tolerance 1e-6: the dense Green-operator TT-SVD in complex64): C_eff of
    the 16^3 sphere within 1e-4 of the FP64 path with FP64 operators."""
    N = 16
    C0 = MS.iso_voigt(0.5 * (LAM1 + LAM2), 0.5 * (MU1 + MU2))
    geo = Q.Ellipsoids(I.sphere_rows(0.2), (N, N, N))
    kw = dict(load_mask=0b1, interleaved=False, max_iter=200, max_rank=512)
    C64, _ = Q.ms_homogenize(ctx, geo, "elastic", (LAM1, MU1, LAM2, MU2), C0, tol=1e-8, eps=1e-9,
                             prec=Q.PREC_F64, **kw)
    Cf, rf = Q.ms_homogenize(ctx, geo, "elastic", (LAM1, MU1, LAM2, MU2), C0, tol=5e-5, eps=1e-6,
                             op_tol=1e-6, prec=Q.PREC_F32, **kw)
    rel = np.linalg.norm(Cf[:, 0] - C64[:, 0]) / np.linalg.norm(C64[:, 0])
    print("\nelastic sphere 16^3, float operators: vs FP64 %.2e (setup %.0f ms)" % (rel, rf.setup_ms))
    assert rf.iterations[0] < 200 and rel < 1e-4

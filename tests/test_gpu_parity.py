"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances: placement work (tt_add with exactly representable scales) is
bit-exact; FP64 arithmetic is compared at 1e-12 relative on gauge-invariant
quantities (contracted tensors, norms of difference trains computed by the
oracle, inner products, singular-value ranks); FP32 storage at 1e-5.
Sizes span several 64-wide GEMM tiles and ragged tails.
"""
import math

import numpy as np
import pytest

from oracle import ms as MS
from oracle import qft as QF
from oracle import randround as RR
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


def cplx_tt(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((ranks[k], n, ranks[k + 1]))
             + 1j * rng.standard_normal((ranks[k], n, ranks[k + 1]))) / math.sqrt(2 * max(ranks))
            for k, n in enumerate(dims)]


def rel_diff(a, b):
    """||a - b|| / ||b|| computed by the oracle on the difference train."""
    nb = T.tt_norm(b)
    return T.tt_norm(T.tt_add(a, b, 1.0, -1.0)) / (nb if nb > 0 else 1.0)


DIMS = [2, 3, 2, 2, 5, 2, 2, 3]
RA = [1, 2, 6, 12, 70, 9, 6, 3, 1]
RB = [1, 3, 5, 65, 8, 10, 4, 3, 1]


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, -1.0), (2.0, 0.5), (0.5j, -4.0)])
def test_tt_add_bit_exact(Q, ctx, a, b):
    x, y = cplx_tt(DIMS, RA, 1), cplx_tt(DIMS, RB, 2)
    z = Q.tt_add(ctx, a, Q.TT.from_cores(ctx, x), b, Q.TT.from_cores(ctx, y))
    ref = T.tt_add(x, y, a, b)
    assert z.ranks == T.tt_ranks(ref)
    for g, r in zip(z.cores(), ref):
        assert np.array_equal(g, r)


def test_tt_hadamard(Q, ctx):
    x, y = cplx_tt(DIMS, RA, 3), cplx_tt(DIMS, RB, 4)
    z = Q.tt_hadamard(ctx, Q.TT.from_cores(ctx, x), Q.TT.from_cores(ctx, y))
    ref = T.tt_hadamard(x, y)
    assert z.ranks == T.tt_ranks(ref)
    for g, r in zip(z.cores(), ref):
        np.testing.assert_allclose(g, r, rtol=0, atol=4e-16 * np.abs(r).max())


def test_tt_mpo_apply(Q, ctx):
    rng = np.random.default_rng(5)
    gr = [1, 2, 3, 4, 2, 3, 2, 2, 1]
    mpo = [(rng.standard_normal((gr[k], n + (k % 2), n, gr[k + 1]))
            + 1j * rng.standard_normal((gr[k], n + (k % 2), n, gr[k + 1]))) for k, n in enumerate(DIMS)]
    x = cplx_tt(DIMS, RA, 6)
    z = Q.tt_mpo_apply(ctx, Q.MPO.from_cores(ctx, mpo), Q.TT.from_cores(ctx, x))
    ref = T.tt_mpo_apply(mpo, x)
    assert z.ranks == T.tt_ranks(ref)
    for g, r in zip(z.cores(), ref):
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-14 * np.abs(r).max())


def test_tt_dot_and_norm(Q, ctx):
    x, y = cplx_tt(DIMS, RA, 7), cplx_tt(DIMS, RB, 8)
    gx, gy = Q.TT.from_cores(ctx, x), Q.TT.from_cores(ctx, y)
    v = Q.tt_dot(ctx, gx, gy)
    ref = T.tt_dot(x, y)
    assert abs(v - ref) <= 1e-12 * T.tt_norm(x) * T.tt_norm(y)
    assert math.isclose(Q.tt_norm(ctx, gx), T.tt_norm(x), rel_tol=1e-12)


def test_round_gapped_spectrum_matches_oracle(Q, ctx):
    """A rank-k train written at rank 2k: unique truncation ranks, 1e-12 parity."""
    base = I.random_tt_cores(16, 2, 24, seed=11, dtype=np.complex128)
    x = T.tt_add(base, base, 1.0, 0.75)
    g = Q.TT.from_cores(ctx, x)
    y, info = Q.tt_round(ctx, g, 1e-10)
    ref, rinfo = T.tt_round(x, 1e-10)
    assert y.ranks == T.tt_ranks(ref) == T.tt_ranks(base)
    assert math.isclose(info.norm, rinfo["norm"], rel_tol=1e-12)
    assert rel_diff(y.cores(), ref) < 1e-12


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_round_bound_and_oracle_agreement(Q, ctx, eps):
    rng = np.random.default_rng(12)
    dims = [2] * 14
    low = I.random_tt_cores(14, 2, 40, seed=13, dtype=np.complex128)
    noise = I.random_tt_cores(14, 2, 20, seed=14, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    y, info = Q.tt_round(ctx, Q.TT.from_cores(ctx, x), eps)
    yc = y.cores()
    err = rel_diff(yc, x)
    assert err <= eps * (1 + 1e-9)
    ref, _ = T.tt_round(x, eps)
    # where the oracle and the GPU chose the same ranks, the results agree
    if y.ranks == T.tt_ranks(ref):
        assert rel_diff(yc, ref) < 1e-10
    # right-orthonormal cores 2..d
    for c in yc[1:]:
        M = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(c.shape[0]), atol=1e-12)


def test_round_forced_by_max_rank(Q, ctx):
    x = I.random_tt_cores(12, 2, 32, seed=15, dtype=np.complex128)
    y, info = Q.tt_round(ctx, Q.TT.from_cores(ctx, x), 1e-12, max_rank=9)
    ref, rinfo = T.tt_round(x, 1e-12, max_rank=9)
    assert info.capped == 1 and rinfo["capped"]
    assert y.ranks == T.tt_ranks(ref)
    assert rel_diff(y.cores(), ref) < 1e-10


@pytest.mark.parametrize("k,n0,n1", [(17, 39, 100), (25, 55, 150), (50, 300, 300), (64, 140, 256), (100, 205, 500),
                                     (128, 300, 512)])
@pytest.mark.parametrize("fp32", [False, True])
def test_round_factorisation_shapes(Q, ctx, k, n0, n1, fp32):
    """Two cores (1, n0, 2k) and (2k, n1, 1) holding 1.75 x a rank-k train:
    the left sweep factors an n0 x 2k matrix, the truncation SVD a
    (n1 x 2k) C^H, so the cases reach the block-cyclic Jacobi with odd block
    widths and 4 or 8 CTAs, 8 and 16 rows per lane, the shared-memory limit
    (2k = 200, 500 rows), the panel QR beyond 256 rows, and a 512 x 256 C^H
    that no single-launch Jacobi kernel takes (QR first, then Jacobi on the
    256 x 256 factor).  The rank-k
    truncation is unique: ranks equal, 1e-12 (FP64) / 1e-5 (FP32) parity."""
    rng = np.random.default_rng(100 + k)
    a = (rng.standard_normal((1, n0, k)) + 1j * rng.standard_normal((1, n0, k))) / math.sqrt(2 * k)
    b = (rng.standard_normal((k, n1, 1)) + 1j * rng.standard_normal((k, n1, 1))) / math.sqrt(2 * k)
    x = T.tt_add([a, b], [a, b], 1.0, 0.75)
    eps = 1e-5 if fp32 else 1e-10
    g = Q.TT.from_cores(ctx, x, dtype=Q.C64 if fp32 else Q.C128)
    y, info = Q.tt_round(ctx, g, eps)
    ref, _ = T.tt_round(x, eps)
    assert y.ranks == T.tt_ranks(ref) == [1, k, 1]
    err = rel_diff([c.astype(np.complex128) for c in y.cores()], ref)
    assert err < (1e-5 if fp32 else 1e-12)


def test_round_fp32(Q, ctx):
    base = I.random_tt_cores(14, 2, 20, seed=16, dtype=np.complex128)
    x = T.tt_add(base, base, 1.0, 1.0)
    g = Q.TT.from_cores(ctx, x, dtype=Q.C64)
    y, info = Q.tt_round(ctx, g, 1e-4)
    assert y.ranks == T.tt_ranks(base)
    assert rel_diff([c.astype(np.complex128) for c in y.cores()], T.tt_scale(2.0, base)) < 1e-5


def test_round_edge_cases(Q, ctx):
    # one core
    x = [np.arange(5, dtype=np.complex128).reshape(1, 5, 1)]
    y, info = Q.tt_round(ctx, Q.TT.from_cores(ctx, x), 1e-8)
    np.testing.assert_array_equal(y.cores()[0], x[0])
    # zero train rounds to rank 1 zero
    z = [np.zeros((1, 2, 3)), np.zeros((3, 2, 3)), np.zeros((3, 2, 1))]
    y, info = Q.tt_round(ctx, Q.TT.from_cores(ctx, z), 1e-8)
    assert y.ranks == [1, 1, 1, 1] and info.norm == 0.0
    assert all(np.count_nonzero(c) == 0 for c in y.cores()[:1])
    # ranks limited by mode products (rank-deficient R factors)
    w = I.random_tt_cores(6, 3, 50, seed=17, dtype=np.complex128, ranks=[1, 3, 9, 27, 9, 3, 1])
    y, _ = Q.tt_round(ctx, Q.TT.from_cores(ctx, w), 1e-13)
    assert rel_diff(y.cores(), w) < 1e-12


def test_sketched_rounding_matches_oracle(Q, ctx):
    """Same Gaussian sketch on both sides: the projected trains agree to 1e-11."""
    dims = [2] * 12
    x = I.random_tt_cores(12, 2, 16, seed=21, dtype=np.complex128)
    rng = np.random.default_rng(22)
    gr = [1] + [3] * 11 + [1]
    mpo = [(rng.standard_normal((gr[k], 2, 2, gr[k + 1])) + 1j * rng.standard_normal((gr[k], 2, 2, gr[k + 1])))
           / 2.0 for k in range(12)]
    y = I.random_tt_cores(12, 2, 5, seed=23, dtype=np.complex128)
    ell = 30
    sr = RR.sketch_ranks(12, dims, ell)
    S = [rng.standard_normal((sr[k], 2, sr[k + 1])).astype(np.complex128) for k in range(12)]
    s_full = T.tt_add(T.tt_mpo_apply(mpo, x), y, 1.5, -0.5)
    P = RR.rand_orth(s_full, S)
    ref, _ = T.tt_round(P, 1e-12)
    g, info = Q.tt_round_sketched(ctx, [(1.5, Q.MPO.from_cores(ctx, mpo), Q.TT.from_cores(ctx, x)),
                                        (-0.5, None, Q.TT.from_cores(ctx, y))],
                                  Q.TT.from_cores(ctx, S), 1e-12)
    assert rel_diff(g.cores(), ref) < 1e-11
    # and the result is close to the exact sum (the sketch width covers rank 16*3+5)
    assert rel_diff(g.cores(), s_full) < 0.5


def test_sketched_exact_for_low_rank_sum(Q, ctx):
    x = I.random_tt_cores(10, 2, 6, seed=24, dtype=np.complex128)
    rng = np.random.default_rng(25)
    sr = RR.sketch_ranks(10, [2] * 10, 14)
    S = [rng.standard_normal((sr[k], 2, sr[k + 1])).astype(np.complex128) for k in range(10)]
    g, info = Q.tt_round_sketched(ctx, [(1.0, None, Q.TT.from_cores(ctx, x)), (2.0, None, Q.TT.from_cores(ctx, x))],
                                  Q.TT.from_cores(ctx, S), 1e-12)
    assert rel_diff(g.cores(), T.tt_scale(3.0, x)) < 1e-12
    assert g.ranks == T.tt_ranks(x)


def test_tt_from_dense_matches_tt_svd(Q, ctx):
    import torch
    rng = np.random.default_rng(26)
    low = cplx_tt([4, 2, 3, 2, 2, 4, 2], [1, 3, 5, 7, 6, 4, 2, 1], 27)
    F = T.tt_full(low) + 1e-9 * (rng.standard_normal(T.tt_full(low).shape))
    dev = torch.from_numpy(np.ascontiguousarray(F.astype(np.complex128))).cuda()
    g = Q.tt_from_dense(ctx, dev.data_ptr(), list(F.shape), 1e-6)
    ref = T.tt_svd(F, 1e-6)
    assert g.ranks == T.tt_ranks(ref)
    np.testing.assert_allclose(T.tt_full(g.cores()), F, atol=1e-6 * np.linalg.norm(F))


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_qft_mpo_is_bitreversed_dft(Q, ctx, n):
    A = Q.qtt_qft_mpo(ctx, n, -1, 1e-12)
    M = T.mpo_full(A.cores())
    N = 1 << n
    F = np.fft.fft(np.eye(N), norm="ortho", axis=0)
    np.testing.assert_allclose(M, F[QF.bit_reverse_indices(n)], atol=1e-10)
    assert max(A.ranks) <= 16


def test_ms_scalar_laminate_32cubed_15_sites(Q, ctx):
    """32^3 laminate, 15 interleaved bit sites: the exact 20/11 and 11/2."""
    ind = I.laminate_indicator(32)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), tol=1e-12, max_rank=64,
                             eps=1e-8, max_iter=50, prec=Q.PREC_F64)
    np.testing.assert_allclose(C, MS.scalar_laminate_keff(1.0, 10.0, 0.5), atol=1e-10)
    assert max(rep.iterations[:3]) <= 3
    assert rep.sigma_imag_max < 1e-10


def test_ms_elastic_laminate_backus(Q, ctx):
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    ind = I.laminate_indicator(8)
    C0 = MS.iso_voigt(0.5 * (lam1 + lam2), 0.5 * (mu1 + mu2))
    C, rep = Q.ms_homogenize(ctx, ind, "elastic", (lam1, mu1, lam2, mu2), C0, tol=1e-13, max_rank=32,
                             eps=1e-12, max_iter=200, prec=Q.PREC_F64)
    Cx = MS.elastic_laminate_ceff([lam2, lam1], [mu2, mu1], [0.5, 0.5])
    np.testing.assert_allclose(C, Cx, atol=1e-9 * np.abs(Cx).max())


def test_ms_scalar_sphere_matches_dense_oracle(Q, ctx):
    pb = MS.scalar_problem(I.sphere_indicator(8, 0.2), 1.0, 10.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-10, max_iter=500)
    C, rep = Q.ms_homogenize(ctx, pb.indicator, "scalar", (1.0, 10.0), pb.C0, tol=1e-10, max_rank=200,
                             eps=1e-10, max_iter=200, oversample=16, prec=Q.PREC_F64)
    assert np.linalg.norm(C - Cd.real) / np.linalg.norm(Cd.real) < 1e-7


def test_ms_plane_laminate_closed_form(Q, ctx):
    """32 x 32 x 1 laminate (10 spatial sites, none along z): the plane
    laminate's k_eff = diag(20/11, 11/2, 11/2) to 1e-10 in FP64."""
    ind = I.laminate_indicator_2d(32)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), tol=1e-13, max_rank=32,
                             eps=1e-10, max_iter=20, prec=Q.PREC_F64)
    np.testing.assert_allclose(C, np.diag([20.0 / 11.0, 5.5, 5.5]), atol=1e-10)


def test_ms_plane_elastic_laminate_backus(Q, ctx):
    """16 x 16 x 1 elastic laminate in plane strain: the Backus averages."""
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    C0 = MS.iso_voigt(0.5 * (lam1 + lam2), 0.5 * (mu1 + mu2))
    C, rep = Q.ms_homogenize(ctx, I.laminate_indicator_2d(16), "elastic", (lam1, mu1, lam2, mu2), C0, tol=1e-13,
                             max_rank=32, eps=1e-12, max_iter=200, prec=Q.PREC_F64)
    Cx = MS.elastic_laminate_ceff([lam2, lam1], [mu2, mu1], [0.5, 0.5])
    np.testing.assert_allclose(C, Cx, atol=1e-9 * np.abs(Cx).max())


def test_ms_plane_box_matches_dense_oracle(Q, ctx):
    pb = MS.scalar_problem(I.box_indicator_2d(16, 0.25), 1.0, 10.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-11, max_iter=500)
    C, rep = Q.ms_homogenize(ctx, pb.indicator, "scalar", (1.0, 10.0), pb.C0, tol=1e-11, max_rank=64,
                             eps=1e-11, max_iter=300, oversample=16, prec=Q.PREC_F64)
    assert np.linalg.norm(C - Cd.real) / np.linalg.norm(Cd.real) < 1e-7


@pytest.mark.parametrize("interleaved", [True, False])
def test_ms_anisotropic_grid_matches_dense_oracle(Q, ctx, interleaved):
    """8 x 4 x 2 grid (3 + 2 + 1 bits): both site orders reach the dense result."""
    rng = np.random.default_rng(8)
    ind = (rng.random((8, 4, 2)) < 0.3).astype(np.float64)
    pb = MS.scalar_problem(ind, 1.0, 5.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-12, max_iter=500)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 5.0), pb.C0, tol=1e-12, max_rank=64, eps=1e-12,
                             max_iter=300, oversample=16, prec=Q.PREC_F64, interleaved=interleaved)
    assert np.linalg.norm(C - Cd.real) / np.linalg.norm(Cd.real) < 1e-8


def test_ms_fp32_laminate(Q, ctx):
    ind = I.laminate_indicator(16)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), tol=1e-6, max_rank=32,
                             eps=1e-6, max_iter=20, prec=Q.PREC_F32)
    Cx = MS.scalar_laminate_keff(1.0, 10.0, 0.5)
    assert np.abs(C - Cx).max() / np.abs(Cx).max() < 1e-5


@pytest.mark.parametrize("n", [13, 20])
def test_qft_layer_route_matches_fft(Q, ctx, n):
    """Beyond 12 bits the transform is built from circuit layers; applied to a
    random rank-3 train it must equal numpy's unitary FFT with bit-reversed output."""
    A = Q.qtt_qft_mpo(ctx, n, -1, 1e-12)
    assert max(A.ranks) <= 24
    rng = np.random.default_rng(40 + n)
    ranks = [1] + [3] * (n - 1) + [1]
    x = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) + 0j for k in range(n)]
    y = Q.tt_mpo_apply(ctx, A, Q.TT.from_cores(ctx, x))
    v = T.tt_full(x).reshape(-1)
    got = T.tt_full(y.cores()).reshape(-1)
    want = np.fft.fft(v, norm="ortho")[QF.bit_reverse_indices(n)]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-9


def test_mpo_diag_is_hadamard(Q, ctx):
    x, y = cplx_tt(DIMS, RA, 30), cplx_tt(DIMS, RB, 31)
    gx, gy = Q.TT.from_cores(ctx, x), Q.TT.from_cores(ctx, y)
    z = Q.tt_mpo_apply(ctx, Q.qtt_mpo_diag(ctx, gx), gy)
    assert rel_diff(z.cores(), T.tt_hadamard(x, y)) < 1e-13


@pytest.mark.parametrize("fp32", [False, True])
def test_dot_structured_matches_oracle(Q, ctx, fp32):
    """<y, 0.7 A x1 + (-0.3 + 0.2i) x2> without forming the sum equals the
    dense inner product of the oracle's explicit sum."""
    d = 8
    x1 = cplx_tt([2] * d, I.capped_ranks(d, 2, 5), 41)
    x2 = cplx_tt([2] * d, I.capped_ranks(d, 2, 3), 42)
    y = cplx_tt([2] * d, I.capped_ranks(d, 2, 4), 43)
    A = I.random_mpo_cores(d, 2, 3, seed=44)
    c1, c2 = 0.7, -0.3 + 0.2j
    s = c1 * T.tt_full(T.tt_mpo_apply(A, x1)) + c2 * T.tt_full(x2)
    ref = np.vdot(T.tt_full(y), s)
    dt = Q.C64 if fp32 else Q.C128
    got = Q.tt_dot_structured(ctx, [(c1, Q.MPO.from_cores(ctx, A, dt), Q.TT.from_cores(ctx, x1, dt)),
                                    (c2, None, Q.TT.from_cores(ctx, x2, dt))], Q.TT.from_cores(ctx, y, dt))
    assert abs(got - ref) <= (2e-5 if fp32 else 1e-12) * np.linalg.norm(s) * np.linalg.norm(T.tt_full(y))


def test_profile_shapes_sum_to_class_totals(Q, ctx):
    """The per-shape profiler rows of each kernel class add up to the class
    totals (launches, time, model flops), and every GEMM row names a shape."""
    x = Q.TT.from_cores(ctx, I.random_tt_cores(12, 2, 24, seed=71, dtype=np.complex128), Q.C64)
    y = Q.TT.from_cores(ctx, I.random_tt_cores(12, 2, 24, seed=72, dtype=np.complex128), Q.C64)
    ctx.profile(True)
    try:
        z = Q.tt_add(ctx, 1.0, x, 0.5, y)
        Q.tt_round(ctx, z, 1e-6)
        for cls in ["gemm", "qr", "jacobi"]:
            tot = ctx.profile_read(cls)
            rows = ctx.profile_shapes(cls, 4096)
            assert sum(r["launches"] for r in rows) == tot["launches"]
            assert abs(sum(r["ms"] for r in rows) - tot["ms"]) <= 1e-9 * max(1.0, tot["ms"])
            assert abs(sum(r["flops"] for r in rows) - tot["flops"]) <= 1e-9 * max(1.0, tot["flops"])
            assert all(r["ms"] >= rows[i + 1]["ms"] for i, r in enumerate(rows[:-1]))
            if cls == "gemm":
                assert tot["launches"] > 0
                assert all(min(r["dims"]) > 0 and r["batch"] > 0 and r["variant"] >= 3200 for r in rows)
    finally:
        ctx.profile(False)

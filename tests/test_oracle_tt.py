"""Pins for the oracle's tensor-train algebra (Sec. 2 of the paper).

Every check compares against something other than the oracle itself:
explicit loops over multi-indices (the definition Eq. tt_format), dense
NumPy arithmetic on the contracted tensors, the Eckart-Young optimum, or
invariants of the construction.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import tt as T
from oracle import randround as RR
from paper_2512_07811_gb300 import inputs as I


def brute_full(cores):
    """x(i_1..i_d) = A_1(i_1) ... A_d(i_d), one multi-index at a time."""
    dims = [c.shape[1] for c in cores]
    out = np.zeros(dims, dtype=np.result_type(*cores))
    for idx in itertools.product(*[range(n) for n in dims]):
        m = np.eye(1, dtype=out.dtype)
        for c, i in zip(cores, idx):
            m = m @ c[:, i, :]
        out[idx] = m[0, 0]
    return out


def brute_mpo(cores):
    dims_o = [c.shape[1] for c in cores]
    dims_i = [c.shape[2] for c in cores]
    R = int(np.prod(dims_o))
    C = int(np.prod(dims_i))
    out = np.zeros((R, C), dtype=np.result_type(*cores))
    for ri, io in enumerate(itertools.product(*[range(n) for n in dims_o])):
        for ci, ii in enumerate(itertools.product(*[range(n) for n in dims_i])):
            m = np.eye(1, dtype=out.dtype)
            for c, a, b in zip(cores, io, ii):
                m = m @ c[:, a, b, :]
            out[ri, ci] = m[0, 0]
    return out


def rand_tt(dims, ranks, seed, cplx=True):
    rng = np.random.default_rng(seed)
    cores = []
    for k, n in enumerate(dims):
        shape = (ranks[k], n, ranks[k + 1])
        a = rng.standard_normal(shape)
        if cplx:
            a = a + 1j * rng.standard_normal(shape)
        cores.append(a)
    return cores


DIMS = [2, 3, 2, 2, 3]
RA = [1, 2, 3, 4, 2, 1]
RB = [1, 3, 2, 2, 3, 1]


def test_full_matches_definition():
    x = rand_tt(DIMS, RA, 1)
    np.testing.assert_allclose(T.tt_full(x), brute_full(x), rtol=1e-13, atol=1e-13)


def test_rank_one_is_outer_product():
    vs = [np.arange(1, n + 1, dtype=float) * (k + 1) for k, n in enumerate(DIMS)]
    x = [v.reshape(1, -1, 1) for v in vs]
    dense = vs[0]
    for v in vs[1:]:
        dense = np.multiply.outer(dense, v)
    np.testing.assert_array_equal(T.tt_full(x), dense)


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (2.0, -1.0), (0.5 + 1j, -3.0)])
def test_add_is_elementwise_sum(a, b):
    x = rand_tt(DIMS, RA, 2)
    y = rand_tt(DIMS, RB, 3)
    z = T.tt_add(x, y, a, b)
    assert T.tt_ranks(z) == [1] + [p + q for p, q in zip(RA[1:-1], RB[1:-1])] + [1]
    np.testing.assert_allclose(T.tt_full(z), a * brute_full(x) + b * brute_full(y),
                               rtol=1e-12, atol=1e-12)


def test_add_block_placement_exact():
    """Inner cores are exactly diag(A, B): placement is pure indexing."""
    x = rand_tt(DIMS, RA, 4)
    y = rand_tt(DIMS, RB, 5)
    z = T.tt_add(x, y)
    k = 2
    A, B, C = x[k], y[k], z[k]
    assert np.array_equal(C[:A.shape[0], :, :A.shape[2]], A)
    assert np.array_equal(C[A.shape[0]:, :, A.shape[2]:], B)
    assert np.count_nonzero(C[:A.shape[0], :, A.shape[2]:]) == 0
    assert np.count_nonzero(C[A.shape[0]:, :, :A.shape[2]]) == 0


def test_hadamard_is_elementwise_product():
    x = rand_tt(DIMS, RA, 6)
    y = rand_tt(DIMS, RB, 7)
    z = T.tt_hadamard(x, y)
    assert T.tt_ranks(z) == [p * q for p, q in zip(RA, RB)]
    np.testing.assert_allclose(T.tt_full(z), brute_full(x) * brute_full(y),
                               rtol=1e-12, atol=1e-12)


def test_mpo_apply_is_matvec():
    rng = np.random.default_rng(8)
    g = [1, 2, 3, 2, 2, 1]
    mpo = []
    for k, n in enumerate(DIMS):
        no = n + (k % 2)          # rectangular operator cores too
        mpo.append(rng.standard_normal((g[k], no, n, g[k + 1]))
                   + 1j * rng.standard_normal((g[k], no, n, g[k + 1])))
    x = rand_tt(DIMS, RA, 9)
    y = T.tt_mpo_apply(mpo, x)
    M = brute_mpo(mpo)
    np.testing.assert_allclose(T.mpo_full(mpo), M, rtol=1e-12, atol=1e-12)
    expect = M @ brute_full(x).reshape(-1)
    np.testing.assert_allclose(T.tt_full(y).reshape(-1), expect, rtol=1e-11, atol=1e-11)
    assert T.tt_ranks(y) == [p * q for p, q in zip(g, RA)]


def test_mpo_product_and_adjoint():
    rng = np.random.default_rng(10)
    mk = lambda: [rng.standard_normal((a, 2, 2, b)) + 1j * rng.standard_normal((a, 2, 2, b))
                  for a, b in [(1, 2), (2, 3), (3, 1)]]
    A, B = mk(), mk()
    np.testing.assert_allclose(T.mpo_full(T.mpo_mpo(A, B)), brute_mpo(A) @ brute_mpo(B),
                               rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(T.mpo_full(T.mpo_adjoint(A)), brute_mpo(A).conj().T,
                               rtol=1e-12, atol=1e-12)


def test_dot_and_norm():
    x = rand_tt(DIMS, RA, 11)
    y = rand_tt(DIMS, RB, 12)
    fx, fy = brute_full(x), brute_full(y)
    assert abs(T.tt_dot(x, y) - np.vdot(fx, fy)) <= 1e-11 * np.linalg.norm(fx) * np.linalg.norm(fy)
    assert math.isclose(T.tt_norm(x), np.linalg.norm(fx), rel_tol=1e-12)


def test_left_orthogonal_isometry():
    x = rand_tt(DIMS, RA, 13)
    q = T.tt_left_orthogonalize(x)
    for c in q[:-1]:
        r0, n, r1 = c.shape
        M = c.reshape(r0 * n, r1)
        np.testing.assert_allclose(M.conj().T @ M, np.eye(r1), atol=1e-13)
    np.testing.assert_allclose(T.tt_full(q), brute_full(x), rtol=1e-12, atol=1e-12)


def test_truncation_rank_rule():
    s = np.array([4.0, 3.0, 1e-3, 1e-4])
    tail = lambda t: math.sqrt(float(np.sum(s[t:] ** 2)))
    for delta in [0.0, 1e-5, 1.1e-4, tail(2), tail(2) * 0.999, 3.5, 10.0]:
        t, _ = T.truncation_rank(s, delta)
        assert t >= 1
        assert tail(t) <= delta or t == len(s)
        if t > 1:
            assert tail(t - 1) > delta
    assert T.truncation_rank(s, 1e-9, max_rank=2) == (2, True)
    assert T.bucket_rank(17, 16, 100) == 32
    assert T.bucket_rank(17, 16, 20) == 20


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-8])
def test_round_error_bound(eps):
    """||x - round(x)|| <= eps ||x|| (Sec. 2.2, Eq. rounding_condition_tt)."""
    rng = np.random.default_rng(14)
    dims = [2] * 8
    x = rand_tt(dims, [1, 2, 4, 8, 8, 8, 4, 2, 1], 15)
    # make a spectrum with decay: scale a low-rank part and add a small perturbation
    y = rand_tt(dims, [1, 2, 2, 2, 2, 2, 2, 2, 1], 16)
    x = T.tt_add(y, x, 1.0, 1e-3)
    fx = brute_full(x)
    z, info = T.tt_round(x, eps)
    err = np.linalg.norm(T.tt_full(z) - fx)
    assert err <= eps * np.linalg.norm(fx) * (1 + 1e-10)
    assert math.isclose(info["norm"], np.linalg.norm(fx), rel_tol=1e-12)


def test_round_matrix_case_is_eckart_young():
    """d = 2: the rounding is the truncated SVD of the matrix."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((6, 7)) + 1j * rng.standard_normal((6, 7))
    x = [A.reshape(1, 6, 7), np.eye(7).reshape(7, 7, 1)]
    s = np.linalg.svd(A, compute_uv=False)
    z, info = T.tt_round(x, 0.0, max_rank=3)
    err = np.linalg.norm(T.tt_full(z) - A)
    assert math.isclose(err, math.sqrt(float(np.sum(s[3:] ** 2))), rel_tol=1e-10)


def test_round_recovers_padded_low_rank():
    """A rank-k train written at rank 2k (x + x) rounds back to rank k, exactly."""
    x = rand_tt([2] * 10, [1, 2, 4, 5, 5, 5, 5, 4, 2, 2, 1], 18)
    z, info = T.tt_round(T.tt_add(x, x), 1e-12)
    assert T.tt_ranks(z) == T.tt_ranks(x)
    fx = T.tt_full(x)
    assert np.linalg.norm(T.tt_full(z) - 2 * fx) <= 1e-13 * np.linalg.norm(fx) * 2 * 10


def test_round_right_orthogonal_cores():
    x = rand_tt([2] * 7, [1, 2, 4, 6, 4, 3, 2, 1], 19)
    z, _ = T.tt_round(x, 1e-10)
    for c in z[1:]:
        r0, n, r1 = c.shape
        M = c.reshape(r0, n * r1)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(r0), atol=1e-13)


def test_tt_svd_reconstruction():
    rng = np.random.default_rng(20)
    low = rand_tt([2, 3, 2, 4, 2], [1, 2, 3, 2, 2, 1], 21)
    F = brute_full(low)
    cores = T.tt_svd(F, 1e-13)
    assert max(T.tt_ranks(cores)) <= 3
    np.testing.assert_allclose(T.tt_full(cores), F, rtol=1e-11, atol=1e-11)
    G = rng.standard_normal((2, 2, 2, 2, 2, 2, 2))
    for eps in [0.3, 0.05]:
        c = T.tt_svd(G, eps)
        assert np.linalg.norm(T.tt_full(c) - G) <= eps * np.linalg.norm(G) * (1 + 1e-12)


def test_random_tt_generator_shapes():
    cores = I.random_tt_cores(30, 2, 64, seed=1064)
    ranks = T.tt_ranks(cores)
    assert ranks[0] == ranks[-1] == 1 and max(ranks) == 64
    assert ranks[3] == 8 and ranks[27] == 8


def test_rand_orth_exact_when_sketch_covers_rank():
    dims = [2] * 9
    x = rand_tt(dims, [1, 2, 4, 5, 5, 5, 5, 4, 2, 1], 22)
    x = T.tt_add(x, x, 1.0, 0.5)          # rank 10 representation of a rank-5 tensor
    rng = np.random.default_rng(23)
    ranks = RR.sketch_ranks(len(dims), dims, 8)
    R = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(len(dims))]
    y = RR.rand_orth(x, R)
    fx = T.tt_full(x)
    assert np.linalg.norm(T.tt_full(y) - fx) <= 1e-12 * np.linalg.norm(fx)
    z, info = RR.rand_round(x, R, 1e-10)
    assert info["err"] <= 1e-12
    assert max(T.tt_ranks(z)) <= 5


def test_rand_orth_is_projection_error_exact():
    """The randomized result is an orthogonal projection: ||x||^2 = ||y||^2 + ||x-y||^2."""
    dims = [2] * 8
    x = rand_tt(dims, [1, 2, 4, 8, 8, 8, 4, 2, 1], 24)
    rng = np.random.default_rng(25)
    ranks = RR.sketch_ranks(len(dims), dims, 3)
    R = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(len(dims))]
    y = RR.rand_orth(x, R)
    fx, fy = T.tt_full(x), T.tt_full(y)
    lhs = np.linalg.norm(fx) ** 2
    rhs = np.linalg.norm(fy) ** 2 + np.linalg.norm(fx - fy) ** 2
    assert math.isclose(lhs, rhs, rel_tol=1e-11)


def test_sketch_with_exact_right_part_is_stable_in_single_precision():
    """A train at its full (mode-capped) ranks rounded by the randomized
    projection in complex64: with Gaussian sketch cores on the bonds whose
    width is capped by the product of the modes to the right, the projection
    error grows with the condition number of square Gaussian matrices; with
    the identity unfolding there (inputs.sketch_cores) it stays at the
    single-precision level.  The projection runs in single precision by
    casting the oracle's inputs."""
    dims = [6] + [2] * 9
    ranks = [1]
    for k in range(1, 10):
        ranks.append(min(int(np.prod(dims[:k])), int(np.prod(dims[k:]))))
    ranks.append(1)
    x = rand_tt(dims, ranks, 31)
    fx = T.tt_full(x)
    x32 = [c.astype(np.complex64) for c in x]
    errs = {}
    for kind in ["gaussian", "exact_right"]:
        worst = 0.0
        for seed in range(6):
            rng = np.random.default_rng(100 + seed)
            if kind == "exact_right":
                R, _ = I.sketch_cores(rng, len(dims), dims, 56)
            else:
                rk = RR.sketch_ranks(len(dims), dims, 56)
                R = [rng.standard_normal((rk[k], dims[k], rk[k + 1])) / math.sqrt(dims[k] * rk[k + 1])
                     for k in range(len(dims))]
            y = RR.rand_orth(x32, [c.astype(np.complex64) for c in R])
            worst = max(worst, np.linalg.norm(T.tt_full([c.astype(np.complex128) for c in y]) - fx)
                        / np.linalg.norm(fx))
        errs[kind] = worst
    print(errs)
    assert errs["exact_right"] < 1e-5
    assert errs["gaussian"] > 10 * errs["exact_right"]

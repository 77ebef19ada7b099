"""Pins of the polar-based compression oracle (Sec. 2.2): the polar factors
and the sign function by their defining properties and closed forms, the
truncation by a matrix of known singular values, and the train rounding by
the rounding bound and by agreement with the SVD rounding where the spectrum
has a gap (then both keep exactly the same singular values)."""
import math

import numpy as np
import pytest

from oracle import polar as P
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_polar_worked_example():
    """A = Q D with Q a known unitary and D = diag(3, 2) positive: U = Q, H = D."""
    c, s = math.cos(0.7), math.sin(0.7)
    Q = np.array([[c, -s * 1j], [-s * 1j, c]])        # unitary
    D = np.diag([3.0, 2.0])
    U, H = P.polar(Q @ D)
    np.testing.assert_allclose(U, Q, atol=1e-14)
    np.testing.assert_allclose(H, D, atol=1e-14)


@pytest.mark.parametrize("m,q,rank", [(9, 5, 5), (6, 6, 6), (10, 6, 3)])
def test_polar_properties(m, q, rank):
    rng = np.random.default_rng(m * 10 + q)
    A = crandn(rng, m, rank) @ crandn(rng, rank, q)
    U, H = P.polar(A)
    np.testing.assert_allclose(U @ H, A, atol=1e-12 * np.linalg.norm(A))
    np.testing.assert_allclose(H, H.conj().T, atol=1e-13 * np.linalg.norm(A))
    assert np.linalg.eigvalsh(H).min() > -1e-12 * np.linalg.norm(A)
    # U is an isometry on the range of H (exactly an isometry at full rank)
    w, V = np.linalg.eigh(H)
    Vr = V[:, w > 1e-10 * w.max()]
    np.testing.assert_allclose((U @ Vr).conj().T @ (U @ Vr), np.eye(Vr.shape[1]), atol=1e-12)


def test_sign_hermitian_closed_form():
    """B = V diag(-2, 0.5, 3) V^H: sign(B) = V diag(-1, 1, 1) V^H; S^2 = I; SB = BS."""
    rng = np.random.default_rng(3)
    V, _ = np.linalg.qr(crandn(rng, 3, 3))
    B = (V * np.array([-2.0, 0.5, 3.0])) @ V.conj().T
    S = P.sign_hermitian(B)
    np.testing.assert_allclose(S, (V * np.array([-1.0, 1.0, 1.0])) @ V.conj().T, atol=1e-13)
    np.testing.assert_allclose(S @ S, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(S @ B, B @ S, atol=1e-12)


def test_polar_truncate_known_spectrum():
    """A = W diag(5, 2, 1e-3, 1e-6) V^H cut at 1e-2: rank 2, F G = the rank-2
    truncation, tail = sqrt(1e-6 + 1e-12), F orthonormal."""
    rng = np.random.default_rng(4)
    W, _ = np.linalg.qr(crandn(rng, 7, 4))
    V, _ = np.linalg.qr(crandn(rng, 4, 4))
    s = np.array([5.0, 2.0, 1e-3, 1e-6])
    A = (W * s) @ V.conj().T
    F, G, l, tail = P.polar_truncate(A, 1e-2)
    assert l == 2
    np.testing.assert_allclose(F @ G, (W[:, :2] * s[:2]) @ V[:, :2].conj().T, atol=1e-12)
    assert math.isclose(tail, math.sqrt(1e-6 + 1e-12), rel_tol=1e-8)
    np.testing.assert_allclose(F.conj().T @ F, np.eye(2), atol=1e-13)


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_round_polar_bound_and_orthonormal_cores(eps):
    low = I.random_tt_cores(10, 2, 12, seed=31, dtype=np.complex128)
    noise = I.random_tt_cores(10, 2, 6, seed=32, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    y, info = P.tt_round_polar(x, eps)
    err = T.tt_norm(T.tt_add(y, x, 1.0, -1.0))
    assert err <= eps * T.tt_norm(x) * (1 + 1e-9)
    for c in y[1:]:
        M = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(c.shape[0]), atol=1e-12)
    # the absolute cutoff delta / q is conservative: no bond below the SVD rounding's rank
    ref, _ = T.tt_round(x, eps)
    assert all(a >= b for a, b in zip(T.tt_ranks(y), T.tt_ranks(ref)))


def test_round_polar_gapped_equals_svd_rounding():
    """A rank-k train written at rank 2k has singular values either O(1) or
    zero: both roundings keep exactly the nonzero ones."""
    base = I.random_tt_cores(12, 2, 10, seed=33, dtype=np.complex128)
    x = T.tt_add(base, base, 1.0, 0.5)
    y, _ = P.tt_round_polar(x, 1e-8)
    ref, _ = T.tt_round(x, 1e-8)
    assert T.tt_ranks(y) == T.tt_ranks(ref) == T.tt_ranks(base)
    assert T.tt_norm(T.tt_add(y, ref, 1.0, -1.0)) < 1e-11 * T.tt_norm(ref)

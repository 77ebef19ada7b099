"""Pins for the superfast Fourier transform Q_n (Sec. 3.2, Fig. 1).

Q_n = R_n^{-1} QFT_n: the DFT with its output bits reversed.  The oracle
builds it as a product of circuit layers; these tests check it against the
direct DFT from numpy.fft and against an independently written bit formula.
"""
import math

import numpy as np
import pytest

from oracle import qft as QF
from oracle import tt as T


def dft_bitrev(n):
    """numpy's unitary forward DFT with rows permuted by bit reversal."""
    N = 1 << n
    F = np.fft.fft(np.eye(N), norm="ortho", axis=0)
    rev = [int(format(m, "0%db" % n)[::-1], 2) for m in range(N)]
    return F[rev]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 10])
def test_qft_mpo_matches_bitreversed_dft(n):
    Q = QF.qft_mpo(n)
    M = T.mpo_full(Q)
    np.testing.assert_allclose(M, dft_bitrev(n), atol=1e-11)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_qft_closed_form(n):
    np.testing.assert_allclose(QF.qft_closed_form(n), dft_bitrev(n), atol=1e-12)


def test_bit_reverse_permutation_exact():
    for n in range(1, 9):
        rev = QF.bit_reverse_indices(n)
        assert sorted(rev.tolist()) == list(range(1 << n))
        assert np.array_equal(rev[rev], np.arange(1 << n))
        assert rev[1] == 1 << (n - 1)


def test_qft_bond_dimension_small():
    """The bond of Q_n stays small (<= 16) for n up to 12 at 1e-12."""
    for n in [8, 10, 12]:
        Q = QF.qft_mpo(n)
        assert max(D.shape[3] for D in Q) <= 16


def test_qft_unitary_and_inverse():
    n = 6
    Q = QF.qft_mpo(n)
    Qi = T.mpo_adjoint(Q)
    P = T.mpo_full(T.mpo_mpo(Qi, Q))
    np.testing.assert_allclose(P, np.eye(1 << n), atol=1e-11)


def test_qft_on_tt_matches_fft():
    """Apply Q to a random rank-3 train and compare with the FFT of the vector."""
    n = 7
    rng = np.random.default_rng(3)
    ranks = [1] + [3] * (n - 1) + [1]
    x = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(n)]
    v = T.tt_full(x).reshape(-1)
    y = T.tt_mpo_apply(QF.qft_mpo(n), x)
    np.testing.assert_allclose(T.tt_full(y).reshape(-1), dft_bitrev(n) @ v, atol=1e-10)

"""Pins of the AMEn oracle y ~ A x (Sec. 2.1 / 3.2): exact products where the
product's TT rank is within reach (identity, diagonal and random operator
trains, the Green operator applied to a transformed polarisation field of
the homogenisation), the rounding bound on products with a decaying
spectrum, and ranks no larger than those of the SVD rounding of the exact
product (plus nothing: the final rounding strips the enrichment)."""
import numpy as np
import pytest

from oracle import amen as AM
from oracle import ms as MS
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I


def _rand_mpo(d, n, g, seed):
    rng = np.random.default_rng(seed)
    ranks = [1] + [g] * (d - 1) + [1]
    return [rng.standard_normal((ranks[k], n, n, ranks[k + 1])) + 1j * rng.standard_normal((ranks[k], n, n, ranks[k + 1]))
            for k in range(d)]


def _rel(y, ref):
    return np.linalg.norm(T.tt_full(y) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("which", ["identity", "diagonal", "random"])
def test_amen_exact_products(which):
    d = 9
    x = I.random_tt_cores(d, 2, 4, seed=1, dtype=np.complex128)
    if which == "identity":
        A = T.identity_mpo([2] * d)
    elif which == "diagonal":
        A = T.diag_mpo_from_tt(I.random_tt_cores(d, 2, 3, seed=2, dtype=np.complex128))
    else:
        A = _rand_mpo(d, 2, 3, seed=3)
    exact = T.tt_mpo_apply(A, x)
    y, info = AM.amen_mv(A, x, 1e-12)
    assert _rel(y, T.tt_full(exact)) < 1e-12
    assert T.tt_ranks(y) == T.tt_ranks(T.tt_round(exact, 1e-12)[0])


@pytest.mark.parametrize("eps", [1e-3, 1e-2])
def test_amen_rounding_bound_on_decaying_spectrum(eps):
    d = 10
    low = I.random_tt_cores(d, 2, 5, seed=4, dtype=np.complex128)
    noise = I.random_tt_cores(d, 2, 5, seed=5, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    A = T.diag_mpo_from_tt(I.random_tt_cores(d, 2, 3, seed=6, dtype=np.complex128))
    exact = T.tt_mpo_apply(A, x)
    y, info = AM.amen_mv(A, x, eps)
    assert _rel(y, T.tt_full(exact)) <= eps
    assert max(T.tt_ranks(y)) <= max(T.tt_ranks(T.tt_round(exact, eps)[0]))


def test_amen_green_operator_on_polarisation_field():
    """The Green step of the QTT homogenisation on a 16 x 16 plane box:
    AMEn equals the exact MPO x TT product."""
    pb = MS.scalar_problem(I.box_indicator_2d(16, 0.25), 1.0, 10.0)
    ops = MS.build_operators(pb)
    tau = T.tt_round(T.tt_mpo_apply(ops.dC, MS.e_tt(np.array([1.0, 0.0, 0.0]), 8)), 1e-12)[0]
    for q in ops.qft:
        if q is not None:
            tau = T.tt_round(T.tt_mpo_apply(q, tau), 1e-12)[0]
    exact = T.tt_mpo_apply(ops.gamma, tau)
    y, info = AM.amen_mv(ops.gamma, tau, 1e-10)
    assert _rel(y, T.tt_full(exact)) < 1e-10


def test_ms_with_amen_green_step_equals_rounded_product():
    """4 x 4 x 2 random grid: Algorithm 2 with the Green step by AMEn
    reaches the effective-tensor column of the rounded-product version."""
    rng = np.random.default_rng(21)
    ind = (rng.random((4, 4, 2)) < 0.3).astype(np.float64)
    pb = MS.scalar_problem(ind, 1.0, 5.0)
    E = np.array([1.0, 0.0, 0.0])
    ops = MS.build_operators(pb)
    a = MS.ms_qtt(pb, E, ops=ops, eps=1e-11, tol=1e-10, max_iter=300)
    b = MS.ms_qtt(pb, E, ops=ops, eps=1e-11, tol=1e-10, max_iter=300, green_amen=True)
    assert np.abs(a.sigma - b.sigma).max() < 1e-8 * np.abs(a.sigma).max()

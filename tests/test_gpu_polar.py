"""Parity of the polar-based compression (Sec. 2.2) on the GPU (Newton-Schulz
iterations, matrix products only) with the oracle's plain-definition version:
equal ranks and trains on gapped spectra; the rounding bound, conservative
ranks and right-orthonormal cores on noisy ones; the same in FP32 and with
the products on the tensor cores (TC32)."""
import numpy as np
import pytest

from oracle import polar as P
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


def rel(a, b):
    return T.tt_norm(T.tt_add(a, b, 1.0, -1.0)) / T.tt_norm(b)


def test_polar_gapped_matches_oracle_and_svd(Q, ctx):
    base = I.random_tt_cores(10, 2, 12, seed=41, dtype=np.complex128)
    x = T.tt_add(base, base, 1.0, 0.5)
    y, info = Q.tt_round_polar(ctx, Q.TT.from_cores(ctx, x), 1e-8)
    ref, _ = P.tt_round_polar(x, 1e-8)
    svd, _ = T.tt_round(x, 1e-8)
    assert y.ranks == T.tt_ranks(ref) == T.tt_ranks(svd) == T.tt_ranks(base)
    assert rel(y.cores(), ref) < 1e-10
    assert rel(y.cores(), svd) < 1e-10


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_polar_bound_ranks_orthonormal(Q, ctx, eps):
    low = I.random_tt_cores(10, 2, 16, seed=42, dtype=np.complex128)
    noise = I.random_tt_cores(10, 2, 8, seed=43, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    y, info = Q.tt_round_polar(ctx, Q.TT.from_cores(ctx, x), eps)
    yc = y.cores()
    assert rel(yc, x) <= eps * (1 + 1e-8)
    svd, _ = T.tt_round(x, eps)
    assert all(a >= b for a, b in zip(y.ranks, T.tt_ranks(svd)))
    ref, _ = P.tt_round_polar(x, eps)
    if y.ranks == T.tt_ranks(ref):
        assert rel(yc, ref) < 1e-9
    for c in yc[1:]:
        M = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(c.shape[0]), atol=1e-10)


@pytest.mark.parametrize("prec", ["f32", "tc32"])
def test_polar_low_precision(Q, ctx, prec):
    """complex64 storage; FP32 CUDA-core or TF32-split tensor-core products.
    The cutoff delta / q must sit above the arithmetic's resolution (eps 1e-2
    here): bound within that resolution, ranks of the FP64 polar rounding."""
    low = I.random_tt_cores(10, 2, 16, seed=44, dtype=np.complex128)
    noise = I.random_tt_cores(10, 2, 8, seed=45, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    p = Q.PREC_TC32 if prec == "tc32" else Q.PREC_F32
    y, _ = Q.tt_round_polar(ctx, Q.TT.from_cores(ctx, x, Q.C64), 1e-2, prec=p)
    yc = [c.astype(np.complex128) for c in y.cores()]
    assert rel(yc, x) <= 1e-2 + 1e-4
    ref, _ = P.tt_round_polar(x, 1e-2)
    assert y.ranks == T.tt_ranks(ref)
    assert rel(yc, ref) < 1e-4

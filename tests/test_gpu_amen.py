"""Parity of the device AMEn product y ~ A x (Sec. 2.1 / 3.2) with the
oracle's definitions: exact products where the rank is within reach
(identity, diagonal, random operator trains; FP64 and FP32), the rounding
bound and ranks on a decaying spectrum, the Green step of the plane box, a
warm start from the answer, and the homogenisation with its Green step by
AMEn against the dense FFT oracle."""
import numpy as np
import pytest

from oracle import amen as AM
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


def _rand_mpo(d, n, g, seed):
    rng = np.random.default_rng(seed)
    ranks = [1] + [g] * (d - 1) + [1]
    return [rng.standard_normal((ranks[k], n, n, ranks[k + 1])) + 1j * rng.standard_normal((ranks[k], n, n, ranks[k + 1]))
            for k in range(d)]


def _rel(cores, ref):
    return np.linalg.norm(T.tt_full(cores) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("which", ["identity", "diagonal", "random"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_amen_exact_products(Q, ctx, which, dtype):
    d = 9
    x = I.random_tt_cores(d, 2, 4, seed=1, dtype=np.complex128)
    if which == "identity":
        A = T.identity_mpo([2] * d)
    elif which == "diagonal":
        A = T.diag_mpo_from_tt(I.random_tt_cores(d, 2, 3, seed=2, dtype=np.complex128))
    else:
        A = _rand_mpo(d, 2, 3, seed=3)
    exact = T.tt_full(T.tt_mpo_apply(A, x))
    dt = Q.C128 if dtype == "c128" else Q.C64
    eps = 1e-12 if dtype == "c128" else 1e-5
    y, info = Q.tt_amen_mv(ctx, Q.MPO.from_cores(ctx, A, dt), Q.TT.from_cores(ctx, x, dt), eps)
    yc = [c.astype(np.complex128) for c in y.cores()]
    assert _rel(yc, exact) < (1e-11 if dtype == "c128" else 2e-5)
    ref, _ = AM.amen_mv(A, x, 1e-12)
    if dtype == "c128":
        assert y.ranks == T.tt_ranks(ref)


@pytest.mark.parametrize("eps", [1e-3, 1e-2])
def test_amen_rounding_bound_on_decaying_spectrum(Q, ctx, eps):
    d = 10
    low = I.random_tt_cores(d, 2, 5, seed=4, dtype=np.complex128)
    noise = I.random_tt_cores(d, 2, 5, seed=5, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-3)
    A = T.diag_mpo_from_tt(I.random_tt_cores(d, 2, 3, seed=6, dtype=np.complex128))
    exact = T.tt_mpo_apply(A, x)
    y, info = Q.tt_amen_mv(ctx, Q.MPO.from_cores(ctx, A), Q.TT.from_cores(ctx, x), eps)
    assert _rel(y.cores(), T.tt_full(exact)) <= eps
    assert max(y.ranks) <= max(T.tt_ranks(T.tt_round(exact, eps)[0]))


def _green_step_inputs():
    pb = MS.scalar_problem(I.box_indicator_2d(16, 0.25), 1.0, 10.0)
    ops = MS.build_operators(pb)
    tau = T.tt_round(T.tt_mpo_apply(ops.dC, MS.e_tt(np.array([1.0, 0.0, 0.0]), 8)), 1e-12)[0]
    for q in ops.qft:
        if q is not None:
            tau = T.tt_round(T.tt_mpo_apply(q, tau), 1e-12)[0]
    return ops.gamma, tau


def test_amen_green_step_and_warm_start(Q, ctx):
    G, tau = _green_step_inputs()
    exact = T.tt_mpo_apply(G, tau)
    Gd, td = Q.MPO.from_cores(ctx, G), Q.TT.from_cores(ctx, tau)
    y, info = Q.tt_amen_mv(ctx, Gd, td, 1e-10)
    assert _rel(y.cores(), T.tt_full(exact)) < 1e-10
    # started from the answer, one sweep finds nothing to change
    y2, info2 = Q.tt_amen_mv(ctx, Gd, td, 1e-10, y0=y)
    assert info2.sweeps <= 2
    assert _rel(y2.cores(), T.tt_full(exact)) < 1e-10


def test_ms_green_step_by_amen_matches_dense_oracle(Q, ctx):
    """16 x 16 plane box: the solve with eps^ = Gamma0 tau^ by AMEn reaches
    the dense FFT oracle's effective tensor."""
    pb = MS.scalar_problem(I.box_indicator_2d(16, 0.25), 1.0, 10.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-11, max_iter=500)
    C, rep = Q.ms_homogenize(ctx, pb.indicator, "scalar", (1.0, 10.0), pb.C0, tol=1e-11, max_rank=64,
                             eps=1e-11, max_iter=300, oversample=16, prec=Q.PREC_F64, green_amen=True,
                             load_mask=1)
    assert np.linalg.norm(C[:, 0] - Cd.real[:, 0]) / np.linalg.norm(Cd.real[:, 0]) < 1e-7

"""Pins for the oracle's Moulinec-Suquet solvers (Algorithms 1 and 2, Appendix A).

Closed forms: laminates (Reuss/Voigt for conduction, Backus-type averages for
elasticity); Green-operator identities (Gamma C0 Gamma = Gamma, and Gamma C0
reproduces compatible fields); Voigt/Reuss and Hashin-Shtrikman bounds and
cubic symmetry for a centred sphere; invariance of the QTT result under the
site ordering; agreement of the QTT solver with the dense FFT solver.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import ms as MS
from oracle import tt as T
from paper_2512_07811_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

E_MAT, E_INC, NU = 1.0, 10.0, 0.3
LAM1, MU1 = I.lame_from_young(E_MAT, NU)
LAM2, MU2 = I.lame_from_young(E_INC, NU)


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_lame_constants_of_the_sphere_phases():
    assert math.isclose(LAM1, 0.576923076923, rel_tol=1e-11)
    assert math.isclose(MU1, 0.384615384615, rel_tol=1e-11)
    assert math.isclose(LAM2, 5.76923076923, rel_tol=1e-11)
    assert math.isclose(MU2, 3.84615384615, rel_tol=1e-11)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_scalar_laminate_dense(N):
    g = load_golden("scalar_laminate_keff.json")
    pb = MS.scalar_problem(I.laminate_indicator(N), g["k1"], g["k2"])
    C, its = MS.effective_tensor_dense(pb, tol=1e-13)
    np.testing.assert_allclose(C.real, np.array(g["keff"]), atol=1e-12)
    assert np.abs(C.imag).max() < 1e-12
    # the fixed point is reached after one iteration (second only confirms)
    assert max(its) <= 2


def test_elastic_laminate_dense_backus():
    N = 8
    pb = MS.elastic_problem(I.laminate_indicator(N), LAM1, MU1, LAM2, MU2)
    C, _ = MS.effective_tensor_dense(pb, tol=1e-14, max_iter=500)
    Cx = MS.elastic_laminate_ceff([LAM2, LAM1], [MU2, MU1], [0.5, 0.5])
    np.testing.assert_allclose(C.real, Cx, atol=1e-10 * np.abs(Cx).max())


def _rand_dirs(rng, count=20):
    out = []
    for _ in range(count):
        xi = rng.integers(-7, 8, size=3).astype(float)
        if not xi.any():
            xi[0] = 1.0
        out.append(xi)
    return out


def _green_at(pb, xi):
    """Evaluate the dense Green operator at one wave vector by placing xi on a grid."""
    N = 16
    f = MS.frequencies(N)
    idx = [int(np.where(f == v)[0][0]) for v in xi]
    G = MS.green_dense(MS.Problem(pb.kind, np.zeros((N, N, N)), pb.C1, pb.C2, pb.C0,
                                  pb.k0, pb.lam0, pb.mu0))
    return G[:, :, idx[0], idx[1], idx[2]]


def test_green_is_c0_projector_elastic():
    pb = MS.elastic_problem(np.zeros((2, 2, 2)), LAM1, MU1, LAM2, MU2)
    rng = np.random.default_rng(0)
    for xi in _rand_dirs(rng, 6):
        G = _green_at(pb, xi)
        np.testing.assert_allclose(G @ pb.C0 @ G, G, atol=1e-12)
        # a compatible strain sym(xi (x) u), written with engineering shears
        u = rng.standard_normal(3)
        e = 0.5 * (np.outer(xi, u) + np.outer(u, xi))
        ev = np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])
        np.testing.assert_allclose(G @ pb.C0 @ ev, ev, atol=1e-11)


def test_green_is_k0_projector_scalar():
    pb = MS.scalar_problem(np.zeros((2, 2, 2)), 1.0, 10.0)
    rng = np.random.default_rng(1)
    for xi in _rand_dirs(rng, 6):
        G = _green_at(pb, xi)
        np.testing.assert_allclose(G @ pb.C0 @ G, G, atol=1e-13)
        np.testing.assert_allclose(G @ pb.C0 @ xi, xi, atol=1e-12)


@pytest.fixture(scope="module")
def sphere16():
    pb = MS.elastic_problem(I.sphere_indicator(16, 0.2), LAM1, MU1, LAM2, MU2)
    C, its = MS.effective_tensor_dense(pb, tol=1e-10, max_iter=500)
    return pb, C


def test_sphere_bounds_and_symmetry(sphere16):
    pb, C = sphere16
    C = C.real
    f2 = float(pb.indicator.mean())
    np.testing.assert_allclose(C, C.T, atol=1e-8)
    V, R = MS.voigt_reuss(pb.C1, pb.C2, f2)
    assert np.linalg.eigvalsh(V - C).min() > -1e-9
    assert np.linalg.eigvalsh(C - R).min() > -1e-9
    # cubic symmetry of a centred sphere on a symmetric voxel grid
    for a, b in [((0, 0), (1, 1)), ((0, 0), (2, 2)), ((0, 1), (0, 2)), ((0, 1), (1, 2)),
                 ((3, 3), (4, 4)), ((3, 3), (5, 5))]:
        assert math.isclose(C[a], C[b], rel_tol=1e-7)
    K = (C[0, 0] + 2 * C[0, 1]) / 3.0
    K1, K2 = LAM1 + 2 * MU1 / 3, LAM2 + 2 * MU2 / 3
    lo, hi = MS.hs_bulk_bounds(K1, MU1, K2, MU2, f2)
    assert lo <= K <= hi


def test_qtt_laminate_32cubed_15_sites():
    """32^3 scalar laminate, 15 interleaved bit sites + one control site."""
    g = load_golden("scalar_laminate_keff.json")
    pb = MS.scalar_problem(I.laminate_indicator(32), g["k1"], g["k2"])
    ops = MS.build_operators(pb, "interleaved")
    assert len(ops.chi) == 15 and max(T.tt_ranks(ops.chi)) == 1
    C = np.zeros((3, 3), dtype=complex)
    for k in range(3):
        E = np.zeros(3)
        E[k] = 1.0
        r = MS.ms_qtt(pb, E, ops, eps=1e-8, max_rank=64, tol=1e-12, max_iter=4)
        C[:, k] = r.sigma
        assert r.residuals[-1] < 1e-12
    np.testing.assert_allclose(C.real, np.array(g["keff"]), atol=1e-10)


def test_momentum_convention_of_green_train():
    """Contracted momentum train at site bits m equals G at k = sum_a m_a 2^(a-1) per dim."""
    pb = MS.scalar_problem(np.zeros((8, 8, 8)), 1.0, 10.0)
    n = 3
    G = MS.green_dense(pb).reshape(9, 8, 8, 8)
    for ordering in ["interleaved", "grouped"]:
        S = MS.spatial_to_sites(G, n, ordering, momentum=True, lead=1)
        rng = np.random.default_rng(2)
        perm = MS.site_permutation(n, ordering)
        for _ in range(20):
            bits = rng.integers(0, 2, size=3 * n)
            k = [0, 0, 0]
            for s, ax in enumerate(perm):
                dim, pos = divmod(ax, n)          # pos: MSB-first position
                # site holds bit of weight 2^(position counted LSB first)
                lsb_pos = pos                     # after reversal the a-th site is weight 2^a
                k[dim] += int(bits[s]) << lsb_pos
            c = int(rng.integers(0, 9))
            assert S[(c,) + tuple(bits)] == G[c, k[0], k[1], k[2]]


def _qtt_effective(pb, ordering, eps, max_iter=60, tol=1e-9):
    ops = MS.build_operators(pb, ordering)
    n = pb.ncomp
    C = np.zeros((n, n), dtype=complex)
    for k in range(n):
        E = np.zeros(n)
        E[k] = 1.0
        r = MS.ms_qtt(pb, E, ops, eps=eps, tol=tol, max_iter=max_iter)
        C[:, k] = r.sigma
    return C


@pytest.mark.slow
def test_qtt_matches_dense_small_sphere_and_ordering_invariance():
    pb = MS.elastic_problem(I.sphere_indicator(4, 0.2), LAM1, MU1, LAM2, MU2)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-9, max_iter=500)
    Ci = _qtt_effective(pb, "interleaved", 1e-10)
    Cg = _qtt_effective(pb, "grouped", 1e-10)
    rel = lambda A, B: np.linalg.norm(A - B) / np.linalg.norm(B)
    assert rel(Ci, Cd) < 1e-7
    assert rel(Cg, Ci) < 1e-7


def test_qtt_scalar_sphere_matches_dense():
    pb = MS.scalar_problem(I.sphere_indicator(8, 0.2), 1.0, 10.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-10, max_iter=500)
    Cq = _qtt_effective(pb, "interleaved", 1e-10, max_iter=80, tol=1e-10)
    assert np.linalg.norm(Cq - Cd) / np.linalg.norm(Cd) < 1e-7


# ------------------------------------------------------------ plane (2D) and anisotropic grids

def test_plane_scalar_laminate_closed_form():
    """32 x 32 x 1 laminate (15 bits in the plane, none along z): the QTT
    solve gives the plane laminate's harmonic mean 20/11 across the layers
    and the arithmetic mean 11/2 along them and along z, and agrees with the
    dense solve."""
    pb = MS.scalar_problem(I.laminate_indicator_2d(32), 1.0, 10.0)
    ops = MS.build_operators(pb, "interleaved")
    assert ops.n == (5, 5, 0) and len(ops.chi) == 10 and ops.qft[2] is None
    expect = np.diag([20.0 / 11.0, 5.5, 5.5])
    for k in range(3):
        E = np.zeros(3)
        E[k] = 1.0
        r = MS.ms_qtt(pb, E, ops, eps=1e-8, max_rank=64, tol=1e-12, max_iter=4)
        np.testing.assert_allclose(r.sigma.real, expect[:, k], atol=1e-10)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-12)
    np.testing.assert_allclose(Cd.real, expect, atol=1e-10)


def test_plane_elastic_laminate_backus():
    """16 x 16 x 1 elastic laminate in plane strain (every field uniform along
    z): the dense solve reproduces the Backus averages."""
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    pb = MS.elastic_problem(I.laminate_indicator_2d(16), lam1, mu1, lam2, mu2)
    C, _ = MS.effective_tensor_dense(pb, tol=1e-12, max_iter=400)
    ref = MS.elastic_laminate_ceff(np.array([lam1, lam2]), np.array([mu1, mu2]), np.array([0.5, 0.5]))
    np.testing.assert_allclose(C.real, ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("ordering", ["interleaved", "grouped"])
def test_plane_box_qtt_matches_dense(ordering):
    pb = MS.scalar_problem(I.box_indicator_2d(8, 0.25), 1.0, 10.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-12)
    ops = MS.build_operators(pb, ordering)
    for k in range(2):
        E = np.zeros(3)
        E[k] = 1.0
        r = MS.ms_qtt(pb, E, ops, eps=1e-12, tol=1e-12, max_iter=200)
        np.testing.assert_allclose(r.sigma, Cd[:, k], atol=1e-8)


def test_anisotropic_grid_qtt_matches_dense():
    """8 x 4 x 2 grid (3 + 2 + 1 bits, interleaved level by level)."""
    rng = np.random.default_rng(8)
    ind = (rng.random((8, 4, 2)) < 0.3).astype(np.float64)
    pb = MS.scalar_problem(ind, 1.0, 5.0)
    Cd, _ = MS.effective_tensor_dense(pb, tol=1e-12)
    for ordering in ("interleaved", "grouped"):
        ops = MS.build_operators(pb, ordering)
        assert ops.n == (3, 2, 1)
        E = np.array([0.3, -1.0, 0.5])
        r = MS.ms_qtt(pb, E, ops, eps=1e-12, tol=1e-12, max_iter=300)
        np.testing.assert_allclose(r.sigma, Cd @ E, atol=1e-8)


def test_multibox_plane_geometry():
    img = I.multibox_indicator_2d(64, count=8, area_fraction=0.2, seed=3)
    assert img.shape == (64, 64, 1)
    assert 0.1 < img.mean() < 0.3


def test_contract_local_strain_laminate_closed_form():
    """Algorithm 2's contract() on the 8^3 laminate, E = e_x: the local
    gradient is 20/11 in phase 1 and 2/11 in phase 2 (constant flux 20/11),
    zero across the layers."""
    ind = I.laminate_indicator(8)
    pb = MS.scalar_problem(ind, 1.0, 10.0)
    res = MS.ms_qtt(pb, np.array([1.0, 0.0, 0.0]), eps=1e-12, tol=1e-13, max_iter=10)
    loc = MS.contract(res.eps_field, (3, 3, 3))
    want = np.where(ind == 1.0, 2.0 / 11.0, 20.0 / 11.0)
    np.testing.assert_allclose(loc[0].real, want, atol=1e-10)
    np.testing.assert_allclose(np.abs(loc[1:]), 0.0, atol=1e-10)


@pytest.mark.parametrize("ordering", ["interleaved", "grouped"])
def test_contract_equals_dense_local_field(ordering):
    """8 x 8 x 2 random two-phase grid: the QTT local strain equals the dense
    FFT solver's local field (Algorithm 1)."""
    rng = np.random.default_rng(12)
    ind = (rng.random((8, 8, 2)) < 0.3).astype(np.float64)
    pb = MS.scalar_problem(ind, 1.0, 5.0)
    E = np.array([1.0, 0.0, 0.0])
    dense = MS.ms_dense(pb, E, tol=1e-12, max_iter=500, keep_field=True)
    res = MS.ms_qtt(pb, E, ops=MS.build_operators(pb, ordering), eps=1e-12, tol=1e-12, max_iter=500,
                    ordering=ordering)
    loc = MS.contract(res.eps_field, (3, 3, 1), ordering)
    np.testing.assert_allclose(loc, dense.eps_field, atol=1e-8)

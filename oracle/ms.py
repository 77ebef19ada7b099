"""Moulinec-Suquet homogenisation: dense FFT (Algorithm 1) and QTT (Algorithm 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Problems
--------
* scalar conductivity: the field is the gradient e (3 components), flux k e;
  Green operator G(xi) = xi xi^T / (k0 |xi|^2), G(0) = 0.
* isotropic linear elasticity in Voigt notation, order (11, 22, 33, 23, 13, 12),
  engineering shear strains (factor 2, Appendix A); Green operator of
  Moulinec & Suquet (1998) mapped to Voigt with the factors below.

Readings (the paper is silent or garbled on these):
* frequencies xi_k = k for k < N/2, else k - N (the numpy.fft.fftfreq
  convention, Nyquist = -N/2); only directions matter since G is homogeneous
  of degree 0;
* reference medium C0 = arithmetic mean of the two phases' moduli;
* stop test ||eps_{m+1} - eps_m||_F / ||E 1||_F < tol with ||E 1||_F =
  ||E|| sqrt(#voxels);
* the fields stay complex; C_eff = Re(sigma_eff), |Im| is a diagnostic;
* QTT site order: one control site first (3 or 6 components), then the
  spatial bits either interleaved (x1 y1 z1 x2 y2 z2 ...) or grouped by
  dimension (x1..xn y1..yn z1..zn), every bit MSB first in position space;
* in momentum space every dimension's bits are reversed (Sec. 3.2, the SFFT
  convention); conjugation is a no-op for the real, even Green operator;
* the 3D SFFT is applied one dimension at a time (x, then y, then z), each
  operator application followed by a rounding; the inverse uses the adjoint
  trains in the reverse order (z, y, x);
* grids may have a different power of two per dimension, including 2^0 = 1:
  a grid one voxel thick along z is the two-dimensional problem (for
  conductivity exactly; for elasticity in plane strain), every field
  uniform along z, xi_z = 0, and that dimension holds no QTT sites.
  Interleaved order with unequal bit counts: level by level (the a-th bit of
  x, then of y, then of z, skipping a dimension whose bits are used up).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import tt as T
from . import qft as QF

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
VOIGT_W = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


# --------------------------------------------------------- materials --

def iso_voigt(lam: float, mu: float) -> np.ndarray:
    """Isotropic stiffness in Voigt form acting on engineering strains."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2 * mu
    for i in range(3, 6):
        C[i, i] = mu
    return C


@dataclass
class Problem:
    kind: str                    # "scalar" or "elastic"
    indicator: np.ndarray        # (Nx, Ny, Nz) 0/1, 1 = phase 2 (powers of two, Nz = 1 allowed)
    C1: np.ndarray               # phase-1 tensor (3x3 or 6x6)
    C2: np.ndarray               # phase-2 tensor
    C0: np.ndarray               # reference tensor
    k0: float = 0.0              # scalar reference conductivity
    lam0: float = 0.0            # elastic reference Lame constants
    mu0: float = 0.0

    @property
    def N(self) -> int:
        return self.indicator.shape[0]

    @property
    def ncomp(self) -> int:
        return self.C1.shape[0]


def scalar_problem(indicator, k1: float, k2: float) -> Problem:
    k0 = 0.5 * (k1 + k2)
    return Problem("scalar", indicator, k1 * np.eye(3), k2 * np.eye(3), k0 * np.eye(3), k0=k0)


def elastic_problem(indicator, lam1, mu1, lam2, mu2) -> Problem:
    lam0 = 0.5 * (lam1 + lam2)
    mu0 = 0.5 * (mu1 + mu2)
    return Problem("elastic", indicator, iso_voigt(lam1, mu1), iso_voigt(lam2, mu2),
                   iso_voigt(lam0, mu0), lam0=lam0, mu0=mu0)


# ---------------------------------------------------- Green operators --

def frequencies(N: int) -> np.ndarray:
    """xi_k = k below the Nyquist index, else k - N (numpy.fft.fftfreq times N;
    the single frequency of a one-voxel dimension is 0)."""
    k = np.arange(N)
    return np.where(k < (N + 1) // 2, k, k - N).astype(np.float64)


def grid_shape(pb: Problem):
    return tuple(pb.indicator.shape)


def grid_bits(shape) -> tuple:
    nb = tuple(int(round(math.log2(N))) for N in shape)
    assert all(1 << b == N for b, N in zip(nb, shape)), shape
    return nb


def green_components(pb: Problem, xi) -> np.ndarray:
    """Green operator G[I, J, ...] at the frequency vectors xi = (xi_x, xi_y,
    xi_z) (float arrays of one shape), G = 0 where xi = 0."""
    xi = [np.asarray(x, dtype=np.float64) for x in xi]
    q2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    zero = q2 == 0
    q2s = np.where(zero, 1.0, q2)
    shape = q2.shape
    if pb.kind == "scalar":
        G = np.zeros((3, 3) + shape)
        for i in range(3):
            for j in range(3):
                G[i, j] = xi[i] * xi[j] / (pb.k0 * q2s)
        G[:, :, zero] = 0.0
        return G
    lam0, mu0 = pb.lam0, pb.mu0
    coef = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0))
    d = np.eye(3)
    G = np.zeros((6, 6) + shape)
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, h) in enumerate(VOIGT):
            g = (d[k, i] * xi[h] * xi[j] + d[h, i] * xi[k] * xi[j]
                 + d[k, j] * xi[h] * xi[i] + d[h, j] * xi[k] * xi[i]) / (4 * mu0 * q2s)
            g = g - coef * xi[i] * xi[j] * xi[k] * xi[h] / (q2s * q2s)
            # eps_V[I] = w_I eps_ij ; sum_kh G_ijkh tau_kh = sum_J w_J G_ij(kh) tau_V[J]
            G[I, J] = VOIGT_W[I] * VOIGT_W[J] * g
    G[:, :, zero] = 0.0
    return G


def green_dense(pb: Problem) -> np.ndarray:
    """Dense Green operator G[I, J, kx, ky, kz] in the natural frequency order."""
    Nx, Ny, Nz = grid_shape(pb)
    ones = np.ones((Nx, Ny, Nz))
    xi = [frequencies(Nx)[:, None, None] * ones,
          frequencies(Ny)[None, :, None] * ones,
          frequencies(Nz)[None, None, :] * ones]
    return green_components(pb, xi)


# --------------------------------------------- Algorithm 1 (dense FFT) --

@dataclass
class MSResult:
    sigma: np.ndarray             # complex macroscopic stress / flux (ncomp,)
    iterations: int
    residuals: list = field(default_factory=list)
    rank_trace: list = field(default_factory=list)
    eps_field: object = None


def _apply_dC(pb: Problem, eps: np.ndarray) -> np.ndarray:
    """tau = (C(x) - C0) eps with C(x) = C1 (1 - chi) + C2 chi."""
    A = pb.C1 - pb.C0
    B = pb.C2 - pb.C1
    return (np.einsum("IJ,Jxyz->Ixyz", A, eps)
            + pb.indicator[None] * np.einsum("IJ,Jxyz->Ixyz", B, eps))


def mean_stress(pb: Problem, eps: np.ndarray) -> np.ndarray:
    """sigma_eff = < C(x) eps(x) > (Appendix A)."""
    s = (np.einsum("IJ,Jxyz->Ixyz", pb.C1, eps)
         + pb.indicator[None] * np.einsum("IJ,Jxyz->Ixyz", pb.C2 - pb.C1, eps))
    return s.mean(axis=(1, 2, 3))


def ms_dense(pb: Problem, E: np.ndarray, tol: float = 1e-10, max_iter: int = 1000,
             G: np.ndarray | None = None, keep_field: bool = False) -> MSResult:
    """Algorithm 1: tau = (C - C0) eps; tau^ = F[tau]; eps^ = G tau^;
    eps_{m+1} = E - F^{-1}[eps^]; stop when the relative change is < tol."""
    shape = grid_shape(pb)
    if G is None:
        G = green_dense(pb)
    E = np.asarray(E, dtype=np.complex128)
    eps = np.broadcast_to(E[:, None, None, None], (pb.ncomp,) + shape).astype(np.complex128)
    normE = float(np.linalg.norm(E)) * math.sqrt(float(np.prod(shape)))
    res = []
    it = 0
    for it in range(1, max_iter + 1):
        tau = _apply_dC(pb, eps)
        tau_h = np.fft.fftn(tau, axes=(1, 2, 3), norm="ortho")
        eps_h = np.einsum("IJxyz,Jxyz->Ixyz", G, tau_h)
        eps_new = E[:, None, None, None] - np.fft.ifftn(eps_h, axes=(1, 2, 3), norm="ortho")
        r = float(np.linalg.norm(eps_new - eps)) / normE
        res.append(r)
        eps = eps_new
        if r < tol:
            break
    return MSResult(mean_stress(pb, eps), it, res, [], eps if keep_field else None)


def effective_tensor_dense(pb: Problem, tol=1e-10, max_iter=1000):
    """C_eff column by column: load case E = e_k gives column k (Appendix A)."""
    G = green_dense(pb)
    n = pb.ncomp
    C = np.zeros((n, n), dtype=np.complex128)
    iters = []
    for k in range(n):
        E = np.zeros(n)
        E[k] = 1.0
        r = ms_dense(pb, E, tol, max_iter, G)
        C[:, k] = r.sigma
        iters.append(r.iterations)
    return C, iters


# ---------------------------------------------- QTT representations --

def _bits3(n) -> tuple:
    """Bits per dimension: an int means a cube."""
    return (n, n, n) if isinstance(n, (int, np.integer)) else tuple(n)


def site_permutation(n, ordering: str) -> list:
    """Axis permutation from (x bits, y bits, z bits) to the chosen site order;
    n: bits per dimension (an int for a cube)."""
    nb = _bits3(n)
    start = [0, nb[0], nb[0] + nb[1]]
    if ordering == "grouped":
        return list(range(sum(nb)))
    if ordering == "interleaved":
        perm = []
        for a in range(max(nb)):
            for dim in range(3):
                if a < nb[dim]:
                    perm.append(start[dim] + a)
        return perm
    raise ValueError(ordering)


def dim_positions(n, ordering: str, dim: int) -> list:
    """Spatial site numbers (0-based, control site excluded) holding the bits of `dim`."""
    nb = _bits3(n)
    lo = sum(nb[:dim])
    perm = site_permutation(nb, ordering)
    return [s for s, ax in enumerate(perm) if lo <= ax < lo + nb[dim]]


def spatial_to_sites(field: np.ndarray, n, ordering: str, momentum: bool = False,
                     lead: int = 0) -> np.ndarray:
    """Reshape a field (..., Nx, Ny, Nz) with `lead` leading axes into one axis
    per bit in site order.  Position space: MSB first; momentum space: the
    bits of every dimension reversed (LSB first)."""
    nb = _bits3(n)
    d = sum(nb)
    lead_shape = field.shape[:lead]
    a = field.reshape(lead_shape + (2,) * d)
    axes = list(range(d))
    if momentum:
        start = [0, nb[0], nb[0] + nb[1]]
        axes = [start[dim] + (nb[dim] - 1 - b) for dim in range(3) for b in range(nb[dim])]
    a = a.transpose(list(range(lead)) + [lead + ax for ax in axes])
    perm = site_permutation(nb, ordering)
    return a.transpose(list(range(lead)) + [lead + p for p in perm])


def sites_to_spatial(arr: np.ndarray, n, ordering: str, lead: int = 0) -> np.ndarray:
    """Inverse of spatial_to_sites (position space)."""
    nb = _bits3(n)
    perm = site_permutation(nb, ordering)
    inv = np.argsort(perm)
    a = arr.transpose(list(range(lead)) + [lead + i for i in inv])
    return a.reshape(arr.shape[:lead] + tuple(1 << b for b in nb))


@dataclass
class QTTOperators:
    n: tuple                      # bits per dimension
    ordering: str
    ncomp: int
    chi: list                     # phase indicator TT (spatial sites only)
    dC: list                      # operator train of C(x) - C0 (control + spatial)
    gamma: list                   # Green operator train in momentum convention
    qft: list                     # per-dimension forward SFFT trains [x, y, z] (None: no bits)
    qft_inv: list                 # adjoints
    ones: list                    # all-ones spatial TT


def build_operators(pb: Problem, ordering: str = "interleaved", op_tol: float = 1e-10,
                    qft_tol: float = 1e-12, op_cross: bool = False, boxes=None,
                    ellipsoids=None) -> QTTOperators:
    """The operator trains of Algorithm 2.  By default the phase indicator
    and the Green operator are compressed from their dense arrays (TT-SVD);
    op_cross samples the Green operator by TT-cross instead (Sec. 3), and a
    box list (rows cx, cy, cz, hx, hy, hz) or an ellipsoid list (rows as in
    inputs.ellipsoids_value) samples the phase indicator by TT-cross; every
    cross is rounded at op_tol."""
    from . import cross as X
    shape = grid_shape(pb)
    n = grid_bits(shape)
    nc = pb.ncomp
    d_sp = sum(n)
    if boxes is not None:
        chi, _ = X.tt_cross(X.boxes_fn(boxes, n, ordering), [2] * d_sp, op_tol, kick=8, init_rank=8,
                            max_half_sweeps=24, init_points=X.box_centre_points(boxes, n, ordering))
        chi = T.tt_round(chi, op_tol)[0]
    elif ellipsoids is not None:
        chi, _ = X.tt_cross(X.ellipsoids_fn(ellipsoids, n, ordering), [2] * d_sp, op_tol, kick=8, init_rank=8,
                            max_half_sweeps=24, init_points=X.ellipsoid_centre_points(ellipsoids, n, ordering))
        chi = T.tt_round(chi, op_tol)[0]
    else:
        chi = T.tt_svd(spatial_to_sites(pb.indicator.astype(np.complex128), n, ordering), op_tol)
    ones = T.ones_tt([2] * d_sp)
    ctrl_a = (pb.C1 - pb.C0).astype(np.complex128).reshape(1, nc, nc, 1)
    ctrl_b = (pb.C2 - pb.C1).astype(np.complex128).reshape(1, nc, nc, 1)
    part_a = [ctrl_a] + T.identity_mpo([2] * d_sp)
    part_b = [ctrl_b] + T.diag_mpo_from_tt(chi)
    dC = T.mpo_add(part_a, part_b)
    # Green operator in the momentum convention: TT-SVD of G[(I J), bits...]
    # or TT-cross of its entries
    if op_cross:
        g_tt, _ = X.tt_cross(X.green_fn(pb, n, ordering), [nc * nc] + [2] * d_sp, op_tol, kick=4,
                             max_half_sweeps=24)
        g_tt = T.tt_round(g_tt, op_tol)[0]
    else:
        G = green_dense(pb).reshape((nc * nc,) + shape).astype(np.complex128)
        Gs = spatial_to_sites(G, n, ordering, momentum=True, lead=1)
        g_tt = T.tt_svd(Gs, op_tol)
    c0 = g_tt[0]
    gamma = [c0.reshape(1, nc, nc, c0.shape[2])] + T.diag_mpo_from_tt(g_tt[1:])
    # SFFT, one dimension at a time, embedded with identities elsewhere
    dims = [nc] + [2] * d_sp
    qft, qinv = [], []
    for dim in range(3):
        if n[dim] == 0:
            qft.append(None)
            qinv.append(None)
            continue
        q1 = QF.qft_mpo(n[dim], -1.0, qft_tol)
        pos = [1 + s for s in dim_positions(n, ordering, dim)]
        full = QF.embed_1d_mpo(q1, pos, 1 + d_sp, dims)
        qft.append(full)
        qinv.append(T.mpo_adjoint(full))
    return QTTOperators(n, ordering, nc, chi, dC, gamma, qft, qinv, ones)


def e_tt(E, d_sp: int):
    ctrl = np.asarray(E, dtype=np.complex128).reshape(1, -1, 1)
    return [ctrl] + T.ones_tt([2] * d_sp)


def qtt_mean_stress(pb: Problem, ops: QTTOperators, eps_tt) -> np.ndarray:
    """sigma = C1 <eps> + (C2 - C1) <chi eps>, the means by inner products with
    e_I (x) ones and e_I (x) chi (Appendix A)."""
    nc = ops.ncomp
    Nvox = float(2 ** sum(ops.n))
    m1 = np.zeros(nc, dtype=np.complex128)
    m2 = np.zeros(nc, dtype=np.complex128)
    for I in range(nc):
        e = np.zeros((1, nc, 1), dtype=np.complex128)
        e[0, I, 0] = 1.0
        m1[I] = T.tt_dot([e] + ops.ones, eps_tt) / Nvox
        m2[I] = T.tt_dot([e] + ops.chi, eps_tt) / Nvox
    return pb.C1 @ m1 + (pb.C2 - pb.C1) @ m2


def ms_qtt(pb: Problem, E, ops: QTTOperators | None = None, eps: float = 1e-8,
           max_rank: int | None = None, tol: float = 1e-10, max_iter: int = 50,
           ordering: str = "interleaved", min_iter: int = 1, r0: int = 1, green_amen: bool = False) -> MSResult:
    """Algorithm 2 with operator application + SVD rounding after every step:
      tau = round(dC eps);  tau^ = S tau (three applications, each rounded);
      eps^ = round(Gamma tau^) (or AMEn(Gamma, tau^), warm-started from the
      previous iteration's eps^, with green_amen);  eps_{m+1} = round(E - S^{-1} eps^);
      stop when ||eps_{m+1} - eps_m|| / ||E 1|| < tol (after min_iter)."""
    if ops is None:
        ops = build_operators(pb, ordering)
    d_sp = sum(ops.n)
    Et = e_tt(E, d_sp)
    normE = T.tt_norm(Et)
    x = [c.copy() for c in Et]
    res, trace = [], []

    def rnd(y, tag):
        z, info = T.tt_round(y, eps, max_rank, r0)
        trace.append((tag, info["ranks"]))
        return z

    it = 0
    ghat = None
    for it in range(1, max_iter + 1):
        tau = rnd(T.tt_mpo_apply(ops.dC, x), "dC")
        h = tau
        for dim in range(3):
            if ops.qft[dim] is not None:
                h = rnd(T.tt_mpo_apply(ops.qft[dim], h), "S%d" % dim)
        if green_amen:
            from . import amen as AM
            h, _ = AM.amen_mv(ops.gamma, h, eps, y0=ghat, seed=it)
            ghat = h
        else:
            h = rnd(T.tt_mpo_apply(ops.gamma, h), "G")
        for dim in (2, 1, 0):
            if ops.qft_inv[dim] is not None:
                h = rnd(T.tt_mpo_apply(ops.qft_inv[dim], h), "Si%d" % dim)
        x_new = rnd(T.tt_add(Et, h, 1.0, -1.0), "E")
        r = T.tt_norm(T.tt_add(x_new, x, 1.0, -1.0)) / normE
        res.append(r)
        x = x_new
        if r < tol and it >= min_iter:
            break
    return MSResult(qtt_mean_stress(pb, ops, x), it, res, trace, x)


def contract(x, n, ordering: str = "interleaved") -> np.ndarray:
    """The local field of a strain train (Algorithm 2's final contract()):
    the full tensor, control index first, in the position-space voxel order
    (ncomp, Nx, Ny, Nz)."""
    nb = _bits3(n)
    full = T.tt_full(x)
    nc = x[0].shape[1]
    return sites_to_spatial(full.reshape((nc,) + (2,) * sum(nb)), nb, ordering, lead=1)


# ------------------------------------------------------ closed forms --

def scalar_laminate_keff(k1, k2, f2, axis=0):
    """Layers normal to `axis`: harmonic mean across, arithmetic mean along."""
    f1 = 1.0 - f2
    K = np.eye(3) * (f1 * k1 + f2 * k2)
    K[axis, axis] = 1.0 / (f1 / k1 + f2 / k2)
    return K


def elastic_laminate_ceff(lam, mu, fr):
    """Layers normal to x: Backus-type averages <.> over the phases (fractions fr)."""
    lam = np.asarray(lam, float)
    mu = np.asarray(mu, float)
    fr = np.asarray(fr, float)
    M = lam + 2 * mu
    avg = lambda v: float(np.sum(fr * v))
    iM = 1.0 / avg(1.0 / M)
    lM = avg(lam / M)
    C = np.zeros((6, 6))
    C[0, 0] = iM
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = lM * iM
    C[1, 1] = C[2, 2] = avg(M - lam ** 2 / M) + lM ** 2 * iM
    C[1, 2] = C[2, 1] = avg(lam - lam ** 2 / M) + lM ** 2 * iM
    C[3, 3] = avg(mu)                       # yz
    C[4, 4] = C[5, 5] = 1.0 / avg(1.0 / mu)  # xz, xy
    return C


def voigt_reuss(C1, C2, f2):
    f1 = 1.0 - f2
    V = f1 * C1 + f2 * C2
    R = np.linalg.inv(f1 * np.linalg.inv(C1) + f2 * np.linalg.inv(C2))
    return V, R


def hs_bulk_bounds(K_a, mu_a, K_b, mu_b, f_b):
    """Hashin-Shtrikman bulk bounds for a two-phase isotropic composite:
    K_HS = K_a + f_b / (1/(K_b - K_a) + 3 f_a / (3 K_a + 4 mu_a)), with (a, b)
    = (softer, stiffer) for the lower and swapped for the upper bound."""
    f_a = 1.0 - f_b

    def hs(Ka, mua, Kb, fb):
        fa = 1.0 - fb
        return Ka + fb / (1.0 / (Kb - Ka) + 3.0 * fa / (3.0 * Ka + 4.0 * mua))
    lo = hs(K_a, mu_a, K_b, f_b)
    hi = hs(K_b, mu_b, K_a, f_a)
    return min(lo, hi), max(lo, hi)

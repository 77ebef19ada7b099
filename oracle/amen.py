"""AMEn approximation of an operator-train times train product, y ~ A x
(Sec. 2.1, the optimisation-based alternative to MPO x TT plus rounding, and
Sec. 3.2, where the Green operator is applied this way), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names the method (Dolgov & Savostyanov's alternating minimal
energy with residual enrichment) without details; this oracle takes its
matrix-vector form:

* y (the approximation) and z (a low-rank approximation of the residual
  A x - y) are trains; before every sweep both are right-orthogonalised;
* sweeping k = 0..d-1, core k of y is replaced by the projection of A x
  onto the interface of y's left (orthonormal) and right (orthonormal)
  parts, the optimal core for the others fixed:
      Y_k = Phi_k A_k X_k Psi_{k+1},
  with Phi_k = y_{<k}^H A_{<k} x_{<k} and Psi_{k+1} = y_{>k}^H A_{>k} x_{>k};
* the new core is truncated by SVD at eps ||Y_k|| / sqrt(d - 1); the residual
  A x - y projected onto z's interfaces gives z's core k (its leading left
  singular vectors, rank `kick`), and the residual projected onto y's left
  and z's right interface enriches the kept basis of y's core k before it is
  orthonormalised (the product y is unchanged: the enrichment directions get
  zero weight in the next core);
* sweeps repeat until no core changes by more than eps (relative), or
  `max_sweeps`; the result is rounded at eps (the enrichment adds rank).

Every contraction is written out with einsum over its named indices.
"""
from __future__ import annotations

import math

import numpy as np

from . import tt as T


def _right_orth(cores):
    """Right-orthogonalise a train (every core but the first has orthonormal rows)."""
    cores = [c.copy() for c in cores]
    for k in range(len(cores) - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0, n * r1).conj().T)   # M^H = Q R
        cores[k] = Q.conj().T.reshape(Q.shape[1], n, r1)              # M = R^H Q^H
        cores[k - 1] = np.einsum("anb,bc->anc", cores[k - 1], R.conj().T)
    return cores


def _phi_next(phi, Y, A, X):
    """Phi_{k+1}[a', g', b'] = sum conj(Y[a, i, a']) phi[a, g, b] A[g, i, j, g'] X[b, j, b']."""
    return np.einsum("agb,aic,gijh,bjd->chd", phi, Y.conj(), A, X)


def _psi_prev(psi, Y, A, X):
    """Psi_k[a, g, b] = sum conj(Y[a, i, a']) A[g, i, j, g'] X[b, j, b'] psi[a', g', b']."""
    return np.einsum("aic,gijh,bjd,chd->agb", Y.conj(), A, X, psi)


def _proj(phi, A, X, psi):
    """Local core phi_k A_k X_k psi_{k+1}: [a, i, a'] = sum phi[a, g, b] A[g, i, j, g'] X[b, j, b'] psi[a', g', b']."""
    return np.einsum("agb,gijh,bjd,chd->aic", phi, A, X, psi)


def _phi_zy_next(phi, Z, Y):
    """[c', a'] = sum conj(Z[c, i, c']) phi[c, a] Y[a, i, a']."""
    return np.einsum("ca,cid,aie->de", phi, Z.conj(), Y)


def _psi_zy_prev(psi, Z, Y):
    """[c, a] = sum conj(Z[c, i, c']) Y[a, i, a'] psi[c', a']."""
    return np.einsum("cid,aie,de->ca", Z.conj(), Y, psi)


def amen_mv(A, x, eps: float, y0=None, kick: int = 4, max_sweeps: int = 20, init_rank: int = 4, seed: int = 0):
    """y ~ A x for an operator train A (cores (g, m, n, g')) and a train x
    (cores (r, n, r')).  y0: initial guess (default: a Gaussian train of rank
    init_rank).  Returns (y cores, info) with info = dict(sweeps, dx, ranks)."""
    d = len(x)
    rng = np.random.default_rng(seed)
    m = [a.shape[1] for a in A]

    def gauss(r):
        ranks = [1] + [r] * (d - 1) + [1]
        return [rng.standard_normal((ranks[k], m[k], ranks[k + 1])) + 0j for k in range(d)]

    y = [np.asarray(c, dtype=np.complex128) for c in (y0 if y0 is not None else gauss(init_rank))]
    z = gauss(kick)
    A = [np.asarray(a, dtype=np.complex128) for a in A]
    x = [np.asarray(c, dtype=np.complex128) for c in x]
    dx = math.inf
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        y = _right_orth(y)
        z = _right_orth(z)
        one = np.ones((1, 1, 1), dtype=np.complex128)
        psi = [None] * (d + 1)
        psiz = [None] * (d + 1)
        psizy = [None] * (d + 1)
        psi[d] = one
        psiz[d] = one
        psizy[d] = np.ones((1, 1), dtype=np.complex128)
        for k in range(d - 1, 0, -1):
            psi[k] = _psi_prev(psi[k + 1], y[k], A[k], x[k])
            psiz[k] = _psi_prev(psiz[k + 1], z[k], A[k], x[k])
            psizy[k] = _psi_zy_prev(psizy[k + 1], z[k], y[k])
        phi, phiz, phizy = one, one, np.ones((1, 1), dtype=np.complex128)
        dx = 0.0
        for k in range(d):
            Yn = _proj(phi, A[k], x[k], psi[k + 1])
            nrm = np.linalg.norm(Yn)
            dx = max(dx, np.linalg.norm(Yn - y[k]) / nrm if nrm > 0 else 0.0)
            if k == d - 1:
                y[k] = Yn
                break
            r0, n, r1 = Yn.shape
            U, s, Vh = np.linalg.svd(Yn.reshape(r0 * n, r1), full_matrices=False)
            t, _ = T.truncation_rank(s, eps * nrm / math.sqrt(d - 1))
            Ycur = (U[:, :t] * s[:t]) @ Vh[:t]                       # truncated core, (r0 n) x r1
            # residual core of z: (A x - y) on z's interfaces
            Zk = _proj(phiz, A[k], x[k], psiz[k + 1]) - np.einsum("ca,aie,de->cid", phizy,
                                                                    Ycur.reshape(r0, n, r1), psizy[k + 1])
            rz0, _, rz1 = Zk.shape
            Uz, sz, _ = np.linalg.svd(Zk.reshape(rz0 * n, rz1), full_matrices=False)
            kz = min(kick, Uz.shape[1])
            z[k] = Uz[:, :kz].reshape(rz0, n, kz)
            z[k + 1] = z[k + 1][:kz]          # only its shape matters: core k+1 is recomputed next
            # enrichment: (A x - y) on y's left and z's right interface
            Ek = _proj(phi, A[k], x[k], psiz[k + 1]) - np.einsum("aie,de->aid", Ycur.reshape(r0, n, r1),
                                                                  psizy[k + 1])
            # orthonormal basis of [U_t, E_k]: its left singular vectors, the
            # discarded tail at most 100 u ||[U_t, E_k]|| (E_k may repeat
            # directions of U_t)
            Uaug = np.hstack([U[:, :t], Ek.reshape(r0 * n, -1)])
            Qs, sq, _ = np.linalg.svd(Uaug, full_matrices=False)
            keep, _ = T.truncation_rank(sq, 100 * np.finfo(np.float64).eps * np.linalg.norm(Uaug))
            Q = Qs[:, :keep]
            carry = Q.conj().T @ Ycur                                  # keep x r1
            y[k] = Q.reshape(r0, n, keep)
            y[k + 1] = np.einsum("ab,bjc->ajc", carry, y[k + 1])
            phi = _phi_next(phi, y[k], A[k], x[k])
            phiz = _phi_next(phiz, z[k], A[k], x[k])
            phizy = _phi_zy_next(phizy, z[k], y[k])
        if dx <= eps:
            break
    y, _ = T.tt_round(y, eps)
    return y, dict(sweeps=sweeps, dx=dx, ranks=T.tt_ranks(y))

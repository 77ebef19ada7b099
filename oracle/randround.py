"""Randomize-then-orthogonalize TT rounding (not in the
paper).  TEST INFRASTRUCTURE ONLY (see the package docstring).

Published method: Al Daas, Ballard, Cazeaux, Hallman, Miedlar, Pasha, Reid,
Saibaba, "Randomized algorithms for rounding in the tensor-train format",
SIAM J. Sci. Comput. 45 (2023), the randomize-then-orthogonalize variant:

1. draw a Gaussian sketch TT R with bond ranks l_k (l_0 = l_d = 1);
2. right-to-left partial contractions W_{d+1} = 1,
   W_k = sum_i X_k(i) W_{k+1} R_k(i)^T       (r_{k-1} x l_{k-1});
3. left-to-right: with the running core Y_1 = X_1, for k = 1..d-1
   Z_k = unfold_L(Y_k) W_{k+1} ((s_{k-1} n) x l_k), Q_k = qr(Z_k),
   M_k = Q_k^H unfold_L(Y_k) (l_k x r_k), Y_{k+1} = M_k X_{k+1};
   the result has cores Q_1..Q_{d-1}, Y_d.
The result is an orthogonal projection of x, so the a-posteriori error is
computed exactly on the difference train in FP64.  A deterministic SVD
rounding of the (already small) result then enforces the tolerance.

The random sketch cores are inputs (drawn by the caller from a seeded
generator), so the GPU path and this oracle can use the same sketch.
"""
from __future__ import annotations

import numpy as np

from . import tt as T


def sketch_ranks(d: int, n_dims, ell: int):
    """l_0 = l_d = 1; l_k = min(ell, prod n_1..n_k, prod n_{k+1}..n_d)."""
    ranks = [1]
    left = 1
    for k in range(1, d):
        left = min(left * n_dims[k - 1], 1 << 40)
        right = 1
        for m in n_dims[k:]:
            right = min(right * m, 1 << 40)
        ranks.append(int(min(ell, left, right)))
    ranks.append(1)
    return ranks


def right_partials(x, R):
    """W_k for k = 1..d (index k-1 in the list); W_{d+1} = [[1]]."""
    d = len(x)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1), dtype=np.result_type(x[0], R[0]))
    for k in range(d - 1, -1, -1):
        X = x[k]
        Rk = R[k]
        # W_k[a, l] = sum_{i, b, m} X[a, i, b] W_{k+1}[b, m] R[l, i, m]
        W[k] = np.einsum("aib,bm,lim->al", X, W[k + 1], Rk)
    return W


def rand_orth(x, R):
    """Randomize-then-orthogonalize projection of x with sketch R."""
    d = len(x)
    W = right_partials(x, R)
    out = []
    Y = x[0].copy()
    for k in range(d - 1):
        s0, n, r1 = Y.shape
        YL = Y.reshape(s0 * n, r1)
        Z = YL @ W[k + 1]
        Q, _ = np.linalg.qr(Z, mode="reduced")
        out.append(Q.reshape(s0, n, Q.shape[1]))
        M = np.conj(Q.T) @ YL
        Y = np.tensordot(M, x[k + 1], axes=(1, 0))
    out.append(Y)
    return out


def rand_round(x, R, eps: float, max_rank: int | None = None):
    """Sketch, then deterministic rounding of the sketched train; returns
    (cores, info) with info['err'] = ||x - result|| / ||x|| exact in FP64."""
    y = rand_orth(x, R)
    z, info = T.tt_round(y, eps, max_rank)
    nx = T.tt_norm(x)
    err = T.tt_norm(T.tt_add(x, z, 1.0, -1.0)) / nx if nx > 0 else 0.0
    info = dict(info)
    info["err"] = err
    return z, info

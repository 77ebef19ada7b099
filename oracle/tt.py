"""Tensor-train (TT) and tensor-train-operator (TTO / MPO) algebra in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Storage convention: a TT is a list of NumPy arrays, core k of shape
(r_{k-1}, n_k, r_k) with r_0 = r_d = 1, so that
    x(i_1..i_d) = A_1(i_1) A_2(i_2) ... A_d(i_d)          (Sec. 2, Eq. tt_format)
with A_k(i) = core[:, i, :].  The paper writes cores as (r_k x p x r_{k-1});
the index order is immaterial.  An operator train is a list of arrays of
shape (chi_{k-1}, n_out, n_in, chi_k)                   (Sec. 2, Eq. tto_format).

Combined bonds are always ordered with the FIRST operand's bond index as the
slow (major) index: Hadamard bond (alpha_x, alpha_y); operator application
bond (gamma, alpha); addition bond [x block, y block].
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------ basics --

def tt_ranks(cores):
    return [cores[0].shape[0]] + [c.shape[2] for c in cores]


def tt_full(cores) -> np.ndarray:
    """Contract all bonds: the definition of the TT format (Sec. 2, Eq. tt_format;
    also the final `contract` of Algorithm 2)."""
    dims = [c.shape[1] for c in cores]
    res = cores[0].reshape(cores[0].shape[0] * cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        r0, n, r1 = c.shape
        res = (res @ c.reshape(r0, n * r1)).reshape(-1, r1)
    return res.reshape(dims)


def mpo_full(cores) -> np.ndarray:
    """Operator train contracted to a matrix M[i, j] with i = (i_1..i_d), j = (j_1..j_d),
    each multi-index row-major with i_1 slowest (Sec. 2, Eq. tto_format)."""
    d = len(cores)
    res = np.ones((1, 1, 1), dtype=np.result_type(*cores))  # (rows, cols, bond)
    for c in cores:
        g0, no, ni, g1 = c.shape
        R, C, _ = res.shape
        res = np.einsum("abg,gijh->aibjh", res, c).reshape(R * no, C * ni, g1)
    return res[:, :, 0]


def tt_scale(c, cores):
    """Constant multiplication: rescale the first core (Sec. 2.1, Eq. tt_const_multiplication)."""
    out = [x.copy() for x in cores]
    out[0] = c * out[0]
    return out


def tt_add(x, y, a=1.0, b=1.0):
    """z = a*x + b*y by block-diagonal placement (Sec. 2.1, Addition).

    Inner cores are diag(A_k, B_k); the first core is the row [A_1 B_1], the
    last the column [A_d; B_d].  The scalars a, b scale the first cores
    (Sec. 2.1, constant multiplication; subtraction is b = -1)."""
    d = len(x)
    assert len(y) == d
    dt = np.result_type(x[0], y[0], np.asarray(a), np.asarray(b))
    if d == 1:
        return [(a * x[0] + b * y[0]).astype(dt)]
    z = []
    for k in range(d):
        A, B = x[k], y[k]
        ra0, n, ra1 = A.shape
        rb0, nb, rb1 = B.shape
        assert n == nb
        if k == 0:
            C = np.zeros((1, n, ra1 + rb1), dtype=dt)
            C[:, :, :ra1] = a * A
            C[:, :, ra1:] = b * B
        elif k == d - 1:
            C = np.zeros((ra0 + rb0, n, 1), dtype=dt)
            C[:ra0] = A
            C[ra0:] = B
        else:
            C = np.zeros((ra0 + rb0, n, ra1 + rb1), dtype=dt)
            C[:ra0, :, :ra1] = A
            C[ra0:, :, ra1:] = B
        z.append(C)
    return z


def tt_hadamard(x, y):
    """Elementwise product: C_k(i) = A_k(i) (x) B_k(i), the Kronecker product of the
    slice matrices (Sec. 2.1, Hadamard product); ranks multiply."""
    z = []
    for A, B in zip(x, y):
        ra0, n, ra1 = A.shape
        rb0, _, rb1 = B.shape
        C = np.empty((ra0 * rb0, n, ra1 * rb1), dtype=np.result_type(A, B))
        for i in range(n):
            C[:, i, :] = np.kron(A[:, i, :], B[:, i, :])
        z.append(C)
    return z


def tt_mpo_apply(mpo, x):
    """y = A x for an operator train A: B_k(i) = sum_j D_k(i, j) (x) A_k(j)
    (Sec. 2.1, TT-TTO contraction); ranks multiply, operator bond major."""
    out = []
    for D, A in zip(mpo, x):
        g0, no, ni, g1 = D.shape
        a0, n, a1 = A.shape
        assert n == ni
        B = np.zeros((g0 * a0, no, g1 * a1), dtype=np.result_type(D, A))
        for i in range(no):
            acc = np.zeros((g0 * a0, g1 * a1), dtype=B.dtype)
            for j in range(ni):
                acc += np.kron(D[:, i, j, :], A[:, j, :])
            B[:, i, :] = acc
        out.append(B)
    return out


def mpo_mpo(a, b):
    """Operator product (A B) with A applied after B: core (gamma eta, i, j, gamma' eta')
    = sum_k A(i, k) (x) B(k, j)."""
    out = []
    for A, B in zip(a, b):
        ga0, no, nk, ga1 = A.shape
        gb0, nk2, ni, gb1 = B.shape
        assert nk == nk2
        C = np.einsum("aikb,ckjd->acijbd", A, B).reshape(ga0 * gb0, no, ni, ga1 * gb1)
        out.append(C)
    return out


def mpo_adjoint(mpo):
    """Conjugate transpose of an operator train (swap in/out, conjugate)."""
    return [np.conj(D.transpose(0, 2, 1, 3)) for D in mpo]


def tt_entries(cores, idx) -> np.ndarray:
    """Entries of the train at the multi-indices idx (M x d): the product of
    the core slices G_k[:, i_k, :]."""
    idx = np.asarray(idx)
    v = np.ones((idx.shape[0], 1), dtype=np.complex128)
    for k, c in enumerate(cores):
        v = np.einsum("ma,amb->mb", v, c[:, idx[:, k], :])
    return v[:, 0]


def tt_dot(x, y):
    """<x, y> = sum_i conj(x(i)) y(i) by the transfer-matrix chain
    W_k = sum_i A_k(i)^H W_{k-1} B_k(i)."""
    W = np.ones((1, 1), dtype=np.result_type(x[0], y[0]))
    for A, B in zip(x, y):
        W = np.einsum("aib,ac,cid->bd", np.conj(A), W, B)
    return W[0, 0]


# ----------------------------------------- orthogonalisation / rounding --

def tt_left_orthogonalize(x):
    """Left-to-right QR sweep (Sec. 2.2, Orthogonalization): keep Q_k as core k,
    absorb R_k into core k+1.  Returns the cores; the last one is the
    orthogonality centre."""
    cores = [c.copy() for c in x]
    for k in range(len(cores) - 1):
        r0, n, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0 * n, r1), mode="reduced")
        cores[k] = Q.reshape(r0, n, Q.shape[1])
        cores[k + 1] = np.tensordot(R, cores[k + 1], axes=(1, 0))
    return cores


def tt_norm(x) -> float:
    """Frobenius norm as the norm of the orthogonality centre after the QR sweep."""
    return float(np.linalg.norm(tt_left_orthogonalize(x)[-1]))


def truncation_rank(s: np.ndarray, delta: float, max_rank: int | None = None):
    """Smallest t >= 1 with sqrt(sum_{j>t} s_j^2) <= delta (Sec. 2.2, the
    sufficient condition for Eq. rounding_condition_tt), then capped at
    max_rank.  Returns (t, capped) where capped says the cap cut a rank that
    the tolerance asked for."""
    q = len(s)
    if q == 0:
        return 0, False
    tail2 = np.concatenate([np.cumsum((s[::-1].astype(np.float64)) ** 2)[::-1], [0.0]])
    # tail2[t] = sum_{j >= t} s_j^2 (0-based), t = number kept
    t = q
    for cand in range(1, q + 1):
        if math.sqrt(tail2[cand]) <= delta:
            t = cand
            break
    capped = False
    if max_rank is not None and t > max_rank:
        t = max_rank
        capped = True
    return t, capped


def rounding_delta(eps: float, norm: float, d: int) -> float:
    """Per-bond threshold delta = eps ||x||_F / sqrt(d - 1).  The paper prints
    eps/sqrt(1-n)||x|| (Sec. 2.2, Eq. optimal_delta), imaginary for n > 1;
    the cited source (Oseledets 2011) has sqrt(d-1), which is read here."""
    if d <= 1:
        return 0.0
    return eps * norm / math.sqrt(d - 1)


def bucket_rank(t: int, r0: int, limit: int) -> int:
    """Coarse-grained rank n*r0 >= t (Sec. 5.1), never above `limit`."""
    if r0 <= 1:
        return t
    return min(int(math.ceil(t / r0)) * r0, limit)


def tt_round(x, eps: float, max_rank: int | None = None, r0: int = 1,
             forced_ranks=None):
    """SVD-based compression (Sec. 2.2): left-to-right QR sweep, ||x|| from the
    orthogonality centre, delta = eps ||x|| / sqrt(d-1), then a right-to-left
    sweep of truncated SVDs of the centre; U_k S_k is absorbed into core k-1
    and V_k^H stays as core k.

    `forced_ranks` (list of d+1 ints) replaces the adaptive rule (used to
    compare implementations on one rank trace).  Returns (cores, info) where
    info = dict(norm, delta, ranks, capped, tail) and tail[k] is the
    discarded singular-value mass at bond k."""
    d = len(x)
    cores = tt_left_orthogonalize(x)
    nrm = float(np.linalg.norm(cores[-1]))
    delta = rounding_delta(eps, nrm, d)
    capped = False
    tails = [0.0] * (d + 1)
    for k in range(d - 1, 0, -1):
        r0_, n, r1 = cores[k].shape
        U, s, Vh = np.linalg.svd(cores[k].reshape(r0_, n * r1), full_matrices=False)
        if forced_ranks is not None:
            t = min(forced_ranks[k], len(s))
        else:
            t, c = truncation_rank(s, delta, max_rank)
            capped = capped or c
            t = bucket_rank(t, r0, len(s) if max_rank is None else min(len(s), max_rank))
        tails[k] = float(np.sqrt(np.sum(s[t:] ** 2)))
        cores[k] = Vh[:t].reshape(t, n, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], U[:, :t] * s[:t], axes=(2, 0))
    info = dict(norm=nrm, delta=delta, ranks=tt_ranks(cores), capped=capped, tail=tails)
    return cores, info


def tt_svd(full: np.ndarray, eps: float, max_rank: int | None = None):
    """Dense tensor to TT by sequential truncated SVDs of the unfoldings
    (TT-SVD, Oseledets 2011, Algorithm 1), with the same per-bond threshold
    delta = eps ||A||_F / sqrt(d-1)."""
    dims = full.shape
    d = len(dims)
    if d == 1:
        return [full.reshape(1, dims[0], 1).copy()]
    delta = rounding_delta(eps, float(np.linalg.norm(full)), d)
    C = full.reshape(dims[0], -1)
    r_prev = 1
    cores = []
    for k in range(d - 1):
        C = C.reshape(r_prev * dims[k], -1)
        U, s, Vh = np.linalg.svd(C, full_matrices=False)
        t, _ = truncation_rank(s, delta, max_rank)
        cores.append(U[:, :t].reshape(r_prev, dims[k], t))
        C = s[:t, None] * Vh[:t]
        r_prev = t
    cores.append(C.reshape(r_prev, dims[-1], 1))
    return cores


def mpo_round(mpo, eps: float, max_rank: int | None = None):
    """Round an operator train by viewing each core as a TT core with the
    combined physical index (i, j)."""
    shapes = [D.shape for D in mpo]
    as_tt = [D.reshape(D.shape[0], D.shape[1] * D.shape[2], D.shape[3]) for D in mpo]
    rounded, info = tt_round(as_tt, eps, max_rank)
    out = [c.reshape(c.shape[0], s[1], s[2], c.shape[2]) for c, s in zip(rounded, shapes)]
    return out, info


def diag_mpo_from_tt(cores):
    """Operator with D(i, j) = B(i) delta(i, j) (Sec. 2.1, Eq. tt_to_tto)."""
    out = []
    for B in cores:
        r0, n, r1 = B.shape
        D = np.zeros((r0, n, n, r1), dtype=B.dtype)
        for i in range(n):
            D[:, i, i, :] = B[:, i, :]
        out.append(D)
    return out


def identity_mpo(dims, dtype=np.complex128):
    return [np.eye(n, dtype=dtype).reshape(1, n, n, 1) for n in dims]


def mpo_add(a, b):
    """Sum of two operator trains by the block rule of Sec. 2.1 applied to the
    combined physical index."""
    ta = [D.reshape(D.shape[0], D.shape[1] * D.shape[2], D.shape[3]) for D in a]
    tb = [D.reshape(D.shape[0], D.shape[1] * D.shape[2], D.shape[3]) for D in b]
    s = tt_add(ta, tb)
    return [c.reshape(c.shape[0], D.shape[1], D.shape[2], c.shape[2]) for c, D in zip(s, a)]


def ones_tt(dims, dtype=np.complex128):
    return [np.ones((1, n, 1), dtype=dtype) for n in dims]

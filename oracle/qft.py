"""The superfast Fourier transform: Q_n of QFT_n = R_n Q_n as an operator train.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (Sec. 3.2 and Fig. 1 of the paper; sign and normalisation are a
reading, the paper is silent on them):
* Input index j = sum_a j_a 2^(n-a): site a carries bit j_a, MSB first.
* Forward transform = unitary DFT, F[k, j] = exp(-2 pi i k j / N) / sqrt(N)
  (numpy.fft with norm="ortho").
* Q_n drops the final bit reversal R_n, so output site a carries the bit m_a
  of the frequency k with weight 2^(a-1) (LSB first):  Q[m, j] = F[rev(m), j].
* Written out, Q(m, j) = N^(-1/2) exp(-2 pi i sum_{b <= a} j_a m_b 2^(b-a-1)).

Construction: the QFT circuit without its swaps, one layer per qubit b:
a Hadamard on qubit b followed by the phase gates controlled by qubit b on
every later qubit a > b.  Each layer is an operator train of bond 2 (the bond
carries the control bit m_b); the layers are multiplied in circuit order and
the running product is rounded after each layer.
"""
from __future__ import annotations

import math

import numpy as np

from . import tt as T


def _layer(n: int, b: int, sign: float):
    """Layer b (0-based) of the circuit: H on site b, then the controlled phases
    exp(sign * 2 pi i m_b j_a 2^(b-a-1)) for every a > b (1-based exponents
    translate to 0-based b, a unchanged)."""
    cores = []
    for a in range(n):
        if a < b:
            cores.append(np.eye(2, dtype=np.complex128).reshape(1, 2, 2, 1))
        elif a == b:
            # core[0, m, j, c] = (-1)^(m j)/sqrt(2) * delta(c, m)
            last = (b == n - 1)
            core = np.zeros((1, 2, 2, 1 if last else 2), dtype=np.complex128)
            for m in range(2):
                for j in range(2):
                    h = (-1.0) ** (m * j) / math.sqrt(2.0)
                    core[0, m, j, 0 if last else m] = h
            cores.append(core)
        else:
            last = (a == n - 1)
            core = np.zeros((2, 2, 2, 1 if last else 2), dtype=np.complex128)
            theta = sign * 2.0 * math.pi * 2.0 ** (b - a - 1)
            for c in range(2):
                for j in range(2):
                    core[c, j, j, 0 if last else c] = np.exp(1j * theta * c * j)
            cores.append(core)
    return cores


def qft_mpo(n: int, sign: float = -1.0, tol: float = 1e-12, max_rank: int | None = None):
    """Operator train of Q_n (n sites, bond <= chi_Q after rounding at `tol`)."""
    Q = T.identity_mpo([2] * n)
    for b in range(n):
        L = _layer(n, b, sign)
        Q = T.mpo_mpo(L, Q)          # layer b acts after the earlier layers
        if n > 1:
            Q, _ = T.mpo_round(Q, tol, max_rank)
    return Q


def bit_reverse_indices(n: int) -> np.ndarray:
    N = 1 << n
    out = np.zeros(N, dtype=np.int64)
    for m in range(N):
        r = 0
        for a in range(n):
            if (m >> a) & 1:
                r |= 1 << (n - 1 - a)
        out[m] = r
    return out


def qft_closed_form(n: int, sign: float = -1.0) -> np.ndarray:
    """Dense Q[m, j] from the bit-level closed form (m, j as MSB-first site strings)."""
    N = 1 << n
    M = np.zeros((N, N), dtype=np.complex128)
    for m in range(N):
        mb = [(m >> (n - 1 - a)) & 1 for a in range(n)]  # bit at site a
        for j in range(N):
            jb = [(j >> (n - 1 - a)) & 1 for a in range(n)]
            ph = 0.0
            for a in range(n):
                for b in range(a + 1):
                    ph += jb[a] * mb[b] * 2.0 ** (b - a - 1)
            M[m, j] = np.exp(sign * 2j * math.pi * ph) / math.sqrt(N)
    return M


def embed_1d_mpo(mpo1d, positions, total_sites, dims):
    """Place a one-dimensional operator train on `positions` (increasing site
    numbers) of a longer train of `total_sites` sites with physical
    dimensions `dims`; every other site gets the identity, carrying the bond
    through unchanged."""
    out = []
    pos = list(positions)
    bond = 1
    q = 0
    for s in range(total_sites):
        n = dims[s]
        if q < len(pos) and s == pos[q]:
            D = mpo1d[q]
            out.append(D)
            bond = D.shape[3]
            q += 1
        else:
            core = np.zeros((bond, n, n, bond), dtype=np.complex128)
            for g in range(bond):
                core[g, :, :, g] = np.eye(n)
            out.append(core)
    return out

"""Compression via polar decomposition (Sec. 2.2, "Compression via Polar
Decomposition") in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper replaces the truncated SVD of the orthogonality centre by:
  1. the polar decomposition of the centre, T = U H (U isometric, H Hermitian
     positive semidefinite, its eigenvalues the singular values of T);
  2. the polar decomposition of H - delta~ I, whose unitary factor U' has
     eigenvalue +1 on the eigenvectors of H with sigma > delta~ and -1 on the
     others (U' is the matrix sign function of H - delta~ I);
  3. the projectors P_+- = (1 +- U') / 2 and the truncated centre
     T~ = U (P_+ H P_+);
  4. an orthonormal basis C_+ of the range of P_+ (subspace iteration), and
     the factors F = U C_+, G = C_+^H H with T~ = F G;
with the absolute cutoff delta~ = delta / q, q the number of untruncated
singular values, so that the discarded mass of every bond is at most
sqrt(q) delta~ <= delta and the TT rounding bound still holds (with ranks at
least those of the SVD rounding).

Every step here is its plain definition: the polar factors from an SVD, the
sign function from an eigendecomposition, the basis from a QR of P_+ applied
to a starting block.  The sweep structure is that of oracle.tt.tt_round:
left-orthogonalise, then right to left, truncating the bond between cores
k-1 and k with T the (n_k r_k) x r_{k-1} matrix C_k^H, F^H becoming core k
and the rest (H C_+)(r_{k-1} x l) absorbed into core k-1.
"""
from __future__ import annotations

import numpy as np

from . import tt as T


def polar(A: np.ndarray):
    """A = U H with U = W V^H (isometric on the range of A) and H = V S V^H,
    from the thin SVD A = W S V^H."""
    W, s, Vh = np.linalg.svd(A, full_matrices=False)
    U = W @ Vh
    H = (Vh.conj().T * s) @ Vh
    return U, 0.5 * (H + H.conj().T)


def sign_hermitian(B: np.ndarray) -> np.ndarray:
    """Matrix sign function of a Hermitian matrix: eigenvalues mapped to +1
    (> 0) and -1 (<= 0); it is the unitary polar factor of B when B is
    nonsingular."""
    w, V = np.linalg.eigh(0.5 * (B + B.conj().T))
    sgn = np.where(w > 0, 1.0, -1.0)
    return (V * sgn) @ V.conj().T


def polar_truncate(A: np.ndarray, delta_t: float, rng=None):
    """Truncate the columns of A (m x q) at the absolute cutoff delta_t by the
    polar steps.  Returns (F, G, l, tail): A~ = F G, F (m x l) with
    orthonormal columns, G (l x q), l = the number of singular values above
    delta_t (at least 1), tail = ||A - A~||_F."""
    m, q = A.shape
    U, H = polar(A)
    Up = sign_hermitian(H - delta_t * np.eye(q))
    Pp = 0.5 * (np.eye(q) + Up)
    l = int(round(float(np.real(np.trace(Pp)))))
    l = max(1, min(l, q))
    # subspace iteration on the projector from a fixed Gaussian block
    rng = np.random.default_rng(0) if rng is None else rng
    Om = rng.standard_normal((q, l)) + 1j * rng.standard_normal((q, l))
    Cp, _ = np.linalg.qr(Pp @ Om)
    Cp, _ = np.linalg.qr(Pp @ Cp)
    F = U @ Cp
    G = Cp.conj().T @ H
    tail = float(np.linalg.norm(A - F @ G))
    return F, G, l, tail


def tt_round_polar(x, eps: float):
    """Polar-based compression of a train (Sec. 2.2): the sweeps of
    oracle.tt.tt_round with polar_truncate in place of the truncated SVD and
    delta~ = delta / q at every bond.  Returns (cores, info) with info =
    dict(norm, delta, ranks, tail)."""
    d = len(x)
    cores = T.tt_left_orthogonalize(x)
    nrm = float(np.linalg.norm(cores[-1]))
    delta = T.rounding_delta(eps, nrm, d)
    tails = [0.0] * (d + 1)
    for k in range(d - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        A = cores[k].reshape(r0, n * r1).conj().T           # (n r1) x r0: the bond r0 on the columns
        F, G, l, tail = polar_truncate(A, delta / min(A.shape))   # q: the number of singular values
        tails[k] = tail
        cores[k] = F.conj().T.reshape(l, n, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], G.conj().T, axes=(2, 0))
    info = dict(norm=nrm, delta=delta, ranks=T.tt_ranks(cores), tail=tails)
    return cores, info

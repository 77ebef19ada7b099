"""TT-cross approximation (Sec. 3: the phase and Green operator trains are
built by sampling, not by a dense TT-SVD) in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper separates the cores of its discretised operands with the TT-cross
approximation of Oseledets & Tyrtyshnikov (2010).  It gives no further
detail; this oracle takes the rank-adaptive two-site form of that method
(Savostyanov & Oseledets 2011), in which the ranks follow from truncated SVDs
of sampled two-site blocks:

* index sets: for every bond k a set I_k of "left" multi-indices over sites
  0..k-1 and a set J_k of "right" multi-indices over sites k..d-1, nested
  (every left index of I_{k+1} extends one of I_k by a value of site k, and
  likewise from the right);
* a forward half-sweep visits the bonds k = 0..d-2: it samples the
  superblock S[(a, i), (j, b)] = f(I_k[a], i, j, J_{k+2}[b]), keeps the
  leading singular vectors U of S whose discarded tail is at most
  eps ||S||_F / sqrt(d - 1) (at most max_rank of them), appends `kick`
  Gaussian columns (so that the index sets keep exploring), chooses the rows
  of the result by the maximum-volume rule (maxvol), and takes those rows as
  I_{k+1}; core k is the interpolation matrix A A[rows]^-1, and at the last
  bond core d-1 is the sampled rows S[rows, :];
* a backward half-sweep does the same from the right with the right singular
  vectors, building J and the interpolation cores (A A[rows]^-1)^H; at bond 0
  core 0 is the sampled columns S[:, cols];
* the half-sweeps alternate until the train changes by at most 10 eps
  (relative, in the Frobenius norm) from one half-sweep to the next (two
  approximations that each meet the eps truncation rule differ by a few eps),
  or a sweep limit is met; the start is a right index set drawn from
  `init_rank` random points and any given `init_points` (for a box geometry
  the voxels holding the box centres, box_centre_points: points inside the
  phase-2 region, which random points may all miss).

The sampled operands: the Green operator train (momentum convention), the
phase indicator of a union of axis-aligned boxes, and the phase indicator of
a union of ellipsoids (spheres, random ellipsoids and aligned fibres, the
geometries of the 3D workloads), each a pointwise function of the site
values pinned entry by entry to the dense voxelisation of the input
generators.

maxvol (Goreinov, Oseledets, Savostyanov et al. 2010): start from the rows of
Gaussian elimination with partial pivoting, then, while some entry of
B = A A[rows]^-1 exceeds `tol` in modulus, replace the row of its column by
its row.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import ms as MS
from . import tt as T
from paper_2512_07811_gb300 import inputs as IN


def maxvol(A: np.ndarray, tol: float = 1.05, max_iters: int = 100):
    """Rows `rows` of the tall full-column-rank A (m x r) with a dominant
    r x r submatrix: every entry of B = A A[rows]^-1 has modulus <= tol (or
    max_iters swaps were made).  Returns (rows, B)."""
    m, r = A.shape
    assert m >= r
    P, _, _ = scipy.linalg.lu(A)                # A = P L U, partial pivoting over rows
    rows = list(np.argmax(P, axis=0)[:r])        # row perm[i] of A becomes row i of L U
    B = None
    for _ in range(max_iters + 1):
        B = np.linalg.solve(A[rows].T, A.T).T    # B = A A[rows]^-1
        i, j = np.unravel_index(int(np.argmax(np.abs(B))), B.shape)
        if abs(B[i, j]) <= tol:
            break
        rows[j] = int(i)
    return rows, B


def _superblock(f, Il, Jr, n0, n1):
    """S[(a, i), (j, b)] = f(Il[a], i, j, Jr[b]) as an (rl n0) x (n1 rr) matrix."""
    rl, rr = Il.shape[0], Jr.shape[0]
    a, i, j, b = np.meshgrid(np.arange(rl), np.arange(n0), np.arange(n1), np.arange(rr), indexing="ij")
    a, i, j, b = a.ravel(), i.ravel(), j.ravel(), b.ravel()
    idx = np.concatenate([Il[a], i[:, None], j[:, None], Jr[b]], axis=1)
    return np.asarray(f(idx)).reshape(rl * n0, n1 * rr).astype(np.complex128)


def _kept(S, eps, d, max_rank, kick, rng, right: bool):
    """Leading singular vectors of S (left, or right as the columns of V)
    with the eps ||S|| / sqrt(d - 1) tail rule and `kick` Gaussian columns."""
    U, s, Vh = np.linalg.svd(S, full_matrices=False)
    delta = eps * np.linalg.norm(S) / math.sqrt(max(d - 1, 1))
    t, _ = T.truncation_rank(s, delta, max_rank)
    V = Vh.conj().T if right else U
    A = V[:, :t]
    extra = min(kick, A.shape[0] - t)
    if extra > 0:
        Z = rng.standard_normal((A.shape[0], extra)) + 0j
        A = np.hstack([A, Z])
    return A


def tt_cross(f, modes, eps: float, max_rank: int | None = None, kick: int = 2, max_half_sweeps: int = 12,
             init_rank: int = 2, seed: int = 0, init_points=None):
    """TT-cross approximation of the tensor with entries f(idx) (idx an
    integer array (M, d) of multi-indices, f returning M values) and mode
    sizes `modes`.  Returns (cores, info), info = dict(half_sweeps,
    evaluations, rel_change, ranks)."""
    d = len(modes)
    rng = np.random.default_rng(seed)
    if d == 1:
        idx = np.arange(modes[0])[:, None]
        return [np.asarray(f(idx), dtype=np.complex128).reshape(1, modes[0], 1)], \
            dict(half_sweeps=0, evaluations=modes[0], rel_change=0.0, ranks=[1, 1])
    pts = np.stack([rng.integers(0, n, size=init_rank) for n in modes], axis=1)
    if init_points is not None:
        pts = np.concatenate([pts, np.asarray(init_points, dtype=pts.dtype).reshape(-1, d)], axis=0)
    I = [np.zeros((1, 0), dtype=np.int64) for _ in range(d + 1)]
    J = [np.zeros((1, 0), dtype=np.int64) for _ in range(d + 1)]
    for k in range(1, d):
        J[k] = np.unique(pts[:, k:], axis=0)
    cores = [None] * d
    prev = None
    evals = 0
    rel = math.inf
    h = 0
    for h in range(1, max_half_sweeps + 1):
        if h % 2 == 1:                                   # forward
            for k in range(d - 1):
                n0, n1 = modes[k], modes[k + 1]
                S = _superblock(f, I[k], J[k + 2], n0, n1)
                evals += S.size
                A = _kept(S, eps, d, max_rank, kick, rng, right=False)
                rows, B = maxvol(A)
                cores[k] = B.reshape(I[k].shape[0], n0, len(rows))
                I[k + 1] = np.array([list(I[k][r // n0]) + [r % n0] for r in rows], dtype=np.int64)
                if k == d - 2:
                    cores[d - 1] = S[rows, :].reshape(len(rows), n1, 1)
        else:                                            # backward
            for k in range(d - 2, -1, -1):
                n0, n1 = modes[k], modes[k + 1]
                S = _superblock(f, I[k], J[k + 2], n0, n1)
                evals += S.size
                A = _kept(S, eps, d, max_rank, kick, rng, right=True)
                cols, B = maxvol(A)
                rr = J[k + 2].shape[0]
                cores[k + 1] = B.conj().T.reshape(len(cols), n1, rr)
                J[k + 1] = np.array([[c // rr] + list(J[k + 2][c % rr]) for c in cols], dtype=np.int64)
                if k == 0:
                    cores[0] = S[:, cols].reshape(1, n0, len(cols))
        cur = [c.copy() for c in cores]
        if prev is not None:
            nrm = T.tt_norm(cur)
            rel = T.tt_norm(T.tt_add(cur, prev, 1.0, -1.0)) / nrm if nrm > 0 else 0.0
            if rel <= 10 * eps:
                break
        prev = cur
    return cores, dict(half_sweeps=h, evaluations=evals, rel_change=rel, ranks=T.tt_ranks(cores))


# ----------------------------------------------- the sampled operands --

def _site_bits(idx_sites, nb, ordering, momentum: bool):
    """Integer coordinates per dimension from the spatial site values
    idx_sites (M, sum(nb)): position space MSB first, momentum space LSB
    first (each dimension's bits reversed, the SFFT convention)."""
    coords = []
    for dim in range(3):
        pos = MS.dim_positions(nb, ordering, dim)
        v = np.zeros(idx_sites.shape[0], dtype=np.int64)
        for a, s in enumerate(pos):
            shift = a if momentum else nb[dim] - 1 - a
            v |= idx_sites[:, s].astype(np.int64) << shift
        coords.append(v)
    return coords


def green_fn(pb: MS.Problem, nb, ordering: str = "interleaved"):
    """Entries of the Green operator train: site 0 the control index
    I * ncomp + J, then the spatial sites in the momentum convention."""
    nc = pb.ncomp
    shape = tuple(1 << b for b in nb)

    def f(idx):
        idx = np.asarray(idx)
        k = _site_bits(idx[:, 1:], nb, ordering, momentum=True)
        xi = [np.where(k[a] < (shape[a] + 1) // 2, k[a], k[a] - shape[a]).astype(np.float64) for a in range(3)]
        G = MS.green_components(pb, xi)                       # (nc, nc, M)
        c = idx[:, 0]
        return G[c // nc, c % nc, np.arange(idx.shape[0])]
    return f


def box_centre_points(boxes, nb, ordering: str = "interleaved") -> np.ndarray:
    """Site values (position convention) of the voxel holding each box centre."""
    boxes = np.asarray(boxes, dtype=np.float64).reshape(-1, 6)
    pts = np.zeros((boxes.shape[0], sum(nb)), dtype=np.int64)
    for i, b in enumerate(boxes):
        for dim in range(3):
            N = 1 << nb[dim]
            x = min(int((b[dim] - math.floor(b[dim])) * N), N - 1)
            for a, s in enumerate(MS.dim_positions(nb, ordering, dim)):
                pts[i, s] = (x >> (nb[dim] - 1 - a)) & 1
    return pts


def boxes_fn(boxes, nb, ordering: str = "interleaved"):
    """Entries of the phase indicator train of a union of boxes (position
    convention, spatial sites only)."""
    shape = tuple(1 << b for b in nb)

    def f(idx):
        x = _site_bits(np.asarray(idx), nb, ordering, momentum=False)
        return IN.boxes_value(boxes, x[0], x[1], x[2], shape)
    return f


def ellipsoid_centre_points(rows, nb, ordering: str = "interleaved") -> np.ndarray:
    """Site values (position convention) of the voxel holding each ellipsoid
    centre (rows as in inputs.ellipsoids_value)."""
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, IN.ELLIPSOID_ROW)
    pts = np.zeros((rows.shape[0], sum(nb)), dtype=np.int64)
    for i, e in enumerate(rows):
        for dim in range(3):
            N = 1 << nb[dim]
            x = min(int((e[dim] - math.floor(e[dim])) * N), N - 1)
            for a, s in enumerate(MS.dim_positions(nb, ordering, dim)):
                pts[i, s] = (x >> (nb[dim] - 1 - a)) & 1
    return pts


def ellipsoids_fn(rows, nb, ordering: str = "interleaved"):
    """Entries of the phase indicator train of a union of ellipsoids (spheres,
    random ellipsoids, fibres with an infinite semi-axis), position
    convention, spatial sites only."""
    shape = tuple(1 << b for b in nb)

    def f(idx):
        x = _site_bits(np.asarray(idx), nb, ordering, momentum=False)
        return IN.ellipsoids_value(rows, x[0], x[1], x[2], shape)
    return f

"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the homogenisation method: it only draws
random numbers and voxelises simple geometries.  Everything that the method
computes (tensor-train algebra, rounding, Fourier operators, Green operator,
fixed-point iteration) lives elsewhere.

Conventions
-----------
* A voxel grid has N = 2**n points per side; voxel (i, j, k) has its centre at
  ((i + 1/2)/N, (j + 1/2)/N, (k + 1/2)/N) in the unit cell.  Points exactly on
  an inclusion boundary count as inside.
* Phase indicators are float64 arrays of shape (N, N, N) holding 0.0 (matrix,
  phase 1) or 1.0 (inclusion / second phase, phase 2).
* Random tensor-train cores have shape (r_{k-1}, p, r_k) with r_0 = r_d = 1 and
  bond caps r_k <= min(r, p**k, p**(d-k)).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- geometry --

def voxel_centres(N: int) -> np.ndarray:
    return (np.arange(N, dtype=np.float64) + 0.5) / N


def laminate_indicator(N: int, axis: int = 0, fraction: float = 0.5) -> np.ndarray:
    """Two-phase laminate, layers normal to `axis`; phase 2 where coordinate < fraction."""
    c = voxel_centres(N)
    ind1d = (c < fraction).astype(np.float64)
    shape = [1, 1, 1]
    shape[axis] = N
    return np.broadcast_to(ind1d.reshape(shape), (N, N, N)).copy()


def prism(ind2d: np.ndarray) -> np.ndarray:
    """A two-dimensional phase image (Nx, Ny) as a grid one voxel thick along
    z (Nx, Ny, 1): the plane problem in the three-dimensional solver."""
    return np.ascontiguousarray(ind2d, dtype=np.float64)[:, :, None].copy()


def laminate_indicator_2d(N: int, axis: int = 0, fraction: float = 0.5) -> np.ndarray:
    """Plane laminate (N, N, 1): layers normal to `axis` (0 or 1)."""
    c = voxel_centres(N)
    ind1d = (c < fraction).astype(np.float64)
    img = ind1d[:, None] * np.ones((1, N)) if axis == 0 else np.ones((N, 1)) * ind1d[None, :]
    return prism(img)


def box_indicator_2d(N: int, area_fraction: float = 0.2, centre=(0.5, 0.5)) -> np.ndarray:
    """Square inclusion of the given area fraction in the plane (N, N, 1) --
    the box geometry of the paper's Fig. 4."""
    h = 0.5 * math.sqrt(area_fraction)
    c = voxel_centres(N)
    img = (np.abs(c - centre[0]) <= h)[:, None] & (np.abs(c - centre[1]) <= h)[None, :]
    return prism(img.astype(np.float64))


def boxes_value(boxes, ix, iy, iz, shape) -> np.ndarray:
    """Phase value (0.0 / 1.0) at voxels (ix, iy, iz) (integer arrays of one
    shape) of an (Nx, Ny, Nz) grid for a union of axis-aligned boxes, rows
    (cx, cy, cz, hx, hy, hz) in unit-cell coordinates: a voxel is in phase 2
    when, along every axis, the periodic (minimum image) distance
    |((c - cx + 1/2) mod 1) - 1/2| of its centre c = (i + 1/2)/N from some
    box centre is at most that box's half width."""
    boxes = np.asarray(boxes, dtype=np.float64).reshape(-1, 6)
    idx = [np.asarray(ix), np.asarray(iy), np.asarray(iz)]
    cen = [(idx[a].astype(np.float64) + 0.5) / shape[a] for a in range(3)]
    out = np.zeros(np.broadcast(*idx).shape, dtype=bool)
    for b in boxes:
        inside = np.ones_like(out)
        for a in range(3):
            inside &= np.abs((cen[a] - b[a] + 0.5) % 1.0 - 0.5) <= b[3 + a]
        out |= inside
    return out.astype(np.float64)


def boxes_indicator(boxes, shape) -> np.ndarray:
    """The union of boxes voxelised on the whole (Nx, Ny, Nz) grid (see boxes_value)."""
    ix, iy, iz = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return boxes_value(boxes, ix, iy, iz, shape)


def multibox_boxes_2d(N: int, count: int = 8, area_fraction: float = 0.2, seed: int = 0) -> np.ndarray:
    """`count` non-overlapping axis-aligned squares of random sizes and
    positions (periodic minimum image, at least one voxel of an N x N grid
    apart) filling about `area_fraction` of the plane, as box rows
    (cx, cy, 1/2, h, h, 1/2) spanning the single voxel along z: a synthetic
    look-alike of the paper's multibox images."""
    rng = np.random.default_rng(seed)
    placed = []
    target = area_fraction / count
    tries = 0
    while len(placed) < count and tries < 10000:
        tries += 1
        h = 0.5 * math.sqrt(target * rng.uniform(0.5, 1.5))
        x0, y0 = rng.uniform(0, 1, 2)
        ok = True
        for (x1, y1, h1) in placed:
            dx = abs((x0 - x1 + 0.5) % 1.0 - 0.5)
            dy = abs((y0 - y1 + 0.5) % 1.0 - 0.5)
            if dx < h + h1 + 1.0 / N and dy < h + h1 + 1.0 / N:
                ok = False
                break
        if not ok:
            continue
        placed.append((x0, y0, h))
    return np.array([[x0, y0, 0.5, h, h, 0.5] for (x0, y0, h) in placed], dtype=np.float64)


def multibox_indicator_2d(N: int, count: int = 8, area_fraction: float = 0.2, seed: int = 0) -> np.ndarray:
    """The multibox image of multibox_boxes_2d voxelised on (N, N, 1)."""
    return boxes_indicator(multibox_boxes_2d(N, count, area_fraction, seed), (N, N, 1))


def laminate_boxes_2d(fraction: float = 0.5) -> np.ndarray:
    """The plane laminate of laminate_indicator_2d (axis 0) as one box: phase 2
    where the x coordinate of the voxel centre is below `fraction`."""
    return np.array([[0.5 * fraction, 0.5, 0.5, 0.5 * fraction, 0.5, 0.5]])


def box_indicator(N: int, volume_fraction: float = 0.2, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Axis-aligned cubic inclusion of the given volume fraction (the 3D
    counterpart of the box geometry of the paper's Fig. 4)."""
    h = 0.5 * volume_fraction ** (1.0 / 3.0)
    c = voxel_centres(N)
    inx = (np.abs(c - centre[0]) <= h)[:, None, None]
    iny = (np.abs(c - centre[1]) <= h)[None, :, None]
    inz = (np.abs(c - centre[2]) <= h)[None, None, :]
    return (inx & iny & inz).astype(np.float64)


def sphere_radius(volume_fraction: float) -> float:
    """Radius of a sphere of the given volume fraction in the unit cell."""
    return (3.0 * volume_fraction / (4.0 * math.pi)) ** (1.0 / 3.0)


def sphere_indicator(N: int, volume_fraction: float = 0.2,
                     centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Single centred spherical inclusion of the given (continuum) volume fraction."""
    R = sphere_radius(volume_fraction)
    c = voxel_centres(N)
    dx = (c - centre[0])[:, None, None]
    dy = (c - centre[1])[None, :, None]
    dz = (c - centre[2])[None, None, :]
    return ((dx * dx + dy * dy + dz * dz) <= R * R).astype(np.float64)


# Ellipsoid rows: (cx, cy, cz, a0, a1, a2, R00, R01, R02, R10, R11, R12, R20,
# R21, R22) -- centre, semi-axes and the rotation R (row-major) whose column i
# is the direction of semi-axis i.  A semi-axis may be +inf (a cylinder along
# that direction: a fibre).  Spheres, random ellipsoids and aligned fibres
# all use this one description and the one voxelisation rule below.
ELLIPSOID_ROW = 15


def ellipsoids_value(rows, ix, iy, iz, shape) -> np.ndarray:
    """Phase value (0.0 / 1.0) at voxels (ix, iy, iz) (integer arrays of one
    shape) of an (Nx, Ny, Nz) grid for a union of ellipsoids (rows as above):
    with the voxel centre c_j = (i_j + 1/2)/N_j, the periodic offsets
    D_j = (c_j - centre_j) - round(c_j - centre_j) (round half to even), the
    body-frame coordinates u_i = (R[0, i] D_0 + R[1, i] D_1) + R[2, i] D_2 and
    t_i = u_i / a_i, a voxel is in phase 2 when
    (t_0 t_0 + t_1 t_1) + t_2 t_2 <= 1 for some row.  Every operation is one
    IEEE double operation in exactly this order (no fused multiply-add), so
    any implementation that follows it voxelises bit for bit alike."""
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, ELLIPSOID_ROW)
    idx = [np.asarray(ix), np.asarray(iy), np.asarray(iz)]
    cen = [(idx[a].astype(np.float64) + 0.5) / shape[a] for a in range(3)]
    out = np.zeros(np.broadcast(*idx).shape, dtype=bool)
    for e in rows:
        D = []
        for a in range(3):
            t = cen[a] - e[a]
            D.append(t - np.round(t))
        R = e[6:15].reshape(3, 3)
        s = None
        for i in range(3):
            u = R[0, i] * D[0] + R[1, i] * D[1]
            u = u + R[2, i] * D[2]
            t = u / e[3 + i]
            s = t * t if s is None else s + t * t
        out |= s <= 1.0
    return out.astype(np.float64)


def ellipsoids_indicator(rows, shape) -> np.ndarray:
    """The union of ellipsoids voxelised on the whole (Nx, Ny, Nz) grid (see ellipsoids_value)."""
    ix, iy, iz = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return ellipsoids_value(rows, ix, iy, iz, shape)


def sphere_rows(volume_fraction: float = 0.2, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """One sphere of the given continuum volume fraction as an ellipsoid row."""
    R = sphere_radius(volume_fraction)
    return np.array([[centre[0], centre[1], centre[2], R, R, R, 1, 0, 0, 0, 1, 0, 0, 0, 1]], dtype=np.float64)


def fibre_rows(rng: np.random.Generator, count: int = 32, fibre_fraction: float = 0.3,
               max_tries: int = 100000) -> np.ndarray:
    """`count` aligned cylindrical fibres (axis along z), non-overlapping under
    the periodic minimum-image distance, radius sqrt(fraction / (count pi)) so
    that they fill `fibre_fraction` of the cell, as ellipsoid rows with an
    infinite third semi-axis."""
    radius = math.sqrt(fibre_fraction / (count * math.pi))
    centres = []
    for _ in range(max_tries):
        if len(centres) == count:
            break
        p = rng.uniform(0.0, 1.0, size=2)
        ok = True
        for q in centres:
            d = p - q
            d -= np.round(d)
            if d @ d < (2.0 * radius) ** 2:
                ok = False
                break
        if ok:
            centres.append(p)
    if len(centres) < count:
        raise RuntimeError("fibre_rows: could not place all fibres")
    return np.array([[p[0], p[1], 0.5, radius, radius, math.inf, 1, 0, 0, 0, 1, 0, 0, 0, 1] for p in centres],
                    dtype=np.float64)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _periodic_delta(c: np.ndarray, centre: float) -> np.ndarray:
    d = c - centre
    return d - np.round(d)


def ellipsoid_rve_rows(N: int, rng: np.random.Generator, max_tries: int = 400):
    """Random RVE of 1..8 non-overlapping, randomly oriented ellipsoids.

    The count is drawn from 1..8, the semi-axes from U[0.05, 0.2] (units of
    the cell side) and the orientation from a uniform quaternion; a target
    phase fraction f is drawn from U[0.12, 0.28] and all semi-axes are scaled
    by one common factor so that the ellipsoids' continuum volume is f (drawn
    as specified, 1-8 such ellipsoids rarely reach the required fraction of
    0.1-0.3).  An ellipsoid that overlaps an earlier one on the voxel grid
    (periodic) is redrawn; the whole RVE is redrawn until the voxel phase
    fraction lies in [0.1, 0.3].  Returns (rows, indicator, contrast): the
    ellipsoid rows, their voxelisation on the N^3 grid (ellipsoids_value) and
    the contrast, log-uniform in [5, 100].
    """
    shape = (N, N, N)
    ix, iy, iz = np.meshgrid(*[np.arange(N)] * 3, indexing="ij")
    for _ in range(max_tries):
        count = int(rng.integers(1, 9))
        f = rng.uniform(0.12, 0.28)
        axes_all = rng.uniform(0.05, 0.2, size=(count, 3))
        vol = float(np.sum(4.0 / 3.0 * math.pi * np.prod(axes_all, axis=1)))
        axes_all *= (f / vol) ** (1.0 / 3.0)
        ind = np.zeros(shape, dtype=bool)
        rows = []
        for e in range(count):
            axes = axes_all[e]
            for _ in range(50):
                rot = _random_rotation(rng)
                ctr = rng.uniform(0.0, 1.0, size=3)
                row = np.concatenate([ctr, axes, rot.reshape(-1)])
                inside = ellipsoids_value(row, ix, iy, iz, shape) > 0
                if np.any(inside & ind):
                    continue
                ind |= inside
                rows.append(row)
                break
        frac = ind.mean()
        if len(rows) == count and 0.1 <= frac <= 0.3:
            contrast = float(np.exp(rng.uniform(np.log(5.0), np.log(100.0))))
            return np.array(rows), ind.astype(np.float64), contrast
    raise RuntimeError("ellipsoid_rve: no admissible draw")


def ellipsoid_rve(N: int, rng: np.random.Generator, max_tries: int = 400):
    """The RVE of ellipsoid_rve_rows as (indicator, contrast)."""
    _, ind, contrast = ellipsoid_rve_rows(N, rng, max_tries)
    return ind, contrast


def fibre_rve(N: int, rng: np.random.Generator, count: int = 32,
              fibre_fraction: float = 0.3, max_tries: int = 100000) -> np.ndarray:
    """Aligned cylindrical fibres (axis parallel to z), non-overlapping under the
    periodic minimum-image distance, radius chosen so that `count` fibres fill
    `fibre_fraction` of the cell."""
    radius = math.sqrt(fibre_fraction / (count * math.pi))
    centres = []
    for _ in range(max_tries):
        if len(centres) == count:
            break
        p = rng.uniform(0.0, 1.0, size=2)
        ok = True
        for q in centres:
            d = p - q
            d -= np.round(d)
            if d @ d < (2.0 * radius) ** 2:
                ok = False
                break
        if ok:
            centres.append(p)
    if len(centres) < count:
        raise RuntimeError("fibre_rve: could not place all fibres")
    c = voxel_centres(N)
    ind2 = np.zeros((N, N), dtype=bool)
    for p in centres:
        dx = _periodic_delta(c, p[0])[:, None]
        dy = _periodic_delta(c, p[1])[None, :]
        ind2 |= dx * dx + dy * dy <= radius * radius
    return np.broadcast_to(ind2[:, :, None], (N, N, N)).astype(np.float64)


def batched_rve_set(count: int = 64, seed: int = 4, log2_min: int = 6, log2_max: int = 9):
    """The mixed-resolution ellipsoid RVE batch: side 2**u with u uniform in
    [log2_min, log2_max]; RVE i uses the i-th child generator spawned from
    `default_rng(seed)`.  Returns a list of (n_bits, child_rng) pairs; the
    indicator itself is drawn lazily with `ellipsoid_rve(2**n, rng)`."""
    master = np.random.default_rng(seed)
    children = master.spawn(count)
    sizes = master.integers(log2_min, log2_max + 1, size=count)
    return [(int(s), ch) for s, ch in zip(sizes, children)]


# ------------------------------------------------------ isotropic moduli --

def lame_from_young(E: float, nu: float):
    """(lambda, mu) of an isotropic material from Young's modulus and Poisson ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


# ------------------------------------------------------ random TT cores --

def capped_ranks(d: int, p: int, r: int) -> list[int]:
    """Bond ranks r_0..r_d for a uniform target rank r with boundary caps."""
    ranks = [1]
    for k in range(1, d):
        ranks.append(int(min(r, p ** min(k, 30), p ** min(d - k, 30))))
    ranks.append(1)
    return ranks


def random_tt_cores(d: int, p: int, r: int, seed: int, dtype=np.float64,
                    ranks: list[int] | None = None) -> list[np.ndarray]:
    """Gaussian cores N(0,1)/sqrt(r) with shapes (r_{k-1}, p, r_k).

    For complex dtypes the real and imaginary parts are drawn independently
    and scaled by 1/sqrt(2) so that E|z|^2 matches the real case."""
    rng = np.random.default_rng(seed)
    if ranks is None:
        ranks = capped_ranks(d, p, r)
    cores = []
    scale = 1.0 / math.sqrt(r)
    cplx = np.issubdtype(np.dtype(dtype), np.complexfloating)
    for k in range(d):
        shape = (ranks[k], p, ranks[k + 1])
        if cplx:
            a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
            a *= scale / math.sqrt(2.0)
        else:
            a = rng.standard_normal(shape) * scale
        cores.append(a.astype(dtype))
    return cores


def sketch_cores(rng: np.random.Generator, d: int, modes, ell: int):
    """Sketch train of width `ell` for sketched rounding: ranks
    l_k = min(ell, prod of the modes left of bond k, prod right of it); real
    Gaussian cores N(0, 1/(n_k l_{k+1})), except cores whose left rank is the
    full product of the modes to their right (l_k = n_k l_{k+1}), which are
    the identity unfolding (the M x M identity, M = n_k l_{k+1}).  Returns
    (cores, ranks)."""
    ranks = [1]
    left = 1
    for k in range(1, d):
        left = min(left * modes[k - 1], 1 << 60)
        right = 1
        for m in modes[k:]:
            right = min(right * m, 1 << 60)
        ranks.append(int(min(ell, left, right)))
    ranks.append(1)
    cores = []
    for k in range(d):
        M = modes[k] * ranks[k + 1]
        if k > 0 and ranks[k] == M:
            cores.append(np.eye(M).reshape(M, modes[k], ranks[k + 1]))
        else:
            cores.append(rng.standard_normal((ranks[k], modes[k], ranks[k + 1])) / math.sqrt(M))
    return cores, ranks


def random_mpo_cores(d: int, p: int, chi: int, seed: int, dtype=np.complex128) -> list[np.ndarray]:
    """Gaussian operator cores of shape (chi_{k-1}, p_out, p_in, chi_k)."""
    rng = np.random.default_rng(seed)
    ranks = capped_ranks(d, p * p, chi)
    cores = []
    for k in range(d):
        shape = (ranks[k], p, p, ranks[k + 1])
        a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        cores.append((a / math.sqrt(2.0 * chi)).astype(dtype))
    return cores

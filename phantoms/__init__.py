"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module draws volumes, seed masks and label points; it contains none of the
random walker's arithmetic (no weights, no Laplacian, no solve, no pyramid).
Every random number comes from a counter-based hash (splitmix64 of a key derived
from ``(seed, stream)`` xor the element index), so a value depends only on
``(seed, stream, index)``: generation order, slab size and machine do not matter.

Shapes follow the synthetic workloads of the paper (Sec. V-B): "cells" are
spheres/ellipsoids on a darker background, "vessels" are bifurcating cylinders
whose branches split at five radii with area-preserving radii, foreground
labels on the centre line and background labels two radii outside.  The
paper's datasets (CT-ORG, the microscopy volumes) are not available; these
phantoms stand in for them.

Array convention: dense ``[z][y][x]`` (x fastest), numpy shape ``(nz, ny, nx)``.
Seed masks: ``code`` uint8 (0 = free, 1 = seed), ``value`` float32 (seed value).
Label points: continuous leaf-voxel coordinates ``(x, y, z)``; voxel ``i``
covers ``[i, i+1)`` so its centre is ``i + 0.5``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "hash_u64", "uniform", "normal", "Stream",
    "ball_case", "plain_ball", "plain_ellipsoids", "vessel_tree", "adjoint_batch",
    "random_case", "border_faces",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _splitmix_np(z: np.ndarray) -> np.ndarray:
    z = z + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _splitmix_int(z: int) -> int:
    z = (z + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _key(seed: int, stream: int) -> int:
    return _splitmix_int(((seed & 0xFFFFFFFF) << 32) ^ (stream & 0xFFFFFFFF))


def hash_u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """64-bit hash of (seed, stream, idx) — the counter-based generator."""
    with np.errstate(over="ignore"):
        return _splitmix_np(np.uint64(_key(seed, stream)) ^ np.asarray(idx, dtype=np.uint64))


def uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits of the hash."""
    h = hash_u64(seed, stream, idx)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Standard normal by Box-Muller from two independent hash streams."""
    u1 = 1.0 - uniform(seed, 2 * stream + 1000, idx)          # (0, 1]
    u2 = uniform(seed, 2 * stream + 1001, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _hash_torch(seed: int, stream: int, idx):
    """hash_u64 on a torch int64 tensor (two's-complement wrap-around; logical
    shifts emulated with masks): the same bits as the numpy path."""
    import torch

    def srl(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    def s64(v):
        return v - (1 << 64) if v >= (1 << 63) else v

    z = idx ^ s64(_key(seed, stream))
    z = z + s64(0x9E3779B97F4A7C15)
    z = (z ^ srl(z, 30)) * s64(0xBF58476D1CE4E5B9)
    z = (z ^ srl(z, 27)) * s64(0x94D049BB133111EB)
    return z ^ srl(z, 31)


def uniform_torch(seed: int, stream: int, idx):
    return (((_hash_torch(seed, stream, idx) >> 11) & ((1 << 53) - 1)).double()) * (1.0 / 9007199254740992.0)


def normal_torch(seed: int, stream: int, idx):
    import math as _m
    u1 = 1.0 - uniform_torch(seed, 2 * stream + 1000, idx)
    u2 = uniform_torch(seed, 2 * stream + 1001, idx)
    return (-2.0 * u1.log()).sqrt() * (2.0 * _m.pi * u2).cos()


class Stream:
    """Scalar draws from the same counter-based generator (host-side geometry)."""

    def __init__(self, seed: int, stream: int):
        self.key = _key(seed, stream)
        self.i = 0

    def u64(self) -> int:
        v = _splitmix_int(self.key ^ self.i)
        self.i += 1
        return v

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.u64() >> 11) * (1.0 / 9007199254740992.0))

    def normal(self) -> float:
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def unit_vector(self) -> np.ndarray:
        v = np.array([self.normal(), self.normal(), self.normal()])
        return v / max(np.linalg.norm(v), 1e-12)

    def rotation(self) -> np.ndarray:
        q = np.array([self.normal() for _ in range(4)])
        q /= np.linalg.norm(q)
        a, b, c, d = q
        return np.array([
            [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
            [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
            [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
        ])


def _centres(shape):
    nz, ny, nx = shape
    z = np.arange(nz, dtype=np.float64)[:, None, None] + 0.5
    y = np.arange(ny, dtype=np.float64)[None, :, None] + 0.5
    x = np.arange(nx, dtype=np.float64)[None, None, :] + 0.5
    return x, y, z


def border_faces(shape) -> np.ndarray:
    """Boolean mask of the six border faces of a box."""
    m = np.zeros(shape, dtype=bool)
    m[0, :, :] = m[-1, :, :] = True
    m[:, 0, :] = m[:, -1, :] = True
    m[:, :, 0] = m[:, :, -1] = True
    return m


def _voxel_noise(seed, stream, shape, sigma, slab=1 << 22):
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, slab):
        e = min(n, s + slab)
        out[s:e] = sigma * normal(seed, stream, np.arange(s, e, dtype=np.uint64))
    return out.reshape(shape)


def ball_case(n: int = 64, seed: int = 0, radius: float = 20.0, bg: float = 0.3, fg: float = 0.7,
              sigma: float = 0.1, ellipsoid: bool = False, shape=None):
    """Ball (or one random ellipsoid) on a background with i.i.d. Gaussian noise.

    Foreground seeds: a 9-voxel line along x through the centre voxel row
    ``y = z = n // 2``; background seeds: every voxel of the six border faces.
    ``shape`` (z, y, x), when given, replaces the n^3 box: the object is
    centred in it and the seed line runs through its centre row.
    Returns a dict with ``volume`` (float32, clamped to [0, 1]), ``code``,
    ``value`` and the analytic ``mask`` (voxel centre inside the object).
    """
    if shape is None:
        shape = (n, n, n)
    x, y, z = _centres(shape)
    c = n / 2.0
    if shape != (n, n, n):
        cz, cy, cx = (d / 2.0 for d in shape)
        x, y, z = x - (cx - c), y - (cy - c), z - (cz - c)
    if ellipsoid:
        st = Stream(seed, 7)
        R = st.rotation()
        ax = np.array([st.uniform(20.0, 40.0) for _ in range(3)]) * (n / 96.0)
        dx, dy, dz = x - c, y - c, z - c
        q = [R[0, 0] * dx + R[1, 0] * dy + R[2, 0] * dz,
             R[0, 1] * dx + R[1, 1] * dy + R[2, 1] * dz,
             R[0, 2] * dx + R[1, 2] * dy + R[2, 2] * dz]
        mask = (q[0] / ax[0]) ** 2 + (q[1] / ax[1]) ** 2 + (q[2] / ax[2]) ** 2 <= 1.0
    else:
        mask = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 <= radius * radius
    vol = np.where(mask, fg, bg) + _voxel_noise(seed, 1, shape, sigma)
    vol = np.clip(vol, 0.0, 1.0).astype(np.float32)
    code = np.zeros(shape, dtype=np.uint8)
    value = np.zeros(shape, dtype=np.float32)
    code[border_faces(shape)] = 1
    hz, hy, hx = (d // 2 for d in shape)
    a, b = max(hx - 4, 1), min(hx + 5, shape[2] - 1)
    if 0 < hz < shape[0] - 1 and 0 < hy < shape[1] - 1:
        code[hz, hy, a:b] = 1
        value[hz, hy, a:b] = 1.0
    return {"volume": vol, "code": code, "value": value, "mask": mask, "beta": 130.0}


def plain_ball(n: int = 64, seed: int = 0):
    """Plain random walker workload on a 64^3 ball (radius 20, bg 0.3, fg 0.7, sigma 0.1)."""
    return ball_case(n=n, seed=seed, radius=20.0 * n / 64.0)


def pocket_case(n: int = 24, seed: int = 0, n_pairs: int = 6, bridge: float = 0.6075):
    """Weakly attached salt pairs: a numerically hard but determined system.

    Background N(0.3, 0.02), clamped; `n_pairs` pairs of adjacent voxels at 1.0
    (joined by a weight-1 edge at beta = 130), each with one neighbour at
    `bridge` (edge weight exp(-130 (1 - bridge)^2) ~ 2e-9) and all other exits
    at ~1e-28.  The common mode of a pair has a Jacobi-scaled eigenvalue
    ~1e-9: below FP32 resolution, well inside FP64's.  Seeds: the x = 0 face
    (value 0) and the x = n - 1 face (value 1).  Returns the plain-solve dict
    plus ``pairs`` (the (z, y, x) of each pair's first voxel)."""
    shape = (n, n, n)
    vol = np.clip(0.3 + _voxel_noise(seed, 1, shape, 0.02), 0.0, 1.0)
    st = Stream(seed, 11)
    pairs = []
    for _ in range(n_pairs):
        z, y, x = (int(st.uniform(3, n - 4)) for _ in range(3))
        vol[z, y, x] = vol[z, y + 1, x] = 1.0
        vol[z, y, x + 1] = bridge
        pairs.append((z, y, x))
    code = np.zeros(shape, dtype=np.uint8)
    value = np.zeros(shape, dtype=np.float32)
    code[:, :, 0] = code[:, :, -1] = 1
    value[:, :, -1] = 1.0
    return {"volume": vol.astype(np.float32), "code": code, "value": value, "pairs": pairs, "beta": 130.0}


def poisson_ball(n: int = 64, seed: int = 0, lam_fg: float = 100.0, lam_bg: float = 50.0):
    """Photon-count ball for the Poisson weight function: counts with mean
    lam_fg inside a ball of radius 0.3 n, lam_bg outside, drawn as
    round(lam + sqrt(lam) N(0, 1)) clamped at 0 (the normal approximation of
    Poisson noise), uint16.  Seeds as in ball_case (9-voxel foreground line,
    border faces background)."""
    shape = (n, n, n)
    x, y, z = _centres(shape)
    c = n / 2.0
    r = 0.3 * n
    mask = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 <= r * r
    lam = np.where(mask, lam_fg, lam_bg)
    cnt = np.clip(np.rint(lam + np.sqrt(lam) * _voxel_noise(seed, 5, shape, 1.0)), 0, 65535).astype(np.uint16)
    code = np.zeros(shape, dtype=np.uint8)
    value = np.zeros(shape, dtype=np.float32)
    code[border_faces(shape)] = 1
    h = n // 2
    a, b = max(h - 4, 1), min(h + 5, n - 1)
    code[h, h, a:b] = 1
    value[h, h, a:b] = 1.0
    return {"volume": cnt, "code": code, "value": value, "mask": mask}


def _polyline(st: Stream, inside, shape, length=40, max_tries=4000):
    nz, ny, nx = shape
    for _ in range(max_tries):
        p = np.array([st.uniform(0, nx), st.uniform(0, ny), st.uniform(0, nz)])
        if inside(p):
            break
    else:
        return []
    d = st.unit_vector()
    pts = [tuple(np.floor(p).astype(int))]
    pos = p.copy()
    tries = 0
    while len(pts) < length and tries < 50 * length:
        tries += 1
        if tries % 10 == 0:
            d = d + 0.5 * st.unit_vector()
            d /= np.linalg.norm(d)
        nxt = pos + 0.5 * d
        v = tuple(np.floor(nxt).astype(int))
        ok = (0 < v[0] < nx - 1) and (0 < v[1] < ny - 1) and (0 < v[2] < nz - 1) and inside(nxt)
        if not ok:
            d = st.unit_vector()
            continue
        pos = nxt
        if v != pts[-1] and v not in pts:
            pts.append(v)
    return pts


def plain_ellipsoids(n: int = 256, seed: int = 0):
    """Three overlapping random ellipsoids with bias field (the 256^3 plain workload).

    Semi-axes U(20, 80), random rotations, centres within +-30 voxels of the
    volume centre (all scaled by n/256), intensities U(0.55, 0.8) on 0.25, overlaps
    take the maximum, noise sigma 0.08, additive bias b*x/(n-1) with b ~ U(0, 0.1).
    Foreground seeds: 5 polylines of 40 voxels inside ellipsoid 0; background:
    border faces plus 5 polylines of 40 voxels outside ellipsoid 0.
    """
    shape = (n, n, n)
    sc = n / 256.0
    st = Stream(seed, 11)
    x, y, z = _centres(shape)
    c = n / 2.0
    ells = []
    for _ in range(3):
        R = st.rotation()
        ax = np.array([st.uniform(20.0, 80.0) for _ in range(3)]) * sc
        ctr = np.array([c + st.uniform(-30, 30) * sc for _ in range(3)])
        inten = st.uniform(0.55, 0.8)
        ells.append((R, ax, ctr, inten))
    vol = np.full(shape, 0.25, dtype=np.float64)
    masks = []
    for R, ax, ctr, inten in ells:
        dx, dy, dz = x - ctr[0], y - ctr[1], z - ctr[2]
        q0 = R[0, 0] * dx + R[1, 0] * dy + R[2, 0] * dz
        q1 = R[0, 1] * dx + R[1, 1] * dy + R[2, 1] * dz
        q2 = R[0, 2] * dx + R[1, 2] * dy + R[2, 2] * dz
        m = (q0 / ax[0]) ** 2 + (q1 / ax[1]) ** 2 + (q2 / ax[2]) ** 2 <= 1.0
        masks.append(m)
        vol = np.where(m, np.maximum(vol, inten), vol)
    b = st.uniform(0.0, 0.1)
    xi = np.arange(n, dtype=np.float64)[None, None, :]
    vol = vol + _voxel_noise(seed, 2, shape, 0.08) + b * xi / max(n - 1, 1)
    vol = np.clip(vol, 0.0, 1.0).astype(np.float32)

    def ell_inside(p, k=0):
        R, ax, ctr, _ = ells[k]
        q = R.T @ (p - ctr)
        return float(np.sum((q / ax) ** 2)) <= 1.0

    code = np.zeros(shape, dtype=np.uint8)
    value = np.zeros(shape, dtype=np.float32)
    code[border_faces(shape)] = 1
    for _ in range(5):
        for (vx, vy, vz) in _polyline(st, lambda p: ell_inside(p), shape):
            code[vz, vy, vx] = 1
            value[vz, vy, vx] = 1.0
    for _ in range(5):
        for (vx, vy, vz) in _polyline(st, lambda p: not ell_inside(p), shape):
            code[vz, vy, vx] = 1
            value[vz, vy, vx] = 0.0
    return {"volume": vol, "code": code, "value": value, "mask": masks[0], "beta": 130.0}


def _seg_dist2(px, py, pz, a, b):
    ab = b - a
    L2 = float(ab @ ab)
    t = ((px - a[0]) * ab[0] + (py - a[1]) * ab[1] + (pz - a[2]) * ab[2]) / max(L2, 1e-12)
    t = np.clip(t, 0.0, 1.0)
    dx = px - (a[0] + t * ab[0])
    dy = py - (a[1] + t * ab[1])
    dz = pz - (a[2] + t * ab[2])
    return dx * dx + dy * dy + dz * dz


def _vessel_geometry(shape, seed, n_segments, r_max, r_min):
    """Segments, rasterised mask and the geometry stream (it continues into
    the label placement) of the branching vessel tree."""
    nz, ny, nx = shape
    dims = np.array([nx, ny, nz], dtype=np.float64)
    sc = min(dims) / 1024.0
    st = Stream(seed, 21)
    segs = []          # (a, b, r)

    def new_root():
        axis = int(st.uniform(0, 3)) % 3
        side = 0 if st.uniform() < 0.5 else 1
        p = np.array([st.uniform(0.3, 0.7) * dims[i] for i in range(3)])
        p[axis] = 0.5 if side == 0 else dims[axis] - 0.5
        d = np.zeros(3)
        d[axis] = 1.0 if side == 0 else -1.0
        d = d + 0.3 * st.unit_vector()
        return (p, d / np.linalg.norm(d), r_max * max(sc, 0.25))

    queue = [new_root()]
    guard = 0
    while len(segs) < n_segments and guard < 50 * n_segments:
        guard += 1
        if not queue:
            queue.append(new_root())
        a, d, r = queue.pop(0)
        b = a + 5.0 * r * d
        if np.any(b < 0) or np.any(b >= dims):
            continue
        segs.append((a, b, r))
        rc = max(r / math.sqrt(2.0), r_min * max(sc, 0.25))
        perp = np.cross(d, st.unit_vector())
        perp /= max(np.linalg.norm(perp), 1e-12)
        for sgn in (1.0, -1.0):
            ang = math.radians(st.uniform(15.0, 60.0))
            dc = math.cos(ang) * d + sgn * math.sin(ang) * perp
            queue.append((b, dc / np.linalg.norm(dc), rc))

    mask = np.zeros(shape, dtype=bool)
    for a, b, r in segs:
        lo = np.floor(np.minimum(a, b) - r - 1).astype(int)
        hi = np.ceil(np.maximum(a, b) + r + 1).astype(int)
        lo = np.maximum(lo, 0)
        hi = np.minimum(hi, [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        px = np.arange(lo[0], hi[0], dtype=np.float64)[None, None, :] + 0.5
        py = np.arange(lo[1], hi[1], dtype=np.float64)[None, :, None] + 0.5
        pz = np.arange(lo[2], hi[2], dtype=np.float64)[:, None, None] + 0.5
        dist2 = np.minimum(_seg_dist2(px, py, pz, a, b),
                           (px - b[0]) ** 2 + (py - b[1]) ** 2 + (pz - b[2]) ** 2)
        mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= dist2 <= r * r

    return segs, mask, st


def vessel_tree(n=1024, seed=0, n_segments=200, r_max=12.0, r_min=2.0, shape=None,
                fg=(3000.0, 400.0), bg=(800.0, 300.0), salt=0.01, salt_value=5000, device=None):
    """Branching vessel tree phantom (uint16) with labels.

    Breadth-first bifurcation from a root at a random border point: each segment
    has length 5 x radius, splits into two children of radius r/sqrt(2) (area
    preserving, clamped to r_min) at random angles of 15-60 degrees, with a
    sphere at every joint.  Intensities: vessel N(3000, 400), background
    N(800, 300), then a fraction ``salt`` of voxels set to ``salt_value``.
    Labels: two centre-line points per segment (value 1) and two points two
    radii away, outside every vessel (value 0).  Radii and lengths scale with
    n/1024 so that smaller volumes keep the same structure.
    Returns ``volume`` (uint16), ``labels_xyz`` (float64, (N, 3)),
    ``labels_value`` (float32), ``mask`` (bool), ``lo``/``hi`` window (0, 5000).
    """
    if shape is None:
        shape = (n, n, n)
    nz, ny, nx = shape
    dims = np.array([nx, ny, nz], dtype=np.float64)
    segs, mask, st = _vessel_geometry(shape, seed, n_segments, r_max, r_min)

    plane = nx * ny
    if device is not None:
        # same values drawn on the GPU (torch), returned as a uint16 tensor there
        import torch
        vol_t = torch.empty(shape, dtype=torch.int32, device=device)
        mask_t = torch.from_numpy(mask).to(device)
        zslab = max(1, (1 << 25) // plane)
        for z0 in range(0, nz, zslab):
            z1 = min(nz, z0 + zslab)
            idx = torch.arange(z0 * plane, z1 * plane, dtype=torch.int64, device=device)
            gn = normal_torch(seed, 3, idx)
            m = mask_t[z0:z1].reshape(-1)
            v = torch.where(m, fg[0] + fg[1] * gn, bg[0] + bg[1] * gn)
            sl = uniform_torch(seed, 4, idx) < salt
            v = torch.where(sl, torch.full_like(v, float(salt_value)), v)
            vol_t[z0:z1] = v.round().clamp(0, 65535).to(torch.int32).reshape(z1 - z0, ny, nx)
        vol = vol_t.to(torch.uint16) if hasattr(torch, "uint16") else vol_t
    else:
        vol = np.empty(shape, dtype=np.uint16)
    zslab = max(1, (1 << 22) // plane)
    for z0 in (range(0, nz, zslab) if device is None else []):
        z1 = min(nz, z0 + zslab)
        idx = np.arange(z0 * plane, z1 * plane, dtype=np.uint64)
        g = normal(seed, 3, idx)
        m = mask[z0:z1].reshape(-1)
        v = np.where(m, fg[0] + fg[1] * g, bg[0] + bg[1] * g)
        s = uniform(seed, 4, idx) < salt
        v = np.where(s, float(salt_value), v)
        vol[z0:z1] = np.clip(np.rint(v), 0, 65535).astype(np.uint16).reshape(z1 - z0, ny, nx)

    def outside_all(p):
        for a, b, r in segs:
            if _seg_dist2(p[0], p[1], p[2], a, b) <= (r + 1.0) ** 2:
                return False
        return True

    lx, lv = [], []
    for a, b, r in segs:
        for t in (1.0 / 3.0, 2.0 / 3.0):
            lx.append(a + t * (b - a))
            lv.append(1.0)
        mid = 0.5 * (a + b)
        d = (b - a) / max(np.linalg.norm(b - a), 1e-12)
        placed = 0
        for _ in range(24):
            if placed == 2:
                break
            perp = np.cross(d, st.unit_vector())
            nrm = np.linalg.norm(perp)
            if nrm < 1e-6:
                continue
            q = mid + 2.0 * r * perp / nrm
            if np.all(q >= 0.5) and np.all(q < dims - 0.5) and outside_all(q):
                lx.append(q)
                lv.append(0.0)
                placed += 1
    return {"volume": vol, "labels_xyz": np.array(lx, dtype=np.float64).reshape(-1, 3),
            "labels_value": np.array(lv, dtype=np.float32), "mask": mask,
            "lo": 0.0, "hi": 5000.0, "beta": 130.0, "segments": segs}


def multiclass_case(shape=(128, 128, 128), seed=0, n_segments=40, n_blobs=60, strokes_per_class=3,
                    stroke_len=200, n_updates=10, device=None):
    """Three-class phantom for multi-class labelling (shape z, y, x).

    Classes: 0 background, 1 branching vessel tree (as in vessel_tree, radii
    scaled with the smallest dim), 2 cell blobs (random rotated ellipsoids,
    semi-axes U(4, 15) times min(max(4 m / 1024, 0.5), 4) for the smallest
    dim m -- large enough to hold a 200-voxel stroke from m = 1024 on --
    vessels take precedence).  Intensities per
    class N(800, 250), N(3000, 250), N(2000, 250) (sigma = 5 % of the window
    [0, 5000]), rounded to uint16.  Strokes: `strokes_per_class` polylines of
    `stroke_len` voxels inside each class, then `n_updates` further strokes
    in random classes (for incremental updates).  Each stroke is (xyz voxel
    centres (L, 3) float64, class).  Returns ``volume`` (uint16, a torch
    tensor on `device` when given), ``classes`` (uint8), ``strokes``,
    ``updates``, ``lo``/``hi``."""
    nz, ny, nx = shape
    segs, vmask, _ = _vessel_geometry(shape, seed, n_segments, 12.0, 2.0)
    classes = np.zeros(shape, dtype=np.uint8)
    st = Stream(seed, 31)
    sc = min(shape) / 1024.0
    for _ in range(n_blobs):
        c = np.array([st.uniform(0, nx), st.uniform(0, ny), st.uniform(0, nz)])
        ax = np.array([st.uniform(4.0, 15.0) for _ in range(3)]) * min(max(sc * 4.0, 0.5), 4.0)
        R = st.rotation()
        r = float(ax.max())
        lo = np.maximum(np.floor(c - r - 1).astype(int), 0)
        hi = np.minimum(np.ceil(c + r + 1).astype(int), [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        px = np.arange(lo[0], hi[0], dtype=np.float64)[None, None, :] + 0.5 - c[0]
        py = np.arange(lo[1], hi[1], dtype=np.float64)[None, :, None] + 0.5 - c[1]
        pz = np.arange(lo[2], hi[2], dtype=np.float64)[:, None, None] + 0.5 - c[2]
        q = [R[0, k] * px + R[1, k] * py + R[2, k] * pz for k in range(3)]
        inside = (q[0] / ax[0]) ** 2 + (q[1] / ax[1]) ** 2 + (q[2] / ax[2]) ** 2 <= 1.0
        sub = classes[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = 2
    classes[vmask] = 1
    means = np.array([800.0, 3000.0, 2000.0])
    plane = nx * ny
    if device is not None:
        import torch
        cl_t = torch.from_numpy(classes).to(device)
        mean_t = torch.tensor(means, device=device)
        vol_t = torch.empty(shape, dtype=torch.int32, device=device)
        zslab = max(1, (1 << 25) // plane)
        for z0 in range(0, nz, zslab):
            z1 = min(nz, z0 + zslab)
            idx = torch.arange(z0 * plane, z1 * plane, dtype=torch.int64, device=device)
            v = mean_t[cl_t[z0:z1].reshape(-1).long()] + 250.0 * normal_torch(seed, 3, idx)
            vol_t[z0:z1] = v.round().clamp(0, 65535).to(torch.int32).reshape(z1 - z0, ny, nx)
        vol = vol_t.to(torch.uint16) if hasattr(torch, "uint16") else vol_t
    else:
        vol = np.empty(shape, dtype=np.uint16)
        zslab = max(1, (1 << 22) // plane)
        for z0 in range(0, nz, zslab):
            z1 = min(nz, z0 + zslab)
            idx = np.arange(z0 * plane, z1 * plane, dtype=np.uint64)
            v = means[classes[z0:z1].reshape(-1)] + 250.0 * normal(seed, 3, idx)
            vol[z0:z1] = np.clip(np.rint(v), 0, 65535).astype(np.uint16).reshape(z1 - z0, ny, nx)
    ss = Stream(seed, 41)

    def stroke(c):
        inside = lambda p: classes[int(p[2]), int(p[1]), int(p[0])] == c
        pts = _polyline(ss, inside, shape, length=stroke_len)
        return np.array([(x + 0.5, y + 0.5, z + 0.5) for (x, y, z) in pts], dtype=np.float64).reshape(-1, 3)

    strokes = [(stroke(c), c) for c in range(3) for _ in range(strokes_per_class)]
    updates = []
    for _ in range(n_updates):
        c = int(ss.uniform(0, 3)) % 3
        updates.append((stroke(c), c))
    return {"volume": vol, "classes": classes, "strokes": strokes, "updates": updates, "lo": 0.0, "hi": 5000.0,
            "beta": 130.0}


def class_labels(strokes, c):
    """Labels of the class-c problem: (xyz, value, class) with class-c stroke
    points 1 and the others 0."""
    if not strokes:
        return np.zeros((0, 3)), np.zeros(0, dtype=np.float32), np.zeros(0, dtype=np.int32)
    xyz = np.concatenate([s for s, _ in strokes], axis=0)
    val = np.concatenate([np.full(len(s), 1.0 if k == c else 0.0, dtype=np.float32) for s, k in strokes])
    cls = np.concatenate([np.full(len(s), k, dtype=np.int32) for s, k in strokes])
    return xyz, val, cls


def adjoint_batch(n: int = 96, batch: int = 32, seed0: int = 0):
    """Batch for the differentiable solve: ball (even seeds, r = 30 n/96) or one
    random ellipsoid (odd seeds, semi-axes U(20, 40) n/96), config-1 seeding."""
    vols, codes, values, masks = [], [], [], []
    for b in range(batch):
        s = seed0 + b
        c = ball_case(n=n, seed=s, radius=30.0 * n / 96.0, ellipsoid=(s % 2 == 1))
        vols.append(c["volume"]); codes.append(c["code"]); values.append(c["value"]); masks.append(c["mask"])
    return {"volume": np.stack(vols), "code": np.stack(codes), "value": np.stack(values),
            "mask": np.stack(masks), "beta": 130.0}


def random_case(shape, seed: int = 0, seed_frac: float = 0.1, beta: float = 30.0, levels=None):
    """Small random volume with random seeds (values 0/1, or in [0, 1] when
    ``levels`` is None and seed values are drawn continuously)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint64)
    vol = uniform(seed, 51, idx).reshape(shape).astype(np.float32)
    is_seed = uniform(seed, 52, idx) < seed_frac
    if not is_seed.any():
        is_seed[0] = True
    if levels is None:
        val = uniform(seed, 53, idx)
    else:
        val = np.asarray(levels, dtype=np.float64)[(hash_u64(seed, 54, idx) % np.uint64(len(levels))).astype(np.int64)]
    code = is_seed.reshape(shape).astype(np.uint8)
    value = np.where(is_seed, val, 0.0).reshape(shape).astype(np.float32)
    return {"volume": vol, "code": code, "value": value, "beta": beta}

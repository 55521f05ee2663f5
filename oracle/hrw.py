"""Hierarchical random walker H / H_p — oracle (TEST INFRASTRUCTURE ONLY).

Plain Python/numpy driver over the FP64 brick solve ``oracle.rw_solve``.
Steps follow the paper in order:

* Sec. III-A — LOD pyramid, bricks of s^3 voxels, uneven border bricks (Sec. IV-A).
* Eq. 1 — the root is the plain random walker on the coarsest level with the
  transformed labels T_n(l).
* Eq. 2 / Eq. 3 — every other node is solved on its neighbourhood N(n) of side
  s_e = floor(e s) with user seeds plus continuous seeds sampled from the
  parent level on the border of N(n); the result is contracted back (N^-1).
* Sec. IV-D1 — hom, dt, cfl, prunable and H_p; sampling through pruned holes
  falls back to the nearest transitive parent (here: the filled field of the
  previous level, which already holds that parent's upsampled values).
* Sec. IV-D2 — each solve starts from the upsampled parent solution.
* Sec. IV-E — incremental labelling: re-solve top-down, keep the old node and
  its whole subtree where the new result is similar (max |diff| < t_inc) and no
  conflict involves an added label.

Readings of points the paper leaves open (each mirrored by the CUDA path):
* label point q (leaf coordinates, voxel i spans [i, i+1)) rasterises at
  level k to voxel floor(q / 2^(K-k)); equal voxel + different values =
  conflict, the voxel stays unseeded;
* expansion margins m_lo = floor((s_e - s)/2), m_hi = s_e - s - m_lo, box clipped
  to the level volume; border seeds on the one-voxel outer layer of the clipped
  box, only on faces that are not on the volume boundary; user seeds override
  border seeds;
* upsampling is trilinear at u = (i + 0.5)/2 - 0.5 with clamp-to-edge;
* a node whose box holds no seed at all keeps its initial guess.

Pins (tests/test_oracle_hier_pins.py): every node problem, decision and
field of tiny trees (s = 4 with e = 1.25, 1.5, 1.75; uneven dims; conflicts;
user seeds on border layers; hom and dt pruning; absent nodes) and of
incremental passes is rebuilt there independently -- neighbourhoods as index
ranges, the border layer as the voxels with a neighbour outside N(n), the
upsampling as tent functions, every node solved by dense Cholesky -- and must
match this module to 1e-12 and decision for decision; hand cases fix the
margins, the strict hom / dt predicates, a conflict with an added label that
forces a re-solve, and a similar node whose subtree is kept bit for bit while
its siblings re-solve; planted one-line mistakes in margins, _region,
_solve_node (border faces, precedence), upsample, _flags and update each fail
them.  The readings themselves (trilinear upsampling, the border layer, the
fill of pruned holes, similarity against the filled old field) are choices
where the paper is silent; the pins fix that this module computes them as
stated above.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ABSENT, FREE, SEED, W_MIN, rw_solve


@dataclass
class Opts:
    brick_size: int = 32
    expand: float = 1.25
    beta: float = 130.0
    w_min: float = W_MIN
    t_hom: float = 0.3
    t_bin: float = 0.01
    t_inc: float = 0.01
    prune_hom: bool = True
    prune_dt: bool = True
    tol: float = 1e-13
    max_iter: int = 200000
    weight: str = "gaussian"    # edge weight function (oracle.rw_solve kind)


@dataclass
class NodeInfo:
    solved: bool = False
    mn: float = 0.0
    mx: float = 0.0
    hom: bool = False
    dt: bool = False
    cfl: bool = False
    cfl_added: bool = False
    prunable: bool = False
    similar: bool = False
    maxdiff: float = 0.0
    iters: int = 0
    free: int = 0


@dataclass
class Tree:
    levels: list                # FP32 intensity levels, root .. leaf
    P: list                     # filled FP64 probability fields, root .. leaf
    info: list                  # per level: dict brick index -> NodeInfo
    labels_xyz: np.ndarray
    labels_value: np.ndarray
    opts: Opts
    stats: dict = field(default_factory=dict)
    labels_cls: np.ndarray | None = None   # class of each label (multi-class), or None


def margins(s: int, e: float):
    se = int(np.floor(e * s))
    m_lo = (se - s) // 2
    return se, m_lo, se - s - m_lo


def brick_counts(shape, s):
    return tuple((d + s - 1) // s for d in shape)


def upsample(prev: np.ndarray, shape) -> np.ndarray:
    """Trilinear upsample of level k-1 onto the voxel grid of level k
    (u = (i + 0.5)/2 - 0.5 per axis, clamp-to-edge), separable, FP64."""
    out = np.asarray(prev, dtype=np.float64)
    for axis in range(3):
        n_out = shape[axis]
        n_in = out.shape[axis]
        i = np.arange(n_out, dtype=np.float64)
        u = (i + 0.5) / 2.0 - 0.5
        i0 = np.floor(u)
        t = u - i0
        ia = np.clip(i0.astype(np.int64), 0, n_in - 1)
        ib = np.clip(i0.astype(np.int64) + 1, 0, n_in - 1)
        a = np.take(out, ia, axis=axis)
        b = np.take(out, ib, axis=axis)
        sh = [1, 1, 1]
        sh[axis] = n_out
        t = t.reshape(sh)
        out = (1.0 - t) * a + t * b
    return out


def rasterize(xyz: np.ndarray, val: np.ndarray, K: int, k: int, shape, added=None, cls=None):
    """T_k of Sec. IV-A: map label points to level-k voxels.  A voxel holding
    labels of different values (or, with `cls`, of different classes: the
    multi-class reading, the same unseeded voxels in every class problem) is
    a conflict.  Returns (seeds: {(z,y,x): value}, conflicts: {(z,y,x):
    involves_added})."""
    scale = 2.0 ** (-(K - k))
    groups = {}
    for n in range(len(val)):
        v = np.floor(np.asarray(xyz[n], dtype=np.float64) * scale).astype(np.int64)
        x, y, z = int(v[0]), int(v[1]), int(v[2])
        if not (0 <= x < shape[2] and 0 <= y < shape[1] and 0 <= z < shape[0]):
            continue
        groups.setdefault((z, y, x), []).append((float(val[n]), bool(added[n]) if added is not None else False,
                                                 int(cls[n]) if cls is not None else -1))
    seeds, conflicts = {}, {}
    for key, items in groups.items():
        vals = {a for a, _, _ in items}
        classes = {c for _, _, c in items if c >= 0}
        if len(vals) == 1 and len(classes) <= 1:
            seeds[key] = items[0][0]
        else:
            conflicts[key] = any(f for _, f, _ in items)
    return seeds, conflicts


def _region(b, shape, s, se, m_lo, m_hi):
    """Brick box and clipped expanded box R (per axis z, y, x): (lo, hi)."""
    box, reg = [], []
    for a in range(3):
        lo = b[a] * s
        hi = min(lo + s, shape[a])
        box.append((lo, hi))
        reg.append((max(lo - m_lo, 0), min(lo + s + m_hi, shape[a])))
    return box, reg


def _solve_node(k, b, level, Up, init, seeds, conflicts, opts, shape):
    s = opts.brick_size
    se, m_lo, m_hi = margins(s, opts.expand)
    box, reg = _region(b, shape, s, se, m_lo, m_hi)
    (z0, z1), (y0, y1), (x0, x1) = reg
    g = np.asarray(level[z0:z1, y0:y1, x0:x1], dtype=np.float64)
    code = np.full(g.shape, FREE, dtype=np.uint8)
    xin = np.array(init[z0:z1, y0:y1, x0:x1], dtype=np.float64)
    if Up is not None:
        # continuous border seeds (Eq. 2, Eq. 3): the outer layer of R on
        # faces that lie inside the level volume
        upr = Up[z0:z1, y0:y1, x0:x1]
        lay = np.zeros(g.shape, dtype=bool)
        if z0 > 0: lay[0, :, :] = True
        if z1 < shape[0]: lay[-1, :, :] = True
        if y0 > 0: lay[:, 0, :] = True
        if y1 < shape[1]: lay[:, -1, :] = True
        if x0 > 0: lay[:, :, 0] = True
        if x1 < shape[2]: lay[:, :, -1] = True
        code[lay] = SEED
        xin[lay] = upr[lay]
    cfl = False
    cfl_added = False
    for (z, y, x), added_flag in conflicts.items():
        if z0 <= z < z1 and y0 <= y < y1 and x0 <= x < x1:
            cfl = True
            cfl_added = cfl_added or added_flag
    for (z, y, x), v in seeds.items():
        if z0 <= z < z1 and y0 <= y < y1 and x0 <= x < x1:
            code[z - z0, y - y0, x - x0] = SEED
            xin[z - z0, y - y0, x - x0] = v
    if not np.any(code == SEED):
        x = xin.copy()
        iters = 0
    else:
        x, iters, _, st = rw_solve(g, code, xin, opts.beta, w_min=opts.w_min, tol=opts.tol,
                                   max_iter=opts.max_iter, kind=opts.weight)
    (bz0, bz1), (by0, by1), (bx0, bx1) = box
    out = x[bz0 - z0:bz1 - z0, by0 - y0:by1 - y0, bx0 - x0:bx1 - x0]
    nfree = int(np.count_nonzero(code == FREE))
    return out, box, cfl, cfl_added, iters, nfree


def _flags(out, cfl, opts, info):
    mn, mx = float(out.min()), float(out.max())
    info.mn, info.mx = mn, mx
    info.hom = (mx - mn) < opts.t_hom                                   # Sec. IV-D1, hom
    info.dt = (mn - 0.5 > opts.t_bin) or (0.5 - mx > opts.t_bin)        # Sec. IV-D1, dt
    info.cfl = cfl
    info.prunable = ((info.hom and opts.prune_hom) or (info.dt and opts.prune_dt)) and not cfl


def _children(b, shape_next, s):
    nb = brick_counts(shape_next, s)
    out = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = (2 * b[0] + dz, 2 * b[1] + dy, 2 * b[2] + dx)
                if c[0] < nb[0] and c[1] < nb[1] and c[2] < nb[2]:
                    out.append(c)
    return out


def run(levels, labels_xyz, labels_value, opts: Opts | None = None, labels_cls=None) -> Tree:
    """Full top-down run of H_p (Eqs. 1-3 with pruning).  Returns the tree with
    the filled probability field of every level; P[-1] is the result."""
    opts = opts or Opts()
    K = len(levels) - 1
    s = opts.brick_size
    P, info = [], []
    active = [(0, 0, 0)]
    st = {"bricks_solved": 0, "bricks_pruned": 0, "bricks_conflict": 0, "voxel_iters": 0}
    for k in range(K + 1):
        shape = levels[k].shape
        Up = upsample(P[k - 1], shape) if k > 0 else None
        seeds, conflicts = rasterize(labels_xyz, labels_value, K, k, shape, cls=labels_cls)
        Pk = Up.copy() if Up is not None else np.zeros(shape, dtype=np.float64)
        init = Pk.copy()
        lvl = {}
        nxt = []
        for b in sorted(active):
            out, box, cfl, _, iters, nfree = _solve_node(k, b, levels[k], Up, init, seeds, conflicts, opts, shape)
            (z0, z1), (y0, y1), (x0, x1) = box
            Pk[z0:z1, y0:y1, x0:x1] = out
            ni = NodeInfo(solved=True, iters=iters, free=nfree)
            _flags(out, cfl, opts, ni)
            lvl[b] = ni
            st["bricks_solved"] += 1
            st["bricks_pruned"] += int(ni.prunable)
            st["bricks_conflict"] += int(cfl)
            st["voxel_iters"] += iters * nfree
            if k < K and not ni.prunable:
                nxt.extend(_children(b, levels[k + 1].shape, s))
        P.append(Pk)
        info.append(lvl)
        active = sorted(set(nxt))
    return Tree(levels=levels, P=P, info=info, labels_xyz=np.asarray(labels_xyz, dtype=np.float64).reshape(-1, 3),
                labels_value=np.asarray(labels_value, dtype=np.float64), opts=opts, stats=st,
                labels_cls=None if labels_cls is None else np.asarray(labels_cls, dtype=np.int64).reshape(-1))


def update(old: Tree, add_xyz, add_value, add_cls=None) -> Tree:
    """Incremental labelling (Sec. IV-E).  The root is re-solved (initialised
    with the old root); at every level the children of re-solved nodes that are
    neither similar nor prunable are re-solved (initialised with the old filled
    field); a similar node keeps its old values and its whole old subtree."""
    opts = old.opts
    levels = old.levels
    K = len(levels) - 1
    s = opts.brick_size
    add_xyz = np.asarray(add_xyz, dtype=np.float64).reshape(-1, 3)
    add_value = np.asarray(add_value, dtype=np.float64).reshape(-1)
    xyz = np.concatenate([old.labels_xyz, add_xyz])
    val = np.concatenate([old.labels_value, add_value])
    added = np.concatenate([np.zeros(len(old.labels_value), bool), np.ones(len(add_value), bool)])
    cls = None
    if old.labels_cls is not None or add_cls is not None:
        oc = old.labels_cls if old.labels_cls is not None else np.full(len(old.labels_value), -1)
        ac = np.asarray(add_cls).reshape(-1) if add_cls is not None else np.full(len(add_value), -1)
        cls = np.concatenate([oc, ac]).astype(np.int64)
    P, info = [], []
    resolve = [(0, 0, 0)]
    reused = []
    st = {"bricks_solved": 0, "bricks_pruned": 0, "bricks_reused": 0, "bricks_conflict": 0, "voxel_iters": 0}
    for k in range(K + 1):
        shape = levels[k].shape
        Up = upsample(P[k - 1], shape) if k > 0 else None
        seeds, conflicts = rasterize(xyz, val, K, k, shape, added, cls)
        Pk = Up.copy() if Up is not None else np.zeros(shape, dtype=np.float64)
        Pold = old.P[k]
        for b in reused:
            box, _ = _region(b, shape, s, *margins(s, opts.expand))
            (z0, z1), (y0, y1), (x0, x1) = box
            Pk[z0:z1, y0:y1, x0:x1] = Pold[z0:z1, y0:y1, x0:x1]
        lvl = {}
        nxt_resolve, nxt_reused = [], []
        for b in reused:
            lvl[b] = NodeInfo(solved=False)
            st["bricks_reused"] += 1
            if k < K:
                nxt_reused.extend(_children(b, levels[k + 1].shape, s))
        for b in sorted(resolve):
            out, box, cfl, cfl_added, iters, nfree = _solve_node(k, b, levels[k], Up, Pold, seeds, conflicts,
                                                                opts, shape)
            (z0, z1), (y0, y1), (x0, x1) = box
            ni = NodeInfo(solved=True, iters=iters, free=nfree)
            _flags(out, cfl, opts, ni)
            ni.cfl_added = cfl_added
            prev = Pold[z0:z1, y0:y1, x0:x1]
            ni.maxdiff = float(np.max(np.abs(out - prev)))
            ni.similar = (ni.maxdiff < opts.t_inc) and not cfl_added
            st["bricks_solved"] += 1
            st["voxel_iters"] += iters * nfree
            st["bricks_conflict"] += int(cfl)
            if ni.similar:
                Pk[z0:z1, y0:y1, x0:x1] = prev
                if k < K:
                    nxt_reused.extend(_children(b, levels[k + 1].shape, s))
            else:
                Pk[z0:z1, y0:y1, x0:x1] = out
                st["bricks_pruned"] += int(ni.prunable)
                if k < K and not ni.prunable:
                    nxt_resolve.extend(_children(b, levels[k + 1].shape, s))
            lvl[b] = ni
        P.append(Pk)
        info.append(lvl)
        resolve = sorted(set(nxt_resolve))
        reused = sorted(set(nxt_reused))
    return Tree(levels=levels, P=P, info=info, labels_xyz=xyz, labels_value=val, opts=opts, stats=st,
                labels_cls=cls)

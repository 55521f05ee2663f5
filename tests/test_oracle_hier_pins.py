"""Independent pins of the oracle's hierarchical procedure on tiny trees.

Every node problem of H_p (Eqs. 1-3), its pruning statistics (Sec. IV-D1), the
fill of absent nodes and the incremental pass (Sec. IV-E) are rebuilt here from
the definitions alone, with constructions that differ from the oracle's:

* the neighbourhood N(n) (Eq. 3) as per-axis index ranges, s_e = floor(e s)
  voxels wide with the brick centred (the odd voxel of the split on the high
  side), clipped to the level;
* the continuous border seeds (Eq. 2) as the voxels of N(n) that have a
  6-neighbour inside the level but outside N(n) -- so faces on the volume
  boundary carry none -- valued by the upsampled parent field;
* the upsampling as a matrix of tent (hat) functions centred on the coarse
  voxel centres, the fine centre clamped to the outermost coarse centres
  (the oracle lerps between floor/ceil indices);
* label rasterisation T_k by integer shifts of floor(q);
* user seeds override border seeds; a voxel holding labels of different
  values is unseeded (cfl);
* children as the next-level bricks whose index halves to the parent's;
* every node solved directly: the Dirichlet energy's normal equations on the
  free voxels, by dense Cholesky (the oracle uses Jacobi-PCG).

The tiny trees (s = 4, e = 1.25 -> s_e = 5 with margins 0 / 1; e = 1.5 and
1.75 for symmetric and 1 / 2 margins; uneven dims) are small enough for dense
solves.  The oracle's fields must agree to 1e-12 at every level and its node
decisions exactly.  A last test plants one-line mistakes in the oracle and
checks that these pins catch each of them.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

import oracle as O
import phantoms as P
from oracle import hrw

W_MIN = 1e-30
FIELD_TOL = 1e-12
MARGIN = 1e-9        # a statistic this close to its threshold would make the case fragile


# ----------------------------------------------------------------------------
# the independent restatement
# ----------------------------------------------------------------------------

def dense_dirichlet(g, is_seed, seed_val, beta, w_min=W_MIN):
    """Minimiser of 1/2 sum_edges w_pq (x_p - x_q)^2 with x fixed on the seeds
    (Sec. III-B), w_pq = max(exp(-beta (g_p - g_q)^2), w_min) over the
    6-neighbour pairs of the box.  Solved by Cholesky on the free voxels."""
    g = np.asarray(g, dtype=np.float64)
    n = g.size
    idx = np.arange(n).reshape(g.shape)
    L = np.zeros((n, n))
    for axis in range(3):
        a = np.take(idx, np.arange(g.shape[axis] - 1), axis=axis).ravel()
        b = np.take(idx, np.arange(1, g.shape[axis]), axis=axis).ravel()
        w = np.maximum(np.exp(-beta * (g.ravel()[a] - g.ravel()[b]) ** 2), w_min)
        np.add.at(L, (a, a), w)
        np.add.at(L, (b, b), w)
        np.add.at(L, (a, b), -w)
        np.add.at(L, (b, a), -w)
    fix = np.asarray(is_seed, bool).ravel()
    fr = ~fix
    xm = np.asarray(seed_val, dtype=np.float64).ravel()[fix]
    x = np.zeros(n)
    x[fix] = xm
    if fr.any():
        c = np.linalg.cholesky(L[np.ix_(fr, fr)])
        rhs = -L[np.ix_(fr, fix)] @ xm
        x[fr] = np.linalg.solve(c.T, np.linalg.solve(c, rhs))
    return x.reshape(g.shape)


def tent_upsample(coarse, shape):
    """Voxel-centre aligned linear interpolation of the parent level onto the
    next level's grid, one axis at a time, as a matrix of hat functions."""
    out = np.asarray(coarse, dtype=np.float64)
    for axis in range(3):
        nc, nf = out.shape[axis], shape[axis]
        u = np.clip((np.arange(nf) + 0.5) / 2.0, 0.5, nc - 0.5)        # fine centre, coarse units
        W = np.maximum(0.0, 1.0 - np.abs(u[:, None] - (np.arange(nc) + 0.5)[None, :]))
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, axis, 0), axes=1), 0, axis)
    return out


def raster(xyz, val, cls, added, shift, shape):
    """Labels at a level `shift` halvings above the leaf: voxel floor(q) >> shift.
    Returns ({voxel: value} of unconflicted voxels, {voxel: conflict involves an
    added label})."""
    per = {}
    for n in range(len(val)):
        v = tuple(int(math.floor(c)) >> shift for c in xyz[n][::-1])          # (z, y, x)
        if all(0 <= v[a] < shape[a] for a in range(3)):
            per.setdefault(v, []).append((float(val[n]), -1 if cls is None else int(cls[n]), bool(added[n])))
    seeds, cfl = {}, {}
    for v, items in per.items():
        if len({it[0] for it in items}) == 1 and len({it[1] for it in items}) == 1:
            seeds[v] = items[0][0]
        else:
            cfl[v] = any(it[2] for it in items)
    return seeds, cfl


def brick_ranges(b, shape, s):
    return [range(b[a] * s, min(b[a] * s + s, shape[a])) for a in range(3)]


def hood_ranges(b, shape, s, e):
    """N(n): s_e = floor(e s) voxels per axis around the brick, the brick
    centred and the odd voxel of the split on the high side, clipped."""
    se = int(math.floor(e * s))
    lo_pad = (se - s) // 2
    return [range(max(b[a] * s - lo_pad, 0), min(b[a] * s - lo_pad + se, shape[a])) for a in range(3)]


def outer_layer(reg, shape):
    """Voxels of the box `reg` with a 6-neighbour inside the level but outside the box."""
    inside = np.zeros(shape, bool)
    inside[reg[0].start:reg[0].stop, reg[1].start:reg[1].stop, reg[2].start:reg[2].stop] = True
    lay = np.zeros(shape, bool)
    for a in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        lo, hi = tuple(lo), tuple(hi)
        lay[lo] |= inside[lo] & ~inside[hi]
        lay[hi] |= inside[hi] & ~inside[lo]
    return lay[reg[0].start:reg[0].stop, reg[1].start:reg[1].stop, reg[2].start:reg[2].stop]


def node_problem(k, b, g_level, up, init, seeds, cfl, s, e, beta):
    """Solve node b of level k on N(b); return (values on the brick, cfl, cfl_added,
    border-seed voxels that a user seed replaced)."""
    shape = g_level.shape
    reg = hood_ranges(b, shape, s, e)
    sl = tuple(slice(r.start, r.stop) for r in reg)
    is_seed = np.zeros(g_level[sl].shape, bool)
    val = np.array(init[sl], dtype=np.float64)
    if k > 0:
        lay = outer_layer(reg, shape)
        is_seed |= lay
        val[lay] = up[sl][lay]
    else:
        lay = np.zeros(is_seed.shape, bool)
    overridden = 0
    has_cfl = has_cfl_added = False
    for (z, y, x), added in cfl.items():
        if z in reg[0] and y in reg[1] and x in reg[2]:
            has_cfl = True
            has_cfl_added |= added
    for (z, y, x), v in seeds.items():
        if z in reg[0] and y in reg[1] and x in reg[2]:
            p = (z - reg[0].start, y - reg[1].start, x - reg[2].start)
            overridden += int(lay[p] and val[p] != v)
            is_seed[p] = True
            val[p] = v
    x = dense_dirichlet(g_level[sl], is_seed, val, beta) if is_seed.any() else val
    br = brick_ranges(b, shape, s)
    out = x[br[0].start - reg[0].start:br[0].stop - reg[0].start,
            br[1].start - reg[1].start:br[1].stop - reg[1].start,
            br[2].start - reg[2].start:br[2].stop - reg[2].start]
    return out, has_cfl, has_cfl_added, overridden


def decide(out, has_cfl, o):
    mn, mx = float(out.min()), float(out.max())
    hom = (mx - mn) < o.t_hom
    dt = bool(np.all(out > 0.5 + o.t_bin) or np.all(out < 0.5 - o.t_bin))
    prunable = ((hom and o.prune_hom) or (dt and o.prune_dt)) and not has_cfl
    # the case must not sit on a threshold (strictness is pinned by hand cases)
    for stat, thr in ((mx - mn, o.t_hom), (mn - 0.5, o.t_bin), (0.5 - mx, o.t_bin)):
        assert abs(stat - thr) > MARGIN, "tiny-tree case too close to a pruning threshold"
    return {"hom": hom, "dt": dt, "cfl": has_cfl, "prunable": prunable}


def bricks_of(shape, s):
    n = [(d + s - 1) // s for d in shape]
    return [(z, y, x) for z in range(n[0]) for y in range(n[1]) for x in range(n[2])]


def put(field, b, s, vals):
    br = brick_ranges(b, field.shape, s)
    field[br[0].start:br[0].stop, br[1].start:br[1].stop, br[2].start:br[2].stop] = vals


def take(field, b, s):
    br = brick_ranges(b, field.shape, s)
    return field[br[0].start:br[0].stop, br[1].start:br[1].stop, br[2].start:br[2].stop]


def tiny_run(levels, xyz, val, o, cls=None):
    """H_p top down: root (Eq. 1), then the children of solved, non-prunable
    nodes (Eqs. 2-3); absent nodes take the upsampled parent field."""
    K = len(levels) - 1
    added = np.zeros(len(val), bool)
    fields, nodes, overridden = [], [], 0
    active = {(0, 0, 0)}
    for k in range(K + 1):
        shape = levels[k].shape
        up = tent_upsample(fields[-1], shape) if k else np.zeros(shape)
        seeds, cfl = raster(xyz, val, cls, added, K - k, shape)
        f = up.copy()
        info = {}
        for b in sorted(active):
            out, c, ca, ov = node_problem(k, b, levels[k], up, up, seeds, cfl, o.brick_size, o.expand, o.beta)
            overridden += ov
            put(f, b, o.brick_size, out)
            info[b] = decide(out, c, o)
        fields.append(f)
        nodes.append(info)
        if k < K:
            active = {c for c in bricks_of(levels[k + 1].shape, o.brick_size)
                      if tuple(v // 2 for v in c) in info and not info[tuple(v // 2 for v in c)]["prunable"]}
    return fields, nodes, overridden


def tiny_update(levels, old_fields, xyz, val, n_old, o, cls=None):
    """Sec. IV-E: re-solve from the root; a re-solved node whose new values
    differ from the old filled field by less than t_inc everywhere on its
    brick, and whose neighbourhood holds no conflict involving an added label,
    keeps its old values and its whole old subtree; otherwise its new values
    are stored and its children re-solved unless it is prunable."""
    K = len(levels) - 1
    added = np.arange(len(val)) >= n_old
    fields, nodes = [], []
    redo, keep = {(0, 0, 0)}, set()
    for k in range(K + 1):
        shape = levels[k].shape
        up = tent_upsample(fields[-1], shape) if k else np.zeros(shape)
        seeds, cfl = raster(xyz, val, cls, added, K - k, shape)
        old = old_fields[k]
        f = up.copy()
        info = {}
        for b in keep:
            put(f, b, o.brick_size, take(old, b, o.brick_size))
            info[b] = {"reused": True}
        next_redo, next_keep = set(), set()
        for b in sorted(redo):
            out, c, ca, _ = node_problem(k, b, levels[k], up, old, seeds, cfl, o.brick_size, o.expand, o.beta)
            d = decide(out, c, o)
            d["maxdiff"] = float(np.max(np.abs(out - take(old, b, o.brick_size))))
            assert abs(d["maxdiff"] - o.t_inc) > MARGIN
            d["cfl_added"] = ca
            d["similar"] = d["maxdiff"] < o.t_inc and not ca
            info[b] = d
            if d["similar"]:
                put(f, b, o.brick_size, take(old, b, o.brick_size))
                next_keep.add(b)
            else:
                put(f, b, o.brick_size, out)
                if not d["prunable"]:
                    next_redo.add(b)
        next_keep |= keep
        fields.append(f)
        nodes.append(info)
        if k < K:
            kids = bricks_of(levels[k + 1].shape, o.brick_size)
            redo = {c for c in kids if tuple(v // 2 for v in c) in next_redo}
            keep = {c for c in kids if tuple(v // 2 for v in c) in next_keep}
    return fields, nodes


# ----------------------------------------------------------------------------
# tiny cases
# ----------------------------------------------------------------------------

def tiny_case(shape, seed, kind):
    """A tiny volume (FP32 levels, s = 4) and label points.
    kind "ball": a bright ball on a dark background with mild noise (beta 130);
    kind "noise": uniform intensities (beta 20); labels: random points, a
    cluster of foreground labels and one conflicting pair."""
    nz, ny, nx = shape
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint64)
    if kind == "ball":
        z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
        c = np.array([nz, ny, nx]) * np.array([0.45, 0.55, 0.5])
        r = 0.3 * min(shape)
        inside = (z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2 <= r * r
        vol = np.where(inside, 0.7, 0.3) + 0.03 * P.normal(seed, 61, idx).reshape(shape)
        beta = 130.0
    else:
        vol = P.uniform(seed, 62, idx).reshape(shape)
        beta = 20.0
    vol = np.clip(vol, 0.0, 1.0).astype(np.float32)
    st = P.Stream(seed, 63)
    pts, vals = [], []
    for _ in range(max(6, n // 40)):
        p = [st.uniform(0, nx), st.uniform(0, ny), st.uniform(0, nz)]
        pts.append(p)
        if kind == "ball":
            vals.append(1.0 if inside[int(p[2]), int(p[1]), int(p[0])] else 0.0)
        else:
            vals.append(float(st.uniform() < 0.5))
    if kind == "ball":
        cz, cy, cx = (int(v) for v in c)
        for dx in (-1, 0, 1):                     # a foreground cluster at the centre
            pts.append([cx + dx + 0.5, cy + 0.5, cz + 0.5])
            vals.append(1.0)
    pts.append([0.25, 0.5, 0.75])                 # a conflicting pair in one leaf voxel
    vals.append(1.0)
    pts.append([0.75, 0.5, 0.25])
    vals.append(0.0)
    return vol, np.array(pts, dtype=np.float64), np.array(vals), beta


CASES = [((8, 8, 8), 1, "ball", 1.25), ((12, 12, 12), 2, "ball", 1.25), ((16, 11, 9), 3, "ball", 1.25),
         ((9, 12, 7), 4, "noise", 1.25), ((12, 12, 12), 5, "noise", 1.5), ((13, 10, 15), 6, "ball", 1.75),
         ((16, 16, 16), 7, "ball", 1.25)]


def _levels(vol, s):
    return O.pyramid(vol, s)


def _compare_run(levels, t, fields, nodes, prune_info=True):
    assert len(t.P) == len(fields)
    for k in range(len(fields)):
        err = np.max(np.abs(t.P[k] - fields[k]))
        assert err <= FIELD_TOL, f"level {k}: max |oracle - restatement| = {err}"
        assert set(t.info[k]) == set(nodes[k]), f"level {k}: node sets differ"
        for b, d in nodes[k].items():
            ni = t.info[k][b]
            if d.get("reused"):
                assert not ni.solved, (k, b)
                continue
            assert ni.solved, (k, b)
            for key in ("hom", "dt", "cfl", "prunable", "similar", "cfl_added"):
                if key in d:
                    assert getattr(ni, key) == d[key], (k, b, key)


@pytest.mark.parametrize("shape,seed,kind,e", CASES)
def test_tiny_tree_run_matches_restatement(shape, seed, kind, e):
    vol, xyz, val, beta = tiny_case(shape, seed, kind)
    o = hrw.Opts(brick_size=4, expand=e, beta=beta)
    levels = _levels(vol, 4)
    t = hrw.run(levels, xyz, val, o)
    fields, nodes, _ = tiny_run(levels, xyz, val, o)
    _compare_run(levels, t, fields, nodes)


def test_tiny_trees_exercise_every_branch():
    """The cases above reach what the pins are meant to cover: three levels,
    pruned nodes by hom and by dt, absent nodes filled from the parent, user
    seeds replacing border seeds, border layers on some faces only, and a
    conflicted node."""
    seen = {"levels3": False, "hom": False, "dt_only": False, "absent": False, "override": 0, "cfl": False}
    for shape, seed, kind, e in CASES:
        vol, xyz, val, beta = tiny_case(shape, seed, kind)
        o = hrw.Opts(brick_size=4, expand=e, beta=beta)
        levels = _levels(vol, 4)
        fields, nodes, ov = tiny_run(levels, xyz, val, o)
        seen["levels3"] |= len(levels) >= 3
        seen["override"] += ov
        for k, info in enumerate(nodes):
            for d in info.values():
                seen["hom"] |= d["hom"] and d["prunable"]
                seen["dt_only"] |= d["dt"] and not d["hom"] and d["prunable"]
                seen["cfl"] |= d["cfl"]
            if k:
                seen["absent"] |= len(info) < len(bricks_of(levels[k].shape, 4))
    assert seen["levels3"] and seen["hom"] and seen["dt_only"] and seen["absent"] and seen["cfl"], seen
    assert seen["override"] > 0, seen


@pytest.mark.parametrize("shape,seed,kind,e", CASES[:4])
def test_tiny_tree_no_pruning_matches_restatement(shape, seed, kind, e):
    vol, xyz, val, beta = tiny_case(shape, seed, kind)
    o = hrw.Opts(brick_size=4, expand=e, beta=beta, prune_hom=False, prune_dt=False)
    levels = _levels(vol, 4)
    t = hrw.run(levels, xyz, val, o)
    fields, nodes, _ = tiny_run(levels, xyz, val, o)
    _compare_run(levels, t, fields, nodes)
    assert len(t.info[-1]) == len(bricks_of(levels[-1].shape, 4))


# ----------------------------------------------------------------------------
# margins and the pruning predicates by hand
# ----------------------------------------------------------------------------

def test_margins_hand_values():
    # s_e = floor(e s); the extra voxels split evenly, the odd one on the high side
    assert hrw.margins(32, 1.25) == (40, 4, 4)
    assert hrw.margins(64, 1.25) == (80, 8, 8)
    assert hrw.margins(4, 1.25) == (5, 0, 1)
    assert hrw.margins(4, 1.75) == (7, 1, 2)
    assert hrw.margins(8, 1.5) == (12, 2, 2)
    assert hrw.margins(16, 1.0) == (16, 0, 0)


def _flags_of(vals, **kw):
    o = hrw.Opts(**kw)
    ni = hrw.NodeInfo()
    hrw._flags(np.asarray(vals, dtype=np.float64), False, o, ni)
    return ni


def test_dt_predicate_strict_both_ways():
    # hom off: only dt can prune.  Thresholds t_bin = 0.25 and values exact in
    # binary, so "min - 0.5 > t_bin" is decided without rounding.
    kw = dict(t_bin=0.25, prune_hom=False)
    assert not _flags_of([0.75, 0.875, 1.0], **kw).dt         # min - 0.5 == t_bin: not determined
    assert _flags_of([0.78125, 0.875, 1.0], **kw).dt          # min - 0.5 > t_bin
    assert _flags_of([0.78125, 0.875, 1.0], **kw).prunable
    assert not _flags_of([0.0, 0.125, 0.25], **kw).dt         # 0.5 - max == t_bin
    assert _flags_of([0.0, 0.125, 0.21875], **kw).dt          # 0.5 - max > t_bin
    assert not _flags_of([0.0, 0.125, 0.75], **kw).dt         # straddles 0.5
    assert not _flags_of([0.21875, 0.78125], **kw).dt
    ni = _flags_of([0.0, 0.1], **kw)
    assert ni.dt and ni.hom and ni.prunable                    # hom computed, dt prunes
    assert not _flags_of([0.0, 0.1], t_bin=0.25, prune_hom=False, prune_dt=False).prunable


def test_hom_predicate_strict_and_conflict_blocks():
    kw = dict(t_hom=0.25, prune_dt=False)
    assert not _flags_of([0.5, 0.75], **kw).hom                # max - min == t_hom
    assert _flags_of([0.5, 0.71875], **kw).hom
    o = hrw.Opts(t_hom=0.25)
    ni = hrw.NodeInfo()
    hrw._flags(np.array([0.5, 0.5]), True, o, ni)              # a conflict keeps the node
    assert ni.hom and not ni.prunable and ni.cfl


# ----------------------------------------------------------------------------
# incremental labelling (Sec. IV-E)
# ----------------------------------------------------------------------------

UPDATE_CASES = [((12, 12, 12), 2, "ball", 1.25), ((16, 11, 9), 3, "ball", 1.25), ((9, 12, 7), 4, "noise", 1.25),
                ((16, 16, 16), 7, "ball", 1.25)]


def _added_labels(shape, seed, n_add):
    st = P.Stream(seed, 64)
    nz, ny, nx = shape
    return (np.array([[st.uniform(0, nx), st.uniform(0, ny), st.uniform(0, nz)] for _ in range(n_add)]),
            np.array([float(st.uniform() < 0.5) for _ in range(n_add)]))


@pytest.mark.parametrize("shape,seed,kind,e", UPDATE_CASES)
def test_tiny_tree_update_matches_restatement(shape, seed, kind, e):
    vol, xyz, val, beta = tiny_case(shape, seed, kind)
    o = hrw.Opts(brick_size=4, expand=e, beta=beta)
    levels = _levels(vol, 4)
    t = hrw.run(levels, xyz, val, o)
    axyz, aval = _added_labels(shape, seed, 2)
    u = hrw.update(t, axyz, aval)
    fields, nodes = tiny_update(levels, t.P, np.concatenate([xyz, axyz]), np.concatenate([val, aval]), len(val), o)
    _compare_run(levels, u, fields, nodes)


def _cluster_case():
    """Constant volume 16^3 (levels 4^3, 8^3, 16^3 for s = 4); foreground
    labels on every leaf voxel of the block [4, 14]^3, so that the voxels
    around (9, 9, 9) are foreground seeds at every level; background labels in
    three far corners."""
    vol = np.full((16, 16, 16), 0.5, np.float32)
    r = np.arange(4, 15) + 0.5
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    pts = [np.stack([x.ravel(), y.ravel(), z.ravel()], 1)]
    vals = [np.ones(x.size)]
    pts.append(np.array([[0.5, 0.5, 0.5], [15.5, 15.5, 0.5], [0.5, 15.5, 15.5]]))
    vals.append(np.zeros(3))
    return vol, np.concatenate(pts), np.concatenate(vals)


def test_conflict_with_added_label_forces_resolve():
    # an added background label inside the foreground block: its leaf voxel
    # (and the coarse voxels above it) become conflicts involving an added
    # label.  The voxel is surrounded by foreground seeds, so the solutions
    # barely move (max |new - old| < t_inc), yet no node containing the
    # conflict may be kept: its children are re-solved.
    vol, xyz, val = _cluster_case()
    o = hrw.Opts(brick_size=4, beta=130.0, t_inc=0.01, prune_hom=False, prune_dt=False)
    levels = _levels(vol, 4)
    t = hrw.run(levels, xyz, val, o)
    u = hrw.update(t, np.array([[9.5, 9.5, 9.5]]), np.array([0.0]))
    root = u.info[0][(0, 0, 0)]
    assert root.cfl_added and root.maxdiff < o.t_inc and not root.similar
    assert any(ni.solved for ni in u.info[1].values())
    # the leaf brick holding the conflict is re-solved, never reused
    assert u.info[-1][(2, 2, 2)].solved and u.info[-1][(2, 2, 2)].cfl_added
    fields, nodes = tiny_update(levels, t.P, np.concatenate([xyz, [[9.5, 9.5, 9.5]]]), np.concatenate([val, [0.0]]),
                                len(val), o)
    _compare_run(levels, u, fields, nodes)
    # the same label added outside any conflict: the root is similar, nothing below is re-solved
    v = hrw.update(t, np.array([[9.5, 9.5, 10.5]]), np.array([1.0]))
    assert v.info[0][(0, 0, 0)].similar and v.stats["bricks_solved"] == 1


def test_similar_node_keeps_subtree_while_sibling_resolves():
    # an added background label between the foreground block and the volume
    # face (no conflict) changes the nearby bricks by more than t_inc; a far
    # level-1 node is similar and keeps its whole old subtree bit for bit
    # while its siblings re-solve
    vol, xyz, val = _cluster_case()
    o = hrw.Opts(brick_size=4, beta=130.0, t_inc=0.01, prune_hom=False, prune_dt=False)
    levels = _levels(vol, 4)
    t = hrw.run(levels, xyz, val, o)
    add_xyz, add_val = np.array([[2.5, 9.5, 9.5]]), np.array([0.0])
    u = hrw.update(t, add_xyz, add_val)
    root = u.info[0][(0, 0, 0)]
    assert not root.similar and not root.cfl_added and root.maxdiff > o.t_inc
    lvl1 = u.info[1]
    similar = [b for b, ni in lvl1.items() if ni.solved and ni.similar]
    redone = [b for b, ni in lvl1.items() if ni.solved and not ni.similar]
    assert similar and redone
    for b in similar:
        kids = [c for c in u.info[2] if tuple(v // 2 for v in c) == b]
        assert kids and all(not u.info[2][c].solved for c in kids)
        for c in kids:                                   # bit for bit the old leaf values
            assert np.array_equal(take(u.P[2], c, 4), take(t.P[2], c, 4))
    for b in redone:
        kids = [c for c in u.info[2] if tuple(v // 2 for v in c) == b]
        assert kids and all(u.info[2][c].solved for c in kids)
    fields, nodes = tiny_update(levels, t.P, np.concatenate([xyz, add_xyz]), np.concatenate([val, add_val]),
                                len(val), o)
    _compare_run(levels, u, fields, nodes)


# ----------------------------------------------------------------------------
# planted mistakes: each one-line change to the oracle fails a pin above
# ----------------------------------------------------------------------------

def _planted(fn_name, old, new):
    """A copy of hrw.<fn_name> with one source line changed (the change must apply)."""
    src = textwrap.dedent(inspect.getsource(getattr(hrw, fn_name)))
    assert old in src, f"planted mistake no longer applies to {fn_name}"
    ns = dict(vars(hrw))
    exec(compile(src.replace(old, new, 1), f"<planted {fn_name}>", "exec"), ns)
    return ns[fn_name]


MISTAKES = [
    ("margins", "m_lo = (se - s) // 2", "m_lo = (se - s + 1) // 2"),                 # odd voxel on the low side
    ("_solve_node", "if z0 > 0: lay[0, :, :] = True", "lay[0, :, :] = True"),       # border on the volume face
    ("_solve_node", "if x1 < shape[2]: lay[:, :, -1] = True", "pass"),              # a missing border face
    ("upsample", "u = (i + 0.5) / 2.0 - 0.5", "u = i / 2.0"),                       # corner- instead of centre-aligned
    ("_flags", "info.dt = (mn - 0.5 > opts.t_bin) or (0.5 - mx > opts.t_bin)",
     "info.dt = (mn - 0.5 > opts.t_bin) or (mx - 0.5 > opts.t_bin)"),               # a sign in dt
    ("_region", "reg.append((max(lo - m_lo, 0), min(lo + s + m_hi, shape[a])))",
     "reg.append((max(lo - m_hi, 0), min(lo + s + m_lo, shape[a])))"),               # margins swapped
]


def _precedence_mistake():
    # border seeds written after the user seeds: a border seed wins
    src = textwrap.dedent(inspect.getsource(hrw._solve_node))
    a = src.index("    if Up is not None:")
    b = src.index("    cfl = False")
    c = src.index("    if not np.any(code == SEED):")
    moved = src[:a] + src[b:c] + src[a:b] + src[c:]
    assert moved != src
    ns = dict(vars(hrw))
    exec(compile(moved, "<planted _solve_node>", "exec"), ns)
    return ns["_solve_node"]


def _run_pins(monkeypatch):
    """Run the tiny-tree pins against the current (possibly planted) oracle;
    returns True when they all pass."""
    try:
        for shape, seed, kind, e in CASES:
            vol, xyz, val, beta = tiny_case(shape, seed, kind)
            o = hrw.Opts(brick_size=4, expand=e, beta=beta)
            levels = _levels(vol, 4)
            _compare_run(levels, hrw.run(levels, xyz, val, o), *tiny_run(levels, xyz, val, o)[:2])
        test_dt_predicate_strict_both_ways()
        test_margins_hand_values()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("which", list(range(len(MISTAKES))) + ["precedence", "similar_ignores_cfl", "no_reuse"])
def test_pins_catch_planted_mistakes(monkeypatch, which):
    if which == "precedence":
        monkeypatch.setattr(hrw, "_solve_node", _precedence_mistake())
        assert not _run_pins(monkeypatch)
        return
    if which in ("similar_ignores_cfl", "no_reuse"):
        if which == "similar_ignores_cfl":
            bad = _planted("update", "ni.similar = (ni.maxdiff < opts.t_inc) and not cfl_added",
                           "ni.similar = (ni.maxdiff < opts.t_inc)")
        else:
            bad = _planted("update", "nxt_reused.extend(_children(b, levels[k + 1].shape, s))\n            else:",
                           "nxt_resolve.extend(_children(b, levels[k + 1].shape, s))\n            else:")
        monkeypatch.setattr(hrw, "update", bad)
        with pytest.raises(AssertionError):
            test_conflict_with_added_label_forces_resolve()
            test_similar_node_keeps_subtree_while_sibling_resolves()
        return
    fn, old, new = MISTAKES[which]
    monkeypatch.setattr(hrw, fn, _planted(fn, old, new))
    assert not _run_pins(monkeypatch)

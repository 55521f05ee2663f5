"""Parity of the CUDA pyramid and hierarchical procedure (rw_build_pyramid,
rw_refine_level, rw_update_seeds) with the oracle's H_p."""
import numpy as np
import pytest

import oracle as O
import phantoms as P
from conftest import determined_mask
from oracle import hrw

pytestmark = pytest.mark.gpu
# Brick systems can hold weakly coupled pockets (isolated eigenvalues of the
# Jacobi-scaled matrix near 1e-6): there a relative residual of 1e-9 still
# allows 1e-3 of error.  The parity runs solve every brick to 1e-10, the
# tolerance the hierarchical benchmarks run at.
TOL = 1e-4
HIER_TOL = 1e-10
NEAR = 1e-4      # a pruning decision may differ only this close to its threshold


@pytest.fixture(scope="module")
def rw():
    import torch
    assert torch.cuda.is_available()
    import paper_2103_09564_gb300 as m
    m.load()
    return m


def _near_threshold(ni, opts):
    return (abs((ni.mx - ni.mn) - opts.t_hom) < NEAR or abs((ni.mn - 0.5) - opts.t_bin) < NEAR or
            abs((0.5 - ni.mx) - opts.t_bin) < NEAR)


def _compare(rw, tree, otree, opts, s, incremental=False):
    """Compare level by level: node sets and decisions must agree unless the
    oracle's statistic sits within NEAR of a threshold; fields within TOL
    outside subtrees below such near-threshold nodes."""
    K = len(otree.P) - 1
    excluded = []     # (level, brick) roots of subtrees where decisions may differ
    for k in range(K + 1):
        fl, mn, mx, md = tree.node_stats(k)
        gpu_solved = {tuple(int(v) for v in b) for b in np.argwhere(fl & rw.RW_NODE_SOLVED)}
        or_solved = {b for b, ni in otree.info[k].items() if ni.solved}

        def under_excluded(b):
            for (kk, e) in excluded:
                sh = k - kk
                if tuple(v >> sh for v in b) == e:
                    return True
            return False
        for b in gpu_solved ^ or_solved:
            assert under_excluded(b), f"level {k}: node {b} solved on one side only"
        for b in gpu_solved & or_solved:
            if under_excluded(b):
                continue
            ni = otree.info[k][b]
            gp = bool(fl[b] & rw.RW_NODE_PRUNABLE)
            if gp != ni.prunable:
                assert _near_threshold(ni, opts), f"level {k}: prunable differs at {b}"
                excluded.append((k, b))
            if incremental:
                gs = bool(fl[b] & rw.RW_NODE_SIMILAR)
                if gs != ni.similar:
                    assert abs(ni.maxdiff - opts.t_inc) < NEAR, f"level {k}: similar differs at {b}"
                    excluded.append((k, b))
        field = tree.read_level(k).astype(np.float64)
        # trapped pockets (salt clusters behind w_min edges) are undetermined
        if opts.weight == "poisson":
            mask = determined_mask(np.sqrt(otree.levels[k]), opts.beta / 2.0)
        else:
            mask = determined_mask(otree.levels[k], opts.beta)
        for (kk, e) in excluded:
            sh = k - kk
            lo = [v * s * (1 << sh) for v in e]
            hi = [(v + 1) * s * (1 << sh) for v in e]
            # the upsampling of the next levels reaches one parent voxel further
            mask[max(lo[0] - 2 * s, 0):hi[0] + 2 * s, max(lo[1] - 2 * s, 0):hi[1] + 2 * s,
                 max(lo[2] - 2 * s, 0):hi[2] + 2 * s] = False
        err = np.max(np.abs(field - otree.P[k])[mask]) if mask.any() else 0.0
        assert err <= TOL, f"level {k}: max |gpu - oracle| = {err}"
        # thresholded labels agree wherever the oracle is clear of 0.5
        clear = mask & (np.abs(otree.P[k] - 0.5) > 1e-3)
        assert np.array_equal(field[clear] > 0.5, otree.P[k][clear] > 0.5), f"level {k}: labels differ"
    return excluded


def test_pyramid_bit_exact(rw):
    ph = P.vessel_tree(shape=(37, 50, 70), seed=5, n_segments=10)
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    lv = O.pyramid(O.leaf_level(q), 8)
    assert pyr.levels == len(lv)
    for k in range(len(lv)):
        assert np.array_equal(pyr.read_level(k), lv[k]), k


@pytest.mark.parametrize("n,s,seed", [(64, 8, 2), (96, 16, 3), ((40, 72, 56), 8, 4)])
def test_full_run_parity(rw, n, s, seed):
    if isinstance(n, tuple):
        ph = P.vessel_tree(shape=n, seed=seed, n_segments=25)
    else:
        ph = P.vessel_tree(n=n, seed=seed, n_segments=30)
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL)
    tree = rw.Tree(pyr, opts)
    st = tree.run(ph["labels_xyz"], ph["labels_value"])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), s)
    oo = hrw.Opts(brick_size=s, beta=130.0)
    ot = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], oo)
    exc = _compare(rw, tree, ot, oo, s)
    if not exc:
        assert st["bricks_solved"] == ot.stats["bricks_solved"]
        assert st["bricks_pruned"] == ot.stats["bricks_pruned"]


def test_brick_64_parity(rw):
    # the 64^3 brick variant: 80^3 expanded neighbourhoods (two brick tiles
    # across x), root 64^3, one leaf level of 8 bricks
    ph = P.vessel_tree(n=128, seed=6, n_segments=20)
    s = 64
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    tree = rw.Tree(pyr, rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL))
    st = tree.run(ph["labels_xyz"], ph["labels_value"])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), s)
    oo = hrw.Opts(brick_size=s, beta=130.0)
    ot = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], oo)
    exc = _compare(rw, tree, ot, oo, s)
    if not exc:
        assert st["bricks_solved"] == ot.stats["bricks_solved"]
        assert st["bricks_pruned"] == ot.stats["bricks_pruned"]


def test_single_brick_equals_plain(rw):
    c = P.random_case((12, 10, 14), seed=5, seed_frac=0.05, levels=[0.0, 1.0])
    z, y, x = np.nonzero(c["code"] == 1)
    xyz = np.stack([x + 0.5, y + 0.5, z + 0.5], 1)
    val = c["value"][z, y, x]
    pyr = rw.rw_build_pyramid(c["volume"], 16)
    tree = rw.Tree(pyr, rw.Opts(brick_size=16, beta=30.0, tol=HIER_TOL))
    tree.run(xyz, val)
    leaf = O.leaf_level(O.quantize(c["volume"]))
    xo, _, _, _ = O.rw_solve(leaf.astype(np.float64), c["code"], c["value"], 30.0)
    assert np.max(np.abs(tree.read_level(0) - xo)) <= 1e-6


@pytest.mark.parametrize("seed", [2, 6])
def test_no_pruning_parity_and_agreement(rw, seed):
    # Table IV: pruning leaves the segmentation essentially unchanged.  Both
    # GPU trees (pruned, unpruned) match the oracle's, and the share of labels
    # that pruning flips on the GPU equals the method's own (the oracle's) on
    # this phantom.  On seed 2 that share is below 0.1 % (the oracle pin's
    # bound); on seed 6 (64^3, brick 8: thin vessels that coarse levels blur)
    # the method itself flips 0.43 % of the labels.
    ph = P.vessel_tree(n=64, seed=seed, n_segments=30)
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    t1 = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL, prune_hom=0, prune_dt=0))
    t1.run(ph["labels_xyz"], ph["labels_value"])
    t2 = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL))
    s2 = t2.run(ph["labels_xyz"], ph["labels_value"])
    a, b = t1.read_level(pyr.levels - 1), t2.read_level(pyr.levels - 1)
    assert s2["bricks_pruned"] > 0
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0, prune_hom=False, prune_dt=False)
    ot = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], oo)
    op = hrw.Opts(brick_size=8, beta=130.0)
    ot2 = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], op)
    _compare(rw, t1, ot, oo, 8)
    _compare(rw, t2, ot2, op, 8)
    agree = np.mean((a > 0.5) == (b > 0.5))
    o_agree = np.mean((ot.P[-1] > 0.5) == (ot2.P[-1] > 0.5))
    assert abs(agree - o_agree) <= 1e-4
    if seed == 2:
        assert agree >= 0.999


def test_incremental_update_parity(rw):
    ph = P.vessel_tree(n=64, seed=7, n_segments=30)
    n0 = len(ph["labels_value"]) - 6
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL)
    tree = rw.Tree(pyr, opts)
    tree.run(ph["labels_xyz"][:n0], ph["labels_value"][:n0])
    su = tree.update_seeds(ph["labels_xyz"][n0:], ph["labels_value"][n0:])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0)
    ot = hrw.run(levels, ph["labels_xyz"][:n0], ph["labels_value"][:n0], oo)
    ou = hrw.update(ot, ph["labels_xyz"][n0:], ph["labels_value"][n0:])
    exc = _compare(rw, tree, ou, oo, 8, incremental=True)
    if not exc:
        assert su["bricks_solved"] == ou.stats["bricks_solved"]
        assert su["bricks_reused"] == ou.stats["bricks_reused"]


def test_chained_updates_parity(rw):
    # three successive incremental passes against the oracle's chained
    # updates: the level fill rewrites only the absent nodes whose parent
    # footprint changed, which must still give the oracle's fields
    ph = P.vessel_tree(n=64, seed=11, n_segments=30)
    xyz, val = ph["labels_xyz"], ph["labels_value"]
    cuts = [len(val) - 9, len(val) - 6, len(val) - 3, len(val)]
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL)
    tree = rw.Tree(pyr, opts)
    tree.run(xyz[:cuts[0]], val[:cuts[0]])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0)
    ot = hrw.run(levels, xyz[:cuts[0]], val[:cuts[0]], oo)
    kept = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        tree.update_seeds(xyz[a:b], val[a:b])
        ot = hrw.update(ot, xyz[a:b], val[a:b])
        fl = tree.node_stats(pyr.levels - 1)[0]
        kept += int(np.count_nonzero((fl & rw.RW_NODE_CHANGED) == 0))
    assert kept > 0
    _compare(rw, tree, ot, oo, 8, incremental=True)


def test_update_without_labels_keeps_everything(rw):
    ph = P.vessel_tree(n=32, seed=3, n_segments=10)
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    tree = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL))
    tree.run(ph["labels_xyz"], ph["labels_value"])
    before = tree.read_level(pyr.levels - 1).copy()
    su = tree.update_seeds(np.zeros((0, 3)), np.zeros(0))
    assert su["bricks_solved"] == 1
    assert np.array_equal(tree.read_level(pyr.levels - 1), before)


def test_per_brick_sequential_equals_batched(rw):
    ph = P.vessel_tree(n=64, seed=8, n_segments=20)
    pyr = rw.rw_build_pyramid(ph["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    a = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL))
    a.run(ph["labels_xyz"], ph["labels_value"])
    b = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL, batch_bricks=0, precision="fp64"))
    b.run(ph["labels_xyz"], ph["labels_value"])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    det = determined_mask(O.leaf_level(q), 130.0)
    assert det.mean() > 0.99
    diff = np.abs(a.read_level(pyr.levels - 1) - b.read_level(pyr.levels - 1))
    assert np.max(diff[det]) <= TOL


def test_leaf_in_host_memory_matches_hbm(rw):
    # out-of-core placement: the leaf level in mapped host memory (the
    # intensities, with the tree's leaf field there too or in HBM; or only the
    # tree's leaf field) gives the same results, bit for bit, through a full
    # run and an incremental update (one fixed tile: no autotuning sweeps)
    ph = P.vessel_tree(n=96, seed=3, n_segments=30)
    xyz, val = ph["labels_xyz"], ph["labels_value"]
    n0 = len(val) // 2
    out = []
    for host, field in ((False, "pyramid"), (True, "pyramid"), (True, "hbm"), (False, "host"), ("all", "pyramid"),
                        (False, "host_all")):
        pyr = rw.rw_build_pyramid(ph["volume"], 16, lo=0.0, hi=5000.0, normalize=True, leaf_in_host=host is True,
                                  all_in_host=host == "all")
        leaf = pyr.read_level(pyr.levels - 1)
        tree = rw.Tree(pyr, rw.Opts(brick_size=16, beta=130.0, tol=1e-10, tile="32x8", leaf_field=field))
        tree.run(xyz[:n0], val[:n0])
        first = tree.read_level(pyr.levels - 1)
        tree.update_seeds(xyz[n0:], val[n0:])
        out.append((leaf, first, tree.read_level(pyr.levels - 1)))
        tree.free()
        pyr.free()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def _class_trees(rw, c, s, tol, prune):
    pyr = rw.rw_build_pyramid(c["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    trees = []
    for k in range(3):
        t = rw.Tree(pyr, rw.Opts(brick_size=s, beta=130.0, tol=tol, prune_hom=int(prune), prune_dt=0))
        t.run(*P.class_labels(c["strokes"], k))
        trees.append(t)
    return pyr, trees


def test_multiclass_argmax_matches_oracle(rw):
    # one tree per class (Sec. III-B), no pruning: the GPU class fields sum to
    # one and the fused argmax agrees with the oracle's per-class hierarchy on
    # every voxel where the two best classes are more than 1e-3 apart
    c = P.multiclass_case((64, 64, 64), seed=1, n_segments=20, n_blobs=30, n_updates=0)
    pyr, trees = _class_trees(rw, c, 8, HIER_TOL, prune=False)
    labels, pmax = rw.trees_argmax(trees, prob=np.empty((64, 64, 64), np.float32))
    fields = np.stack([t.read_level(pyr.levels - 1) for t in trees])
    assert np.array_equal(labels, np.argmax(fields, axis=0).astype(np.uint8))
    assert np.array_equal(pmax, fields.max(axis=0))
    q = O.quantize(c["volume"], 0.0, 5000.0, True)
    seeds = np.zeros(q.shape, bool)
    for xyz, _ in c["strokes"]:
        v = np.floor(xyz).astype(int)
        seeds[v[:, 2], v[:, 1], v[:, 0]] = True
    det = determined_mask(O.leaf_level(q), 130.0, seeds=seeds)
    assert det.mean() > 0.99
    assert np.max(np.abs(fields.sum(axis=0) - 1.0)[det]) <= 1e-4
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0, prune_hom=False, prune_dt=False)
    of = []
    for k in range(3):
        xyz, val, cls = P.class_labels(c["strokes"], k)
        of.append(hrw.run(levels, xyz, val, oo, labels_cls=cls).P[-1])
    of = np.stack(of)
    top2 = np.sort(of, axis=0)
    clear = det & (top2[-1] - top2[-2] > 1e-3)
    assert clear.mean() > 0.9
    assert np.array_equal(labels[clear], np.argmax(of, axis=0)[clear])


def test_argmax_ties_take_the_lowest_class(rw):
    c = P.multiclass_case((32, 32, 32), seed=4, n_segments=8, n_blobs=10, n_updates=0)
    pyr = rw.rw_build_pyramid(c["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    lab = P.class_labels(c["strokes"], 1)
    trees = []
    for _ in range(2):
        t = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=1e-10, tile="32x8"))
        t.run(*lab)
        trees.append(t)
    labels, _ = rw.trees_argmax(trees)
    assert np.array_equal(trees[0].read_level(pyr.levels - 1), trees[1].read_level(pyr.levels - 1))
    assert not labels.any()
    with pytest.raises(rw.RWError):
        rw.trees_argmax(trees, box=[0, 0, 0, 999, 1, 1])


def test_argmax_output_kinds_agree(rw):
    # pageable host memory (staged), device memory and page-locked host memory
    # (written by the kernel) give the same labels and probabilities, on the
    # whole leaf and on a box whose voxel count is not a multiple of 4
    import torch
    shape = (64, 48, 40)
    c = P.multiclass_case(shape, seed=2, n_segments=12, n_blobs=12, n_updates=0)
    pyr, trees = _class_trees(rw, c, 8, 1e-10, prune=True)
    lab, prob = rw.trees_argmax(trees, prob=np.empty(shape, np.float32))
    fields = np.stack([t.read_level(pyr.levels - 1) for t in trees])
    assert np.array_equal(lab, np.argmax(fields, axis=0).astype(np.uint8))
    assert np.array_equal(prob, fields.max(axis=0))
    box = [3, 5, 7, 34, 38, 45]  # x0, y0, z0, x1, y1, z1: 31 x 33 x 38 voxels
    sub = (slice(box[2], box[5]), slice(box[1], box[4]), slice(box[0], box[3]))
    bshape = (box[5] - box[2], box[4] - box[1], box[3] - box[0])
    assert np.prod(bshape) % 4 != 0
    for b, shp, ref_l, ref_p in ((None, shape, lab, prob), (box, bshape, lab[sub], prob[sub])):
        for kind in ("cuda", "pinned", "numpy"):
            if kind == "numpy":
                o, p = np.empty(shp, np.uint8), np.empty(shp, np.float32)
            else:
                kw = {"device": "cuda"} if kind == "cuda" else {"pin_memory": True}
                o = torch.empty(shp, dtype=torch.uint8, **kw)
                p = torch.empty(shp, dtype=torch.float32, **kw)
            rw.trees_argmax(trees, box=b, out=o, prob=p)
            torch.cuda.synchronize()
            o = o.cpu().numpy() if kind != "numpy" else o
            p = p.cpu().numpy() if kind != "numpy" else p
            assert np.array_equal(o, ref_l), (kind, b)
            assert np.array_equal(p, ref_p), (kind, b)


def test_argmax_changed_matches_full_argmax(rw):
    # after each round of updates, relabelling only the changed leaf bricks
    # (device and page-locked outputs) gives the full argmax bit for bit
    import torch
    shape = (64, 64, 64)
    c = P.multiclass_case(shape, seed=3, n_segments=20, n_blobs=20, n_updates=4)
    pyr, trees = _class_trees(rw, c, 8, 1e-10, prune=True)
    lab_d = torch.empty(shape, dtype=torch.uint8, device="cuda")
    prob_d = torch.empty(shape, dtype=torch.float32, device="cuda")
    lab_h = torch.empty(shape, dtype=torch.uint8, pin_memory=True)
    rw.trees_argmax(trees, out=lab_d, prob=prob_d)
    rw.trees_argmax(trees, out=lab_h)
    partial = False
    for xyz, cls in c["updates"]:
        for k, t in enumerate(trees):
            t.update_seeds(xyz, np.full(len(xyz), 1.0 if k == cls else 0.0, np.float32),
                           np.full(len(xyz), cls, np.int32))
        rw.trees_argmax_changed(trees, lab_d, prob_d)
        rw.trees_argmax_changed(trees, lab_h)
        torch.cuda.synchronize()
        ref_l, ref_p = rw.trees_argmax(trees, prob=np.empty(shape, np.float32))
        assert np.array_equal(lab_d.cpu().numpy(), ref_l)
        assert np.array_equal(prob_d.cpu().numpy(), ref_p)
        assert np.array_equal(lab_h.numpy(), ref_l)
        ch = np.zeros_like(trees[0].node_stats(pyr.levels - 1)[0], dtype=bool)
        for t in trees:
            ch |= (t.node_stats(pyr.levels - 1)[0] & rw.RW_NODE_CHANGED) != 0
        partial = partial or not ch.all()
    assert partial
    with pytest.raises(rw.RWError):
        rw.trees_argmax_changed(trees, np.empty(shape, np.uint8))


def test_update_trees_matches_oracle_and_sequential_updates(rw):
    # the class trees updated together (their bricks share batched launches)
    # give every tree the oracle's incremental result, and the same decisions
    # and fields as updating the trees one by one
    c = P.multiclass_case((64, 64, 64), seed=5, n_segments=20, n_blobs=20, n_updates=2)
    pyr = rw.rw_build_pyramid(c["volume"], 8, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=8, beta=130.0, tol=HIER_TOL, prune_hom=1, prune_dt=0)
    joint = [rw.Tree(pyr, opts) for _ in range(3)]
    seq = [rw.Tree(pyr, opts) for _ in range(3)]
    q = O.quantize(c["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0, prune_hom=True, prune_dt=False)
    ot = []
    for k in range(3):
        lab = P.class_labels(c["strokes"], k)
        joint[k].run(*lab)
        seq[k].run(*lab)
        ot.append(hrw.run(levels, lab[0], lab[1], oo, labels_cls=lab[2]))
    for xyz, cu in c["updates"]:
        vals = [np.full(len(xyz), 1.0 if k == cu else 0.0, np.float32) for k in range(3)]
        cl = np.full(len(xyz), cu, np.int32)
        st = rw.update_trees(joint, xyz, vals, cl)
        ss = [seq[k].update_seeds(xyz, vals[k], cl) for k in range(3)]
        assert st["bricks_solved"] == sum(x["bricks_solved"] for x in ss)
        assert st["bricks_reused"] == sum(x["bricks_reused"] for x in ss)
        ot = [hrw.update(ot[k], xyz, vals[k], add_cls=cl) for k in range(3)]
    K = pyr.levels - 1
    seeds = np.zeros(q.shape, bool)
    for xyz, _ in list(c["strokes"]) + list(c["updates"]):
        v = np.floor(xyz).astype(int)
        seeds[v[:, 2], v[:, 1], v[:, 0]] = True
    det = determined_mask(O.leaf_level(q), 130.0, seeds=seeds)
    assert det.mean() > 0.99
    for k in range(3):
        _compare(rw, joint[k], ot[k], oo, 8, incremental=True)
        for lv in range(K + 1):
            assert np.array_equal(joint[k].node_stats(lv)[0], seq[k].node_stats(lv)[0]), (k, lv)
        a, b = joint[k].read_level(K), seq[k].read_level(K)
        assert np.max(np.abs(a - b)[det]) <= TOL
    with pytest.raises(rw.RWError):
        rw.update_trees([joint[0], joint[0]], c["updates"][0][0], [vals[0], vals[0]])
    other = rw.Tree(pyr, rw.Opts(brick_size=8, beta=130.0, tol=1e-9, prune_hom=1, prune_dt=0))
    other.run(*P.class_labels(c["strokes"], 0))
    with pytest.raises(rw.RWError):
        rw.update_trees([joint[0], other], c["updates"][0][0], [vals[0], vals[1]])


def test_poisson_weights_hierarchy_parity(rw):
    S = 255.0
    c = P.poisson_ball(n=64, seed=5)
    h = 32
    xyz = [(x + 0.5, h + 0.5, h + 0.5) for x in range(28, 37)]
    xyz += [(a + 0.5, b + 0.5, d + 0.5) for a in (2, 61) for b in (2, 61) for d in (2, 61)]
    val = np.array([1.0] * 9 + [0.0] * 8, np.float32)
    xyz = np.array(xyz)
    pyr = rw.rw_build_pyramid(c["volume"], 8, lo=0.0, hi=S, normalize=True)
    tree = rw.Tree(pyr, rw.Opts(brick_size=8, beta=S, tol=HIER_TOL, weight="poisson"))
    tree.run(xyz, val)
    q = O.quantize(c["volume"], 0.0, S, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=S, weight="poisson")
    ot = hrw.run(levels, xyz, val, oo)
    _compare(rw, tree, ot, oo, 8)


class _At:
    """A sub-block indexed with the global coordinates of its level (the
    oracle's node solve slices its inputs with level coordinates)."""

    def __init__(self, a, off):
        self.a, self.off = a, off

    def __getitem__(self, sl):
        return self.a[tuple(slice(s.start - o, s.stop - o) for s, o in zip(sl, self.off))]


def test_vessel_tree_1024_sampled_bricks_and_properties(rw):
    """The 1024^3 vessel-tree workload with brick 32, in the benchmark's launch
    configuration (batched levels, autotuned tiles; bricks solved to 1e-10 as
    in the benchmark and every hierarchy parity test).  Properties of the whole result: every
    level within [0, 1] (maximum principle) and every label voxel of the leaf
    exact where its leaf brick was solved (pruned bricks hold the upsampled
    parent).  Sampled parity: leaf bricks equal the oracle's FP64 solve of the
    same brick problem (Eqs. 2-3: expanded box, border seeds from the
    upsampled parent) posed on the GPU's own parent level."""
    import torch
    dev = torch.device("cuda", 0)
    s = 32
    ph = P.vessel_tree(n=1024, seed=0, device=dev)
    xyz = np.asarray(ph["labels_xyz"], dtype=np.float64)
    val = np.asarray(ph["labels_value"], dtype=np.float32)
    vol = ph["volume"]
    pyr = rw.rw_build_pyramid(vol, s, lo=0.0, hi=5000.0, normalize=True)
    tree = rw.Tree(pyr, rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL))
    tree.run(xyz, val)
    K = pyr.levels - 1
    for k in range(K + 1):
        f = torch.empty(tuple(reversed(pyr.dims[k])), dtype=torch.float32, device=dev)
        tree.read_level(k, out=f)
        assert float(f.min()) >= -1e-6 and float(f.max()) <= 1.0 + 1e-6, k
    shape = tuple(reversed(pyr.dims[K]))
    seeds, conflicts = hrw.rasterize(xyz, val, K, K, shape)
    fl, mn, mx, _ = tree.node_stats(K)
    zyx = np.array([v for v in sorted(seeds) if fl[v[0] // s, v[1] // s, v[2] // s] & rw.RW_NODE_SOLVED],
                   dtype=np.int64)
    assert len(zyx) > 100
    got = f[torch.from_numpy(zyx[:, 0]).to(dev), torch.from_numpy(zyx[:, 1]).to(dev),
            torch.from_numpy(zyx[:, 2]).to(dev)].cpu().numpy()
    assert np.array_equal(got, np.array([seeds[tuple(v)] for v in zyx], dtype=np.float32))
    del f

    solved = [tuple(int(v) for v in b) for b in np.argwhere(fl & rw.RW_NODE_SOLVED)]
    assert len(solved) > 50
    solved.sort(key=lambda b: -(mx[b] - mn[b]))
    sample = solved[:2] + solved[len(solved) // 3:len(solved) // 3 + 1] + solved[2 * len(solved) // 3:][:1]
    oo = hrw.Opts(brick_size=s, beta=130.0)
    se, m_lo, m_hi = hrw.margins(s, oo.expand)
    pdims = tuple(reversed(pyr.dims[K - 1]))
    for b in sample:
        box, reg = hrw._region(b, shape, s, se, m_lo, m_hi)
        lo = [r[0] for r in reg]
        hi = [r[1] for r in reg]
        blk = vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].cpu().to(torch.int32).numpy().astype(np.uint16)
        q = O.quantize(blk, 0.0, 5000.0, True)
        g = O.leaf_level(q)
        # the parent sub-block with one voxel of margin: its trilinear upsample
        # equals the whole level's on the region
        p0 = [max(0, lo[a] // 2 - 1) for a in range(3)]
        p1 = [min(pdims[a], (hi[a] + 1) // 2 + 1) for a in range(3)]
        par = tree.read_level(K - 1, box=[p0[2], p0[1], p0[0], p1[2], p1[1], p1[0]]).astype(np.float64)
        up = hrw.upsample(par, tuple(min(2 * p1[a], shape[a]) - 2 * p0[a] for a in range(3)))
        Up = _At(up, [2 * p0[a] for a in range(3)])
        out, box2, _, _, _, _ = hrw._solve_node(K, b, _At(g, lo), Up, Up, seeds, conflicts, oo, shape)
        assert box2 == box
        gpu = tree.read_level(K, box=[box[2][0], box[1][0], box[0][0], box[2][1], box[1][1], box[0][1]])
        # determined voxels of the brick problem: its seeds are the border
        # layer on faces inside the level and the label voxels
        sd = np.zeros(g.shape, bool)
        for a in range(3):
            if lo[a] > 0:
                sd[(slice(None),) * a + (0,)] = True
            if hi[a] < shape[a]:
                sd[(slice(None),) * a + (-1,)] = True
        for (z, y, x) in seeds:
            if lo[0] <= z < hi[0] and lo[1] <= y < hi[1] and lo[2] <= x < hi[2]:
                sd[z - lo[0], y - lo[1], x - lo[2]] = True
        det = determined_mask(g, 130.0, seeds=sd)
        det = det[box[0][0] - lo[0]:box[0][1] - lo[0], box[1][0] - lo[1]:box[1][1] - lo[1],
                  box[2][0] - lo[2]:box[2][1] - lo[2]]
        assert det.mean() > 0.99
        err = np.max(np.abs(gpu.astype(np.float64) - out)[det])
        assert err <= TOL, f"brick {b}: max |gpu - oracle| = {err}"


def test_multiclass_incremental_256_matches_oracle(rw):
    """The incremental three-class workload's generator (vessel tree of 200
    segments, 400 cell blobs, background; three 200-voxel strokes per class,
    then strokes added one at a time) at 256^3, brick 32, hom-only pruning:
    the initial solve and two updates of the three trees together
    (rw_update_seeds_trees, as the benchmark runs them) match the oracle's
    per-class hierarchy and incremental passes level by level, and the leaf
    labels kept up to date on the changed bricks equal the argmax of the
    oracle's fields wherever its two best classes are more than 1e-3 apart."""
    import torch
    shape = (256, 256, 256)
    c = P.multiclass_case(shape, seed=0, n_segments=200, n_blobs=400, n_updates=2)
    s = 32
    pyr = rw.rw_build_pyramid(c["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL, prune_hom=1, prune_dt=0)
    trees = [rw.Tree(pyr, opts) for _ in range(3)]
    q = O.quantize(c["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), s)
    oo = hrw.Opts(brick_size=s, beta=130.0, prune_hom=True, prune_dt=False)
    ot = []
    for k in range(3):
        lab = P.class_labels(c["strokes"], k)
        trees[k].run(*lab)
        ot.append(hrw.run(levels, lab[0], lab[1], oo, labels_cls=lab[2]))
    labels = torch.empty(shape, dtype=torch.uint8, device="cuda")
    rw.trees_argmax(trees, out=labels)
    seeds = np.zeros(q.shape, bool)
    for xyz, _ in list(c["strokes"]) + list(c["updates"]):
        v = np.floor(xyz).astype(int)
        seeds[v[:, 2], v[:, 1], v[:, 0]] = True
    det = determined_mask(O.leaf_level(q), 130.0, seeds=seeds)
    assert det.mean() > 0.99
    for xyz, cu in c["updates"]:
        vals = [np.full(len(xyz), 1.0 if k == cu else 0.0, np.float32) for k in range(3)]
        cl = np.full(len(xyz), cu, np.int32)
        rw.update_trees(trees, xyz, vals, cl)
        rw.trees_argmax_changed(trees, labels)
        ot = [hrw.update(ot[k], xyz, vals[k], add_cls=cl) for k in range(3)]
        for k in range(3):
            _compare(rw, trees[k], ot[k], oo, s, incremental=True)
        of = np.stack([t.P[-1] for t in ot])
        top2 = np.sort(of, axis=0)
        clear = det & (top2[-1] - top2[-2] > 1e-3)
        assert clear.mean() > 0.9
        got = labels.cpu().numpy()
        assert np.array_equal(got[clear], np.argmax(of, axis=0)[clear])


def test_level_sharding_two_trees_match_oracle_and_unsharded(rw):
    """Level sharding through the library on one GPU: two trees on one
    pyramid stand for two ranks (no collective: their exports are imported
    directly; level 2's values move through device memory).  Each level's
    nodes are split into two Morton ranges, each tree solves its range,
    imports the other's nodes and closes the level.  Both trees end up with
    the same fields and node records, which match the oracle's H_p level by
    level and an unsharded tree within the parity tolerance."""
    import torch
    from paper_2103_09564_gb300 import shard
    ph = P.vessel_tree(n=96, seed=3, n_segments=30)
    xyz, val = ph["labels_xyz"], ph["labels_value"]
    s = 16
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    opts = rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL)
    trees = [rw.Tree(pyr, opts) for _ in range(2)]
    sh = [shard.TreeShard(t) for t in trees]
    split = []
    for k in range(pyr.levels):
        ids = sh[0].level_nodes(k)
        assert np.array_equal(ids, sh[1].level_nodes(k))
        nbx, nby = sh[0].brick_grid(k)
        parts = shard.partition(ids, nbx, nby, 2)
        split.append([len(p) for p in parts])
        for r in range(2):
            sh[r].solve(k, parts[r], (xyz, val) if k == 0 else None)
        if k == 2:
            ex = [sh[r].export(k, parts[r], torch.empty((len(parts[r]), s ** 3), device="cuda")) for r in range(2)]
        else:
            ex = [sh[r].export(k, parts[r]) for r in range(2)]
        if k == 1:
            with pytest.raises(rw.RWError):        # the level is incomplete
                sh[0].finish(k)
            with pytest.raises(rw.RWError):        # a level is open
                trees[0].refine_level(k)
        sh[0].import_(k, ex[1])
        sh[1].import_(k, ex[0])
        if k == 1 and len(parts[0]):
            with pytest.raises(rw.RWError):        # already present
                sh[1].import_(k, ex[0])
        for r in range(2):
            sh[r].finish(k)
    assert any(min(a, b) > 0 for a, b in split)
    for k in range(pyr.levels):
        assert np.array_equal(trees[0].read_level(k), trees[1].read_level(k)), k
        for a, b in zip(trees[0].node_stats(k), trees[1].node_stats(k)):
            assert np.array_equal(a, b), k
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), s)
    oo = hrw.Opts(brick_size=s, beta=130.0)
    ot = hrw.run(levels, xyz, val, oo)
    _compare(rw, trees[0], ot, oo, s)
    whole = rw.Tree(pyr, opts)
    whole.run(xyz, val)
    det = determined_mask(levels[-1], 130.0)
    diff = np.abs(whole.read_level(pyr.levels - 1) - trees[0].read_level(pyr.levels - 1))
    assert np.max(diff[det]) <= TOL


def test_all_levels_in_host_memory_match_oracle(rw):
    """Out-of-core placement: every pyramid level and every tree field in
    pinned, mapped host memory (the host input normalised in slabs).  A full
    run and an incremental update match the oracle's H_p level by level, and
    the device memory the pyramid and the tree take is below the size of
    their own leaf field (they live in host memory; HBM holds the batched
    solve's working set)."""
    import torch
    ph = P.vessel_tree(n=128, seed=9, n_segments=40)
    xyz, val = ph["labels_xyz"], ph["labels_value"]
    n0 = len(val) - 6
    s = 16
    torch.cuda.synchronize()
    rw.release_workspace()
    free0 = torch.cuda.mem_get_info()[0]
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True, all_in_host=True)
    opts = rw.Opts(brick_size=s, beta=130.0, tol=HIER_TOL)
    tree = rw.Tree(pyr, opts)
    rw.release_workspace()
    used = free0 - torch.cuda.mem_get_info()[0]
    assert used < 128 ** 3 * 4, used
    tree.run(xyz[:n0], val[:n0])
    tree.update_seeds(xyz[n0:], val[n0:])
    q = O.quantize(ph["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), s)
    for k in range(len(levels)):
        assert np.array_equal(pyr.read_level(k), levels[k]), k
    oo = hrw.Opts(brick_size=s, beta=130.0)
    ot = hrw.run(levels, xyz[:n0], val[:n0], oo)
    ou = hrw.update(ot, xyz[n0:], val[n0:])
    _compare(rw, tree, ou, oo, s, incremental=True)

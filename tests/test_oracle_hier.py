"""Pins of the oracle's pyramid (Sec. III-A) and hierarchical procedure
(Eqs. 1-3, Sec. IV-D1 pruning, Sec. IV-E incremental labelling)."""
import numpy as np
import pytest

import oracle as O
import phantoms as P
from oracle import hrw


def test_downsample_constant_blocks_exact():
    fine = np.full((5, 7, 9), 0.123, dtype=np.float32)
    c = O.downsample(fine)
    assert c.shape == (3, 4, 5)
    assert np.all(c == np.float32(0.123))


def test_downsample_integer_means_exact():
    # small integers: every partial sum is exact in FP32 and the divisor is a
    # power of two, so the FP32 mean equals the exact rational mean
    rng = P.uniform(3, 1, np.arange(9 * 6 * 11, dtype=np.uint64))
    fine = np.floor(rng * 256).astype(np.float32).reshape(9, 6, 11)
    c = O.downsample(fine)
    nz, ny, nx = fine.shape
    for Z in range(c.shape[0]):
        for Y in range(c.shape[1]):
            for X in range(c.shape[2]):
                blk = fine[2 * Z:2 * Z + 2, 2 * Y:2 * Y + 2, 2 * X:2 * X + 2].astype(np.float64)
                assert c[Z, Y, X] == blk.sum() / blk.size


def test_downsample_fixed_pairwise_order():
    # children k = x + 2y + 4z = (1, 2^24, 1, -2^24, 0, 0, 0, 0).  Pairwise:
    # (1 + 2^24) rounds to 2^24 (tie to even), (1 - 2^24) = -16777215 exactly,
    # their sum is 1, so the mean is 1/8.  A left-to-right sum would give 0.
    fine = np.zeros((2, 2, 2), np.float32)
    fine[0, 0, 0], fine[0, 0, 1], fine[0, 1, 0], fine[0, 1, 1] = 1.0, 2.0 ** 24, 1.0, -2.0 ** 24
    assert O.downsample(fine)[0, 0, 0] == np.float32(0.125)


def test_pyramid_level_shapes():
    lv = O.pyramid(np.zeros((37, 70, 129), np.float32), 16)
    assert [l.shape for l in lv] == [(3, 5, 9), (5, 9, 17), (10, 18, 33), (19, 35, 65), (37, 70, 129)]
    assert [l.shape for l in O.pyramid(np.zeros((64, 64, 64), np.float32), 32)] == [(32,) * 3, (64,) * 3]


def _labels_from_mask(code, value):
    z, y, x = np.nonzero(code == 1)
    return np.stack([x + 0.5, y + 0.5, z + 0.5], 1), value[z, y, x].astype(np.float64)


def test_single_brick_equals_plain_solve():
    # Eq. 1 only: a volume that fits in one brick is solved by the plain walker
    c = P.random_case((12, 10, 14), seed=5, seed_frac=0.05, levels=[0.0, 1.0])
    leaf = O.leaf_level(O.quantize(c["volume"]))
    xyz, val = _labels_from_mask(c["code"], c["value"])
    t = hrw.run(O.pyramid(leaf, 16), xyz, val, hrw.Opts(brick_size=16, beta=30.0))
    x, _, _, st = O.rw_solve(leaf.astype(np.float64), c["code"], c["value"], 30.0)
    assert st == 0
    assert len(t.P) == 1 and np.max(np.abs(t.P[0] - x)) == 0.0


def test_constant_volume_all_background():
    vol = np.full((32, 32, 32), 0.4, dtype=np.float32)
    xyz = np.array([[3.5, 4.5, 5.5], [20.5, 20.5, 20.5]])
    val = np.array([0.0, 0.0])
    t = hrw.run(O.pyramid(vol, 8), xyz, val, hrw.Opts(brick_size=8, beta=130.0))
    assert t.stats["bricks_solved"] == 1           # root homogeneous -> pruned
    assert t.info[0][(0, 0, 0)].prunable
    assert np.all(t.P[-1] == 0.0)


def test_hierarchy_invariants_and_label_agreement():
    ph = P.vessel_tree(n=64, seed=2, n_segments=30)
    q = O.quantize(ph["volume"], ph["lo"], ph["hi"], True)
    levels = O.pyramid(O.leaf_level(q), 8)
    opts = hrw.Opts(brick_size=8, beta=130.0)
    t = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], opts)
    out = t.P[-1]
    assert out.shape == (64, 64, 64)
    assert out.min() >= -1e-12 and out.max() <= 1 + 1e-12
    # user labels are exact in every solved leaf brick (no conflicts there);
    # inside pruned regions the leaf holds the upsampled coarse result (H_p)
    seeds, conf = hrw.rasterize(ph["labels_xyz"], ph["labels_value"], len(levels) - 1, len(levels) - 1, out.shape)
    assert not conf
    checked = 0
    for (z, y, x), v in seeds.items():
        if (z // 8, y // 8, x // 8) in t.info[-1]:
            assert out[z, y, x] == v
            checked += 1
    assert checked > 0
    # Table IV of the paper: pruning leaves the binary result essentially unchanged
    full = hrw.run(levels, ph["labels_xyz"], ph["labels_value"],
                   hrw.Opts(brick_size=8, beta=130.0, prune_hom=False, prune_dt=False))
    assert full.stats["bricks_solved"] > t.stats["bricks_solved"]
    agree = np.mean((out > 0.5) == (full.P[-1] > 0.5))
    assert agree >= 0.999


def test_conflict_blocks_pruning_and_stays_unseeded():
    vol = np.full((16, 16, 16), 0.4, dtype=np.float32)
    # two labels 1 voxel apart at the leaf: same voxel at the root (s = 4 -> K = 2)
    xyz = np.array([[8.5, 8.5, 8.5], [9.5, 8.5, 8.5], [1.5, 1.5, 1.5]])
    val = np.array([1.0, 0.0, 0.0])
    levels = O.pyramid(vol, 4)
    K = len(levels) - 1
    seeds, conf = hrw.rasterize(xyz, val, K, 0, levels[0].shape)
    assert (2, 2, 2) in conf and (2, 2, 2) not in seeds
    t = hrw.run(levels, xyz, val, hrw.Opts(brick_size=4, beta=130.0))
    assert t.info[0][(0, 0, 0)].cfl and not t.info[0][(0, 0, 0)].prunable
    assert t.P[-1][8, 8, 8] == 1.0 and t.P[-1][8, 8, 9] == 0.0


def test_surface_bricks_grow_like_two_thirds():
    # Appendix: bricks intersecting a surface grow as O(B^(2/3)).  With the
    # noise-free ball, active leaf bricks hug the sphere; doubling n (B x 8)
    # multiplies them by about 4.
    counts, Bs = [], []
    for n in (32, 64, 128):
        c = P.ball_case(n=n, seed=1, radius=0.3 * n, sigma=0.0)
        h = n // 2
        xyz = np.array([[h + 0.5, h + 0.5, h + 0.5], [1.5, 1.5, 1.5], [n - 1.5, n - 1.5, n - 1.5]])
        val = np.array([1.0, 0.0, 0.0])
        levels = O.pyramid(c["volume"], 4)
        t = hrw.run(levels, xyz, val, hrw.Opts(brick_size=4, beta=130.0))
        counts.append(len(t.info[-1]))
        Bs.append((n // 4) ** 3)
    slope = np.polyfit(np.log(Bs), np.log(counts), 1)[0]
    assert 0.5 < slope < 0.8, (counts, slope)


def test_incremental_without_new_labels_reuses_everything():
    ph = P.vessel_tree(n=32, seed=3, n_segments=10)
    q = O.quantize(ph["volume"], ph["lo"], ph["hi"], True)
    levels = O.pyramid(O.leaf_level(q), 8)
    t = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], hrw.Opts(brick_size=8, beta=130.0))
    u = hrw.update(t, np.zeros((0, 3)), np.zeros(0))
    assert u.stats["bricks_solved"] == 1                # only the root, found similar
    assert u.info[0][(0, 0, 0)].similar
    assert np.all(u.P[-1] == t.P[-1])


def test_incremental_close_to_full_rerun():
    ph = P.vessel_tree(n=64, seed=4, n_segments=30)
    q = O.quantize(ph["volume"], ph["lo"], ph["hi"], True)
    levels = O.pyramid(O.leaf_level(q), 8)
    opts = hrw.Opts(brick_size=8, beta=130.0)
    n0 = len(ph["labels_value"]) - 6
    t = hrw.run(levels, ph["labels_xyz"][:n0], ph["labels_value"][:n0], opts)
    u = hrw.update(t, ph["labels_xyz"][n0:], ph["labels_value"][n0:])
    f = hrw.run(levels, ph["labels_xyz"], ph["labels_value"], opts)
    assert u.stats["bricks_solved"] < f.stats["bricks_solved"] + 1
    assert np.mean((u.P[-1] > 0.5) == (f.P[-1] > 0.5)) >= 0.995


def test_upsample_pins():
    # voxel-centre aligned trilinear 2x upsampling of a linear ramp is exact
    # inside (clamp-to-edge only touches the outermost voxels)
    prev = np.arange(8, dtype=np.float64)[None, None, :] * np.ones((4, 4, 1))
    up = hrw.upsample(prev, (8, 8, 16))
    expect = (np.arange(16) + 0.5) / 2.0 - 0.5
    assert np.allclose(up[0, 0, 1:-1], expect[1:-1], atol=0, rtol=0)
    assert up[0, 0, 0] == 0.0 and up[0, 0, -1] == 7.0


def test_multiclass_hierarchy_sums_to_one():
    # One problem per class (class k's strokes as 1, the others as 0; a voxel
    # with strokes of two classes unseeded in every problem): at the root the
    # class probabilities sum to one (Sec. III-B); the border seeds of every
    # finer neighbourhood are interpolated parent probabilities, so without
    # pruning the sum stays one at every level (to solver tolerance).  The
    # 64^3 case has strokes of different classes in one coarse voxel.
    for shape, kw in (((24, 24, 24), dict(n_segments=6, n_blobs=8, strokes_per_class=2, stroke_len=30)),
                      ((64, 64, 64), dict(n_segments=20, n_blobs=30))):
        _sum_to_one(shape, kw)


def _sum_to_one(shape, kw):
    c = P.multiclass_case(shape, seed=2 if shape[0] == 24 else 1, n_updates=0, **kw)
    q = O.quantize(c["volume"], 0.0, 5000.0, True)
    levels = O.pyramid(O.leaf_level(q), 8)
    oo = hrw.Opts(brick_size=8, beta=130.0, prune_hom=False, prune_dt=False)
    fields = []
    for k in range(3):
        xyz, val, cls = P.class_labels(c["strokes"], k)
        fields.append(hrw.run(levels, xyz, val, oo, labels_cls=cls).P)
    for lev in range(len(levels)):
        total = fields[0][lev] + fields[1][lev] + fields[2][lev]
        assert np.max(np.abs(total - 1.0)) <= 1e-9, lev

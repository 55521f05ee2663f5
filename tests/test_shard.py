"""Level sharding (multi-GPU partition and exchange) on the CPU: the Morton
order and partition by hand, and two gloo ranks refining a tree level by level
through paper_2103_09564_gb300.shard (partition, all_gather exchange, import)
with the oracle's node solve as the per-rank compute.  The two-rank run must
give the single-rank oracle run exactly: the same node sets, decisions and
fields at every level."""
import os

import numpy as np
import pytest

import oracle as O
import phantoms as P
from oracle import hrw

from paper_2103_09564_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _interleave(x, y, z):
    c = 0
    for i in range(21):
        c |= ((x >> i) & 1) << (3 * i) | ((y >> i) & 1) << (3 * i + 1) | ((z >> i) & 1) << (3 * i + 2)
    return c


def test_morton_code_is_the_bit_interleave():
    rs = np.random.default_rng(0)
    pts = rs.integers(0, 1 << 21, size=(200, 3))
    got = shard.morton_code(pts[:, 0], pts[:, 1], pts[:, 2])
    for (x, y, z), g in zip(pts, got):
        assert int(g) == _interleave(int(x), int(y), int(z))
    # the 2 x 2 x 2 block: x fastest
    b = [(x, y, z) for z in range(2) for y in range(2) for x in range(2)]
    assert list(shard.morton_code(*np.array(b).T)) == list(range(8))


def test_partition_contiguous_balanced_and_complete():
    nbx, nby, nbz = 5, 3, 4
    ids = np.arange(nbx * nby * nbz)[::-1]
    order = shard.morton_order(ids, nbx, nby)
    for n in (1, 2, 3, 7):
        parts = shard.partition(ids, nbx, nby, n)
        assert len(parts) == n
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1 and sum(sizes) == len(ids)
        assert np.array_equal(np.concatenate(parts), order)        # contiguous ranges, in order
    assert [len(p) for p in shard.partition(ids[:3], nbx, nby, 5)] == [1, 1, 1, 0, 0]


# flags of the library's node records, reproduced for the oracle backend
SOLVED, PRUNABLE, HOM, DT, CFL = 1, 2, 4, 8, 16


class OracleShard:
    """The per-rank compute of a sharded refinement, done by the oracle's
    node solve (hrw._solve_node) on this rank's copy of the level fields."""

    def __init__(self, levels, opts):
        self.levels, self.o = levels, opts
        self.P, self.info = [], []
        self.active = [(0, 0, 0)]
        self.cur = None
        self.lvl = None

    def brick_grid(self, k):
        nb = hrw.brick_counts(self.levels[k].shape, self.o.brick_size)
        return nb[2], nb[1]

    def _id(self, k, b):
        nbx, nby = self.brick_grid(k)
        return (b[0] * nby + b[1]) * nbx + b[2]

    def _b(self, k, i):
        nbx, nby = self.brick_grid(k)
        return (int(i // (nbx * nby)), int((i // nbx) % nby), int(i % nbx))

    def level_nodes(self, k):
        return np.array(sorted(self._id(k, b) for b in self.active), dtype=np.int64)

    def _open(self, k):
        if self.cur is None:
            shape = self.levels[k].shape
            self.up = hrw.upsample(self.P[k - 1], shape) if k > 0 else None
            self.cur = self.up.copy() if k > 0 else np.zeros(shape)
            self.lvl = {}
            self.seeds, self.cfl = hrw.rasterize(self.xyz, self.val, len(self.levels) - 1, k, shape)

    def solve(self, k, ids, labels=None):
        if labels is not None:
            self.xyz, self.val = np.asarray(labels[0]), np.asarray(labels[1])
        self._open(k)
        init = self.cur.copy()
        for i in ids:
            b = self._b(k, i)
            out, box, cfl, _, _, _ = hrw._solve_node(k, b, self.levels[k], self.up, init, self.seeds, self.cfl,
                                                     self.o, self.levels[k].shape)
            (z0, z1), (y0, y1), (x0, x1) = box
            self.cur[z0:z1, y0:y1, x0:x1] = out
            ni = hrw.NodeInfo(solved=True)
            hrw._flags(out, cfl, self.o, ni)
            self.lvl[b] = ni
        return {}

    def export(self, k, ids):
        s = self.o.brick_size
        vals = np.zeros((len(ids), s ** 3))
        flags = np.zeros(len(ids), np.int32)
        stats = np.zeros((len(ids), 3))
        for j, i in enumerate(ids):
            b = self._b(k, i)
            blk = np.zeros((s, s, s))
            sub = self.cur[b[0] * s:(b[0] + 1) * s, b[1] * s:(b[1] + 1) * s, b[2] * s:(b[2] + 1) * s]
            blk[:sub.shape[0], :sub.shape[1], :sub.shape[2]] = sub
            vals[j] = blk.ravel()
            ni = self.lvl[b]
            flags[j] = SOLVED | PRUNABLE * ni.prunable | HOM * ni.hom | DT * ni.dt | CFL * ni.cfl
            stats[j] = (ni.mn, ni.mx, 0.0)
        return {"nodes": np.asarray(ids, np.int64), "flags": flags, "stats": stats, "values": vals}

    def import_(self, k, part):
        s = self.o.brick_size
        self._open(k)
        for j, i in enumerate(np.asarray(part["nodes"])):
            b = self._b(k, int(i))
            blk = np.asarray(part["values"][j]).reshape(s, s, s)
            sub = self.cur[b[0] * s:(b[0] + 1) * s, b[1] * s:(b[1] + 1) * s, b[2] * s:(b[2] + 1) * s]
            sub[...] = blk[:sub.shape[0], :sub.shape[1], :sub.shape[2]]
            f = int(part["flags"][j])
            st = np.asarray(part["stats"][j])
            self.lvl[b] = hrw.NodeInfo(solved=True, mn=float(st[0]), mx=float(st[1]), hom=bool(f & HOM),
                                       dt=bool(f & DT), cfl=bool(f & CFL), prunable=bool(f & PRUNABLE))

    def finish(self, k):
        self.P.append(self.cur)
        self.info.append(self.lvl)
        nxt = []
        if k + 1 < len(self.levels):
            for b, ni in self.lvl.items():
                if not ni.prunable:
                    nxt.extend(hrw._children(b, self.levels[k + 1].shape, self.o.brick_size))
        self.active = sorted(set(nxt))
        self.cur = None
        return {}


def _case():
    ph = P.vessel_tree(n=64, seed=2, n_segments=30)
    q = O.quantize(ph["volume"], ph["lo"], ph["hi"], True)
    levels = O.pyramid(O.leaf_level(q), 8)
    return levels, ph["labels_xyz"], ph["labels_value"].astype(np.float64), hrw.Opts(brick_size=8, beta=130.0)


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        levels, xyz, val, o = _case()
        sh = OracleShard(levels, o)
        mine = []
        for k in range(len(levels)):
            ids, _ = shard.refine_level_sharded(sh, k, rank, world, labels=(xyz, val) if k == 0 else None)
            mine.append(len(ids))
        np.savez(out_path, *sh.P, counts=np.array(mine),
                 flags=np.array([[k, *b, int(ni.prunable), int(ni.hom), int(ni.dt), int(ni.cfl)]
                                 for k, lvl in enumerate(sh.info) for b, ni in sorted(lvl.items())]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_tree(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_run_rank, args=(r, 2, port, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    levels, xyz, val, o = _case()
    ref = hrw.run(levels, xyz, val, o)
    ref_flags = np.array([[k, *b, int(ni.prunable), int(ni.hom), int(ni.dt), int(ni.cfl)]
                          for k, lvl in enumerate(ref.info) for b, ni in sorted(lvl.items())])
    for path in outs:
        d = np.load(path)
        for k in range(len(levels)):
            assert np.array_equal(d[f"arr_{k}"], ref.P[k]), k
        assert np.array_equal(d["flags"], ref_flags)
    # both ranks solved a share of every level with more than one node
    c0, c1 = np.load(outs[0])["counts"], np.load(outs[1])["counts"]
    per_level = [len(lvl) for lvl in ref.info]
    assert list(c0 + c1) == per_level
    assert all(min(a, b) >= 1 for a, b, n in zip(c0, c1, per_level) if n > 1)


def _run_rank(rank, world, port, out_path):
    import sys
    # the ranks share the host's cores: split the OpenMP threads of the
    # oracle's solves before anything loads the OpenMP runtime
    os.environ["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 2) // world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_shard import _rank_main
    _rank_main(rank, world, port, out_path)

"""Level sharding of the hierarchical walker over several GPUs.

The nodes (bricks) of one level are independent problems once the level above
is final (Sec. IV-D3): every node reads only the filled parent level (border
seeds and initial guess, Eqs. 2-3) and the labels.  So N ranks, each holding
the pyramid and its own copy of the tree, refine a level together:

1. every rank lists the level's nodes (the same list everywhere: every rank
   finished the same parent level);
2. the list, in Morton (Z-order) order of the brick coordinates, is cut into N
   contiguous ranges of equal size (+-1); a rank solves its range;
3. one exchange per level: every rank's solved nodes -- their values (s^3
   floats each), RW_NODE_* flags and min / max / max-diff statistics -- are
   gathered on all ranks (torch.distributed all_gather; NCCL keeps the values
   on the device, gloo on the host);
4. every rank imports the other ranks' nodes and closes the level: the fill of
   absent nodes and the next level's node list are computed identically on
   every rank from identical data.

A contiguous Morton range keeps a rank's bricks spatially close (their
neighbourhoods overlap in the parent level they read).  No kernel waits on
another rank: the only communication is the host-driven collective between
levels.  This module holds the partition and the exchange; the solves run in
the library (rw_refine_level_nodes and its companions, include/rw_api.h).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi, _check, _labels, load

__all__ = ["morton_code", "morton_order", "partition", "exchange", "TreeShard", "refine_level_sharded",
           "run_sharded"]


def _spread3(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the bits of v (21 bits used)."""
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_code(bx, by, bz) -> np.ndarray:
    """Z-order code of brick coordinates: bit i of x, y, z at bits 3i, 3i+1, 3i+2."""
    return _spread3(bx) | (_spread3(by) << np.uint64(1)) | (_spread3(bz) << np.uint64(2))


def morton_order(ids, nbx: int, nby: int) -> np.ndarray:
    """Node ids (brick indices (bz * nby + by) * nbx + bx) sorted by Morton code."""
    ids = np.asarray(ids, dtype=np.int64).reshape(-1)
    bx, by, bz = ids % nbx, (ids // nbx) % nby, ids // (nbx * nby)
    return ids[np.argsort(morton_code(bx, by, bz), kind="stable")]


def partition(ids, nbx: int, nby: int, n_ranks: int) -> list:
    """Contiguous ranges of the Morton order, one per rank, sizes equal +-1
    (the first len % n_ranks ranks take one node more)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = morton_order(ids, nbx, nby)
    q, r = divmod(len(order), n_ranks)
    out, lo = [], 0
    for k in range(n_ranks):
        hi = lo + q + (1 if k < r else 0)
        out.append(order[lo:hi].copy())
        lo = hi
    return out


_KEYS = ("nodes", "flags", "stats", "values")


def exchange(part: dict, group=None) -> list:
    """All-gather one rank's solved nodes {nodes int64 [n], flags int32 [n],
    stats float32 [n, 3], values float32 [n, s^3]} (numpy arrays or torch
    tensors) over `group`; returns every rank's part, in rank order, as torch
    tensors (values on the device for NCCL, on the host for gloo)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    t = {k: torch.as_tensor(part[k]).to(dev) for k in _KEYS}
    n = torch.tensor([t["nodes"].shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    got = [dict() for _ in range(ws)]
    for k in _KEYS:
        x = t[k]
        pad = torch.zeros((m,) + tuple(x.shape[1:]), dtype=x.dtype, device=dev)
        pad[:x.shape[0]] = x
        bufs = [torch.empty_like(pad) for _ in range(ws)]
        dist.all_gather(bufs, pad, group=group)
        for r in range(ws):
            got[r][k] = bufs[r][:counts[r]]
    return got


class TreeShard:
    """A rank's view of a library tree (paper_2103_09564_gb300.Tree) for
    level sharding: list, solve, export, import, finish."""

    def __init__(self, tree):
        self.tree = tree
        self.s = tree.opts.brick_size

    def brick_grid(self, k):
        x, y, z = self.tree.pyr.dims[k]
        return (x + self.s - 1) // self.s, (y + self.s - 1) // self.s

    def level_nodes(self, k) -> np.ndarray:
        n = ctypes.c_int64(0)
        _check(load().rw_tree_level_nodes(self.tree.h, k, ctypes.byref(n), None))
        ids = np.zeros(n.value, dtype=np.int64)
        _check(load().rw_tree_level_nodes(self.tree.h, k, ctypes.byref(n), ids.ctypes.data))
        return ids

    def solve(self, k, ids, labels=None) -> dict:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        st = _abi.rw_stats()
        if labels is not None:
            lab, keep = _labels(*labels)
            _check(load().rw_refine_level_nodes(self.tree.h, k, ctypes.byref(lab), ids.ctypes.data, len(ids),
                                                ctypes.byref(st), None))
        else:
            _check(load().rw_refine_level_nodes(self.tree.h, k, None, ids.ctypes.data, len(ids), ctypes.byref(st),
                                                None))
        return st.as_dict()

    def export(self, k, ids, values_out=None) -> dict:
        """Solved nodes `ids` of the open level; values into `values_out`
        (a [n, s^3] float32 CUDA tensor or numpy array; numpy by default)."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        n = len(ids)
        flags = np.zeros(n, dtype=np.int32)
        stats = np.zeros((n, 3), dtype=np.float32)
        vals = values_out if values_out is not None else np.zeros((n, self.s ** 3), dtype=np.float32)
        vp = vals.data_ptr() if hasattr(vals, "data_ptr") else vals.ctypes.data
        _check(load().rw_tree_export_nodes(self.tree.h, k, ids.ctypes.data, n, flags.ctypes.data, stats.ctypes.data,
                                           vp if n else None, None))
        return {"nodes": ids, "flags": flags, "stats": stats, "values": vals}

    def import_(self, k, part: dict):
        ids = np.ascontiguousarray(_host(part["nodes"]), dtype=np.int64)
        flags = np.ascontiguousarray(_host(part["flags"]), dtype=np.int32)
        stats = np.ascontiguousarray(_host(part["stats"]), dtype=np.float32)
        vals = part["values"]
        if hasattr(vals, "is_cuda") and vals.is_cuda:
            vals = vals.contiguous()
            vp = vals.data_ptr()
        else:
            vals = np.ascontiguousarray(_host(vals), dtype=np.float32)
            vp = vals.ctypes.data
        _check(load().rw_tree_import_nodes(self.tree.h, k, ids.ctypes.data, len(ids), flags.ctypes.data,
                                           stats.ctypes.data, vp if len(ids) else None, None))

    def finish(self, k) -> dict:
        st = _abi.rw_stats()
        _check(load().rw_refine_level_finish(self.tree.h, k, ctypes.byref(st), None))
        return st.as_dict()


def _host(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def refine_level_sharded(shard, k, rank, n_ranks, group=None, labels=None, exchange_fn=None):
    """Refine level k together with the other ranks of `group`: solve this
    rank's Morton range, exchange, import the others' nodes, close the level.
    `shard` offers level_nodes / brick_grid / solve / export / import_ /
    finish (TreeShard for the library).  Returns (this rank's node ids, the
    solve's stats)."""
    ids = shard.level_nodes(k)
    nbx, nby = shard.brick_grid(k)
    mine = partition(ids, nbx, nby, n_ranks)[rank]
    st = shard.solve(k, mine, labels if k == 0 else None)
    parts = (exchange_fn or exchange)(shard.export(k, mine), group)
    for r, part in enumerate(parts):
        if r != rank:
            shard.import_(k, part)
    shard.finish(k)
    return mine, st


def run_sharded(shard, n_levels, xyz, value, cls=None, group=None):
    """A full top-down refinement (Eqs. 1-3 with pruning) by the ranks of
    `group` (torch.distributed initialised): level by level, each rank solving
    its Morton range of the level's nodes.  Returns this rank's solve stats
    per level."""
    import torch.distributed as dist
    rank, n_ranks = dist.get_rank(group), dist.get_world_size(group)
    out = []
    for k in range(n_levels):
        lab = (xyz, value, cls) if k == 0 else None
        out.append(refine_level_sharded(shard, k, rank, n_ranks, group, labels=lab)[1])
    return out

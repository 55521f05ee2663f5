"""GB300 hierarchical random walker — Python binding of librw.so.

Argument marshalling only: every step of the solve runs in the CUDA library
behind include/rw_api.h.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; CUDA tensors are used in place, host arrays are staged by the library.
When librw.so is missing every call raises (there is no CPU fallback).

Names follow the C ABI:
  rw_solve, rw_solve_adjoint                       plain walker (Sec. III-B) and its adjoint
  rw_build_pyramid -> Pyramid                      LOD pyramid (Sec. III-A)
  Tree.refine_level / Tree.update_seeds            H_p (Sec. IV) and incremental labelling (Sec. IV-E)
  RWSolveFn                                        torch.autograd.Function over both solves
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (RW_CODE_ABSENT, RW_CODE_FREE, RW_CODE_SEED, RW_FP64, RW_MIXED, RW_NODE_CFL,  # noqa: F401
                   RW_NODE_CFL_ADDED, RW_NODE_CHANGED, RW_NODE_DT, RW_NODE_HOM, RW_NODE_NO_SEEDS, RW_NODE_PRUNABLE,
                   RW_NODE_REUSED,
                   RW_NODE_SIMILAR, RW_NODE_SOLVED, RW_STORE_F32, RW_STORE_UNORM16, LibraryMissing)

__all__ = ["RWError", "Opts", "rw_solve", "rw_solve_noalloc", "rw_solve_adjoint", "rw_build_pyramid", "Pyramid", "Tree",
           "trees_argmax", "trees_argmax_changed", "update_trees", "load",
           "release_workspace", "version"]


class RWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_abi.STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def load():
    return _abi.load()


def version() -> str:
    return load().rw_version().decode()


def release_workspace():
    _check(load().rw_release_workspace())


def _check(st: int, allow=()):
    if st != _abi.RW_OK and st not in allow:
        raise RWError(st, load().rw_last_error().decode())
    return st


def Opts(**kw) -> _abi.rw_opts:
    """rw_opts with the library defaults, overridden by keyword (precision may
    be 'mixed'/'fp64', tile a name such as '40x8', weight 'gaussian'/'poisson'
    -- for 'poisson', beta is the count that g = 1 stands for --, leaf_field
    'pyramid'/'hbm'/'host'/'host_all')."""
    o = _abi.rw_opts()
    load().rw_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"mixed": RW_MIXED, "fp64": RW_FP64}[v]
        if k == "tile" and isinstance(v, str):
            v = _abi.RW_TILE[v]
        if k == "weight" and isinstance(v, str):
            v = {"gaussian": 0, "poisson": 1}[v]
        if k == "leaf_field" and isinstance(v, str):
            v = {"pyramid": _abi.RW_LEAF_AS_PYRAMID, "hbm": _abi.RW_LEAF_HBM, "host": _abi.RW_LEAF_HOST,
                 "host_all": _abi.RW_FIELDS_HOST}[v]
        if isinstance(v, bool):
            v = int(v)
        setattr(o, k, v)
    return o


def _torch():
    import torch
    return torch


class _Arr:
    """Pointer + lifetime holder for a torch tensor or numpy array."""

    def __init__(self, a, dtype=None):
        self.obj = a
        if a is None:
            self.ptr = None
            self.cuda = False
            return
        if isinstance(a, np.ndarray):
            if dtype is not None and a.dtype != dtype:
                a = a.astype(dtype)
            a = np.ascontiguousarray(a)
            self.obj = a
            self.ptr = a.ctypes.data
            self.cuda = False
        else:
            torch = _torch()
            if dtype is not None:
                td = {np.float32: torch.float32, np.uint16: torch.uint16 if hasattr(torch, "uint16") else None,
                      np.uint8: torch.uint8, np.float64: torch.float64}[dtype]
                if td is not None and a.dtype != td:
                    a = a.to(td)
            a = a.contiguous()
            self.obj = a
            self.ptr = a.data_ptr()
            self.cuda = a.is_cuda


def _stream(*arrs):
    for a in arrs:
        if a is not None and getattr(a, "cuda", False):
            torch = _torch()
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _volume(vol, lo, hi, normalize, storage, batch_dims):
    shape = tuple(vol.shape)
    if batch_dims:
        b, dz, dy, dx = shape
    else:
        b, (dz, dy, dx) = 1, shape
    is_u16 = (vol.dtype == np.uint16) or (str(getattr(vol, "dtype", "")) == "torch.uint16")
    a = _Arr(vol) if is_u16 else _Arr(vol, np.float32)
    v = _abi.rw_volume()
    v.data = a.ptr
    v.dtype = _abi.RW_U16 if is_u16 else _abi.RW_F32
    v.storage = storage
    v.dims[0], v.dims[1], v.dims[2] = dx, dy, dz
    v.batch = b
    v.lo, v.hi, v.normalize = lo, hi, int(normalize)
    return v, a, (b, dz, dy, dx)


def _empty_like_f32(ref, shape):
    if isinstance(ref, np.ndarray):
        return np.empty(shape, dtype=np.float32)
    torch = _torch()
    return torch.empty(shape, dtype=torch.float32, device=ref.device)


def rw_solve(volume, code, value=None, opts=None, x0=None, out=None, *, lo=0.0, hi=1.0, normalize=False,
             storage=RW_STORE_UNORM16, allow_not_converged=False):
    """Plain random walker (Sec. III-B).  volume: (Z,Y,X) or (B,Z,Y,X) float32 or
    uint16; code: uint8 (0 free, 1 seed, 2 absent); value: float32 seed values.
    Returns (x, stats) with x float32 of the volume's shape."""
    batch = len(volume.shape) == 4
    v, va, shp = _volume(volume, lo, hi, normalize, storage, batch)
    c = _Arr(code, np.uint8)
    val = _Arr(value, np.float32)
    xi = _Arr(x0, np.float32)
    if out is None:
        out = _empty_like_f32(volume, tuple(volume.shape))
    o = _Arr(out)
    sm = _abi.rw_seed_mask(c.ptr, val.ptr)
    st = _abi.rw_stats()
    opts = opts if opts is not None else Opts()
    rc = load().rw_solve(ctypes.byref(v), ctypes.byref(sm), ctypes.byref(opts), xi.ptr, o.ptr, ctypes.byref(st),
                         _stream(va, c, val, xi, o))
    _check(rc, allow=(_abi.RW_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    d = st.as_dict()
    d["status"] = rc
    return o.obj, d


def rw_solve_noalloc(volume, code, value=None, opts=None, x0=None, out=None, *, lo=0.0, hi=1.0, normalize=False,
                     stream=None):
    """rw_solve for callers that cannot allocate device memory: every array
    must already live on the volume's GPU (CUDA tensors, `out` included when
    given; without `out` this wrapper allocates the result tensor, the
    library call itself allocates nothing), the scratch is the library's
    fixed device array (at most RW_NOALLOC_MAX_VOXELS voxels).  The call runs
    with the volume's device current, on `stream` (a torch.cuda.Stream or a
    raw cudaStream_t handle; default: that device's current torch stream).
    Returns (x, stats)."""
    torch = _torch()
    batch = len(volume.shape) == 4
    v, va, shp = _volume(volume, lo, hi, normalize, RW_STORE_UNORM16, batch)
    c = _Arr(code, np.uint8)
    val = _Arr(value, np.float32)
    xi = _Arr(x0, np.float32)
    dev = volume.device if hasattr(volume, "device") and getattr(volume, "is_cuda", False) else None
    if out is None:
        out = torch.empty(tuple(volume.shape), dtype=torch.float32, device=dev if dev is not None else "cpu")
    o = _Arr(out)
    sm = _abi.rw_seed_mask(c.ptr, val.ptr)
    st = _abi.rw_stats()
    opts = opts if opts is not None else Opts()
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream if dev is not None else 0
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    if dev is not None:
        with torch.cuda.device(dev):
            rc = load().rw_solve_noalloc(ctypes.byref(v), ctypes.byref(sm), ctypes.byref(opts), xi.ptr, o.ptr,
                                         ctypes.byref(st), ctypes.c_void_p(stream))
    else:
        rc = load().rw_solve_noalloc(ctypes.byref(v), ctypes.byref(sm), ctypes.byref(opts), xi.ptr, o.ptr,
                                     ctypes.byref(st), ctypes.c_void_p(stream))
    _check(rc)
    d = st.as_dict()
    d["status"] = rc
    return o.obj, d


def rw_solve_adjoint(volume, code, x, dloss_dx, opts=None, *, lo=0.0, hi=1.0, normalize=False,
                     storage=RW_STORE_F32, want_dg=True):
    """Adjoint solve: returns (dl/dg, dl/dbeta per volume (float64 numpy), stats)."""
    batch = len(volume.shape) == 4
    v, va, shp = _volume(volume, lo, hi, normalize, storage, batch)
    c = _Arr(code, np.uint8)
    xa = _Arr(x, np.float32)
    dl = _Arr(dloss_dx, np.float32)
    dg = _Arr(_empty_like_f32(volume, tuple(volume.shape))) if want_dg else _Arr(None)
    db = np.zeros(shp[0], dtype=np.float64)
    sm = _abi.rw_seed_mask(c.ptr, None)
    st = _abi.rw_stats()
    opts = opts if opts is not None else Opts()
    rc = load().rw_solve_adjoint(ctypes.byref(v), ctypes.byref(sm), ctypes.byref(opts), xa.ptr, dl.ptr, dg.ptr,
                                 db.ctypes.data, ctypes.byref(st), _stream(va, c, xa, dl, dg))
    _check(rc)
    return dg.obj, db, st.as_dict()


class Pyramid:
    """LOD pyramid owned by the library (Sec. III-A)."""

    def __init__(self, handle):
        self.h = ctypes.c_void_p(handle)
        n = ctypes.c_int32(0)
        _check(load().rw_pyramid_info(self.h, ctypes.byref(n), None))
        dims = np.zeros((n.value, 3), dtype=np.int64)
        _check(load().rw_pyramid_info(self.h, ctypes.byref(n), dims.ctypes.data))
        self.dims = [tuple(int(v) for v in d) for d in dims]   # (x, y, z) per level, root first

    @property
    def levels(self):
        return len(self.dims)

    def shape(self, k):
        x, y, z = self.dims[k]
        return (z, y, x)

    def read_level(self, k, out=None):
        if out is None:
            out = np.empty(self.shape(k), dtype=np.float32)
        o = _Arr(out)
        _check(load().rw_pyramid_read_level(self.h, k, o.ptr, _stream(o)))
        return o.obj

    def free(self):
        if self.h:
            load().rw_pyramid_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


RW_PYR_LEAF_HOST, RW_PYR_HOST_ALL = _abi.RW_PYR_LEAF_HOST, _abi.RW_PYR_HOST_ALL


def rw_build_pyramid(volume, brick_size=32, *, lo=0.0, hi=1.0, normalize=False, leaf_in_host=False,
                     all_in_host=False) -> Pyramid:
    """leaf_in_host: keep the leaf level (and the leaf fields of trees built on
    this pyramid) in mapped host memory, read and written by the GPU in place
    (out-of-core placement for volumes whose leaf does not fit in HBM).
    all_in_host: every level there, and every level's field of the trees built
    on it: HBM holds only the working set of a batched level solve."""
    v, va, _ = _volume(volume, lo, hi, normalize, RW_STORE_UNORM16, False)
    h = ctypes.c_void_p(0)
    flags = (RW_PYR_LEAF_HOST if leaf_in_host else 0) | (RW_PYR_HOST_ALL if all_in_host else 0)
    _check(load().rw_build_pyramid_ex(ctypes.byref(v), brick_size, flags, ctypes.byref(h), _stream(va)))
    return Pyramid(h.value)


RW_MAX_CLASSES = 8


def trees_argmax(trees, level=None, box=None, out=None, prob=None):
    """Multi-class labels: argmax over one refined tree per class (ties: the
    lowest class index) on `level` (default: the leaf).  Returns (labels
    uint8, winning probability float32 or None); host (numpy) arrays unless
    CUDA tensors are passed as `out` / `prob`."""
    if not 2 <= len(trees) <= RW_MAX_CLASSES:
        raise ValueError(f"need 2..{RW_MAX_CLASSES} trees")
    pyr = trees[0].pyr
    if level is None:
        level = pyr.levels - 1
    x, y, z = pyr.dims[level]
    b = np.array(box if box is not None else [0, 0, 0, x, y, z], dtype=np.int64)
    shape = (int(b[5] - b[2]), int(b[4] - b[1]), int(b[3] - b[0]))
    if out is None:
        out = np.empty(shape, dtype=np.uint8)
    o = _Arr(out)
    p = _Arr(prob) if prob is not None else None
    arr = (ctypes.c_void_p * len(trees))(*[t.h.value for t in trees])
    _check(load().rw_trees_argmax(arr, len(trees), level, b.ctypes.data, o.ptr, p.ptr if p else None,
                                  _stream(o, *( [p] if p else []))))
    return o.obj, (p.obj if p else None)


def trees_argmax_changed(trees, out, prob=None):
    """After a round in which every tree ran one pass (update_seeds or run),
    recompute the leaf labels in `out` (and the winning probability in
    `prob`) on the leaf bricks that changed in any tree; the rest of `out`
    keeps the previous round's labels.  `out` / `prob`: CUDA tensors or
    page-locked (pinned) host tensors with the leaf level's shape."""
    if not 2 <= len(trees) <= RW_MAX_CLASSES:
        raise ValueError(f"need 2..{RW_MAX_CLASSES} trees")
    o = _Arr(out)
    p = _Arr(prob) if prob is not None else None
    arr = (ctypes.c_void_p * len(trees))(*[t.h.value for t in trees])
    _check(load().rw_trees_argmax_changed(arr, len(trees), o.ptr, p.ptr if p else None,
                                          _stream(o, *([p] if p else []))))
    return o.obj, (p.obj if p else None)


def update_trees(trees, xyz, values, cls=None):
    """update_seeds on every tree at once (one tree per class): the label
    points `xyz` (and classes `cls`) are shared, values[i] are tree i's label
    values.  The nodes of all trees are solved in shared batches level by
    level; returns the statistics summed over the trees."""
    n = len(trees)
    if len(values) != n:
        raise ValueError("one array of label values per tree")
    labs, keep = [], []
    for v in values:
        lab, hold = _labels(xyz, v, cls)
        labs.append(lab)
        keep.append(hold)
    arr_t = (ctypes.c_void_p * n)(*[t.h.value for t in trees])
    arr_l = (_abi.rw_labels * n)(*labs)
    st = _abi.rw_stats()
    _check(load().rw_update_seeds_trees(arr_t, n, arr_l, ctypes.byref(st), None))
    return st.as_dict()


def _labels(xyz, value, cls=None):
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    val = np.ascontiguousarray(np.asarray(value, dtype=np.float32).reshape(-1))
    c = None if cls is None else np.ascontiguousarray(np.asarray(cls, dtype=np.int32).reshape(-1))
    lab = _abi.rw_labels(xyz.ctypes.data, val.ctypes.data, len(val), c.ctypes.data if c is not None else None)
    return lab, (xyz, val, c)


class Tree:
    """Output tree of H_p over a pyramid (Sec. IV); levels refined in order."""

    def __init__(self, pyramid: Pyramid, opts=None):
        self.pyr = pyramid
        self.opts = opts if opts is not None else Opts(brick_size=32)
        h = ctypes.c_void_p(0)
        _check(load().rw_tree_create(pyramid.h, ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h

    def refine_level(self, level, xyz=None, value=None, cls=None):
        st = _abi.rw_stats()
        if xyz is not None:
            lab, keep = _labels(xyz, value, cls)
            _check(load().rw_refine_level(self.h, level, ctypes.byref(lab), ctypes.byref(st), None))
        else:
            _check(load().rw_refine_level(self.h, level, None, ctypes.byref(st), None))
        return st.as_dict()

    def run(self, xyz, value, cls=None):
        """All levels, root to leaf; returns the summed stats.  cls: the class
        of each label in a multi-class labelling (class-aware conflicts)."""
        tot = {}
        for k in range(self.pyr.levels):
            s = self.refine_level(k, xyz if k == 0 else None, value if k == 0 else None, cls if k == 0 else None)
            for key, v in s.items():
                if key in ("iters", "refine_rounds"):
                    tot[key] = max(tot.get(key, 0), v)
                elif key == "rel_resid":
                    tot[key] = max(tot.get(key, 0.0), v)
                else:
                    tot[key] = tot.get(key, 0) + v
        return tot

    def update_seeds(self, xyz, value, cls=None):
        lab, keep = _labels(xyz, value, cls)
        st = _abi.rw_stats()
        _check(load().rw_update_seeds(self.h, ctypes.byref(lab), ctypes.byref(st), None))
        return st.as_dict()

    def read_level(self, level, box=None, out=None):
        x, y, z = self.pyr.dims[level]
        b = np.array(box if box is not None else [0, 0, 0, x, y, z], dtype=np.int64)
        shape = (int(b[5] - b[2]), int(b[4] - b[1]), int(b[3] - b[0]))
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        o = _Arr(out)
        _check(load().rw_tree_read_level(self.h, level, b.ctypes.data, o.ptr, _stream(o)))
        return o.obj

    def node_stats(self, level):
        n = ctypes.c_int64(0)
        _check(load().rw_tree_node_stats(self.h, level, ctypes.byref(n), None, None, None, None))
        fl = np.zeros(n.value, np.int32)
        mn = np.zeros(n.value, np.float32)
        mx = np.zeros(n.value, np.float32)
        md = np.zeros(n.value, np.float32)
        _check(load().rw_tree_node_stats(self.h, level, ctypes.byref(n), fl.ctypes.data, mn.ctypes.data,
                                         mx.ctypes.data, md.ctypes.data))
        x, y, z = self.pyr.dims[level]
        s = self.opts.brick_size
        nb = ((z + s - 1) // s, (y + s - 1) // s, (x + s - 1) // s)
        return fl.reshape(nb), mn.reshape(nb), mx.reshape(nb), md.reshape(nb)

    def free(self):
        if self.h:
            load().rw_tree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def __getattr__(name):
    if name == "RWSolveFn":
        from .autograd import RWSolveFn
        return RWSolveFn
    raise AttributeError(name)

"""ctypes mirror of include/rw_api.h (structures, enums, prototypes)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librw.so")

RW_OK, RW_ERR_INVALID_ARG, RW_ERR_NO_SEEDS, RW_ERR_NOT_CONVERGED, RW_ERR_TIMEOUT, RW_ERR_OOM, RW_ERR_CUDA, \
    RW_ERR_UNIMPLEMENTED = range(8)
STATUS_NAMES = ["RW_OK", "RW_ERR_INVALID_ARG", "RW_ERR_NO_SEEDS", "RW_ERR_NOT_CONVERGED", "RW_ERR_TIMEOUT",
                "RW_ERR_OOM", "RW_ERR_CUDA", "RW_ERR_UNIMPLEMENTED"]
RW_U16, RW_F32 = 0, 1
RW_STORE_UNORM16, RW_STORE_F32 = 0, 1
RW_MIXED, RW_FP64 = 0, 1
RW_LEAF_AS_PYRAMID, RW_LEAF_HBM, RW_LEAF_HOST, RW_FIELDS_HOST = 0, 1, 2, 3
RW_PYR_LEAF_HOST, RW_PYR_HOST_ALL = 1, 2
RW_CODE_FREE, RW_CODE_SEED, RW_CODE_ABSENT = 0, 1, 2
RW_NODE_SOLVED, RW_NODE_PRUNABLE, RW_NODE_HOM, RW_NODE_DT, RW_NODE_CFL, RW_NODE_SIMILAR, RW_NODE_REUSED, \
    RW_NODE_CFL_ADDED, RW_NODE_NO_SEEDS, RW_NODE_CHANGED = 1, 2, 4, 8, 16, 32, 64, 128, 256, 512
RW_NOALLOC_MAX_VOXELS = 262144
RW_NOALLOC_MAX_BATCH = 64
RW_TILE = {"auto": 0, "40x8": 3, "32x8": 7, "s64x11": 20, "s32x22": 21, "s32x20": 22, "s64x8": 23, "s40x20": 24,
           "s40x8": 25, "s32x20_d3": 31, "s64x8_d3": 32, "s32x22_d1": 33, "s64x8_d1": 34, "s64x14_d1": 35,
           "r64x14_d2": 36, "r64x14_d1": 37, "r64x11_d2": 38, "r64x11_d3": 39, "r32x22_d2": 40, "r32x20_d3": 41,
           "r64x13_d3": 42, "r64x12_d3": 43, "r40x20_d2": 44, "r40x20_d3": 45, "r40x8_d2": 46}

# every function declared in include/rw_api.h
EXPORTS = ["rw_opts_default", "rw_last_error", "rw_version", "rw_release_workspace", "rw_solve", "rw_solve_noalloc",
           "rw_solve_adjoint",
           "rw_build_pyramid", "rw_build_pyramid_ex", "rw_pyramid_info", "rw_pyramid_read_level", "rw_pyramid_free", "rw_tree_create",
           "rw_refine_level", "rw_update_seeds", "rw_tree_read_level", "rw_tree_node_stats", "rw_tree_free",
           "rw_trees_argmax", "rw_trees_argmax_changed", "rw_update_seeds_trees", "rw_tree_level_nodes",
           "rw_refine_level_nodes", "rw_tree_export_nodes", "rw_tree_import_nodes", "rw_refine_level_finish"]


class rw_volume(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("dims", ctypes.c_int64 * 3), ("batch", ctypes.c_int64), ("lo", ctypes.c_float),
                ("hi", ctypes.c_float), ("normalize", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rw_seed_mask(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("value", ctypes.c_void_p)]


class rw_labels(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("value", ctypes.c_void_p), ("n", ctypes.c_int64), ("cls", ctypes.c_void_p)]


class rw_opts(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_float), ("w_min", ctypes.c_float), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32), ("refine_rounds", ctypes.c_int32),
                ("brick_size", ctypes.c_int32), ("expand", ctypes.c_float), ("t_hom", ctypes.c_float),
                ("t_bin", ctypes.c_float), ("t_inc", ctypes.c_float), ("prune_hom", ctypes.c_int32),
                ("prune_dt", ctypes.c_int32), ("iters_per_graph", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("batch_bricks", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("weight", ctypes.c_int32),
                ("leaf_field", ctypes.c_int32)]


class rw_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refine_rounds", ctypes.c_int32), ("rel_resid", ctypes.c_double),
                ("voxel_iters", ctypes.c_int64), ("free_voxels", ctypes.c_int64), ("bricks_active", ctypes.c_int64),
                ("bricks_solved", ctypes.c_int64), ("bricks_pruned", ctypes.c_int64),
                ("bricks_reused", ctypes.c_int64), ("bricks_conflict", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("ms", ctypes.c_double), ("ms_solve", ctypes.c_double), ("ms_sweeps", ctypes.c_double),
                ("launches", ctypes.c_int64), ("tile", ctypes.c_int32), ("iters_per_graph", ctypes.c_int32),
                ("not_converged", ctypes.c_int64), ("fp64_fallbacks", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
PROTOTYPES = {
    "rw_opts_default": (None, [ctypes.POINTER(rw_opts)]),
    "rw_last_error": (ctypes.c_char_p, []),
    "rw_version": (ctypes.c_char_p, []),
    "rw_release_workspace": (ctypes.c_int, []),
    "rw_solve": (ctypes.c_int, [ctypes.POINTER(rw_volume), ctypes.POINTER(rw_seed_mask), ctypes.POINTER(rw_opts),
                                _P, _P, ctypes.POINTER(rw_stats), _P]),
    "rw_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(rw_volume), ctypes.POINTER(rw_seed_mask),
                                        ctypes.POINTER(rw_opts), _P, _P, ctypes.POINTER(rw_stats), _P]),
    "rw_solve_adjoint": (ctypes.c_int, [ctypes.POINTER(rw_volume), ctypes.POINTER(rw_seed_mask),
                                        ctypes.POINTER(rw_opts), _P, _P, _P, _P, ctypes.POINTER(rw_stats), _P]),
    "rw_build_pyramid": (ctypes.c_int, [ctypes.POINTER(rw_volume), ctypes.c_int32, ctypes.POINTER(_P), _P]),
    "rw_trees_argmax": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]),
    "rw_trees_argmax_changed": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _P]),
    "rw_build_pyramid_ex": (ctypes.c_int, [ctypes.POINTER(rw_volume), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P),
                                           _P]),
    "rw_pyramid_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), _P]),
    "rw_pyramid_read_level": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "rw_pyramid_free": (None, [_P]),
    "rw_tree_create": (ctypes.c_int, [_P, ctypes.POINTER(rw_opts), ctypes.POINTER(_P)]),
    "rw_refine_level": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rw_labels), ctypes.POINTER(rw_stats), _P]),
    "rw_update_seeds": (ctypes.c_int, [_P, ctypes.POINTER(rw_labels), ctypes.POINTER(rw_stats), _P]),
    "rw_update_seeds_trees": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(rw_labels),
                                             ctypes.POINTER(rw_stats), _P]),
    "rw_tree_read_level": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "rw_tree_node_stats": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _P, _P, _P, _P]),
    "rw_tree_free": (None, [_P]),
    "rw_tree_level_nodes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _P]),
    "rw_refine_level_nodes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rw_labels), _P, ctypes.c_int64,
                                             ctypes.POINTER(rw_stats), _P]),
    "rw_tree_export_nodes": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "rw_tree_import_nodes": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "rw_refine_level_finish": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rw_stats), _P]),
}

_lib = None


class LibraryMissing(RuntimeError):
    pass


def load(path: str | None = None):
    """Load librw.so; raises LibraryMissing (no fallback) when it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise LibraryMissing(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                             " (nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

"""Host-side checks of the C ABI: the library loads without a GPU and exports
every function that include/rw_api.h declares; struct layouts agree."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rw_api.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rw_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_09564_gb300 import build
    build.build()
    from paper_2103_09564_gb300 import _abi
    return _abi.load()


def test_exports_every_declared_function(lib):
    from paper_2103_09564_gb300 import _abi
    decl = _declared()
    assert decl, "no declarations parsed"
    assert sorted(_abi.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_defaults_without_gpu(lib):
    import paper_2103_09564_gb300 as rw
    o = rw.Opts()
    assert o.beta == 130.0 and o.brick_size == 32 and abs(o.expand - 1.25) < 1e-7
    assert abs(o.t_hom - 0.3) < 1e-7 and abs(o.t_bin - 0.01) < 1e-9 and abs(o.t_inc - 0.01) < 1e-9
    assert o.precision == rw.RW_MIXED and o.iters_per_graph % 2 == 0
    assert rw.version().startswith("rw-gb300")


def test_struct_sizes_match_header(lib, tmp_path):
    # compile a tiny C program against the header and compare sizeof()
    from paper_2103_09564_gb300 import _abi
    src = tmp_path / "sz.c"
    src.write_text('#include "rw_api.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu %zu %zu\\n",'
                   'sizeof(rw_volume),sizeof(rw_seed_mask),sizeof(rw_labels),sizeof(rw_opts),sizeof(rw_stats));}\n')
    exe = tmp_path / "sz"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [ctypes.sizeof(t) for t in (_abi.rw_volume, _abi.rw_seed_mask, _abi.rw_labels, _abi.rw_opts,
                                        _abi.rw_stats)]
    assert [int(v) for v in out] == sizes


def test_invalid_arguments_rejected_on_host(lib):
    import paper_2103_09564_gb300 as rw
    from paper_2103_09564_gb300 import _abi
    st = _abi.rw_stats()
    # NULL volume is rejected before any CUDA call
    rc = lib.rw_solve(None, None, None, None, None, ctypes.byref(st), None)
    assert rc == _abi.RW_ERR_INVALID_ARG
    assert b"NULL" in lib.rw_last_error()
    o = rw.Opts()
    o.max_iter = 0
    v = _abi.rw_volume()
    v.data = 1
    v.dims[0] = v.dims[1] = v.dims[2] = 4
    rc = lib.rw_solve(ctypes.byref(v), None, ctypes.byref(o), None, None, ctypes.byref(st), None)
    assert rc == _abi.RW_ERR_INVALID_ARG
    # tile ids: unassigned values and tiles of the other precision are rejected
    for tile, prec in ((1, rw.RW_MIXED), (26, rw.RW_MIXED), (_abi.RW_TILE["40x8"], rw.RW_MIXED),
                       (_abi.RW_TILE["r64x14_d2"], rw.RW_FP64), (47, rw.RW_MIXED)):
        o = rw.Opts(tile=tile, precision=prec)
        rc = lib.rw_solve(ctypes.byref(v), None, ctypes.byref(o), None, None, ctypes.byref(st), None)
        assert rc == _abi.RW_ERR_INVALID_ARG, (tile, prec)


def test_new_entry_points_reject_bad_arguments_on_host(lib):
    import paper_2103_09564_gb300 as rw
    from paper_2103_09564_gb300 import _abi
    st = _abi.rw_stats()
    # no trees: rejected before any CUDA call
    assert lib.rw_update_seeds_trees(None, 0, None, ctypes.byref(st), None) == _abi.RW_ERR_INVALID_ARG
    assert lib.rw_trees_argmax_changed(None, 3, None, None, None) == _abi.RW_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.rw_trees_argmax_changed(arr, 1, None, None, None) == _abi.RW_ERR_INVALID_ARG
    # leaf placement names map to the header's values; an unknown value is rejected
    assert rw.Opts(leaf_field="hbm").leaf_field == _abi.RW_LEAF_HBM
    assert rw.Opts(leaf_field="host").leaf_field == _abi.RW_LEAF_HOST
    assert rw.Opts().leaf_field == _abi.RW_LEAF_AS_PYRAMID
    o = rw.Opts()
    o.leaf_field = 7
    v = _abi.rw_volume()
    v.data = 1
    v.dims[0] = v.dims[1] = v.dims[2] = 4
    rc = lib.rw_solve(ctypes.byref(v), None, ctypes.byref(o), None, None, ctypes.byref(st), None)
    assert rc == _abi.RW_ERR_INVALID_ARG


def test_noalloc_rejects_65_volumes_on_host(lib):
    # the fixed scratch holds at most RW_NOALLOC_MAX_BATCH volumes: a batch of
    # 65 tiny volumes is refused before any CUDA call
    from paper_2103_09564_gb300 import _abi
    v = _abi.rw_volume()
    h = np.zeros((65, 2, 2, 2), np.float32)
    v.data = h.ctypes.data
    v.dims[0] = v.dims[1] = v.dims[2] = 2
    v.batch = 65
    hc = np.ones((65, 2, 2, 2), np.uint8)
    sm = _abi.rw_seed_mask(hc.ctypes.data, None)
    out = np.zeros((65, 2, 2, 2), np.float32)
    st = _abi.rw_stats()
    rc = lib.rw_solve_noalloc(ctypes.byref(v), ctypes.byref(sm), None, None, out.ctypes.data, ctypes.byref(st), None)
    assert rc == _abi.RW_ERR_INVALID_ARG
    assert b"exceed" in lib.rw_last_error() and b"65 volume" in lib.rw_last_error()

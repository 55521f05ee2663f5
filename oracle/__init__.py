"""FP64 CPU oracle of the hierarchical random walker — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA library
(``paper_2103_09564_gb300``) and never imports it.

Contents
  oracle.c   plain FP64 C: quantisation (normalisation reading), one pyramid
             step (Sec. III-A), the random walker system and its Jacobi-PCG
             solve (Sec. III-B, Sec. IV-D2), residual, adjoint gradient.
  hrw.py     the hierarchical procedure H / H_p (Eqs. 1-3, Sec. IV-D1 pruning,
             Sec. IV-E incremental labelling) in plain Python/numpy, each brick
             solved by ``rw_solve`` below.
  adjoint.py dense adjoint for tiny volumes and the matrix-free adjoint.

Pins (``tests/test_oracle_*.py``): dense Cholesky on <= 8^3 voxels, closed
forms (voltage divider, linear ramp), the discrete maximum principle,
multi-class sum-to-one, symmetry, the residual against a dense operator,
bit-exact pyramid cases, single-brick hierarchy == plain solve, tiny trees
and incremental passes rebuilt independently with dense Cholesky node solves,
pruning agreement, B^(2/3) growth, finite differences for the adjoint.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FREE, SEED, ABSENT = 0, 1, 2
W_MIN = 1e-30


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            L.oracle_quantize_f32.argtypes = [P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_int, P]
            L.oracle_quantize_u16.argtypes = [P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_int, P]
            L.oracle_downsample.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.oracle_weight.argtypes = [ctypes.c_double] * 4
            L.oracle_weight.restype = ctypes.c_double
            L.oracle_rw_solve.argtypes = [ctypes.c_int] * 3 + [P, P, P, P, ctypes.c_double, ctypes.c_double,
                                                               ctypes.c_double, ctypes.c_int, P, P, P]
            L.oracle_rw_solve.restype = ctypes.c_int
            L.oracle_residual.argtypes = [ctypes.c_int] * 3 + [P, P, P, P, ctypes.c_double, ctypes.c_double, P]
            L.oracle_residual.restype = ctypes.c_double
            L.oracle_adjoint_grad.argtypes = [ctypes.c_int] * 3 + [P, P, P, P, ctypes.c_double, ctypes.c_double, P]
            L.oracle_adjoint_grad.restype = ctypes.c_double
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def quantize(v: np.ndarray, lo: float = 0.0, hi: float = 1.0, normalize: bool = False) -> np.ndarray:
    """Normalise to [0, 1] (window [lo, hi] when ``normalize``) and store as unorm16."""
    v = np.ascontiguousarray(v)
    q = np.empty(v.shape, dtype=np.uint16)
    if v.dtype == np.float32:
        lib().oracle_quantize_f32(_p(v), v.size, lo, hi, int(normalize), _p(q))
    elif v.dtype == np.uint16:
        lib().oracle_quantize_u16(_p(v), v.size, lo, hi, int(normalize), _p(q))
    else:
        raise TypeError("volume must be float32 or uint16")
    return q


def dequantize(q: np.ndarray) -> np.ndarray:
    """unorm16 -> FP64 intensity q / 65535 (the plain solve's g)."""
    return q.astype(np.float64) / 65535.0


def leaf_level(q: np.ndarray) -> np.ndarray:
    """unorm16 -> FP32 leaf level of the pyramid, q / 65535 rounded to FP32."""
    return (q.astype(np.float32) / np.float32(65535.0)).astype(np.float32)


def downsample(fine: np.ndarray) -> np.ndarray:
    """One 2^3 mean-filter + downsample step (Sec. III-A), FP32, fixed order."""
    fine = np.ascontiguousarray(fine, dtype=np.float32)
    nz, ny, nx = fine.shape
    out = np.empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), dtype=np.float32)
    lib().oracle_downsample(_p(fine), nx, ny, nz, _p(out))
    return out


def pyramid(leaf: np.ndarray, brick_size: int):
    """LOD pyramid levels [root, ..., leaf] (Sec. III-A): halve (ceil) each axis
    until every axis is <= brick_size; that level is the root."""
    levels = [np.ascontiguousarray(leaf, dtype=np.float32)]
    while max(levels[-1].shape) > brick_size:
        levels.append(downsample(levels[-1]))
    return levels[::-1]


def weight(a: float, b: float, beta: float, w_min: float = W_MIN, kind: str = "gaussian") -> float:
    """Edge weight between intensities a, b (Sec. III-B).  kind "poisson": the
    case-study weight for Poisson noise, exp(-(sqrt(n_a) - sqrt(n_b))^2 / 2)
    on counts n = beta * g, evaluated as the Gaussian form on sqrt(g) with
    beta / 2 (the same expression), clamped at w_min."""
    if kind == "poisson":
        return float(lib().oracle_weight(math.sqrt(a), math.sqrt(b), beta / 2.0, w_min))
    return float(lib().oracle_weight(a, b, beta, w_min))


def _weight_form(g, beta, kind):
    """(intensities, beta) of the Gaussian form that gives weights `kind`."""
    if kind == "poisson":
        return np.sqrt(np.asarray(g, dtype=np.float64)), beta / 2.0
    if kind != "gaussian":
        raise ValueError(f"unknown weight kind {kind!r}")
    return g, beta


def rw_solve(g: np.ndarray, code: np.ndarray, xin: np.ndarray, beta: float, w_min: float = W_MIN,
             tol: float = 1e-13, max_iter: int = 200000, rhs: np.ndarray | None = None, kind: str = "gaussian"):
    """Plain random walker (Sec. III-B) by FP64 Jacobi-PCG.

    g: intensities (FP64), code: 0 free / 1 seed / 2 absent, xin: seed values
    on seeds and the initial guess on free voxels.  Returns (x, iters, relres,
    status) with status 0 ok, 2 no seeds, 3 not converged.  kind: the weight
    function ("gaussian", or "poisson" with beta the count scale)."""
    g, beta = _weight_form(g, beta, kind)
    g = np.ascontiguousarray(g, dtype=np.float64)
    code = np.ascontiguousarray(code, dtype=np.uint8)
    xin = np.ascontiguousarray(xin, dtype=np.float64)
    nz, ny, nx = g.shape
    x = np.zeros_like(g)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rh = None if rhs is None else np.ascontiguousarray(rhs, dtype=np.float64)
    st = lib().oracle_rw_solve(nx, ny, nz, _p(g), _p(code), _p(xin), None if rh is None else _p(rh),
                               beta, w_min, tol, max_iter, _p(x), ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value, st


def residual(g, code, x, beta, w_min=W_MIN, rhs=None):
    """(r, ||b||): r = b - A x on free voxels, FP64."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    code = np.ascontiguousarray(code, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.float64)
    nz, ny, nx = g.shape
    r = np.zeros_like(g)
    rh = None if rhs is None else np.ascontiguousarray(rhs, dtype=np.float64)
    bn = lib().oracle_residual(nx, ny, nz, _p(g), _p(code), _p(x), None if rh is None else _p(rh),
                               beta, w_min, _p(r))
    return r, bn


def adjoint_grad(g, code, x, lam, beta, w_min=W_MIN):
    """(dl/dg, dl/dbeta) from the solution x and the adjoint solution lambda."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    code = np.ascontiguousarray(code, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    nz, ny, nx = g.shape
    dg = np.zeros_like(g)
    db = lib().oracle_adjoint_grad(nx, ny, nz, _p(g), _p(code), _p(x), _p(lam), beta, w_min, _p(dg))
    return dg, db


def solve_volume(volume, code, value, beta, lo=0.0, hi=1.0, normalize=False, tol=1e-13,
                 max_iter=200000, w_min=W_MIN, x0=None, kind="gaussian"):
    """Quantise a raw volume, then solve it (the plain path end to end)."""
    q = quantize(volume, lo, hi, normalize)
    g = dequantize(q)
    xin = np.where(code == SEED, value.astype(np.float64), 0.0 if x0 is None else x0)
    return rw_solve(g, code, xin, beta, w_min=w_min, tol=tol, max_iter=max_iter, kind=kind)

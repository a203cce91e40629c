"""FP64 / uint32 reference of the iterated stencil sweep -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain C, compiled with
gcc, ``-ffp-contract=off``) through ctypes and shares nothing with the CUDA
package: no import in either direction, no common header or helper.

What it computes (paper, Section 1): the naive (d+1)-loop stencil, time
outermost, each point the weighted sum of its neighbours at the previous time
step; Section 3.3 (Algorithm 1) and Section 3.4 reorder these updates without
changing them.  The conventions the paper leaves open are listed in the header
of ``oracle.c``.

Pins (``tests/test_oracle_pins.py``, ``tests/test_oracle_vc_pins.py``): Dirichlet sine eigenmodes,
periodic Fourier modes, the binomial closed form and its method of images,
box separability, T-fold self-correlation, mass conservation, dense-matrix
brute force (FP64 and uint32), the adjoint dot-product identity and finite
differences.  No function here is left unpinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

STAR, BOX = 0, 1
DIRICHLET, PERIODIC = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint32)
        ip = ctypes.POINTER(ctypes.c_int32)
        c_int, c_dbl, c_u32, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_int64
        lib.oracle_npoints.argtypes = [c_int, c_int, c_int]
        lib.oracle_offsets.argtypes = [c_int, c_int, c_int, ip]
        lib.oracle_run_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, c_dbl, dp, c_i64, dp]
        lib.oracle_run_u32.argtypes = [c_int, c_int, c_int, i64p, up, c_int, c_u32, up, c_i64, up]
        lib.oracle_points_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, c_dbl, dp, c_i64, c_i64, i64p, dp]
        lib.oracle_points_u32.argtypes = [c_int, c_int, c_int, i64p, up, c_int, c_u32, up, c_i64, c_i64, i64p, up]
        lib.oracle_transpose_step_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, dp, dp]
        lib.oracle_adjoint_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, c_dbl, dp, dp, c_i64, dp, dp, dp]
        lib.oracle_run_vc_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, c_dbl, dp, c_i64, dp]
        lib.oracle_run_vc_u32.argtypes = [c_int, c_int, c_int, i64p, up, c_int, c_u32, up, c_i64, up]
        lib.oracle_adjoint_vc_f64.argtypes = [c_int, c_int, c_int, i64p, dp, c_int, c_dbl, dp, dp, c_i64, dp, dp, dp]
        lib.oracle_sum_f64.argtypes = [c_i64, dp, dp]
        lib.oracle_sumsq_f64.argtypes = [c_i64, dp, dp]
        lib.oracle_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def npoints(d: int, r: int, pattern: int) -> int:
    return _load().oracle_npoints(d, r, pattern)


def offsets(d: int, r: int, pattern: int) -> np.ndarray:
    """Offsets in compact weight order, shape (npoints, d)."""
    np_ = npoints(d, r, pattern)
    out = np.zeros(np_ * d, dtype=np.int32)
    _load().oracle_offsets(d, r, pattern, _p(out, ctypes.c_int32))
    return out.reshape(np_, d)


def _shape(shape):
    return np.ascontiguousarray(np.asarray(shape, dtype=np.int64))


def run(d, r, pattern, shape, w, bkind, bval, u0, T) -> np.ndarray:
    """u_T after T Jacobi steps from u0, FP64."""
    n = _shape(shape)
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(tuple(shape)))
    out = np.empty_like(u0)
    _check(_load().oracle_run_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(w, ctypes.c_double), bkind,
                                  float(bval), _p(u0, ctypes.c_double), int(T), _p(out, ctypes.c_double)), "run_f64")
    return out


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).astype(np.uint32))


def run_int(d, r, pattern, shape, w, bkind, bval, u0, T) -> np.ndarray:
    """u_T in uint32 wraparound arithmetic, returned as int32 (same bits)."""
    n = _shape(shape)
    wu = _u32(np.asarray(w, dtype=np.float64).astype(np.int64))
    u = np.ascontiguousarray(np.asarray(u0).astype(np.int64).astype(np.uint32).reshape(tuple(shape)))
    out = np.empty_like(u)
    _check(_load().oracle_run_u32(d, r, pattern, _p(n, ctypes.c_int64), _p(wu, ctypes.c_uint32), bkind,
                                  int(bval) & 0xFFFFFFFF, _p(u, ctypes.c_uint32), int(T), _p(out, ctypes.c_uint32)),
           "run_u32")
    return out.view(np.int32)


def points(d, r, pattern, shape, w, bkind, bval, u0, T, pts) -> np.ndarray:
    """u_T at the given points (npts x d indices) from their dependency cones, FP64."""
    n = _shape(shape)
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(tuple(shape)))
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int64).reshape(-1, d))
    out = np.empty(pts.shape[0], dtype=np.float64)
    _check(_load().oracle_points_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(w, ctypes.c_double), bkind,
                                     float(bval), _p(u0, ctypes.c_double), int(T), pts.shape[0],
                                     _p(pts, ctypes.c_int64), _p(out, ctypes.c_double)), "points_f64")
    return out


def points_int(d, r, pattern, shape, w, bkind, bval, u0, T, pts) -> np.ndarray:
    n = _shape(shape)
    wu = _u32(np.asarray(w, dtype=np.float64).astype(np.int64))
    u = np.ascontiguousarray(np.asarray(u0).astype(np.int64).astype(np.uint32).reshape(tuple(shape)))
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int64).reshape(-1, d))
    out = np.empty(pts.shape[0], dtype=np.uint32)
    _check(_load().oracle_points_u32(d, r, pattern, _p(n, ctypes.c_int64), _p(wu, ctypes.c_uint32), bkind,
                                     int(bval) & 0xFFFFFFFF, _p(u, ctypes.c_uint32), int(T), pts.shape[0],
                                     _p(pts, ctypes.c_int64), _p(out, ctypes.c_uint32)), "points_u32")
    return out.view(np.int32)


def transpose_step(d, r, pattern, shape, w, bkind, lam) -> np.ndarray:
    """One application of the transpose of the linear part of a step."""
    n = _shape(shape)
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(tuple(shape)))
    out = np.empty_like(lam)
    _check(_load().oracle_transpose_step_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(w, ctypes.c_double), bkind,
                                             _p(lam, ctypes.c_double), _p(out, ctypes.c_double)), "transpose")
    return out


def adjoint(d, r, pattern, shape, w, bkind, bval, u0, target, T):
    """(loss, grad_u0, grad_w) of loss = 0.5 * ||u_T - target||^2."""
    n = _shape(shape)
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(tuple(shape)))
    tg = np.ascontiguousarray(np.asarray(target, dtype=np.float64).reshape(tuple(shape)))
    gu = np.empty_like(u0)
    gw = np.empty(w.shape[0], dtype=np.float64)
    loss = np.zeros(1, dtype=np.float64)
    _check(_load().oracle_adjoint_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(w, ctypes.c_double), bkind,
                                      float(bval), _p(u0, ctypes.c_double), _p(tg, ctypes.c_double), int(T),
                                      _p(gu, ctypes.c_double), _p(gw, ctypes.c_double), _p(loss, ctypes.c_double)),
           "adjoint")
    return float(loss[0]), gu, gw


def run_vc(d, r, pattern, shape, c, bkind, bval, u0, T) -> np.ndarray:
    """u_T of the variable-coefficient sweep, FP64; c has shape (npoints,
    *shape): coefficient field of each compact offset."""
    n = _shape(shape)
    N = int(np.prod(shape))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, N))
    u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(tuple(shape)))
    out = np.empty_like(u0)
    _check(_load().oracle_run_vc_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(c, ctypes.c_double), bkind,
                                     float(bval), _p(u0, ctypes.c_double), int(T), _p(out, ctypes.c_double)),
           "run_vc_f64")
    return out


def run_vc_int(d, r, pattern, shape, c, bkind, bval, u0, T) -> np.ndarray:
    """The variable-coefficient sweep in uint32 wraparound arithmetic (int32 bits)."""
    n = _shape(shape)
    N = int(np.prod(shape))
    cu = np.ascontiguousarray(np.asarray(c).astype(np.int64).astype(np.uint32).reshape(-1, N))
    u = np.ascontiguousarray(np.asarray(u0).astype(np.int64).astype(np.uint32).reshape(tuple(shape)))
    out = np.empty_like(u)
    _check(_load().oracle_run_vc_u32(d, r, pattern, _p(n, ctypes.c_int64), _p(cu, ctypes.c_uint32), bkind,
                                     int(bval) & 0xFFFFFFFF, _p(u, ctypes.c_uint32), int(T),
                                     _p(out, ctypes.c_uint32)), "run_vc_u32")
    return out.view(np.int32)


def adjoint_vc(d, r, pattern, shape, c, bkind, bval, u0, target, T):
    """(loss, grad_u0, grad_c) of loss = 0.5 * ||u_T - target||^2 for the
    variable-coefficient sweep (grad_c shaped like c)."""
    n = _shape(shape)
    N = int(np.prod(shape))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, N))
    u0 = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(tuple(shape)))
    tg = np.ascontiguousarray(np.asarray(target, dtype=np.float64).reshape(tuple(shape)))
    gu = np.empty_like(u0)
    gc = np.empty_like(c)
    loss = np.zeros(1, dtype=np.float64)
    _check(_load().oracle_adjoint_vc_f64(d, r, pattern, _p(n, ctypes.c_int64), _p(c, ctypes.c_double), bkind,
                                         float(bval), _p(u0, ctypes.c_double), _p(tg, ctypes.c_double), int(T),
                                         _p(gu, ctypes.c_double), _p(gc, ctypes.c_double),
                                         _p(loss, ctypes.c_double)), "adjoint_vc")
    return float(loss[0]), gu, gc.reshape((-1,) + tuple(shape))


def total(u) -> float:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    out = np.zeros(1)
    _check(_load().oracle_sum_f64(u.size, _p(u, ctypes.c_double), _p(out, ctypes.c_double)), "sum")
    return float(out[0])


def sumsq(u) -> float:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    out = np.zeros(1)
    _check(_load().oracle_sumsq_f64(u.size, _p(u, ctypes.c_double), _p(out, ctypes.c_double)), "sumsq")
    return float(out[0])


def threads() -> int:
    return int(_load().oracle_threads())

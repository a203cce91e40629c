"""Python binding of the GB300 iterated-stencil library (``include/stencil.h``).

Argument marshalling only: every step of the sweep runs in the CUDA kernels of
``libstencil_gb300.so``.  Functions carry the C names; tensors are passed as
device pointers (``data_ptr()``) and streams as ``cudaStream_t`` handles.
There is no CPU fallback: if the library is missing, ``load()`` raises.

The method (paper, Sections 1 and 3.3): T Jacobi steps of a star or box
stencil of order r, k steps fused per pass over memory.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libstencil_gb300.so")

STENCIL_OK, STENCIL_ERR_INVALID_ARG, STENCIL_ERR_UNSUPPORTED, STENCIL_ERR_OOM = 0, 1, 2, 3
STENCIL_ERR_CUDA, STENCIL_ERR_TIMEOUT, STENCIL_ERR_INTERNAL = 4, 5, 6
STENCIL_F64, STENCIL_F32, STENCIL_BF16, STENCIL_F16, STENCIL_I32 = 0, 1, 2, 3, 4
STENCIL_STAR, STENCIL_BOX = 0, 1
STENCIL_DIRICHLET, STENCIL_PERIODIC = 0, 1
STENCIL_VARIANT_FUSED, STENCIL_VARIANT_PLAIN, STENCIL_VARIANT_FUSED_PER_PASS, STENCIL_VARIANT_TESSELLATE = 0, 1, 2, 3
STENCIL_REDUCE_SUM, STENCIL_REDUCE_SUMSQ, STENCIL_REDUCE_HALF_SQDIST = 0, 1, 2

# Every symbol include/stencil.h declares (checked by the CPU test suite).
EXPORTS = [
    "stencil_plan_create", "stencil_plan_destroy", "stencil_plan_set_k", "stencil_plan_get_k",
    "stencil_plan_max_k", "stencil_plan_set_variant", "stencil_plan_get_variant", "stencil_plan_set_tile_rows",
    "stencil_plan_get_tile_rows", "stencil_plan_set_block_warps", "stencil_plan_get_block_warps",
    "stencil_plan_tune", "stencil_plan_launch_count",
    "stencil_plan_describe", "stencil_run", "stencil_run_host", "stencil_run_host_many", "stencil_run_inplace",
    "stencil_inplace_workspace_bytes", "stencil_run_vc", "stencil_adjoint_vc", "stencil_batch_create",
    "stencil_batch_destroy", "stencil_batch_run", "stencil_batch_get_device_status", "stencil_batch_set_config",
    "stencil_batch_get_config", "stencil_batch_tune",
    "stencil_batch_launch_count", "stencil_adjoint_run", "stencil_run_checkpointed",
    "stencil_adjoint_from_checkpoints", "stencil_reduce", "stencil_reduce_noalloc",
    "stencil_get_device_status", "stencil_probe_fma_rate", "stencil_tess_counts",
    "stencil_status_string", "stencil_last_error",
]


class StencilError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what}: {detail} (status {status})")
        self.status = status


class stencil_weights_t(ctypes.Structure):
    _fields_ = [("pattern", ctypes.c_int32), ("count", ctypes.c_int32), ("w", ctypes.POINTER(ctypes.c_double))]


class stencil_boundary_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("value", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load libstencil_gb300.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA stencil library not built: {p} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "stencil_plan_create": (st, [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(i64), ctypes.POINTER(stencil_weights_t),
                                     ctypes.POINTER(stencil_boundary_t), i32]),
        "stencil_plan_destroy": (st, [vp]),
        "stencil_plan_set_k": (st, [vp, i32]),
        "stencil_plan_get_k": (st, [vp, ctypes.POINTER(i32)]),
        "stencil_plan_max_k": (st, [vp, ctypes.POINTER(i32)]),
        "stencil_plan_set_variant": (st, [vp, i32]),
        "stencil_plan_get_variant": (st, [vp, ctypes.POINTER(i32)]),
        "stencil_plan_set_tile_rows": (st, [vp, i32]),
        "stencil_plan_get_tile_rows": (st, [vp, ctypes.POINTER(i32)]),
        "stencil_plan_set_block_warps": (st, [vp, i32]),
        "stencil_plan_get_block_warps": (st, [vp, ctypes.POINTER(i32)]),
        "stencil_plan_tune": (st, [vp, i64, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
        "stencil_plan_launch_count": (st, [vp, i64, ctypes.POINTER(i64)]),
        "stencil_plan_describe": (st, [vp, ctypes.c_char_p, i32]),
        "stencil_run": (st, [vp, vp, vp, i64, vp]),
        "stencil_run_host": (st, [vp, vp, vp, i64, vp]),
        "stencil_run_inplace": (st, [vp, vp, i64, vp]),
        "stencil_run_host_many": (st, [vp, i64, ctypes.POINTER(vp), ctypes.POINTER(vp), i64, vp]),
        "stencil_inplace_workspace_bytes": (st, [vp, ctypes.POINTER(i64)]),
        "stencil_run_vc": (st, [vp, vp, vp, vp, i64, vp]),
        "stencil_adjoint_vc": (st, [vp, vp, vp, vp, i64, i32, vp, vp, vp]),
        "stencil_batch_create": (st, [ctypes.POINTER(vp), i32, i32, i32, ctypes.POINTER(i64),
                                      ctypes.POINTER(stencil_weights_t), ctypes.POINTER(i64),
                                      ctypes.POINTER(stencil_boundary_t), i32]),
        "stencil_batch_destroy": (st, [vp]),
        "stencil_batch_run": (st, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]),
        "stencil_batch_get_device_status": (st, [vp]),
        "stencil_batch_set_config": (st, [vp, i32, i32]),
        "stencil_batch_get_config": (st, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "stencil_batch_tune": (st, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.POINTER(dbl)]),
        "stencil_batch_launch_count": (st, [vp, ctypes.POINTER(i64)]),
        "stencil_adjoint_run": (st, [vp, vp, vp, i64, i32, vp, vp, vp]),
        "stencil_run_checkpointed": (st, [vp, vp, vp, i64, i32, vp, vp]),
        "stencil_adjoint_from_checkpoints": (st, [vp, vp, vp, vp, i64, i32, vp, vp, vp]),
        "stencil_reduce": (st, [i32, i64, vp, vp, i32, vp, vp]),
        "stencil_reduce_noalloc": (st, [i32, i64, vp, vp, i32, vp, vp]),
        "stencil_get_device_status": (st, [vp]),
        "stencil_probe_fma_rate": (st, [i32, ctypes.POINTER(dbl), vp]),
        "stencil_tess_counts": (st, [i32, ctypes.POINTER(i64), i32, i32, i32, i32, ctypes.POINTER(i32)]),
        "stencil_status_string": (ctypes.c_char_p, [st]),
        "stencil_batch_test_skip_publish": (st, [vp, i64]),
        "stencil_plan_test_poison_counter": (st, [vp, i64]),
        "stencil_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != STENCIL_OK:
        lib = load()
        raise StencilError(status, what, lib.stencil_last_error().decode(errors="replace"))


def _dtype_code(t) -> int:
    import torch
    m = {torch.float64: STENCIL_F64, torch.float32: STENCIL_F32, torch.bfloat16: STENCIL_BF16,
         torch.float16: STENCIL_F16, torch.int32: STENCIL_I32}
    if t not in m:
        raise TypeError(f"unsupported dtype {t}")
    return m[t]


def torch_dtype(code: int):
    import torch
    return {STENCIL_F64: torch.float64, STENCIL_F32: torch.float32, STENCIL_BF16: torch.bfloat16,
            STENCIL_F16: torch.float16, STENCIL_I32: torch.int32}[code]


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Owns a stencil_plan_t (destroyed with the object)."""

    def __init__(self, handle, dim, radius, shape, pattern, weights, bkind, bval, dtype):
        self.handle = handle
        self.dim, self.radius, self.shape = dim, radius, tuple(int(s) for s in shape)
        self.pattern, self.weights, self.bkind, self.bval, self.dtype = pattern, list(weights), bkind, bval, dtype

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.stencil_plan_destroy(h)
            self.handle = None

    @property
    def torch_dtype(self):
        return torch_dtype(self.dtype)


def stencil_plan_create(dim: int, radius: int, shape, pattern: int, weights, bkind: int = STENCIL_DIRICHLET,
                        bval: float = 0.0, dtype: int = STENCIL_F32) -> Plan:
    lib = load()
    n = (ctypes.c_int64 * dim)(*[int(s) for s in shape])
    warr = (ctypes.c_double * len(weights))(*[float(x) for x in weights])
    w = stencil_weights_t(pattern, len(weights), warr)
    b = stencil_boundary_t(bkind, float(bval))
    h = ctypes.c_void_p()
    _check(lib.stencil_plan_create(ctypes.byref(h), dim, radius, n, ctypes.byref(w), ctypes.byref(b), dtype),
           "stencil_plan_create")
    return Plan(h, dim, radius, shape, pattern, weights, bkind, bval, dtype)


def stencil_plan_set_k(plan: Plan, k: int):
    _check(load().stencil_plan_set_k(plan.handle, int(k)), "stencil_plan_set_k")


def stencil_plan_get_k(plan: Plan) -> int:
    k = ctypes.c_int32()
    _check(load().stencil_plan_get_k(plan.handle, ctypes.byref(k)), "stencil_plan_get_k")
    return k.value


def stencil_plan_max_k(plan: Plan) -> int:
    k = ctypes.c_int32()
    _check(load().stencil_plan_max_k(plan.handle, ctypes.byref(k)), "stencil_plan_max_k")
    return k.value


def stencil_plan_set_variant(plan: Plan, variant: int):
    _check(load().stencil_plan_set_variant(plan.handle, int(variant)), "stencil_plan_set_variant")


def stencil_plan_get_variant(plan: Plan) -> int:
    v = ctypes.c_int32()
    _check(load().stencil_plan_get_variant(plan.handle, ctypes.byref(v)), "stencil_plan_get_variant")
    return v.value


def stencil_plan_set_tile_rows(plan: Plan, rows: int):
    _check(load().stencil_plan_set_tile_rows(plan.handle, int(rows)), "stencil_plan_set_tile_rows")


def stencil_plan_get_tile_rows(plan: Plan) -> int:
    r = ctypes.c_int32()
    _check(load().stencil_plan_get_tile_rows(plan.handle, ctypes.byref(r)), "stencil_plan_get_tile_rows")
    return r.value


def stencil_plan_set_block_warps(plan: Plan, warps: int):
    _check(load().stencil_plan_set_block_warps(plan.handle, int(warps)), "stencil_plan_set_block_warps")


def stencil_plan_get_block_warps(plan: Plan) -> int:
    r = ctypes.c_int32()
    _check(load().stencil_plan_get_block_warps(plan.handle, ctypes.byref(r)), "stencil_plan_get_block_warps")
    return r.value


def stencil_plan_tune(plan: Plan, T: int, stream=None):
    k = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load().stencil_plan_tune(plan.handle, int(T), _stream_handle(stream), ctypes.byref(k), ctypes.byref(ms)),
           "stencil_plan_tune")
    return k.value, ms.value


def stencil_plan_launch_count(plan: Plan, T: int) -> int:
    n = ctypes.c_int64()
    _check(load().stencil_plan_launch_count(plan.handle, int(T), ctypes.byref(n)), "stencil_plan_launch_count")
    return n.value


def stencil_plan_describe(plan: Plan) -> str:
    buf = ctypes.create_string_buffer(256)
    _check(load().stencil_plan_describe(plan.handle, buf, 256), "stencil_plan_describe")
    return buf.value.decode()


def _check_grid(plan: Plan, t, name: str):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if tuple(t.shape) != plan.shape or _dtype_code(t.dtype) != plan.dtype:
        raise ValueError(f"{name} must have shape {plan.shape} and the plan's dtype")


def stencil_run(plan: Plan, u_in, u_out, T: int, stream=None):
    """u_out := T steps applied to u_in (both CUDA tensors of the plan's shape)."""
    _check_grid(plan, u_in, "u_in")
    _check_grid(plan, u_out, "u_out")
    _check(load().stencil_run(plan.handle, ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()),
                              int(T), _stream_handle(stream)), "stencil_run")
    return u_out


def stencil_run_inplace(plan: Plan, u, T: int, stream=None):
    """u := T steps applied to u, in place (2D plans; one grid of memory plus
    two small ring buffers)."""
    _check_grid(plan, u, "u")
    _check(load().stencil_run_inplace(plan.handle, ctypes.c_void_p(u.data_ptr()), int(T), _stream_handle(stream)),
           "stencil_run_inplace")
    return u


def stencil_inplace_workspace_bytes(plan: Plan) -> int:
    n = ctypes.c_int64()
    _check(load().stencil_inplace_workspace_bytes(plan.handle, ctypes.byref(n)), "stencil_inplace_workspace_bytes")
    return n.value


def stencil_run_vc(plan: Plan, coef, u_in, u_out, T: int, stream=None):
    """u_out := T steps of the variable-coefficient sweep; coef is a CUDA
    tensor of shape (npoints, *plan.shape) in the arithmetic type (float32 for
    F32 plans, float64 for F64, int32 for I32), compact offset order."""
    import torch
    _check_grid(plan, u_in, "u_in")
    _check_grid(plan, u_out, "u_out")
    ctype = {STENCIL_F32: torch.float32, STENCIL_F64: torch.float64, STENCIL_I32: torch.int32}.get(plan.dtype)
    if ctype is None:
        raise ValueError("variable coefficients support F32, F64 and I32 plans")
    if (not coef.is_cuda or not coef.is_contiguous() or coef.dtype != ctype or coef.device != u_in.device
            or tuple(coef.shape) != (len(plan.weights),) + plan.shape):
        raise ValueError(f"coef must be a contiguous {ctype} CUDA tensor of shape {(len(plan.weights),) + plan.shape}")
    _check(load().stencil_run_vc(plan.handle, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(u_in.data_ptr()),
                                 ctypes.c_void_p(u_out.data_ptr()), int(T), _stream_handle(stream)), "stencil_run_vc")
    return u_out



def stencil_adjoint_vc(plan: Plan, coef, u0, grad_uT, T: int, ckpt_every: int, grad_u0=None, grad_coef=None,
                       stream=None):
    """(grad_u0, grad_coef) of the variable-coefficient sweep for lam_T =
    grad_uT (F32 / F64 plans); grad_coef has coef's shape and dtype."""
    import torch
    _check_grid(plan, u0, "u0")
    _check_grid(plan, grad_uT, "grad_uT")
    ctype = {STENCIL_F32: torch.float32, STENCIL_F64: torch.float64}.get(plan.dtype)
    if ctype is None:
        raise ValueError("the variable-coefficient adjoint supports F32 and F64 plans")
    if (not coef.is_cuda or not coef.is_contiguous() or coef.dtype != ctype or coef.device != u0.device
            or tuple(coef.shape) != (len(plan.weights),) + plan.shape):
        raise ValueError("coef must be a contiguous CUDA tensor of shape (npoints, *shape) in the arithmetic type")
    grad_u0 = torch.empty_like(u0) if grad_u0 is None else grad_u0
    grad_coef = torch.empty_like(coef) if grad_coef is None else grad_coef
    _check_grid(plan, grad_u0, "grad_u0")
    if grad_coef.shape != coef.shape or grad_coef.dtype != coef.dtype or not grad_coef.is_contiguous() \
            or grad_coef.device != coef.device:
        raise ValueError("grad_coef must be a contiguous tensor like coef")
    _check(load().stencil_adjoint_vc(plan.handle, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(u0.data_ptr()),
                                     ctypes.c_void_p(grad_uT.data_ptr()), int(T), int(ckpt_every),
                                     ctypes.c_void_p(grad_u0.data_ptr()), ctypes.c_void_p(grad_coef.data_ptr()),
                                     _stream_handle(stream)), "stencil_adjoint_vc")
    return grad_u0, grad_coef

def _host_grid(plan: Plan, a, name: str) -> int:
    """Address of a host grid (numpy array or CPU tensor) after checking that
    it is contiguous, on the host and exactly one grid of the plan's dtype."""
    import numpy as np
    npts = int(np.prod(plan.shape))
    size = {STENCIL_F64: 8, STENCIL_F32: 4, STENCIL_BF16: 2, STENCIL_F16: 2, STENCIL_I32: 4}[plan.dtype]
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous() or _dtype_code(a.dtype) != plan.dtype or a.numel() != npts:
            raise ValueError(f"{name} must be a contiguous CPU tensor of {npts} values of the plan's dtype")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous or a.size != npts or a.itemsize != size:
        raise ValueError(f"{name} must be a contiguous array of {npts} values of the plan's dtype")
    return a.ctypes.data


def stencil_run_host(plan: Plan, h_in, h_out, T: int, stream=None):
    """Host-buffer run (numpy arrays or CPU tensors); synchronises."""
    def ptr(a):
        return _host_grid(plan, a, "host grid")
    _check(load().stencil_run_host(plan.handle, ctypes.c_void_p(ptr(h_in)), ctypes.c_void_p(ptr(h_out)), int(T),
                                   _stream_handle(stream)), "stencil_run_host")
    return h_out


def stencil_run_host_many(plan: Plan, h_ins, h_outs, T: int, stream=None):
    """h_outs[i] := T steps of h_ins[i] (host arrays or CPU tensors; pinned
    memory makes the copies overlap the sweeps); synchronises."""
    def ptr(a):
        return _host_grid(plan, a, "host grid")
    n = len(h_ins)
    if len(h_outs) != n:
        raise ValueError("one output per input")
    pin = (ctypes.c_void_p * max(n, 1))(*[ptr(a) for a in h_ins])
    pout = (ctypes.c_void_p * max(n, 1))(*[ptr(a) for a in h_outs])
    _check(load().stencil_run_host_many(plan.handle, n, pin, pout, int(T), _stream_handle(stream)),
           "stencil_run_host_many")
    return h_outs


def stencil_get_device_status(plan: Plan) -> int:
    return int(load().stencil_get_device_status(plan.handle))


def _reduce_args(u, op: int, target, out, what: str):
    """Host-side checks shared by the reduction wrappers: every pointer the C
    call receives must be a contiguous tensor of the right dtype, size and
    device, so that the kernels never read past a buffer or across GPUs."""
    import torch
    if not isinstance(u, torch.Tensor) or not u.is_cuda or not u.is_contiguous():
        raise ValueError(f"{what}: u must be a contiguous CUDA tensor")
    if u.numel() < 1:
        raise ValueError(f"{what}: u must not be empty")
    if int(op) == STENCIL_REDUCE_HALF_SQDIST:
        if target is None:
            raise ValueError(f"{what}: HALF_SQDIST needs a target")
    if target is not None:
        if not isinstance(target, torch.Tensor) or not target.is_cuda or not target.is_contiguous():
            raise ValueError(f"{what}: target must be a contiguous CUDA tensor")
        if target.dtype != u.dtype or target.numel() != u.numel() or target.device != u.device:
            raise ValueError(f"{what}: target must have u's dtype, number of elements and device")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=u.device)
    elif (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or out.device != u.device
          or out.numel() < 1 or not out.is_contiguous()):
        raise ValueError(f"{what}: out must be a contiguous float64 tensor on u's device")
    tp = ctypes.c_void_p(target.data_ptr()) if target is not None else ctypes.c_void_p(0)
    return out, tp


def stencil_reduce(u, op: int, target=None, out=None, stream=None):
    """FP64 reduction of a CUDA tensor; returns the 1-element float64 CUDA tensor."""
    import torch
    out, tp = _reduce_args(u, op, target, out, "stencil_reduce")
    with torch.cuda.device(u.device):
        _check(load().stencil_reduce(_dtype_code(u.dtype), u.numel(), ctypes.c_void_p(u.data_ptr()), tp, int(op),
                                     ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "stencil_reduce")
    return out


def stencil_reduce_noalloc(u, op: int, target=None, out=None, stream=None):
    """stencil_reduce without any device allocation (partial sums in a
    library-static array); `out` defaults to a new 1-element float64 tensor,
    which the caller may preallocate to avoid torch's allocator as well."""
    import torch
    out, tp = _reduce_args(u, op, target, out, "stencil_reduce_noalloc")
    with torch.cuda.device(u.device):
        _check(load().stencil_reduce_noalloc(_dtype_code(u.dtype), u.numel(), ctypes.c_void_p(u.data_ptr()), tp,
                                             int(op), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "stencil_reduce_noalloc")
    return out


def stencil_probe_fma_rate(dtype: int, stream=None) -> float:
    """Measured FMAs per second of the current GPU in F32 or F64."""
    r = ctypes.c_double()
    _check(load().stencil_probe_fma_rate(int(dtype), ctypes.byref(r), _stream_handle(stream)),
           "stencil_probe_fma_rate")
    return r.value


def stencil_tess_counts(shape, radius: int, levels: int, tile: int, periodic: bool):
    """Host-only: (d + 1, *shape) int32 array, the levels at which each stage of
    one tessellation time tile updates each point."""
    import numpy as np
    d = len(shape)
    n = (ctypes.c_int64 * d)(*[int(v) for v in shape])
    out = np.zeros((d + 1,) + tuple(int(v) for v in shape), dtype=np.int32)
    _check(load().stencil_tess_counts(d, n, int(radius), int(levels), int(tile), 1 if periodic else 0,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "stencil_tess_counts")
    return out


def stencil_status_string(status: int) -> str:
    return load().stencil_status_string(int(status)).decode()


def stencil_last_error() -> str:
    return load().stencil_last_error().decode()


class Batch:
    """Owns a stencil_batch_t (destroyed with the object)."""

    def __init__(self, handle, shapes, dtype):
        self.handle, self.shapes, self.dtype = handle, [tuple(s) for s in shapes], dtype

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.stencil_batch_destroy(h)
            self.handle = None


def stencil_batch_create(shapes, weights, T, pattern: int, radius: int = 1, bkind: int = STENCIL_PERIODIC,
                         bval: float = 0.0, dtype: int = STENCIL_F32) -> Batch:
    """A batch of 2D grids (shapes: list of (ny, nx); weights: list of compact
    weight lists; T: list of step counts)."""
    lib = load()
    n = len(shapes)
    sh = (ctypes.c_int64 * (2 * n))(*[int(v) for s in shapes for v in s])
    keep = [(ctypes.c_double * len(w))(*[float(x) for x in w]) for w in weights]
    ws = (stencil_weights_t * n)(*[stencil_weights_t(pattern, len(w), k) for w, k in zip(weights, keep)])
    ts = (ctypes.c_int64 * n)(*[int(t) for t in T])
    b = stencil_boundary_t(bkind, float(bval))
    h = ctypes.c_void_p()
    _check(lib.stencil_batch_create(ctypes.byref(h), n, 2, radius, sh, ws, ts, ctypes.byref(b), dtype),
           "stencil_batch_create")
    return Batch(h, shapes, dtype)


def stencil_batch_run(batch: Batch, u_in, u_out, stream=None):
    """u_out[i] := T[i] steps applied to u_in[i] (lists of CUDA tensors)."""
    n = len(batch.shapes)
    if len(u_in) != n or len(u_out) != n:
        raise ValueError("one input and one output tensor per batch member")
    for i, (a, b) in enumerate(zip(u_in, u_out)):
        for t, nm in ((a, "u_in"), (b, "u_out")):
            if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != batch.shapes[i] or \
                    _dtype_code(t.dtype) != batch.dtype:
                raise ValueError(f"{nm}[{i}] must be a contiguous CUDA tensor of shape {batch.shapes[i]}")
    pin = (ctypes.c_void_p * n)(*[t.data_ptr() for t in u_in])
    pout = (ctypes.c_void_p * n)(*[t.data_ptr() for t in u_out])
    _check(load().stencil_batch_run(batch.handle, pin, pout, _stream_handle(stream)), "stencil_batch_run")
    return u_out


def stencil_batch_set_config(batch: Batch, k: int, tile_rows: int):
    _check(load().stencil_batch_set_config(batch.handle, int(k), int(tile_rows)), "stencil_batch_set_config")


def stencil_batch_get_config(batch: Batch):
    k, rows = ctypes.c_int32(), ctypes.c_int32()
    _check(load().stencil_batch_get_config(batch.handle, ctypes.byref(k), ctypes.byref(rows)), "stencil_batch_get_config")
    return k.value, rows.value


def stencil_batch_tune(batch: Batch, u_in, u_out, stream=None) -> float:
    """Choose the batch's k and tile height by timing runs on these tensors."""
    n = len(batch.shapes)
    pin = (ctypes.c_void_p * n)(*[t.data_ptr() for t in u_in])
    pout = (ctypes.c_void_p * n)(*[t.data_ptr() for t in u_out])
    ms = ctypes.c_double()
    _check(load().stencil_batch_tune(batch.handle, pin, pout, _stream_handle(stream), ctypes.byref(ms)),
           "stencil_batch_tune")
    return ms.value


def stencil_batch_get_device_status(batch: Batch) -> int:
    return int(load().stencil_batch_get_device_status(batch.handle))


def stencil_batch_launch_count(batch: Batch) -> int:
    n = ctypes.c_int64()
    _check(load().stencil_batch_launch_count(batch.handle, ctypes.byref(n)), "stencil_batch_launch_count")
    return n.value


def stencil_adjoint_run(plan: Plan, u0, grad_uT, T: int, ckpt_every: int, grad_u0=None, grad_w=None, stream=None):
    """Reverse-mode derivative of T steps (FP32 plans): returns (grad_u0,
    grad_w) for a loss whose gradient w.r.t. u_T is grad_uT."""
    import torch
    _check_grid(plan, u0, "u0")
    _check_grid(plan, grad_uT, "grad_uT")
    if grad_u0 is None:
        grad_u0 = torch.empty_like(u0)
    if grad_w is None:
        grad_w = torch.empty(len(plan.weights), dtype=torch.float64, device=u0.device)
    _check_grid(plan, grad_u0, "grad_u0")
    _check(load().stencil_adjoint_run(plan.handle, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(grad_uT.data_ptr()),
                                      int(T), int(ckpt_every), ctypes.c_void_p(grad_u0.data_ptr()),
                                      ctypes.c_void_p(grad_w.data_ptr()), _stream_handle(stream)), "stencil_adjoint_run")
    return grad_u0, grad_w


def checkpoint_count(T: int, ckpt_every: int) -> int:
    """Grids stencil_run_checkpointed stores for T steps."""
    return max(0, -(-int(T) // int(ckpt_every)) - 1)


def stencil_run_checkpointed(plan: Plan, u0, u_T, T: int, ckpt_every: int, ckpts=None, stream=None):
    """u_T := T steps of u0, keeping the state every ckpt_every steps in
    `ckpts` (a CUDA tensor of checkpoint_count(T, ckpt_every) grids, allocated
    when None); returns ckpts."""
    import torch
    _check_grid(plan, u0, "u0")
    _check_grid(plan, u_T, "u_T")
    n = checkpoint_count(T, ckpt_every)
    if ckpts is None:
        ckpts = torch.empty((max(n, 1),) + plan.shape, dtype=u0.dtype, device=u0.device)
    if (not ckpts.is_cuda or not ckpts.is_contiguous() or ckpts.dtype != u0.dtype
            or ckpts.numel() < n * u0.numel()):
        raise ValueError(f"ckpts must be a contiguous CUDA tensor of at least {n} grids")
    _check(load().stencil_run_checkpointed(plan.handle, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(u_T.data_ptr()),
                                           int(T), int(ckpt_every), ctypes.c_void_p(ckpts.data_ptr()),
                                           _stream_handle(stream)), "stencil_run_checkpointed")
    return ckpts


def stencil_adjoint_from_checkpoints(plan: Plan, u0, ckpts, grad_uT, T: int, ckpt_every: int, grad_u0=None,
                                     grad_w=None, stream=None):
    """The backward sweep from stencil_run_checkpointed's checkpoints."""
    import torch
    _check_grid(plan, u0, "u0")
    _check_grid(plan, grad_uT, "grad_uT")
    if ckpts.numel() < checkpoint_count(T, ckpt_every) * u0.numel() or not ckpts.is_contiguous():
        raise ValueError("ckpts holds fewer grids than T / ckpt_every needs")
    if grad_u0 is None:
        grad_u0 = torch.empty_like(u0)
    if grad_w is None:
        grad_w = torch.empty(len(plan.weights), dtype=torch.float64, device=u0.device)
    _check_grid(plan, grad_u0, "grad_u0")
    _check(load().stencil_adjoint_from_checkpoints(
        plan.handle, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(ckpts.data_ptr()),
        ctypes.c_void_p(grad_uT.data_ptr()), int(T), int(ckpt_every), ctypes.c_void_p(grad_u0.data_ptr()),
        ctypes.c_void_p(grad_w.data_ptr()), _stream_handle(stream)), "stencil_adjoint_from_checkpoints")
    return grad_u0, grad_w


def _autograd_fn():
    import torch

    class StencilFn(torch.autograd.Function):
        """u_T = T stencil steps of u0 with the plan's weights.  The forward
        keeps a checkpoint every `ckpt_every` steps; backward runs the
        transposed sweep from them and returns the gradients w.r.t. u0 and
        the weights (compact order).  `weights` must hold the plan's
        coefficients (checked)."""

        @staticmethod
        def forward(ctx, u0, weights, plan, T, ckpt_every=8):
            w = weights.detach().double().cpu().tolist()
            if len(w) != len(plan.weights) or any(a != float(b) for a, b in zip(w, plan.weights)):
                raise ValueError("stencil_apply: `weights` differs from the plan's coefficients; create the plan "
                                 "from these weights")
            u0 = u0.contiguous()
            out = torch.empty_like(u0)
            c = int(min(max(1, ckpt_every), max(1, T)))
            ckpts = stencil_run_checkpointed(plan, u0, out, T, c)
            ctx.save_for_backward(u0, ckpts)
            ctx.plan, ctx.T, ctx.ckpt = plan, int(T), c
            ctx.wdtype = weights.dtype
            return out

        @staticmethod
        def backward(ctx, grad_out):
            u0, ckpts = ctx.saved_tensors
            gu, gw = stencil_adjoint_from_checkpoints(ctx.plan, u0, ckpts, grad_out.contiguous(), ctx.T, ctx.ckpt)
            return gu, gw.to(ctx.wdtype), None, None, None

    return StencilFn


_stencil_fn = None


def stencil_apply(u0, weights, plan: Plan, T: int, ckpt_every: int = 8):
    """Differentiable T-step sweep (torch.autograd.Function over the C ABI)."""
    global _stencil_fn
    if _stencil_fn is None:
        _stencil_fn = _autograd_fn()
    return _stencil_fn.apply(u0, weights, plan, T, ckpt_every)

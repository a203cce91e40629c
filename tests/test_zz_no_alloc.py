"""stencil_reduce_noalloc: the reduction for callers that cannot allocate.

Some callers cannot allocate device memory when they reduce: devices or
drivers without stream-ordered memory pools (stencil_reduce takes its
partial-sum buffer with cudaMallocAsync), applications whose caching
allocator already holds nearly all free device memory, and latency-critical
loops that must not enter an allocator.  stencil_reduce_noalloc keeps its
partial sums in a library-static device array instead.  This test calls it
through the C ABI, twice in a row, and checks that each result is
bit-identical to the allocating entry point's: both run the same kernels over
the same partition in the same order, so any difference would be a stale or
missing partial sum in the shared array.  The Python wrapper is exercised too,
including its host-side argument checks.

The file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from synth import uniform01

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


@pytest.mark.parametrize("dtype", ["float64", "float32", "bfloat16"])
def test_noalloc_reduction_matches_allocating_one(dtype):
    sg = sgmod()
    lib = sg.load()
    td = getattr(torch, dtype)
    code = sg._dtype_code(td)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in (1, 4097, 1_000_003, 20_000_000):
        u = torch.from_numpy(uniform01(11, n) - 0.5).to(td).to(DEV)
        t = torch.from_numpy(uniform01(12, n)).to(td).to(DEV)
        for op in (sg.STENCIL_REDUCE_SUM, sg.STENCIL_REDUCE_SUMSQ, sg.STENCIL_REDUCE_HALF_SQDIST):
            ref = sg.stencil_reduce(u, op, target=t).item()
            for _ in range(2):       # the static scratch is reused by consecutive calls
                out = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
                st = lib.stencil_reduce_noalloc(code, n, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                op, ctypes.c_void_p(out.data_ptr()), stream)
                assert st == 0, lib.stencil_last_error()
                got = out.item()
                assert got == ref, (n, op, got, ref)      # same partition, same order: identical
            # the Python wrapper (argument checks, then the same C call)
            again = sg.stencil_reduce_noalloc(u, op, target=t if op == sg.STENCIL_REDUCE_HALF_SQDIST else None)
            assert again.item() == ref, (n, op)


def test_noalloc_wrapper_rejects_mismatched_tensors():
    """Host-side checks: a shorter or differently typed target, an output of
    the wrong dtype or a non-contiguous input raise before any launch."""
    sg = sgmod()
    u = torch.zeros(1000, device=DEV)
    with pytest.raises(ValueError):
        sg.stencil_reduce_noalloc(u, sg.STENCIL_REDUCE_HALF_SQDIST, target=torch.zeros(999, device=DEV))
    with pytest.raises(ValueError):
        sg.stencil_reduce_noalloc(u, sg.STENCIL_REDUCE_HALF_SQDIST, target=torch.zeros(1000, device=DEV,
                                                                                         dtype=torch.float64))
    with pytest.raises(ValueError):
        sg.stencil_reduce_noalloc(u, sg.STENCIL_REDUCE_SUM, out=torch.zeros(1, device=DEV))
    with pytest.raises(ValueError):
        sg.stencil_reduce_noalloc(torch.zeros(10, 10, device=DEV).t(), sg.STENCIL_REDUCE_SUM)
    with pytest.raises(ValueError):
        sg.stencil_reduce_noalloc(u, sg.STENCIL_REDUCE_HALF_SQDIST)


def test_noalloc_reduction_rejects_bad_arguments():
    sg = sgmod()
    lib = sg.load()
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    u = torch.zeros(8, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.stencil_reduce_noalloc(sg.STENCIL_F32, 0, ctypes.c_void_p(u.data_ptr()), None, 0,
                                      ctypes.c_void_p(out.data_ptr()), stream) == sg.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_reduce_noalloc(sg.STENCIL_I32, 8, ctypes.c_void_p(u.data_ptr()), None, 0,
                                      ctypes.c_void_p(out.data_ptr()), stream) == sg.STENCIL_ERR_UNSUPPORTED
    assert lib.stencil_reduce_noalloc(sg.STENCIL_F32, 8, ctypes.c_void_p(u.data_ptr()), None, 2,
                                      ctypes.c_void_p(out.data_ptr()), stream) == sg.STENCIL_ERR_INVALID_ARG

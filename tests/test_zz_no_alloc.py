"""stencil_reduce_noalloc: the reduction for callers that cannot allocate.

Some callers cannot allocate device memory when they reduce: devices or
drivers without stream-ordered memory pools (stencil_reduce takes its
partial-sum buffer with cudaMallocAsync), applications whose caching
allocator already holds nearly all free device memory, and latency-critical
loops that must not enter an allocator.  stencil_reduce_noalloc keeps its
partial sums in a library-static device array instead.  This test calls it
through the C ABI, twice in a row, and checks each result against the
allocating entry point's within the tolerance the reduction tests use.

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
        bound = n * 2.0 ** -52
        for op in (sg.STENCIL_REDUCE_SUM, sg.STENCIL_REDUCE_SUMSQ, sg.STENCIL_REDUCE_HALF_SQDIST):
            ref = sg.stencil_reduce(u, op, target=t).item()
            scale = max(1.0, float(torch.sum(torch.abs(u.double() - (t.double() if op == 2 else 0)) ** (1 if op == 0 else 2))))
            for _ in range(2):       # the static scratch is reused by consecutive calls
                out = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
                st = lib.stencil_reduce_noalloc(code, n, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                op, ctypes.c_void_p(out.data_ptr()), stream)
                assert st == 0, lib.stencil_last_error()
                got = out.item()
                assert abs(got - ref) <= bound * scale, (n, op, got, ref)


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

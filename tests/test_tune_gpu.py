"""The autotuner: its choices give results bit-identical to the plain sweep,
its persistent cache is written and read back, the 2D block size is a free
launch parameter, and fusion depths up to 16 are accepted and exact."""

import os

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FUSED, PLAIN, PER_PASS = 0, 1, 2


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def run(plan, x, T, variant=None):
    sg = sgmod()
    if variant is not None:
        sg.stencil_plan_set_variant(plan, variant)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    return y


def test_tune_cache_written_and_reused(tmp_path, monkeypatch):
    sg = sgmod()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(cache))
    shape, T = (300, 700), 24
    w = [0.5, 0.125, 0.125, 0.125, 0.125]
    x = torch.from_numpy(uniform01(5, shape[0] * shape[1]).reshape(shape).astype(np.float32)).to(DEV)
    ref = run(sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32), x, T, PLAIN)
    p1 = sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    k1, ms1 = sg.stencil_plan_tune(p1, T)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and f"/T{T}" in lines[0]
    assert torch.equal(run(p1, x, T), ref)
    choice1 = (sg.stencil_plan_get_k(p1), sg.stencil_plan_get_variant(p1), sg.stencil_plan_get_tile_rows(p1),
               sg.stencil_plan_get_block_warps(p1))
    # a second plan of the same geometry takes the stored choice without timing
    p2 = sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    k2, ms2 = sg.stencil_plan_tune(p2, T)
    assert (k2, ms2) == (k1, pytest.approx(ms1, rel=1e-5))
    assert len(cache.read_text().splitlines()) == 1
    choice2 = (sg.stencil_plan_get_k(p2), sg.stencil_plan_get_variant(p2), sg.stencil_plan_get_tile_rows(p2),
               sg.stencil_plan_get_block_warps(p2))
    assert choice1 == choice2
    assert torch.equal(run(p2, x, T), ref)
    # another T is another entry
    sg.stencil_plan_tune(p2, T + 1)
    assert len(cache.read_text().splitlines()) == 2


@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_block_warps_do_not_change_results(bkind):
    sg = sgmod()
    shape, T = (513, 1031), 17
    w = [float(v) for v in np.random.default_rng(2).integers(-3, 7, 9)]
    u0 = uniform_u16(8, shape[0] * shape[1]).reshape(shape)
    plan = sg.stencil_plan_create(2, 1, shape, BOX, w, bkind, 9 if bkind == DIRICHLET else 0, sg.STENCIL_I32)
    ref = oracle.run_int(2, 1, BOX, shape, w, bkind, 9 if bkind == DIRICHLET else 0, u0, T)
    x = torch.from_numpy(u0).to(DEV)
    for warps in (1, 2, 3, 8, 0):
        sg.stencil_plan_set_block_warps(plan, warps)
        assert sg.stencil_plan_get_block_warps(plan) == warps
        for k in (1, 4, 7):
            sg.stencil_plan_set_k(plan, k)
            for variant in (FUSED, PER_PASS):
                got = run(plan, x, T, variant).cpu().numpy()
                np.testing.assert_array_equal(got, ref, err_msg=f"warps={warps} k={k} variant={variant}")
    with pytest.raises(sg.StencilError):
        sg.stencil_plan_set_block_warps(plan, 9)


@pytest.mark.parametrize("d,r,pattern,shape", [(2, 1, STAR, (400, 300)), (2, 1, BOX, (300, 260)),
                                               (2, 2, BOX, (200, 300)), (2, 3, STAR, (150, 260)),
                                               (1, 1, STAR, (50003,)), (1, 3, STAR, (9001,))])
def test_deep_fusion_exact(d, r, pattern, shape):
    """Every fusion depth up to the plan's maximum (16 for the 2D and 1D
    radius-1 FP32/int32 kernels) is bit-exact in the integer mode."""
    sg = sgmod()
    n = int(np.prod(shape))
    w = [float(v) for v in np.random.default_rng(d + r).integers(-2, 5, npoints(d, r, pattern))]
    u0 = uniform_u16(9 + n, n).reshape(shape)
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, DIRICHLET, 3, sg.STENCIL_I32)
    kmax = sg.stencil_plan_max_k(plan)
    if r == 1:
        assert kmax == 16
    T = 2 * kmax + 3
    ref = oracle.run_int(d, r, pattern, shape, w, DIRICHLET, 3, u0, T)
    x = torch.from_numpy(u0).to(DEV)
    for k in range(1, kmax + 1):
        sg.stencil_plan_set_k(plan, k)
        np.testing.assert_array_equal(run(plan, x, T, FUSED).cpu().numpy(), ref, err_msg=f"k={k}")
    f32 = sg.stencil_plan_create(d, r, shape, pattern, [v / 16 for v in w], DIRICHLET, 0.5, sg.STENCIL_F32)
    xf = torch.from_numpy(uniform01(4, n).reshape(shape).astype(np.float32)).to(DEV)
    base = run(f32, xf, T, PLAIN)
    assert sg.stencil_plan_max_k(f32) == kmax
    for k in (kmax // 2, kmax):
        sg.stencil_plan_set_k(f32, k)
        assert torch.equal(run(f32, xf, T, FUSED), base), k

"""Tessellate tiling on the GPU (paper Section 3.4): T steps in time tiles of
h levels, d + 1 stages each, no redundant work -- bit-identical to the plain
sweep in FP32/FP64 and exact against the oracle in the integer mode, for
1D/2D/3D, star and box, Dirichlet and periodic, T not a multiple of h."""

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PLAIN, TESS = 1, 3

CASES = [(1, 1, STAR, (4099,), 8, 0), (1, 2, STAR, (1000,), 5, 100), (2, 1, STAR, (300, 517), 8, 0),
         (2, 1, BOX, (130, 200), 6, 32), (2, 2, BOX, (70, 90), 3, 16), (3, 1, STAR, (40, 37, 70), 4, 0),
         (3, 1, BOX, (33, 32, 35), 3, 16)]


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def run(plan, x, T, variant):
    sg = sgmod()
    sg.stencil_plan_set_variant(plan, variant)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    return y


@pytest.mark.parametrize("d,r,pattern,shape,h,tile", CASES)
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_tess_int32_exact(d, r, pattern, shape, h, tile, bkind):
    sg = sgmod()
    n = int(np.prod(shape))
    w = [float(v) for v in np.random.default_rng(d + r).integers(-3, 6, npoints(d, r, pattern))]
    u0 = uniform_u16(60 + n, n).reshape(shape)
    bval = 11 if bkind == DIRICHLET else 0
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
    sg.stencil_plan_set_k(plan, min(h, sg.stencil_plan_max_k(plan)))
    sg.stencil_plan_set_tile_rows(plan, tile)
    x = torch.from_numpy(u0).to(DEV)
    for T in (1, h, 2 * h + 1):
        ref = oracle.run_int(d, r, pattern, shape, w, bkind, bval, u0, T)
        np.testing.assert_array_equal(run(plan, x, T, TESS).cpu().numpy(), ref, err_msg=f"T={T}")


@pytest.mark.parametrize("d,r,pattern,shape,h,tile", CASES[:5])
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_tess_float_bit_identical_to_plain(d, r, pattern, shape, h, tile, dt):
    sg = sgmod()
    code = sg.STENCIL_F32 if dt == "f32" else sg.STENCIL_F64
    n = int(np.prod(shape))
    w = list(np.random.default_rng(7).uniform(0.0, 0.3, npoints(d, r, pattern)))
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, DIRICHLET, 0.2, code)
    sg.stencil_plan_set_k(plan, min(h, sg.stencil_plan_max_k(plan)))
    sg.stencil_plan_set_tile_rows(plan, tile)
    x = torch.from_numpy(uniform01(61, n).reshape(shape)).to(sg.torch_dtype(code)).to(DEV)
    T = 3 * h + 2
    assert torch.equal(run(plan, x, T, TESS), run(plan, x, T, PLAIN))
    # the set-up copy, then d + 1 stage launches per time tile
    sg.stencil_plan_set_variant(plan, TESS)
    assert sg.stencil_plan_launch_count(plan, T) == 1 + (-(-T // sg.stencil_plan_get_k(plan))) * (d + 1)


def test_tess_bench_size_2d():
    """8192^2 2D5P FP32 at h = 8 and 16: bit-identical to the plain sweep."""
    sg = sgmod()
    shape, T = (8192, 8192), 32
    plan = sg.stencil_plan_create(2, 1, shape, STAR, [0.5, 0.125, 0.125, 0.125, 0.125], DIRICHLET, 0.0,
                                  sg.STENCIL_F32)
    x = torch.rand(shape, device=DEV)
    ref = run(plan, x, T, PLAIN)
    for h in (8, 16):
        sg.stencil_plan_set_k(plan, h)
        assert torch.equal(run(plan, x, T, TESS), ref), h

"""Variable-coefficient sweeps (u_{t+1}[x] = sum_o c_o[x] u_t(x+o)) on the GPU
against the pinned variable-coefficient oracle: int32 bit-exact, FP64 within
1e-12 and FP32 within 1e-5 normwise; every fusion depth bit-identical to the
one-step kernel; a constant field bit-identical to stencil_run."""

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FUSED, PLAIN = 0, 1

SHAPES = {1: [(1001,), (7,)], 2: [(67, 300), (5, 9), (130, 17)], 3: [(9, 10, 37), (5, 6, 7)]}


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def run_vc(plan, coef, u0, T, k=None, variant=FUSED):
    sg = sgmod()
    sg.stencil_plan_set_variant(plan, variant)
    if k is not None:
        sg.stencil_plan_set_k(plan, k)
    x = torch.from_numpy(np.ascontiguousarray(u0)).to(DEV)
    y = torch.empty_like(x)
    sg.stencil_run_vc(plan, coef, x, y, T)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def normwise(g, o):
    return float(np.max(np.abs(np.asarray(g, np.float64) - o)) / max(1e-300, np.max(np.abs(o))))


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_vc_int32_exact(d, r, pattern, bkind):
    if d == 3 and r == 3 and pattern == BOX:
        pytest.skip("343 coefficient planes on toy grids: covered by the 2D radius-3 box")
    sg = sgmod()
    for shape in SHAPES[d]:
        n = int(np.prod(shape))
        np_ = npoints(d, r, pattern)
        c = (uniform_u16(70 + d + r, np_ * n).astype(np.int64) % 11 - 5).astype(np.int32).reshape((np_,) + shape)
        u0 = uniform_u16(71 + n, n).reshape(shape)
        bval = 19 if bkind == DIRICHLET else 0
        plan = sg.stencil_plan_create(d, r, shape, pattern, [1.0] * np_, bkind, bval, sg.STENCIL_I32)
        ct = torch.from_numpy(c).to(DEV)
        for T in (1, 6):
            ref = oracle.run_vc_int(d, r, pattern, shape, c, bkind, bval, u0, T)
            np.testing.assert_array_equal(run_vc(plan, ct, u0, T, variant=PLAIN), ref, err_msg=f"plain {shape}")
            if d == 2 and r <= 2:
                for k in range(1, 5 if r == 1 else 3):
                    np.testing.assert_array_equal(run_vc(plan, ct, u0, T, k=min(k, sg.stencil_plan_max_k(plan))),
                                                  ref, err_msg=f"k={k} {shape} T={T}")


@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("pattern", [STAR, BOX])
def test_vc_fp64_fp32_against_oracle(bkind, pattern):
    sg = sgmod()
    shape, T = (97, 301), 9
    n = shape[0] * shape[1]
    np_ = npoints(2, 1, pattern)
    c = (0.02 + 0.18 * uniform01(80, np_ * n)).reshape((np_,) + shape)
    u0 = uniform01(81, n).reshape(shape)
    bval = 0.4 if bkind == DIRICHLET else 0.0
    ref = oracle.run_vc(2, 1, pattern, shape, c, bkind, bval, u0, T)
    p64 = sg.stencil_plan_create(2, 1, shape, pattern, [1.0] * np_, bkind, bval, sg.STENCIL_F64)
    c64 = torch.from_numpy(c).to(DEV)
    base = run_vc(p64, c64, u0, T, variant=PLAIN)
    assert normwise(base, ref) <= 1e-12
    for k in (1, 2, 3, 4):
        np.testing.assert_array_equal(run_vc(p64, c64, u0, T, k=min(k, sg.stencil_plan_max_k(p64))), base)
    c32 = c.astype(np.float32)
    u32 = u0.astype(np.float32)
    ref32 = oracle.run_vc(2, 1, pattern, shape, c32.astype(np.float64), bkind, float(np.float32(bval)),
                          u32.astype(np.float64), T)
    p32 = sg.stencil_plan_create(2, 1, shape, pattern, [1.0] * np_, bkind, bval, sg.STENCIL_F32)
    ct = torch.from_numpy(c32).to(DEV)
    base32 = run_vc(p32, ct, u32, T, variant=PLAIN)
    assert normwise(base32, ref32) <= 1e-5
    for k in (1, 2, 3, 4):
        np.testing.assert_array_equal(run_vc(p32, ct, u32, T, k=k), base32, err_msg=f"k={k}")


def test_vc_constant_field_matches_stencil_run():
    sg = sgmod()
    shape, T = (300, 517), 12
    w = [0.5, 0.125, 0.1, 0.15, 0.125]
    plan = sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.25, sg.STENCIL_F32)
    x = torch.from_numpy(uniform01(90, shape[0] * shape[1]).reshape(shape).astype(np.float32)).to(DEV)
    ref = torch.empty_like(x)
    sg.stencil_plan_set_k(plan, 4)
    sg.stencil_run(plan, x, ref, T)
    coef = torch.stack([torch.full(shape, float(np.float32(v)), device=DEV) for v in w]).contiguous()
    y = torch.empty_like(x)
    sg.stencil_run_vc(plan, coef, x, y, T)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)

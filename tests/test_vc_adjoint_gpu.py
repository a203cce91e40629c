"""The GPU adjoint of the variable-coefficient sweep (stencil_adjoint_vc)
against the pinned FP64 variable-coefficient adjoint of the oracle: gradients
with respect to u0 and to the coefficient field, FP64 within 1e-12 and FP32
within 1e-5 normwise (positive fields and a zero target, so no term cancels),
every checkpoint spacing bit-identical, T = 0 and argument errors."""

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = {1: (37,), 2: (13, 17), 3: (6, 7, 9)}


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def normwise(g, o):
    return float(np.max(np.abs(np.asarray(g, np.float64) - o)) / max(1e-300, np.max(np.abs(o))))


def field(d, r, pattern, shape, seed, lo, hi):
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, npoints(d, r, pattern) * n)).reshape((-1,) + tuple(shape))


def gpu_adjoint(plan, c, u0, g, T, ckpt):
    sg = sgmod()
    ct = torch.from_numpy(np.ascontiguousarray(c)).to(DEV)
    x = torch.from_numpy(np.ascontiguousarray(u0)).to(DEV)
    gt = torch.from_numpy(np.ascontiguousarray(g)).to(DEV)
    gu, gc = sg.stencil_adjoint_vc(plan, ct, x, gt, T, ckpt)
    torch.cuda.synchronize()
    return gu.cpu().numpy(), gc.cpu().numpy()


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r,pattern", [(1, STAR), (1, BOX), (2, STAR)])
@pytest.mark.parametrize("bkind,bval", [(DIRICHLET, 0.3), (PERIODIC, 0.0)])
def test_vc_adjoint_fp64_against_oracle(d, r, pattern, bkind, bval):
    sg = sgmod()
    shape = SHAPES[d]
    n = int(np.prod(shape))
    c = field(d, r, pattern, shape, 700 + d + r, -0.2, 0.5)
    u0 = uniform01(701, n).reshape(shape)
    tg = uniform01(702, n).reshape(shape)
    T = 7
    _, ogu, ogc = oracle.adjoint_vc(d, r, pattern, shape, c, bkind, bval, u0, tg, T)
    uT = oracle.run_vc(d, r, pattern, shape, c, bkind, bval, u0, T)
    w = [1.0] * npoints(d, r, pattern)
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_F64)
    for ckpt in (1, 3, T):
        gu, gc = gpu_adjoint(plan, c, u0, uT - tg, T, ckpt)
        assert normwise(gu, ogu) <= 1e-12, ckpt
        assert normwise(gc, ogc) <= 1e-12, ckpt
        if ckpt == 1:
            ref = (gu, gc)
        else:   # the recomputed states do not depend on the spacing
            np.testing.assert_array_equal(gu, ref[0])
            np.testing.assert_array_equal(gc, ref[1])


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("bkind,bval", [(DIRICHLET, 0.25), (PERIODIC, 0.0)])
def test_vc_adjoint_fp32_against_oracle(d, bkind, bval):
    sg = sgmod()
    r, pattern = 1, STAR
    shape = SHAPES[d]
    n = int(np.prod(shape))
    c = field(d, r, pattern, shape, 710 + d, 0.0, 0.3).astype(np.float32)
    u0 = uniform01(711, n).reshape(shape).astype(np.float32)
    T = 9
    w = [1.0] * npoints(d, r, pattern)
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_F32)
    ct = torch.from_numpy(c).to(DEV)
    x = torch.from_numpy(u0).to(DEV)
    y = torch.empty_like(x)
    sg.stencil_run_vc(plan, ct, x, y, T)
    torch.cuda.synchronize()
    # target 0: lam_T = u_T > 0 and every term of both gradients is positive
    _, ogu, ogc = oracle.adjoint_vc(d, r, pattern, shape, c.astype(np.float64), bkind, float(np.float32(bval)),
                                    u0.astype(np.float64), np.zeros(shape), T)
    gu, gc = gpu_adjoint(plan, c, u0, y.cpu().numpy(), T, 4)
    assert normwise(gu, ogu) <= 1e-5
    assert normwise(gc, ogc) <= 1e-5


def test_vc_adjoint_zero_steps_and_errors():
    sg = sgmod()
    shape = (11, 12)
    n = int(np.prod(shape))
    c = field(2, 1, STAR, shape, 720, 0.0, 0.3)
    u0 = uniform01(721, n).reshape(shape)
    g = uniform01(722, n).reshape(shape)
    plan = sg.stencil_plan_create(2, 1, shape, STAR, [1.0] * 5, DIRICHLET, 0.0, sg.STENCIL_F64)
    gu, gc = gpu_adjoint(plan, c, u0, g, 0, 1)
    np.testing.assert_array_equal(gu, g)
    assert not np.any(gc)
    with pytest.raises(sg.StencilError):
        gpu_adjoint(plan, c, u0, g, 5, 6)   # ckpt_every beyond T
    p32 = sg.stencil_plan_create(2, 1, shape, STAR, [1.0] * 5, DIRICHLET, 0.0, sg.STENCIL_I32)
    ci = torch.zeros((5,) + shape, dtype=torch.int32, device=DEV)
    xi = torch.zeros(shape, dtype=torch.int32, device=DEV)
    with pytest.raises(ValueError):
        sg.stencil_adjoint_vc(p32, ci, xi, xi, 3, 1)

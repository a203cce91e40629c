"""GPU parity at radius 3 in 2D and 3D, the largest order stencil_plan_create
accepts (paper Section 1: a (2r+1)-per-dimension neighbourhood; Table 1 lists
orders 1 and 2, order 3 is the library's upper limit).

Bars: int32 bit-exact against the oracle for star and box, Dirichlet and
periodic; FP64 normwise error <= 1e-12 and FP32 <= 1e-5 against the oracle;
every fusion depth the plan accepts bit-identical to the plain one-step sweep.
Grids are chosen so that several tiles, ragged last tiles and (periodic) halos
wider than a tile's edge are exercised.
"""

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, f32_weights, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FUSED, PLAIN, PER_PASS = 0, 1, 2


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def run(plan, u0, T, k=None, variant=FUSED):
    sg = sgmod()
    sg.stencil_plan_set_variant(plan, variant)
    if k is not None:
        sg.stencil_plan_set_k(plan, k)
    x = torch.from_numpy(np.ascontiguousarray(u0)).to(DEV)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    return y.cpu().numpy()


def normwise(g, o):
    return float(np.max(np.abs(np.asarray(g, np.float64) - o)) / max(1e-300, np.max(np.abs(o))))


def kvalues(plan):
    return list(range(1, sgmod().stencil_plan_max_k(plan) + 1))


SHAPES = {2: [(71, 300), (7, 9), (130, 23)], 3: [(13, 17, 140), (7, 8, 9), (20, 41, 37)]}


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_radius3_int32_bit_exact(d, pattern, bkind):
    sg = sgmod()
    r = 3
    rng = np.random.default_rng(3000 + 10 * d + pattern + 3 * bkind)
    for shape in SHAPES[d]:
        n = int(np.prod(shape))
        w = [float(x) for x in rng.integers(-3, 8, npoints(d, r, pattern))]
        bval = -4321 if bkind == DIRICHLET else 0
        u0 = uniform_u16(3100 + n, n).reshape(shape)
        plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        for T in (1, 5, 9):
            ref = oracle.run_int(d, r, pattern, shape, w, bkind, bval, u0, T)
            np.testing.assert_array_equal(run(plan, u0, T, variant=PLAIN), ref, err_msg=f"plain {shape} T={T}")
            for k in kvalues(plan):
                np.testing.assert_array_equal(run(plan, u0, T, k=k), ref, err_msg=f"k={k} {shape} T={T}")
                np.testing.assert_array_equal(run(plan, u0, T, k=k, variant=PER_PASS), ref,
                                              err_msg=f"per-pass k={k} {shape} T={T}")


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_radius3_fp64_fp32_against_oracle(d, pattern, bkind):
    sg = sgmod()
    r = 3
    rng = np.random.default_rng(3200 + 10 * d + pattern + 3 * bkind)
    for shape in SHAPES[d][:2]:
        n = int(np.prod(shape))
        w = list(rng.uniform(0.0, 1.0, npoints(d, r, pattern)))
        w = [x / sum(w) for x in w]
        bval = 0.35 if bkind == DIRICHLET else 0.0
        u0 = uniform01(3300 + n, n).reshape(shape)
        T = 7
        p64 = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_F64)
        ref = oracle.run(d, r, pattern, shape, w, bkind, bval, u0, T)
        base = run(p64, u0, T, variant=PLAIN)
        assert normwise(base, ref) <= 1e-12
        for k in kvalues(p64):
            np.testing.assert_array_equal(run(p64, u0, T, k=k), base, err_msg=f"f64 k={k} {shape}")
        u32 = u0.astype(np.float32)
        p32 = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_F32)
        ref32 = oracle.run(d, r, pattern, shape, f32_weights(w), bkind, float(np.float32(bval)),
                           u32.astype(np.float64), T)
        base32 = run(p32, u32, T, variant=PLAIN)
        assert normwise(base32, ref32) <= 1e-5
        for k in kvalues(p32):
            np.testing.assert_array_equal(run(p32, u32, T, k=k), base32, err_msg=f"f32 k={k} {shape}")

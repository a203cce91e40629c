"""The in-place sweep (paper Section 3.3, last paragraph: with the time loop
unrolled, a pass's input and output can share one array): results
bit-identical to stencil_run -- and exact against the oracle in the integer
mode -- with the extra device memory a fraction of the one workspace grid
stencil_run needs."""

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [(300, 517), (41, 1000), (5, 7), (129, 130), (1000, 61)]


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_inplace_int32_exact(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(40 + 7 * r + pattern + 3 * bkind)
    for shape in SHAPES:
        n = shape[0] * shape[1]
        w = [float(v) for v in rng.integers(-3, 7, npoints(2, r, pattern))]
        bval = 77 if bkind == DIRICHLET else 0
        u0 = uniform_u16(50 + n, n).reshape(shape)
        plan = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        for k in (1, 2, 3, 4):
            sg.stencil_plan_set_k(plan, min(k, sg.stencil_plan_max_k(plan)))
            for T in (1, 2 * k, 2 * k + 1):
                ref = oracle.run_int(2, r, pattern, shape, w, bkind, bval, u0, T)
                x = torch.from_numpy(u0).to(DEV)
                sg.stencil_run_inplace(plan, x, T)
                torch.cuda.synchronize()
                assert sg.stencil_get_device_status(plan) == 0
                np.testing.assert_array_equal(x.cpu().numpy(), ref, err_msg=f"{shape} k={k} T={T}")


@pytest.mark.parametrize("dt", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_inplace_bit_identical_to_two_grid_run(dt, bkind):
    sg = sgmod()
    code = {"f32": sg.STENCIL_F32, "f64": sg.STENCIL_F64, "bf16": sg.STENCIL_BF16}[dt]
    shape, T = (700, 1100), 13
    w = list(np.random.default_rng(3).uniform(0.0, 0.25, 9))
    plan = sg.stencil_plan_create(2, 1, shape, BOX, w, bkind, 0.3 if bkind == DIRICHLET else 0.0, code)
    x0 = torch.from_numpy(uniform01(9, shape[0] * shape[1]).reshape(shape)).to(sg.torch_dtype(code)).to(DEV)
    for k in (1, 2, 4):
        sg.stencil_plan_set_k(plan, k)
        ref = torch.empty_like(x0)
        sg.stencil_run(plan, x0, ref, T)
        x = x0.clone()
        sg.stencil_run_inplace(plan, x, T)
        torch.cuda.synchronize()
        assert torch.equal(x, ref), f"k={k}"


def test_inplace_footprint_is_a_fraction_of_a_grid():
    """At the benchmark size (8192^2 FP32, k = 2) the ring buffers take well
    under half of the workspace grid the two-grid sweep allocates; the sweep
    agrees with stencil_run bit for bit."""
    sg = sgmod()
    shape, T = (8192, 8192), 8
    plan = sg.stencil_plan_create(2, 1, shape, STAR, [0.5, 0.125, 0.125, 0.125, 0.125], DIRICHLET, 0.0,
                                  sg.STENCIL_F32)
    sg.stencil_plan_set_k(plan, 2)
    grid_bytes = shape[0] * shape[1] * 4
    extra = sg.stencil_inplace_workspace_bytes(plan)
    assert 0 < extra < 0.3 * grid_bytes, extra / grid_bytes
    x0 = torch.rand(shape, device=DEV)
    ref = torch.empty_like(x0)
    sg.stencil_run(plan, x0, ref, T)
    sg.stencil_run_inplace(plan, x0, T)
    torch.cuda.synchronize()
    assert torch.equal(x0, ref)


def test_inplace_rejects_other_dimensions():
    sg = sgmod()
    plan = sg.stencil_plan_create(3, 1, (8, 8, 8), STAR, [0.4] + [0.1] * 6, DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.zeros((8, 8, 8), device=DEV)
    with pytest.raises(sg.StencilError) as e:
        sg.stencil_run_inplace(plan, x, 3)
    assert e.value.status == sg.STENCIL_ERR_UNSUPPORTED

"""Host-buffer entry points and the FMA probe: stencil_run_host_many gives, for
every grid of the list, the result of a device stencil_run bit for bit (pinned
and pageable buffers, odd list lengths, an empty list, T = 0); the wrappers
reject host grids of the wrong size or dtype before any copy; the measured
FP32 / FP64 FMA rates lie in a plausible range for one GPU."""

import numpy as np
import pytest

from synth import BOX, DIRICHLET, PERIODIC, STAR, uniform01

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def device_run(plan, u0, T):
    sg = sgmod()
    x = torch.from_numpy(u0).to(DEV)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_run_host_many_matches_device_runs(n, pinned):
    sg = sgmod()
    shape, T = (257, 390), 11
    plan = sg.stencil_plan_create(2, 1, shape, BOX, [1 / 9] * 9, PERIODIC, 0.0, sg.STENCIL_F32)
    ins = [uniform01(40 + i, shape[0] * shape[1]).reshape(shape).astype(np.float32) for i in range(n)]
    refs = [device_run(plan, u, T) for u in ins]
    h_in = [torch.from_numpy(u) for u in ins]
    h_out = [torch.empty(shape, dtype=torch.float32) for _ in range(n)]
    if pinned:
        h_in = [t.pin_memory() for t in h_in]
        h_out = [t.pin_memory() for t in h_out]
    sg.stencil_run_host_many(plan, h_in, h_out, T)
    for i in range(n):
        np.testing.assert_array_equal(h_out[i].numpy(), refs[i], err_msg=f"grid {i}")
    # numpy buffers, and T = 0 copies through
    outs = [np.empty_like(u) for u in ins]
    sg.stencil_run_host_many(plan, ins, outs, 0)
    for i in range(n):
        np.testing.assert_array_equal(outs[i], ins[i])


def test_run_host_many_empty_and_argument_checks():
    sg = sgmod()
    shape = (64, 96)
    plan = sg.stencil_plan_create(2, 1, shape, STAR, [0.5, 0.125, 0.125, 0.125, 0.125], DIRICHLET, 0.0,
                                  sg.STENCIL_F32)
    sg.stencil_run_host_many(plan, [], [], 4)
    good = np.zeros(shape, np.float32)
    with pytest.raises(ValueError):
        sg.stencil_run_host_many(plan, [good], [], 4)
    with pytest.raises(ValueError):
        sg.stencil_run_host_many(plan, [np.zeros((64, 95), np.float32)], [good], 4)
    with pytest.raises(ValueError):
        sg.stencil_run_host_many(plan, [good], [np.zeros(shape, np.float64)], 4)
    with pytest.raises(ValueError):
        sg.stencil_run_host(plan, good, np.zeros(64 * 96 - 1, np.float32), 4)
    with pytest.raises(ValueError):
        sg.stencil_run_host(plan, torch.zeros(shape, device=DEV), good, 4)


def test_fma_probe_rates_are_plausible():
    sg = sgmod()
    f32 = sg.stencil_probe_fma_rate(sg.STENCIL_F32)
    f64 = sg.stencil_probe_fma_rate(sg.STENCIL_F64)
    # one GPU: between a small part and a few times the nominal FMA rates
    assert 1e12 < f32 < 1e15, f32
    assert 1e10 < f64 < 1e14, f64
    assert f32 > 4 * f64
    with pytest.raises(sg.StencilError):
        sg.stencil_probe_fma_rate(sg.STENCIL_I32)

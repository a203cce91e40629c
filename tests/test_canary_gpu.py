"""Guard bands around every output: no kernel writes outside the grid it owns.

The fused kernels read a few values beyond their dependency windows on
purpose (whole TMA stages, prefetched rows), so a stray *write* would only be
caught by a parity test if it happened to land in a compared value.  Here each
output grid sits in the middle of a larger allocation whose margins hold a
poison pattern, and every launch form (persistent multi-pass, one launch per
pass, plain one-step, batched, adjoint) must leave the margins -- and the
input -- untouched.  Margins are at least one full row (or plane) plus a
16-byte-misaligning offset on both sides.
"""

import numpy as np
import pytest

from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FUSED, PLAIN, PER_PASS = 0, 1, 2
POISON_F = -1.2345e30
POISON_I = -0x5A5A5A5A


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


class Guarded:
    """A grid of `shape` inside an allocation with poisoned margins of `pad`
    elements before and after (pad a multiple of 4 keeps 16-byte alignment
    for 4-byte types; odd pads misalign it)."""

    def __init__(self, shape, dtype, pad, fill=None):
        n = int(np.prod(shape))
        self.n, self.pad, self.shape = n, pad, tuple(shape)
        poison = POISON_I if dtype == torch.int32 else POISON_F
        self.buf = torch.full((n + 2 * pad,), poison, dtype=dtype, device=DEV)
        self.poison = self.buf[:pad].clone()
        if fill is not None:
            self.view.copy_(fill)

    @property
    def view(self):
        return self.buf[self.pad:self.pad + self.n].view(self.shape)

    def margins_intact(self):
        torch.cuda.synchronize()
        lo = self.buf[:self.pad]
        hi = self.buf[self.pad + self.n:]
        return torch.equal(lo, self.poison) and torch.equal(hi, self.poison)


def check_run(sg, plan, x_host, T, k, variant, pad, dtype):
    xin = Guarded(x_host.shape, dtype, pad, torch.from_numpy(x_host).to(DEV))
    before = xin.view.clone()
    out = Guarded(x_host.shape, dtype, pad)
    sg.stencil_plan_set_variant(plan, variant)
    sg.stencil_plan_set_k(plan, k)
    sg.stencil_run(plan, xin.view, out.view, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    assert out.margins_intact(), f"write outside the output: k={k} variant={variant} pad={pad}"
    assert xin.margins_intact() and torch.equal(xin.view, before), f"input written: k={k} variant={variant}"
    return out.view.clone()


CASES = [
    (1, 1, STAR, (4099,)), (1, 3, STAR, (1000,)),
    (2, 1, STAR, (300, 517)), (2, 2, BOX, (131, 260)), (2, 3, BOX, (40, 77)),
    (3, 1, STAR, (21, 37, 141)), (3, 1, BOX, (18, 40, 132)), (3, 2, STAR, (15, 19, 70)), (3, 3, BOX, (9, 11, 30)),
]


@pytest.mark.parametrize("d,r,pattern,shape", CASES)
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_outputs_stay_in_bounds(d, r, pattern, shape, bkind, dt):
    sg = sgmod()
    n = int(np.prod(shape))
    rng = np.random.default_rng(d + 7 * r + 3 * pattern + bkind)
    if dt == "i32":
        w = [float(v) for v in rng.integers(-2, 5, npoints(d, r, pattern))]
        code, tdt = sg.STENCIL_I32, torch.int32
        x = uniform_u16(4000 + n, n).reshape(shape)
        bval = 17
    else:
        w = list(rng.uniform(0.0, 0.3, npoints(d, r, pattern)))
        code, tdt = sg.STENCIL_F32, torch.float32
        x = uniform01(4000 + n, n).reshape(shape).astype(np.float32)
        bval = 0.5
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval if bkind == DIRICHLET else 0, code)
    row = shape[-1] if d == 1 else int(np.prod(shape[1:]))
    ref = None
    for pad in (row + 64, row + 67):     # aligned and misaligned base pointers
        for T in (5, 12):
            ref = check_run(sg, plan, x, T, 1, PLAIN, pad, tdt)
            for k in range(1, sg.stencil_plan_max_k(plan) + 1):
                for variant in (FUSED, PER_PASS):
                    got = check_run(sg, plan, x, T, k, variant, pad, tdt)
                    assert torch.equal(got, ref), f"k={k} variant={variant} T={T}"


def test_batch_outputs_stay_in_bounds():
    import synth
    sg = sgmod()
    rng = np.random.default_rng(91)
    probs = []
    for g in range(12):
        shape = (int(rng.integers(5, 200)), int(rng.integers(5, 300)))
        w = list(rng.uniform(0.05, 1.0, 9))
        w = [v / sum(w) for v in w]
        probs.append(synth.Problem(f"g{g}", 2, 1, BOX, shape, w, PERIODIC, 0.0, int(rng.integers(1, 30)), 200 + g))
    ins = [Guarded(p.shape, torch.float32, p.shape[1] + 33,
                   torch.from_numpy(uniform01(p.seed, p.npts).reshape(p.shape).astype(np.float32)).to(DEV))
           for p in probs]
    outs = [Guarded(p.shape, torch.float32, p.shape[1] + 33) for p in probs]
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX, 1,
                                PERIODIC, 0.0, sg.STENCIL_F32)
    for _ in range(2):          # capture, then replay
        sg.stencil_batch_run(b, [g.view for g in ins], [g.view for g in outs])
        torch.cuda.synchronize()
        assert sg.stencil_batch_get_device_status(b) == 0
        for i, (gi, go) in enumerate(zip(ins, outs)):
            assert go.margins_intact(), f"batch member {i} wrote outside its output"
            assert gi.margins_intact(), f"batch member {i} wrote outside its input"


@pytest.mark.parametrize("d,r,shape", [(3, 1, (20, 33, 40)), (3, 2, (16, 18, 36)), (2, 1, (70, 90))])
def test_adjoint_outputs_stay_in_bounds(d, r, shape):
    sg = sgmod()
    n = int(np.prod(shape))
    w = list(np.random.default_rng(5).uniform(0.02, 0.2, npoints(d, r, STAR)))
    plan = sg.stencil_plan_create(d, r, shape, STAR, w, PERIODIC, 0.0, sg.STENCIL_F32)
    pad = int(np.prod(shape[1:])) + 35
    u0 = Guarded(shape, torch.float32, pad, torch.from_numpy(uniform01(1, n).reshape(shape).astype(np.float32)).to(DEV))
    g = Guarded(shape, torch.float32, pad, torch.from_numpy(uniform01(2, n).reshape(shape).astype(np.float32)).to(DEV))
    gu = Guarded(shape, torch.float32, pad)
    gw = Guarded((len(w),), torch.float64, 9)
    sg.stencil_adjoint_run(plan, u0.view, g.view, 9, 4, gu.view, gw.view)
    torch.cuda.synchronize()
    assert gu.margins_intact() and gw.margins_intact() and u0.margins_intact() and g.margins_intact()

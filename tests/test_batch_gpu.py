"""Batched runs (one persistent, graph-captured kernel over many grids)
against per-grid stencil_run calls and the oracle."""

import time

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, c4_batch, f32_weights, npoints, uniform01, uniform_u16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def single_runs(sg, probs, xs, dtype):
    outs = []
    for p, x in zip(probs, xs):
        plan = sg.stencil_plan_create(2, p.r, p.shape, p.pattern, p.weights, p.bkind, p.bval, dtype)
        y = torch.empty_like(x)
        sg.stencil_run(plan, x, y, p.T)
        outs.append(y)
    torch.cuda.synchronize()
    return outs


def random_batch(n, seed, pattern, bkind, lo=5, hi=300, tmax=21, r=1, integer=False):
    import synth
    rng = np.random.default_rng(seed)
    probs = []
    for g in range(n):
        shape = (int(rng.integers(lo, hi)), int(rng.integers(lo, hi)))
        T = int(rng.integers(0 if g == 3 else 1, tmax))
        npt = npoints(2, r, pattern)
        w = [float(v) for v in rng.integers(-3, 6, npt)] if integer else list(rng.uniform(0.05, 1.0, npt))
        if not integer:
            s = sum(w)
            w = [v / s for v in w]
        probs.append(synth.Problem(f"g{g}", 2, r, pattern, shape, w, bkind, 5 if integer and bkind == DIRICHLET
                                   else 0.0, T, 100 + g))
    return probs


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [PERIODIC, DIRICHLET])
def test_batch_f32_matches_single_runs(pattern, bkind):
    sg = sgmod()
    probs = random_batch(24, 3 + pattern + 2 * bkind, pattern, bkind)
    xs = [torch.from_numpy(uniform01(p.seed, p.npts).reshape(p.shape).astype(np.float32)).to(DEV) for p in probs]
    ref = single_runs(sg, probs, xs, sg.STENCIL_F32)
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], pattern,
                                1, bkind, 0.0, sg.STENCIL_F32)
    ys = [torch.empty_like(x) for x in xs]
    for rep in range(2):     # first call captures the graph, second replays it
        for y in ys:
            y.fill_(-1.0)
        sg.stencil_batch_run(b, xs, ys)
        torch.cuda.synchronize()
        assert sg.stencil_batch_get_device_status(b) == 0
        for g, (y, r) in enumerate(zip(ys, ref)):
            assert torch.equal(y, r), (rep, g, probs[g].shape, probs[g].T)
    assert sg.stencil_batch_launch_count(b) == 1
    # a few members against the FP64 oracle
    for g in range(0, 24, 6):
        p = probs[g]
        o = oracle.run(2, 1, pattern, p.shape, f32_weights(p.weights), bkind, 0.0,
                       xs[g].cpu().numpy().astype(np.float64), p.T)
        assert np.max(np.abs(ys[g].cpu().numpy() - o)) <= 1e-5 * max(1.0, np.max(np.abs(o)))


@pytest.mark.parametrize("r,pattern", [(1, BOX), (1, STAR), (2, STAR), (2, BOX)])
@pytest.mark.parametrize("bkind", [PERIODIC, DIRICHLET])
def test_batch_int32_bit_exact(r, pattern, bkind):
    sg = sgmod()
    probs = random_batch(12, 40 + r + pattern + bkind, pattern, bkind, lo=3, hi=150, tmax=15, r=r, integer=True)
    us = [uniform_u16(p.seed, p.npts).reshape(p.shape) for p in probs]
    xs = [torch.from_numpy(u).to(DEV) for u in us]
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], pattern,
                                r, bkind, 5 if bkind == DIRICHLET else 0.0, sg.STENCIL_I32)
    ys = [torch.empty_like(x) for x in xs]
    sg.stencil_batch_run(b, xs, ys)
    torch.cuda.synchronize()
    assert sg.stencil_batch_get_device_status(b) == 0
    for p, u, y in zip(probs, us, ys):
        ref = oracle.run_int(2, r, pattern, p.shape, p.weights, bkind, p.bval, u, p.T)
        np.testing.assert_array_equal(y.cpu().numpy(), ref, err_msg=f"{p.shape} T={p.T}")


def test_batch_new_buffers_after_capture():
    """Replaying the captured graph with other input/output tensors."""
    sg = sgmod()
    probs = random_batch(8, 99, BOX, PERIODIC)
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX,
                                1, PERIODIC, 0.0, sg.STENCIL_F32)
    for seed in (1, 2, 3):
        xs = [torch.from_numpy(uniform01(seed * 1000 + g, p.npts).reshape(p.shape).astype(np.float32)).to(DEV)
              for g, p in enumerate(probs)]
        ys = [torch.empty_like(x) for x in xs]
        sg.stencil_batch_run(b, xs, ys)
        ref = single_runs(sg, probs, xs, sg.STENCIL_F32)
        for y, r in zip(ys, ref):
            assert torch.equal(y, r)


def test_batch_rejects_aliasing():
    sg = sgmod()
    probs = random_batch(3, 5, BOX, PERIODIC)
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX,
                                1, PERIODIC, 0.0, sg.STENCIL_F32)
    xs = [torch.zeros(p.shape, device=DEV) for p in probs]
    with pytest.raises(sg.StencilError) as e:
        sg.stencil_batch_run(b, xs, [xs[0]] + [torch.empty_like(x) for x in xs[1:]])
    assert e.value.status == sg.STENCIL_ERR_INVALID_ARG


def test_batch_timeout_is_reported_not_hung():
    """Fault injected on the host side: one work item never publishes its
    completion.  The items that depend on it give up their bounded waits
    (about a second), the batch reports STENCIL_ERR_TIMEOUT, and the GPU
    context stays usable."""
    sg = sgmod()
    probs = random_batch(4, 7, BOX, PERIODIC, lo=100, hi=200, tmax=20)
    for p in probs:
        p.T = max(p.T, 9)
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX,
                                1, PERIODIC, 0.0, sg.STENCIL_F32)
    assert sg.load().stencil_batch_test_skip_publish(b.handle, 0) == 0   # item 0: grid 0, pass 0, tile 0
    xs = [torch.rand(p.shape, device=DEV) for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    t0 = time.time()
    sg.stencil_batch_run(b, xs, ys)
    status = sg.stencil_batch_get_device_status(b)
    assert status == sg.STENCIL_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # the context still works
    assert sg.load().stencil_batch_test_skip_publish(b.handle, -1) == 0
    sg.stencil_batch_run(b, xs, ys)
    assert sg.stencil_batch_get_device_status(b) == 0
    ref = single_runs(sg, probs, xs, sg.STENCIL_F32)
    for y, r in zip(ys, ref):
        assert torch.equal(y, r)


def test_batch_full_workload():
    """The batched workload: 256 periodic 2D 9-point grids, sides log-uniform
    in [64, 2048], T uniform in [8, 128], normalised random weights.  Every
    output bit-identical to its own stencil_run; mass conserved."""
    sg = sgmod()
    probs = c4_batch()
    xs = [torch.from_numpy(uniform01(p.seed, p.npts).reshape(p.shape).astype(np.float32)).to(DEV) for p in probs]
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX,
                                1, PERIODIC, 0.0, sg.STENCIL_F32)
    ys = [torch.empty_like(x) for x in xs]
    sg.stencil_batch_run(b, xs, ys)
    torch.cuda.synchronize()
    assert sg.stencil_batch_get_device_status(b) == 0
    ref = single_runs(sg, probs, xs, sg.STENCIL_F32)
    for g, (y, r) in enumerate(zip(ys, ref)):
        assert torch.equal(y, r), g
    for x, y in zip(xs[:16], ys[:16]):
        m0, m1 = x.double().sum().item(), y.double().sum().item()
        assert abs(m1 - m0) <= 1e-4 * abs(m0)


@pytest.mark.parametrize("bkind", [PERIODIC, DIRICHLET])
def test_batch_config_and_tune_keep_results(bkind):
    """Every fusion depth and tile height of the batch, and the tuner's
    choice, give results bit-identical to per-grid stencil_run calls."""
    sg = sgmod()
    probs = random_batch(16, 90 + bkind, BOX, bkind)
    xs = [torch.from_numpy(uniform01(p.seed, p.npts).reshape(p.shape).astype(np.float32)).to(DEV) for p in probs]
    ref = single_runs(sg, probs, xs, sg.STENCIL_F32)
    b = sg.stencil_batch_create([p.shape for p in probs], [p.weights for p in probs], [p.T for p in probs], BOX, 1,
                                bkind, 0.0, sg.STENCIL_F32)
    ys = [torch.empty_like(x) for x in xs]
    for k in (1, 2, 3, 4):
        for rows in (16, 32, 128):
            if rows < 4 * k:
                continue
            sg.stencil_batch_set_config(b, k, rows)
            assert sg.stencil_batch_get_config(b) == (k, rows)
            sg.stencil_batch_run(b, xs, ys)
            torch.cuda.synchronize()
            assert sg.stencil_batch_get_device_status(b) == 0
            for i, (y, r) in enumerate(zip(ys, ref)):
                assert torch.equal(y, r), (k, rows, i)
    ms = sg.stencil_batch_tune(b, xs, ys)
    assert ms > 0
    sg.stencil_batch_run(b, xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, ref):
        assert torch.equal(y, r)

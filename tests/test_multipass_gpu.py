"""GPU parity of the persistent multi-pass 2D kernel (all passes of exactly
k steps in one launch, tiles waiting on their neighbours' previous pass).

Bars: int32 bit-exact against the oracle; FP32 and FP64 bit-identical to the
one-launch-per-pass fused kernels and to the plain one-step sweep (same
per-point operation order), and within 1e-5 / 1e-12 normwise of the oracle.
Grids span many tiles with ragged last bands and chunks, periodic halos that
reach two tiles, unaligned base pointers (register-load path) and repeated
runs (the launch alternates two sets of counters).
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


def run(plan, x, T, k, variant, offset=0):
    """stencil_run on device tensor x; offset > 0 shifts both grids by that
    many elements inside larger allocations (unaligned base pointers)."""
    sg = sgmod()
    sg.stencil_plan_set_variant(plan, variant)
    sg.stencil_plan_set_k(plan, k)
    if offset:
        xin = torch.empty(x.numel() + offset, dtype=x.dtype, device=DEV)
        xin[offset:] = x.reshape(-1)
        xo = torch.empty_like(xin)
        sg.stencil_run(plan, xin[offset:].view(x.shape), xo[offset:].view(x.shape), T)
        y = xo[offset:].view(x.shape)
    else:
        y = torch.empty_like(x)
        sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    return y.clone()


def normwise(g, o):
    return float(np.max(np.abs(np.asarray(g, np.float64) - o)) / max(1e-300, np.max(np.abs(o))))


# shapes: many bands and chunks with ragged last ones, a single band, few rows
SHAPES = [(700, 1000), (257, 4100), (2000, 130), (37, 5003), (9, 300)]


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_int32_bit_exact(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(500 + 10 * r + pattern + 3 * bkind)
    for shape in SHAPES:
        w = [float(x) for x in rng.integers(-3, 8, npoints(2, r, pattern))]
        bval = -777 if bkind == DIRICHLET else 0
        u0 = uniform_u16(900 + shape[1], shape[0] * shape[1]).reshape(shape)
        plan = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        x = torch.from_numpy(u0).to(DEV)
        kmax = sg.stencil_plan_max_k(plan)
        for k in sorted({1, 2, kmax // 2 or 1, kmax}):
            for T in (2 * k, 3 * k + 1, 5 * k):
                ref = oracle.run_int(2, r, pattern, shape, w, bkind, bval, u0, T)
                got = run(plan, x, T, k, FUSED).cpu().numpy()
                np.testing.assert_array_equal(got, ref, err_msg=f"{shape} k={k} T={T}")
                assert sg.stencil_plan_launch_count(plan, T) == 1 + (T % k > 0)


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_fp32_fp64_identical_to_per_pass_and_oracle(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(600 + 10 * r + pattern + 3 * bkind)
    for shape in SHAPES[:3]:
        w = list(rng.uniform(-0.1, 0.4, npoints(2, r, pattern)))
        bval = 0.25 if bkind == DIRICHLET else 0.0
        u0 = uniform01(1002, shape[0] * shape[1]).reshape(shape)
        for dt, tol in ((sg.STENCIL_F32, 1e-5), (sg.STENCIL_F64, 1e-12)):
            plan = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, dt)
            if dt == sg.STENCIL_F32:
                ui = u0.astype(np.float32)
                ref_w, ref_b, ref_u = f32_weights(w), float(np.float32(bval)), ui.astype(np.float64)
            else:
                ui, ref_w, ref_b, ref_u = u0, w, bval, u0
            x = torch.from_numpy(ui).to(DEV)
            kmax = sg.stencil_plan_max_k(plan)
            T = 4 * kmax + 1
            ref = oracle.run(2, r, pattern, shape, ref_w, bkind, ref_b, ref_u, T)
            plain = run(plan, x, T, 1, PLAIN)
            assert normwise(plain.cpu().numpy(), ref) <= tol
            for k in range(1, kmax + 1):
                mp = run(plan, x, T, k, FUSED)
                pp = run(plan, x, T, k, PER_PASS)
                assert torch.equal(mp, pp), f"{shape} dt={dt} k={k}"
                assert torch.equal(mp, plain), f"{shape} dt={dt} k={k}"


@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_unaligned_pointers_register_path(bkind):
    """Base pointers off 16-byte alignment: the register-load producer with
    L2-coherent loads (data written by other SMs within the launch)."""
    sg = sgmod()
    shape, r, pattern = (513, 1031), 1, STAR
    w = [0.5, 0.125, 0.125, 0.125, 0.125]
    plan = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, 0.5 if bkind == DIRICHLET else 0.0,
                                  sg.STENCIL_F32)
    x = torch.from_numpy(uniform01(77, shape[0] * shape[1]).reshape(shape).astype(np.float32)).to(DEV)
    for k in (1, 3, 4, 8):
        T = 6 * k
        plain = run(plan, x, T, 1, PLAIN)
        for off in (1, 3):
            assert torch.equal(run(plan, x, T, k, FUSED, offset=off), plain), f"k={k} offset={off}"


def test_repeated_runs_alternate_counters():
    sg = sgmod()
    shape = (1500, 1500)
    w = [1 / 9] * 9
    plan = sg.stencil_plan_create(2, 1, shape, BOX, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.from_numpy(uniform01(5, shape[0] * shape[1]).reshape(shape).astype(np.float32)).to(DEV)
    first = run(plan, x, 40, 4, FUSED)
    for _ in range(4):
        assert torch.equal(run(plan, x, 40, 4, FUSED), first)
    # a change of k regrows the counters; per-pass launches in between
    assert torch.equal(run(plan, x, 40, 8, FUSED), first)
    assert torch.equal(run(plan, x, 40, 2, PER_PASS), first)
    assert torch.equal(run(plan, x, 40, 5, FUSED), first)


def test_bench_size_many_passes():
    """2048^2 FP32 2D5P, T = 64: the persistent launch against the oracle."""
    sg = sgmod()
    shape, T = (2048, 2048), 64
    w = [0.5, 0.125, 0.125, 0.125, 0.125]
    u0 = uniform01(1002, shape[0] * shape[1]).reshape(shape).astype(np.float32)
    plan = sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.from_numpy(u0).to(DEV)
    ref = oracle.run(2, 1, STAR, shape, f32_weights(w), DIRICHLET, 0.0, u0.astype(np.float64), T)
    for k in (2, 4, 6, 8):
        got = run(plan, x, T, k, FUSED)
        assert normwise(got.cpu().numpy(), ref) <= 1e-5
        assert sg.stencil_plan_launch_count(plan, T) == 1 + (T % k > 0)


def test_tile_rows_do_not_change_results():
    sg = sgmod()
    shape = (1111, 900)
    w = [0.5, 0.125, 0.125, 0.125, 0.125]
    for bkind in (DIRICHLET, PERIODIC):
        plan = sg.stencil_plan_create(2, 1, shape, STAR, w, bkind, 0.0, sg.STENCIL_F32)
        x = torch.from_numpy(uniform01(8, shape[0] * shape[1]).reshape(shape).astype(np.float32)).to(DEV)
        plain = run(plan, x, 24, 1, PLAIN)
        for rows in (1, 16, 17, 50, 333, 5000):
            sg.stencil_plan_set_tile_rows(plan, rows)
            assert sg.stencil_plan_get_tile_rows(plan) == rows
            for k in (2, 4, 8):
                assert torch.equal(run(plan, x, 24, k, FUSED), plain), f"rows={rows} k={k}"
                assert torch.equal(run(plan, x, 24, k, PER_PASS), plain), f"rows={rows} k={k}"
        sg.stencil_plan_set_tile_rows(plan, 0)
        k, ms = sg.stencil_plan_tune(plan, 24)
        assert sg.stencil_plan_get_tile_rows(plan) in (0, 32, 48, 64, 96, 128, 192)
        v = sg.stencil_plan_get_variant(plan)
        assert v in (FUSED, PLAIN, PER_PASS) and (v == PLAIN) == (k == 0)
        y = torch.empty_like(x)
        sg.stencil_run(plan, x, y, 24)      # the tuned configuration as it stands
        torch.cuda.synchronize()
        assert torch.equal(y, plain)


# ------------------------------------------------------------------- 3D
SHAPES_3D = [(40, 70, 300), (23, 33, 129), (9, 100, 37)]


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_3d_int32_bit_exact(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(700 + 10 * r + pattern + 3 * bkind)
    for shape in SHAPES_3D:
        w = [float(x) for x in rng.integers(-2, 5, npoints(3, r, pattern))]
        bval = 4321 if bkind == DIRICHLET else 0
        n = shape[0] * shape[1] * shape[2]
        u0 = uniform_u16(950 + shape[2], n).reshape(shape)
        plan = sg.stencil_plan_create(3, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        x = torch.from_numpy(u0).to(DEV)
        kmax = sg.stencil_plan_max_k(plan)
        for k in sorted({1, kmax}):
            T = 2 * k + 1
            ref = oracle.run_int(3, r, pattern, shape, w, bkind, bval, u0, T)
            got = run(plan, x, T, k, FUSED).cpu().numpy()
            np.testing.assert_array_equal(got, ref, err_msg=f"{shape} k={k} T={T}")
            # the 125-point box has no fused form: one plain launch per step
            expect = T if (r == 2 and pattern == BOX) else 1 + (T % k > 0)
            assert sg.stencil_plan_launch_count(plan, T) == expect


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_3d_fp32_identical_to_per_pass_plain_and_oracle(pattern, bkind):
    sg = sgmod()
    shape = SHAPES_3D[0]
    w = list(np.random.default_rng(77 + pattern + bkind).uniform(-0.05, 0.2, npoints(3, 1, pattern)))
    bval = 0.5 if bkind == DIRICHLET else 0.0
    u0 = uniform01(1003, shape[0] * shape[1] * shape[2]).reshape(shape).astype(np.float32)
    plan = sg.stencil_plan_create(3, 1, shape, pattern, w, bkind, bval, sg.STENCIL_F32)
    x = torch.from_numpy(u0).to(DEV)
    T = 17
    ref = oracle.run(3, 1, pattern, shape, f32_weights(w), bkind, float(np.float32(bval)), u0.astype(np.float64), T)
    plain = run(plan, x, T, 1, PLAIN)
    assert normwise(plain.cpu().numpy(), ref) <= 1e-5
    for k in range(1, sg.stencil_plan_max_k(plan) + 1):
        assert torch.equal(run(plan, x, T, k, FUSED), plain), f"k={k}"
        assert torch.equal(run(plan, x, T, k, PER_PASS), plain), f"k={k}"
        for off in (1,):
            assert torch.equal(run(plan, x, T, k, FUSED, offset=off), plain), f"k={k} offset={off}"
    for planes in (1, 8, 13, 40):
        sg.stencil_plan_set_tile_rows(plan, planes)
        for k in (2, 4):
            assert torch.equal(run(plan, x, T, k, FUSED), plain), f"planes={planes} k={k}"


def test_3d_bench_size_sampled():
    """512^3 FP32 3D7P, T = 32, at the tuned configuration: the persistent
    launch bit-identical to the plain sweep (whose parity against the oracle
    the dependency-cone tests establish)."""
    sg = sgmod()
    shape, T = (512, 512, 512), 32
    w = [0.4] + [0.1] * 6
    plan = sg.stencil_plan_create(3, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.rand(shape, device=DEV)
    plain = run(plan, x, T, 1, PLAIN)
    k, _ = sg.stencil_plan_tune(plan, T)
    for kk in sorted({max(k, 1), 4}):
        assert torch.equal(run(plan, x, T, kk, FUSED), plain), f"k={kk}"


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dependency_timeout_is_reported_and_recovers(dim):
    """Host-side fault injection: tile 0's pass counter is poisoned (a large
    negative value), so the tiles of pass 1 that read it must give up their
    bounded waits (about one second), raise the abort flag and report
    STENCIL_ERR_TIMEOUT; the context stays usable, the aborted launch's last
    worker resets the counters, and the next runs are correct."""
    import time
    sg = sgmod()
    shape = {1: (100003,), 2: (300, 500), 3: (40, 70, 300)}[dim]
    w = {1: [0.25, 0.5, 0.25], 2: [0.5, 0.125, 0.125, 0.125, 0.125], 3: [0.4] + [0.1] * 6}[dim]
    plan = sg.stencil_plan_create(dim, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.rand(shape, device=DEV)
    plain = run(plan, x, 8, 1, PLAIN)
    sg.stencil_plan_set_variant(plan, FUSED)
    sg.stencil_plan_set_k(plan, 2)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, 8)            # allocates the counters
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    assert sg.load().stencil_plan_test_poison_counter(plan.handle, 0) == 0
    t0 = time.time()
    sg.stencil_run(plan, x, y, 8)
    assert sg.stencil_get_device_status(plan) == sg.STENCIL_ERR_TIMEOUT
    assert time.time() - t0 < 30
    for _ in range(2):
        assert torch.equal(run(plan, x, 8, 2, FUSED), plain)



# ------------------------------------------------------------------- 1D
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("n", [5, 300, 257, 4097, 65536, 100003])
def test_1d_int32_bit_exact_and_fp64_identical(r, bkind, n):
    sg = sgmod()
    rng = np.random.default_rng(800 + r + 3 * bkind + n % 97)
    w = [float(x) for x in rng.integers(-3, 8, 2 * r + 1)]
    bval = 99 if bkind == DIRICHLET else 0
    u0 = uniform_u16(960 + n, n)
    plan = sg.stencil_plan_create(1, r, (n,), STAR, w, bkind, bval, sg.STENCIL_I32)
    x = torch.from_numpy(u0).to(DEV)
    for k in (1, 3, 8):
        for T in (2 * k, 3 * k + 2):
            ref = oracle.run_int(1, r, STAR, (n,), w, bkind, bval, u0, T)
            np.testing.assert_array_equal(run(plan, x, T, k, FUSED).cpu().numpy(), ref, err_msg=f"k={k} T={T}")
    wf = list(rng.uniform(0.05, 0.3, 2 * r + 1))
    u = uniform01(961 + n, n)
    pf = sg.stencil_plan_create(1, r, (n,), STAR, wf, bkind, 0.25 if bkind == DIRICHLET else 0.0, sg.STENCIL_F64)
    xf = torch.from_numpy(u).to(DEV)
    T = 37
    ref = oracle.run(1, r, STAR, (n,), wf, bkind, 0.25 if bkind == DIRICHLET else 0.0, u, T)
    plain = run(pf, xf, T, 1, PLAIN)
    assert normwise(plain.cpu().numpy(), ref) <= 1e-12
    for k in (1, 2, 5, 8):
        assert torch.equal(run(pf, xf, T, k, FUSED), plain), f"k={k}"
    for cpj in (1, 13, 40):
        sg.stencil_plan_set_tile_rows(pf, cpj)
        assert torch.equal(run(pf, xf, T, 4, FUSED), plain), f"cpj={cpj}"



@pytest.mark.parametrize("variant", [FUSED, PER_PASS])
def test_cuda_graph_replay(variant):
    """stencil_run captured into a CUDA graph (after one uncaptured call with
    the same settings) and replayed: every launch leaves its ticket and
    dependency counters at zero, so each replay -- the same parameters --
    recomputes the result."""
    sg = sgmod()
    cases = [(1, (100003,), [0.25, 0.5, 0.25], 21, 4), (2, (700, 1000), [0.5, 0.125, 0.125, 0.125, 0.125], 22, 4),
             (3, (40, 70, 300), [0.4] + [0.1] * 6, 13, 3)]
    for dim, shape, w, T, k in cases:
        plan = sg.stencil_plan_create(dim, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
        x = torch.rand(shape, device=DEV)
        plain = run(plan, x, T, 1, PLAIN)
        sg.stencil_plan_set_variant(plan, variant)
        sg.stencil_plan_set_k(plan, k)
        y = torch.empty_like(x)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            sg.stencil_run(plan, x, y, T)          # allocates workspace and counters
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            sg.stencil_run(plan, x, y, T)
        for _ in range(3):
            y.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert sg.stencil_get_device_status(plan) == 0
            assert torch.equal(y, plain), f"dim={dim} variant={variant}"
        # and an ordinary call afterwards
        assert torch.equal(run(plan, x, T, k, variant), plain)

"""GPU parity: the CUDA kernels (through the C ABI) against the FP64/uint32
oracle on the same seeded inputs.

Bars (written here): int32 mode bit-exact; FP64 normwise error <= 1e-12;
FP32 normwise error <= 1e-5 after T steps; every fusion depth k gives results
bit-identical to the plain one-step kernel in FP32, FP64 and int32 (same
per-point operation order); BF16/F16 storage within the bound derived from
one round-to-nearest per pass (unit roundoff 2^-8 / 2^-11) for positive
weights summing to <= 1, which keep the max norm non-increasing.
"""

import numpy as np
import pytest

import oracle
from synth import (BOX, DIRICHLET, PERIODIC, STAR, box_weights, c2_2d5p, c2_2d9p, f32_weights, npoints,
                   sine_mode_1d, star_weights, uniform01, uniform_u16)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def gpu_run(plan, u0, T, k=None, variant=0):
    sg = sgmod()
    sg.stencil_plan_set_variant(plan, variant)
    if k is not None:
        sg.stencil_plan_set_k(plan, k)
    x = torch.from_numpy(np.ascontiguousarray(u0)).to(DEV)
    if plan.dtype in (sg.STENCIL_BF16, sg.STENCIL_F16):
        x = x.to(plan.torch_dtype)
    y = torch.empty_like(x)
    sg.stencil_run(plan, x, y, T)
    torch.cuda.synchronize()
    assert sg.stencil_get_device_status(plan) == 0
    return y


def normwise(g, o):
    return float(np.max(np.abs(np.asarray(g, np.float64) - o)) / max(1e-300, np.max(np.abs(o))))


def kvalues(plan):
    return list(range(1, sgmod().stencil_plan_max_k(plan) + 1))


SHAPES_2D = [(67, 300), (5, 1), (1, 7), (33, 129), (130, 17)]


# ------------------------------------------------------------- int32 mode
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_int32_bit_exact_2d_every_k(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(10 * r + pattern + 3 * bkind)
    for shape in SHAPES_2D:
        w = [float(x) for x in rng.integers(-3, 8, npoints(2, r, pattern))]
        bval = 12345 if bkind == DIRICHLET else 0
        u0 = uniform_u16(700 + shape[0], shape[0] * shape[1]).reshape(shape)
        plan = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        for T in (1, 7, 13):
            ref = oracle.run_int(2, r, pattern, shape, w, bkind, bval, u0, T)
            got = gpu_run(plan, u0, T, variant=1).cpu().numpy()
            np.testing.assert_array_equal(got, ref, err_msg=f"plain {shape} T={T}")
            for k in kvalues(plan):
                got = gpu_run(plan, u0, T, k=k).cpu().numpy()
                np.testing.assert_array_equal(got, ref, err_msg=f"fused k={k} {shape} T={T}")


@pytest.mark.parametrize("d,shape,r", [(1, (1001,), 1), (1, (3,), 2), (1, (257,), 3), (3, (9, 10, 37), 1),
                                       (3, (1, 1, 5), 1), (3, (6, 5, 11), 2)])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_int32_bit_exact_1d_3d(d, shape, r, pattern, bkind):
    sg = sgmod()
    rng = np.random.default_rng(d + r + pattern + bkind)
    w = [float(x) for x in rng.integers(-3, 8, npoints(d, r, pattern))]
    bval = -77 if bkind == DIRICHLET else 0
    u0 = uniform_u16(900 + d, int(np.prod(shape))).reshape(shape)
    plan = sg.stencil_plan_create(d, r, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
    for T in (1, 6):
        ref = oracle.run_int(d, r, pattern, shape, w, bkind, bval, u0, T)
        np.testing.assert_array_equal(gpu_run(plan, u0, T, variant=1).cpu().numpy(), ref)
        for k in kvalues(plan):
            np.testing.assert_array_equal(gpu_run(plan, u0, T, k=k).cpu().numpy(), ref)


# --------------------------------------------------------- floating point
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_f64_f32_2d_against_oracle_and_plain(pattern, r, bkind):
    sg = sgmod()
    rng = np.random.default_rng(40 + r + pattern + bkind)
    for shape in [(67, 300), (130, 17), (2, 3)]:
        w = list(rng.uniform(-0.1, 0.4, npoints(2, r, pattern)))
        bval = 0.3 if bkind == DIRICHLET else 0.0
        u0 = uniform01(1002, shape[0] * shape[1]).reshape(shape)
        T = 13
        # FP64
        p64 = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, sg.STENCIL_F64)
        ref = oracle.run(2, r, pattern, shape, w, bkind, bval, u0, T)
        base = gpu_run(p64, u0, T, variant=1).cpu().numpy()
        assert normwise(base, ref) <= 1e-12
        for k in kvalues(p64):
            np.testing.assert_array_equal(gpu_run(p64, u0, T, k=k).cpu().numpy(), base)
        # FP32
        u32 = u0.astype(np.float32)
        p32 = sg.stencil_plan_create(2, r, shape, pattern, w, bkind, bval, sg.STENCIL_F32)
        ref32 = oracle.run(2, r, pattern, shape, f32_weights(w), bkind, float(np.float32(bval)),
                           u32.astype(np.float64), T)
        base32 = gpu_run(p32, u32, T, variant=1).cpu().numpy()
        assert normwise(base32, ref32) <= 1e-5
        for k in kvalues(p32):
            np.testing.assert_array_equal(gpu_run(p32, u32, T, k=k).cpu().numpy(), base32, err_msg=f"k={k}")


@pytest.mark.parametrize("dt,ur", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)])
@pytest.mark.parametrize("pattern", [STAR, BOX])
def test_half_storage_error_bound(dt, ur, pattern):
    sg = sgmod()
    code = sg.STENCIL_BF16 if dt == "bf16" else sg.STENCIL_F16
    shape, T = (97, 333), 24
    w = star_weights(2, 1, 0.5, 0.125) if pattern == STAR else box_weights(2, 1, 1.0 / 9.0)
    plan = sg.stencil_plan_create(2, 1, shape, pattern, w, DIRICHLET, 0.0, code)
    u0 = uniform01(1002, shape[0] * shape[1]).reshape(shape).astype(np.float32)
    x = torch.from_numpy(u0).to(sg.torch_dtype(code))
    uq = x.float().numpy().astype(np.float64)          # the stored (quantised) input
    ref = oracle.run(2, 1, pattern, shape, f32_weights(w), DIRICHLET, 0.0, uq, T)
    for k in kvalues(plan):
        got = gpu_run(plan, u0, T, k=k)
        passes = -(-T // k)
        err = float(np.max(np.abs(got.float().cpu().numpy().astype(np.float64) - ref)))
        assert err <= (passes * ur + 1e-5) * np.max(np.abs(uq)), (k, err)


# ---------------------------------------------------- full-size workloads
def sample_points(shape, n_random=120, seed=5):
    ny, nx = shape
    rng = np.random.default_rng(seed)
    pts = {(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (ny // 2, 0), (0, nx // 2)}
    for bw in (120, 112, 124, 104, 96):   # band seams of the fused kernel for k = 1..8
        for j in (1, 2, 7, nx // bw - 1):
            for dx in (-1, 0):
                x = j * bw + dx
                if 0 <= x < nx:
                    pts.add((int(rng.integers(0, ny)), x))
    for y in (1, 2, 63, 64, 65, 127, 128, 129, ny - 2):
        pts.add((y, int(rng.integers(0, nx))))
    for _ in range(n_random):
        pts.add((int(rng.integers(0, ny)), int(rng.integers(0, nx))))
    return np.array(sorted(pts), dtype=np.int64)


@pytest.mark.parametrize("maker", [c2_2d5p, c2_2d9p])
def test_full_size_2d_fp32_sampled(maker):
    """8192^2, T=64, FP32, at the plan's default k (the launch configuration
    the benchmark times): sampled outputs against the oracle's dependency
    cones, and the whole grid bit-identical to the plain one-step sweep."""
    sg = sgmod()
    p = maker()
    u0 = uniform01(p.seed, p.npts).reshape(p.shape).astype(np.float32)
    plan = sg.stencil_plan_create(2, 1, p.shape, p.pattern, p.weights, p.bkind, p.bval, sg.STENCIL_F32)
    fused = gpu_run(plan, u0, p.T)
    plain = gpu_run(plan, u0, p.T, variant=1)
    assert torch.equal(fused, plain)
    pts = sample_points(p.shape)
    ref = oracle.points(2, 1, p.pattern, p.shape, f32_weights(p.weights), p.bkind, p.bval,
                        u0.astype(np.float64), p.T, pts)
    got = fused.cpu().numpy()[pts[:, 0], pts[:, 1]].astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(u0))


def test_full_size_eigenmode_fp32():
    """A Dirichlet sine mode on the 8192^2 grid decays by lam^T exactly."""
    sg = sgmod()
    p = c2_2d5p()
    ny, nx = p.shape
    ky, kx = 3, 5
    phi = np.multiply.outer(sine_mode_1d(ny, ky), sine_mode_1d(nx, kx))
    w = f32_weights(p.weights)
    lam = w[0] + (w[1] + w[2]) * np.cos(np.pi * ky / (ny + 1)) + (w[3] + w[4]) * np.cos(np.pi * kx / (nx + 1))
    plan = sg.stencil_plan_create(2, 1, p.shape, STAR, p.weights, DIRICHLET, 0.0, sg.STENCIL_F32)
    got = gpu_run(plan, phi.astype(np.float32), p.T).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - lam ** p.T * phi)) <= 2e-5


# ------------------------------------------------------------- API edges
def test_run_host_matches_device_run():
    sg = sgmod()
    shape, T = (77, 131), 9
    w = box_weights(2, 1, 1 / 9)
    plan = sg.stencil_plan_create(2, 1, shape, BOX, w, PERIODIC, 0.0, sg.STENCIL_F32)
    u0 = uniform01(3, shape[0] * shape[1]).reshape(shape).astype(np.float32)
    dev = gpu_run(plan, u0, T).cpu().numpy()
    h_in = torch.from_numpy(u0).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    sg.stencil_run_host(plan, h_in, h_out, T)
    np.testing.assert_array_equal(h_out.numpy(), dev)


def test_zero_steps_and_ragged_pass_counts():
    sg = sgmod()
    shape = (40, 64)
    w = star_weights(2, 1, 0.5, 0.125)
    plan = sg.stencil_plan_create(2, 1, shape, STAR, w, DIRICHLET, 0.0, sg.STENCIL_F32)
    u0 = uniform01(4, shape[0] * shape[1]).reshape(shape).astype(np.float32)
    np.testing.assert_array_equal(gpu_run(plan, u0, 0).cpu().numpy(), u0)
    base = gpu_run(plan, u0, 11, variant=1).cpu().numpy()
    for k in kvalues(plan):
        np.testing.assert_array_equal(gpu_run(plan, u0, 11, k=k).cpu().numpy(), base)
        # 2D: the passes of exactly k steps share one persistent launch
        full = 11 // k
        assert sg.stencil_plan_launch_count(plan, 11) == (1 + (11 % k > 0) if full >= 2 else -(-11 // k))
        np.testing.assert_array_equal(gpu_run(plan, u0, 11, k=k, variant=sg.STENCIL_VARIANT_FUSED_PER_PASS)
                                      .cpu().numpy(), base)
        assert sg.stencil_plan_launch_count(plan, 11) == -(-11 // k)


def test_errors_are_reported():
    sg = sgmod()
    plan = sg.stencil_plan_create(2, 1, (16, 16), STAR, [1, 0, 0, 0, 0], DIRICHLET, 0.0, sg.STENCIL_F32)
    x = torch.zeros((16, 16), device=DEV)
    with pytest.raises(sg.StencilError) as e:
        sg.stencil_run(plan, x, x, 3)
    assert e.value.status == sg.STENCIL_ERR_INVALID_ARG
    with pytest.raises(sg.StencilError) as e:
        sg.stencil_plan_set_k(plan, 99)
    assert e.value.status == sg.STENCIL_ERR_UNSUPPORTED


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_reductions_against_oracle(dtype):
    sg = sgmod()
    n = 1_000_003
    u = torch.from_numpy(uniform01(8, n) - 0.5).to(dtype).to(DEV)
    t = torch.from_numpy(uniform01(9, n)).to(dtype).to(DEV)
    uh = u.double().cpu().numpy()
    th = t.double().cpu().numpy()
    bound = n * 2.0 ** -52
    got = sg.stencil_reduce(u, sg.STENCIL_REDUCE_SUM).item()
    assert abs(got - oracle.total(uh)) <= bound * np.sum(np.abs(uh))
    got = sg.stencil_reduce(u, sg.STENCIL_REDUCE_SUMSQ).item()
    assert abs(got - oracle.sumsq(uh)) <= bound * np.sum(uh * uh)
    got = sg.stencil_reduce(u, sg.STENCIL_REDUCE_HALF_SQDIST, target=t).item()
    exp = 0.5 * oracle.sumsq(uh - th)
    assert abs(got - exp) <= bound * exp
    again = sg.stencil_reduce(u, sg.STENCIL_REDUCE_HALF_SQDIST, target=t).item()
    assert again == got      # fixed order: deterministic


# ------------------------------------------------------------------- 3D
SHAPES_3D = [(37, 53, 260), (9, 10, 36), (20, 70, 131)]


@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_3d_int32_and_fp32_every_k(pattern, bkind):
    """3D fused kernel (TMA and cp.async paths, several tiles in x, y and z):
    int32 bit-exact against the oracle, FP32 bit-identical to the plain
    sweep and within 1e-5 of the FP64 oracle."""
    sg = sgmod()
    rng = np.random.default_rng(77 + pattern + 2 * bkind)
    for shape in SHAPES_3D:
        n = int(np.prod(shape))
        w = [float(x) for x in rng.integers(-2, 5, npoints(3, 1, pattern))]
        bval = 31 if bkind == DIRICHLET else 0
        u0 = uniform_u16(1300, n).reshape(shape)
        plan = sg.stencil_plan_create(3, 1, shape, pattern, w, bkind, bval, sg.STENCIL_I32)
        T = 9
        ref = oracle.run_int(3, 1, pattern, shape, w, bkind, bval, u0, T)
        for k in kvalues(plan):
            np.testing.assert_array_equal(gpu_run(plan, u0, T, k=k).cpu().numpy(), ref, err_msg=f"{shape} k={k}")
        wf = list(rng.uniform(0.0, 1.0, npoints(3, 1, pattern)))
        wf = [x / sum(wf) for x in wf]
        uf = uniform01(1301, n).reshape(shape).astype(np.float32)
        pf = sg.stencil_plan_create(3, 1, shape, pattern, wf, bkind, 0.2 if bkind == DIRICHLET else 0.0,
                                    sg.STENCIL_F32)
        reff = oracle.run(3, 1, pattern, shape, f32_weights(wf), bkind, float(np.float32(0.2)) if bkind == DIRICHLET
                          else 0.0, uf.astype(np.float64), T)
        base = gpu_run(pf, uf, T, variant=1).cpu().numpy()
        assert normwise(base, reff) <= 1e-5
        for k in kvalues(pf):
            np.testing.assert_array_equal(gpu_run(pf, uf, T, k=k).cpu().numpy(), base, err_msg=f"{shape} k={k}")


@pytest.mark.parametrize("r,pattern", [(2, STAR), (2, BOX)])
def test_3d_radius2(r, pattern):
    sg = sgmod()
    shape, T = (15, 22, 68), 5
    rng = np.random.default_rng(5)
    w = [float(x) for x in rng.integers(-2, 5, npoints(3, r, pattern))]
    u0 = uniform_u16(1400, int(np.prod(shape))).reshape(shape)
    for bkind in (DIRICHLET, PERIODIC):
        plan = sg.stencil_plan_create(3, r, shape, pattern, w, bkind, 4 if bkind == DIRICHLET else 0, sg.STENCIL_I32)
        ref = oracle.run_int(3, r, pattern, shape, w, bkind, 4 if bkind == DIRICHLET else 0, u0, T)
        for k in kvalues(plan):
            np.testing.assert_array_equal(gpu_run(plan, u0, T, k=k).cpu().numpy(), ref)


@pytest.mark.parametrize("dt,ur", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11), ("f64", 0.0)])
def test_3d_other_dtypes(dt, ur):
    sg = sgmod()
    code = {"bf16": sg.STENCIL_BF16, "f16": sg.STENCIL_F16, "f64": sg.STENCIL_F64}[dt]
    shape, T = (33, 40, 136), 12
    w = star_weights(3, 1, 0.4, 0.1)
    plan = sg.stencil_plan_create(3, 1, shape, STAR, w, DIRICHLET, 0.0, code)
    u0 = uniform01(1500, int(np.prod(shape))).reshape(shape)
    if dt == "f64":
        ref = oracle.run(3, 1, STAR, shape, w, DIRICHLET, 0.0, u0, T)
        base = gpu_run(plan, u0, T, variant=1).cpu().numpy()
        assert normwise(base, ref) <= 1e-12
        for k in kvalues(plan):
            np.testing.assert_array_equal(gpu_run(plan, u0, T, k=k).cpu().numpy(), base)
        return
    u32 = u0.astype(np.float32)
    uq = torch.from_numpy(u32).to(sg.torch_dtype(code)).float().numpy().astype(np.float64)
    ref = oracle.run(3, 1, STAR, shape, f32_weights(w), DIRICHLET, 0.0, uq, T)
    for k in kvalues(plan):
        got = gpu_run(plan, u32, T, k=k).float().cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) <= (-(-T // k) * ur + 1e-5) * np.max(np.abs(uq)), k


def sample_points_3d(shape, n_random=40, seed=7):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    pts = {(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, 0), (nz // 2, 0, nx - 1)}
    # seams of the fused 3D tiles: 64-wide windows with a 4-column halo in x
    # (first tile 60 columns, then 56), 64-row windows with a k-row halo in y
    # (first tile 64 - k rows, then 64 - 2k), for k = 1..4
    for x in (59, 60, 115, 116, 171, 172, nx - 61, nx - 60):
        pts.add((int(rng.integers(0, nz)), int(rng.integers(0, ny)), x))
    for k in range(1, 5):
        f, b = 64 - k, 64 - 2 * k
        for y in (f - 1, f, f + b - 1, f + b, ny - f - 1, ny - f):
            pts.add((int(rng.integers(0, nz)), y, int(rng.integers(0, nx))))
    for _ in range(n_random):
        pts.add(tuple(int(rng.integers(0, s)) for s in shape))
    return np.array(sorted(pts), dtype=np.int64)


@pytest.mark.parametrize("maker", ["c3_3d7p", "c3_3d27p"])
def test_full_size_3d_sampled(maker):
    """512^3, T=32, FP32 and BF16 storage at the plan's default k: sampled
    outputs against the oracle's dependency cones; FP32 bit-identical to the
    plain sweep over the whole grid."""
    import synth
    sg = sgmod()
    p = getattr(synth, maker)()
    u0 = synth.u0_modes_plus_noise(p, np.float32)
    plan = sg.stencil_plan_create(3, 1, p.shape, p.pattern, p.weights, p.bkind, p.bval, sg.STENCIL_F32)
    fused = gpu_run(plan, u0, p.T)
    plain = gpu_run(plan, u0, p.T, variant=1)
    assert torch.equal(fused, plain)
    del plain
    pts = sample_points_3d(p.shape)
    ref = oracle.points(3, 1, p.pattern, p.shape, f32_weights(p.weights), p.bkind, p.bval,
                        u0.astype(np.float64), p.T, pts)
    got = fused.cpu().numpy()[pts[:, 0], pts[:, 1], pts[:, 2]].astype(np.float64)
    scale = np.max(np.abs(u0))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    del fused
    pb = sg.stencil_plan_create(3, 1, p.shape, p.pattern, p.weights, p.bkind, p.bval, sg.STENCIL_BF16)
    k = sg.stencil_plan_get_k(pb)
    xb = torch.from_numpy(u0).to(torch.bfloat16)
    uq = xb.float().numpy().astype(np.float64)
    refq = oracle.points(3, 1, p.pattern, p.shape, f32_weights(p.weights), p.bkind, p.bval, uq, p.T, pts)
    gotb = gpu_run(pb, u0, p.T)
    gb = gotb.float().cpu().numpy()[pts[:, 0], pts[:, 1], pts[:, 2]].astype(np.float64)
    assert np.max(np.abs(gb - refq)) <= (-(-p.T // k) * 2.0 ** -8 + 1e-5) * np.max(np.abs(uq))


# ------------------------------------------------------------------- 1D
def test_1d3p_full_config_f64_and_int():
    """The 1D workload at full size: 65536 points, T=100, FP64 (normwise
    1e-12 against the oracle, every k bit-identical to the plain sweep) and
    the int32 mode with weights 1/2/1 (bit-exact)."""
    import synth
    sg = sgmod()
    p = synth.c1_1d3p()
    u0 = synth.u0_uniform(p)
    plan = sg.stencil_plan_create(1, 1, p.shape, STAR, p.weights, DIRICHLET, 0.0, sg.STENCIL_F64)
    ref = oracle.run(1, 1, STAR, p.shape, p.weights, DIRICHLET, 0.0, u0, p.T)
    base = gpu_run(plan, u0, p.T, variant=1).cpu().numpy()
    assert normwise(base, ref) <= 1e-12
    for k in kvalues(plan):
        np.testing.assert_array_equal(gpu_run(plan, u0, p.T, k=k).cpu().numpy(), base, err_msg=f"k={k}")
    pi = synth.c1_1d3p_int()
    ui = synth.u0_int(pi)
    plan_i = sg.stencil_plan_create(1, 1, pi.shape, STAR, pi.weights, DIRICHLET, 0.0, sg.STENCIL_I32)
    refi = oracle.run_int(1, 1, STAR, pi.shape, pi.weights, DIRICHLET, 0, ui, pi.T)
    for k in kvalues(plan_i):
        np.testing.assert_array_equal(gpu_run(plan_i, ui, pi.T, k=k).cpu().numpy(), refi, err_msg=f"k={k}")


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("n", [1, 5, 127, 128, 129, 4097, 100003])
def test_1d_ragged_every_k(r, bkind, n):
    sg = sgmod()
    rng = np.random.default_rng(n + r + bkind)
    w = [float(x) for x in rng.integers(-3, 6, 2 * r + 1)]
    bval = 9 if bkind == DIRICHLET else 0
    u0 = uniform_u16(1600 + n, n)
    plan = sg.stencil_plan_create(1, r, (n,), STAR, w, bkind, bval, sg.STENCIL_I32)
    T = 19
    ref = oracle.run_int(1, r, STAR, (n,), w, bkind, bval, u0, T)
    for k in kvalues(plan):
        np.testing.assert_array_equal(gpu_run(plan, u0, T, k=k).cpu().numpy(), ref, err_msg=f"k={k}")
    wf = [0.2, 0.5, 0.3] if r == 1 else [0.1, 0.2, 0.3, 0.25, 0.15]
    uf = uniform01(1700 + n, n).astype(np.float32)
    pf = sg.stencil_plan_create(1, r, (n,), STAR, wf, bkind, 0.25 if bkind == DIRICHLET else 0.0, sg.STENCIL_F32)
    base = gpu_run(pf, uf, T, variant=1).cpu().numpy()
    reff = oracle.run(1, r, STAR, (n,), f32_weights(wf), bkind, 0.25 if bkind == DIRICHLET else 0.0,
                      uf.astype(np.float64), T)
    assert normwise(base, reff) <= 1e-5
    for k in kvalues(pf):
        np.testing.assert_array_equal(gpu_run(pf, uf, T, k=k).cpu().numpy(), base, err_msg=f"k={k}")

"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each check is computed independently of the oracle's code: a dense matrix
written from the definition (Section 1: each point is a weighted sum of its
neighbours at the previous time step), closed forms (sine and Fourier
eigenmodes, binomial coefficients and their images), separability, T-fold
self-correlation, conservation laws and the adjoint identity.  A dropped
term, a wrong sign or index, a transposed operand or a wrong boundary rule in
the oracle fails at least one of them.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from synth import (BOX, DIRICHLET, PERIODIC, STAR, box_weights, c4_batch, sine_mode_1d,
                   star_weights, uniform01, uniform_u16)


# ----------------------------------------------------------------- helpers
def ref_offsets(d, r, pattern):
    """Offsets in compact weight order, written from the convention."""
    if pattern == BOX:
        return [tuple(o) for o in itertools.product(range(-r, r + 1), repeat=d)]
    out = [tuple([0] * d)]
    for a in range(d):
        for m in list(range(-r, 0)) + list(range(1, r + 1)):
            o = [0] * d
            o[a] = m
            out.append(tuple(o))
    return out


def dense_model(d, r, pattern, shape, w, bkind, bval):
    """(M, c) with u_{t+1} = M u_t + c, built point by point from the definition."""
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    c = np.zeros(N)
    offs = ref_offsets(d, r, pattern)
    for lin, x in enumerate(itertools.product(*[range(s) for s in shape])):
        for j, o in enumerate(offs):
            y = [x[a] + o[a] for a in range(d)]
            if any(y[a] < 0 or y[a] >= shape[a] for a in range(d)):
                if bkind == DIRICHLET:
                    c[lin] += w[j] * bval
                    continue
                y = [y[a] % shape[a] for a in range(d)]
            M[lin, int(np.ravel_multi_index(y, shape))] += w[j]
    return M, c


def dense_model_int(d, r, pattern, shape, w, bkind, bval):
    N = int(np.prod(shape))
    M = np.zeros((N, N), dtype=object)
    c = np.zeros(N, dtype=object)
    offs = ref_offsets(d, r, pattern)
    for lin, x in enumerate(itertools.product(*[range(s) for s in shape])):
        for j, o in enumerate(offs):
            y = [x[a] + o[a] for a in range(d)]
            if any(y[a] < 0 or y[a] >= shape[a] for a in range(d)):
                if bkind == DIRICHLET:
                    c[lin] += int(w[j]) * int(bval)
                    continue
                y = [y[a] % shape[a] for a in range(d)]
            M[lin, int(np.ravel_multi_index(y, shape))] += int(w[j])
    return M, c


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, float(np.max(np.abs(b)))))


SMALL_SHAPES = {1: [(9,), (2,)], 2: [(5, 7), (3, 2)], 3: [(4, 3, 5), (2, 3, 2)]}


# ------------------------------------------------------- compact ordering
def test_offsets_match_convention():
    for d in (1, 2, 3):
        for r in (1, 2, 3):
            for pat in (STAR, BOX):
                got = [tuple(o) for o in oracle.offsets(d, r, pat)]
                assert got == ref_offsets(d, r, pat), (d, r, pat)
    # spelled out once for the 2D 5-point star and 3x3 box
    assert [tuple(o) for o in oracle.offsets(2, 1, STAR)] == [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    assert [tuple(o) for o in oracle.offsets(2, 1, BOX)][:4] == [(-1, -1), (-1, 0), (-1, 1), (0, -1)]


# ------------------------------------------- dense brute force (P-h)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_dense_bruteforce_f64(d, r, pattern, bkind):
    if d == 3 and r == 3 and pattern == BOX:
        shapes = [(2, 3, 2)]
    else:
        shapes = SMALL_SHAPES[d]
    rng = np.random.default_rng(100 * d + 10 * r + 2 * pattern + bkind)
    for shape in shapes:
        npnt = len(ref_offsets(d, r, pattern))
        w = rng.uniform(-0.3, 0.6, npnt)        # asymmetric on purpose
        bval = 0.7 if bkind == DIRICHLET else 0.0
        u0 = rng.uniform(-1, 1, shape)
        T = 3
        M, c = dense_model(d, r, pattern, shape, w, bkind, bval)
        u = u0.ravel().copy()
        for _ in range(T):
            u = M @ u + c
        got = oracle.run(d, r, pattern, shape, w, bkind, bval, u0, T)
        assert relerr(got.ravel(), u) < 1e-13, (shape, relerr(got.ravel(), u))


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_dense_bruteforce_int(d, pattern, bkind):
    r = 1 if d == 3 else 2
    rng = np.random.default_rng(7 + d + pattern + bkind)
    for shape in SMALL_SHAPES[d]:
        npnt = len(ref_offsets(d, r, pattern))
        w = rng.integers(-3, 8, npnt)
        bval = 12345 if bkind == DIRICHLET else 0
        u0 = rng.integers(0, 65536, shape)
        T = 9   # enough steps for the uint32 wraparound to matter
        M, c = dense_model_int(d, r, pattern, shape, w, bkind, bval)
        u = np.array([int(v) for v in u0.ravel()], dtype=object)
        for _ in range(T):
            u = np.array([(int(v)) % (1 << 32) for v in (M.dot(u) + c)], dtype=object)
        got = oracle.run_int(d, r, pattern, shape, w.astype(float), bkind, bval, u0, T)
        exp = np.array([int(v) for v in u], dtype=np.uint64).astype(np.uint32).view(np.int32)
        np.testing.assert_array_equal(got.ravel(), exp)


# ------------------------------------- Dirichlet sine eigenmodes (P-a)
EIG_CASES = [
    (1, STAR, [0.5, 0.25, 0.25], (300,), 100),
    (2, STAR, star_weights(2, 1, 0.5, 0.125), (40, 56), 30),
    (2, BOX, box_weights(2, 1, 1.0 / 9.0), (33, 20), 30),
    (3, STAR, star_weights(3, 1, 0.4, 0.1), (12, 10, 14), 12),
    (3, BOX, box_weights(3, 1, 1.0 / 27.0), (9, 11, 8), 12),
]


@pytest.mark.parametrize("d,pattern,w,shape,T", EIG_CASES)
def test_dirichlet_sine_eigenmode(d, pattern, w, shape, T):
    """phi_k(i) = prod_a sin(pi k_a (i_a+1)/(n_a+1)) is an eigenvector of the
    Dirichlet-0 operator for axis-symmetric r=1 weights, with eigenvalue
    sum_o w_o prod_a cos(pi k_a o_a / (n_a+1))."""
    rng = np.random.default_rng(d * 7 + pattern)
    for _ in range(3):
        ks = [int(rng.integers(1, max(1, s // 6) + 1)) for s in shape]   # |lam| stays near 1
        vecs = [sine_mode_1d(shape[a], ks[a]) for a in range(d)]
        phi = vecs[0]
        for v in vecs[1:]:
            phi = np.multiply.outer(phi, v)
        lam = 0.0
        for j, o in enumerate(ref_offsets(d, 1, pattern)):
            term = w[j]
            for a in range(d):
                term *= math.cos(math.pi * ks[a] * o[a] / (shape[a] + 1))
            lam += term
        got = oracle.run(d, 1, pattern, shape, w, DIRICHLET, 0.0, phi, T)
        exp = (lam ** T) * phi
        err = np.max(np.abs(got - exp))
        assert err < 1e-14 * T                       # rounding only (max|u0| = 1)
        assert err / abs(lam) ** T < 1e-9            # against the surviving signal


# -------------------------------------- periodic Fourier modes (P-b)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("pattern", [STAR, BOX])
def test_periodic_fourier_mode(d, r, pattern):
    """On a periodic grid cos(theta.x) maps to Re(lam^T e^{i theta.x}) with
    lam = sum_o w_o e^{i theta.o}, for any (asymmetric) weights."""
    shape = {1: (37,), 2: (12, 9), 3: (6, 7, 5)}[d]
    rng = np.random.default_rng(31 * d + r + pattern)
    w = rng.uniform(-0.2, 0.5, len(ref_offsets(d, r, pattern)))
    w = w / np.sum(np.abs(w))
    ks = [int(rng.integers(0, s)) for s in shape]
    theta = [2 * math.pi * ks[a] / shape[a] for a in range(d)]
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    phase = sum(theta[a] * grids[a] for a in range(d))
    lam = sum(w[j] * np.exp(1j * sum(theta[a] * o[a] for a in range(d)))
              for j, o in enumerate(ref_offsets(d, r, pattern)))
    T = 7
    got = oracle.run(d, r, pattern, shape, w, PERIODIC, 0.0, np.cos(phase), T)
    exp = np.real(lam ** T * np.exp(1j * phase))
    assert np.max(np.abs(got - exp)) < 1e-13


# -------------------------------------------- binomial closed form (P-c)
def test_binomial_periodic_exact():
    """1D3P (1/4, 1/2, 1/4) from a delta: u_T[j+m] = C(2T, T+m) / 4^T.  All
    values are dyadic with < 53 significant bits, so FP64 is exact."""
    T = 20
    n = 2 * T + 5
    u0 = np.zeros(n)
    u0[3] = 1.0
    got = oracle.run(1, 1, STAR, (n,), [0.5, 0.25, 0.25], PERIODIC, 0.0, u0, T)
    exp = np.zeros(n)
    for m in range(-T, T + 1):
        exp[(3 + m) % n] = math.comb(2 * T, T + m) / 4.0 ** T
    np.testing.assert_array_equal(got, exp)


def test_binomial_int_wraps():
    """Integer weights (1, 2, 1): u_T[j+m] = C(2T, T+m) mod 2^32, bit-exact."""
    T = 40
    n = 2 * T + 3
    u0 = np.zeros(n, dtype=np.int64)
    u0[0] = 1
    got = oracle.run_int(1, 1, STAR, (n,), [2, 1, 1], PERIODIC, 0, u0, T)
    exp = np.zeros(n, dtype=np.uint64)
    for m in range(-T, T + 1):
        exp[m % n] = math.comb(2 * T, T + m) % (1 << 32)
    np.testing.assert_array_equal(got, exp.astype(np.uint32).view(np.int32))


def test_binomial_dirichlet_images_exact():
    """Dirichlet-0 on n points is the odd periodic extension of period 2(n+1):
    u_T[x] = sum_p K(x - y + 2p(n+1)) - K(x + y + 2 + 2p(n+1)), K(m) = C(2T,T+m)/4^T."""
    n, T, y = 7, 12, 2
    u0 = np.zeros(n)
    u0[y] = 1.0

    def K(m):
        return math.comb(2 * T, T + m) / 4.0 ** T if abs(m) <= T else 0.0

    exp = np.zeros(n)
    for x in range(n):
        s = 0.0
        for p in range(-4, 5):
            s += K(x - y + 2 * p * (n + 1)) - K(x + y + 2 + 2 * p * (n + 1))
        exp[x] = s
    got = oracle.run(1, 1, STAR, (n,), [0.5, 0.25, 0.25], DIRICHLET, 0.0, u0, T)
    assert np.max(np.abs(got - exp)) < 1e-15


# ------------------------------------------------- separability (P-d)
def test_box_separability_2d_3d():
    """Box 1/9 (1/27) = tensor product of (1/3, 1/3, 1/3): with Dirichlet 0 the
    operator is A (x) A (x) A, A = tridiag(1/3), applied by matrix powers."""
    def tri(n):
        return (np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)) / 3.0
    rng = np.random.default_rng(5)
    T = 9
    u0 = rng.uniform(0, 1, (11, 13))
    Ay, Ax = np.linalg.matrix_power(tri(11), T), np.linalg.matrix_power(tri(13), T)
    exp = Ay @ u0 @ Ax.T
    got = oracle.run(2, 1, BOX, (11, 13), box_weights(2, 1, 1 / 9), DIRICHLET, 0.0, u0, T)
    assert relerr(got, exp) < 1e-13
    u3 = rng.uniform(0, 1, (6, 7, 5))
    A0, A1, A2 = (np.linalg.matrix_power(tri(s), T) for s in (6, 7, 5))
    exp3 = np.einsum("ia,jb,kc,abc->ijk", A0, A1, A2, u3)
    got3 = oracle.run(3, 1, BOX, (6, 7, 5), box_weights(3, 1, 1 / 27), DIRICHLET, 0.0, u3, T)
    assert relerr(got3, exp3) < 1e-13


# ----------------------------------------------- self-correlation (P-e)
@pytest.mark.parametrize("r,pattern", [(1, BOX), (2, STAR)])
def test_tfold_self_correlation(r, pattern):
    """T steps on a periodic grid = one correlation with the T-fold composed
    kernel K_T, K_{t+1}[o] = sum_{a+b=o} K_t[a] w[b]."""
    d, shape, T = 2, (13, 11), 5
    rng = np.random.default_rng(11 + r)
    offs = ref_offsets(d, r, pattern)
    w = rng.uniform(-0.3, 0.7, len(offs))
    K = {(0, 0): 1.0}
    for _ in range(T):
        nk = {}
        for a, ka in K.items():
            for j, b in enumerate(offs):
                o = (a[0] + b[0], a[1] + b[1])
                nk[o] = nk.get(o, 0.0) + ka * w[j]
        K = nk
    u0 = rng.uniform(-1, 1, shape)
    exp = np.zeros(shape)
    for o, k in K.items():
        exp += k * np.roll(u0, shift=(-o[0], -o[1]), axis=(0, 1))
    got = oracle.run(d, r, pattern, shape, w, PERIODIC, 0.0, u0, T)
    assert relerr(got, exp) < 1e-12


# ------------------------------------------- conservation laws (P-f)
def test_mass_conserved_periodic_normalised():
    """Periodic and sum w = 1: sum_x u_t is invariant (the batched workload)."""
    p = c4_batch(count=3, lo=16, hi=40)[1]
    u0 = uniform01(p.seed, int(np.prod(p.shape))).reshape(p.shape)
    got = oracle.run(2, 1, BOX, p.shape, p.weights, PERIODIC, 0.0, u0, p.T)
    assert abs(math.fsum(got.ravel()) - math.fsum(u0.ravel())) < 1e-11 * math.fsum(u0.ravel())


def test_mass_scales_int_mode():
    """Integer (1,2,1) periodic: sum u_T = 4^T sum u_0 mod 2^32, exactly."""
    n, T = 101, 23
    u0 = uniform_u16(77, n)
    got = oracle.run_int(1, 1, STAR, (n,), [2, 1, 1], PERIODIC, 0, u0, T)
    s = int(np.sum(got.view(np.uint32).astype(np.uint64))) % (1 << 32)
    assert s == (4 ** T * int(np.sum(u0.astype(np.int64)))) % (1 << 32)


# ------------------------------- single points from dependency cones
@pytest.mark.parametrize("d,shape", [(1, (23,)), (2, (9, 14)), (3, (5, 7, 6))])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_cone_points_equal_full_run(d, shape, r, pattern, bkind):
    """u_T at chosen points from their cones is the full run's value, bit for
    bit (same operands, same order); cones wider than the grid included."""
    rng = np.random.default_rng(3 * d + r + 5 * pattern + bkind)
    w = rng.uniform(-0.4, 0.6, len(ref_offsets(d, r, pattern)))
    bval = -0.35 if bkind == DIRICHLET else 0.0
    u0 = rng.uniform(-1, 1, shape)
    T = 6
    full = oracle.run(d, r, pattern, shape, w, bkind, bval, u0, T)
    pts = np.array(list(itertools.product(*[range(s) for s in shape])))
    got = oracle.points(d, r, pattern, shape, w, bkind, bval, u0, T, pts)
    np.testing.assert_array_equal(got, full.reshape(-1))
    wi = rng.integers(-2, 5, len(w)).astype(float)
    ui = rng.integers(0, 65536, shape)
    fi = oracle.run_int(d, r, pattern, shape, wi, bkind, 99 if bkind == DIRICHLET else 0, ui, 11)
    gi = oracle.points_int(d, r, pattern, shape, wi, bkind, 99 if bkind == DIRICHLET else 0, ui, 11, pts)
    np.testing.assert_array_equal(gi, fi.reshape(-1))


# ---------------------------------------------------- adjoint (P-g)
@pytest.mark.parametrize("d,shape", [(1, (17,)), (2, (6, 5)), (3, (4, 3, 5))])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_transpose_dot_product(d, shape, pattern, bkind):
    """<A^T y, x> = <y, A x> for the linear part A of one step (bval = 0)."""
    rng = np.random.default_rng(d + 2 * pattern + 4 * bkind)
    r = 1
    w = rng.uniform(-0.5, 1.0, len(ref_offsets(d, r, pattern)))
    x = rng.uniform(-1, 1, shape)
    y = rng.uniform(-1, 1, shape)
    Ax = oracle.run(d, r, pattern, shape, w, bkind, 0.0, x, 1)
    ATy = oracle.transpose_step(d, r, pattern, shape, w, bkind, y)
    assert abs(np.sum(ATy * x) - np.sum(y * Ax)) < 1e-13 * np.sum(np.abs(y) * np.abs(Ax) + 1)
    M, _ = dense_model(d, r, pattern, shape, w, bkind, 0.0)
    assert relerr(ATy.ravel(), M.T @ y.ravel()) < 1e-13


@pytest.mark.parametrize("bkind,bval", [(DIRICHLET, 0.3), (PERIODIC, 0.0)])
def test_adjoint_against_dense_and_fd(bkind, bval):
    """Gradients of 0.5||u_T - target||^2: w.r.t. u0 against the dense model's
    transpose, w.r.t. the weights against central differences of the dense
    model's loss (h = 1e-6)."""
    d, r, pattern, shape, T = 2, 1, STAR, (5, 6), 6
    rng = np.random.default_rng(42 + bkind)
    w = rng.uniform(-0.2, 0.6, 5)
    u0 = rng.uniform(0, 1, shape)
    tg = rng.uniform(0, 1, shape)

    def dense_loss(wv):
        M, c = dense_model(d, r, pattern, shape, wv, bkind, bval)
        u = u0.ravel().copy()
        for _ in range(T):
            u = M @ u + c
        return 0.5 * np.sum((u - tg.ravel()) ** 2), M, u

    L, M, uT = dense_loss(w)
    loss, gu, gw = oracle.adjoint(d, r, pattern, shape, w, bkind, bval, u0, tg, T)
    assert abs(loss - L) < 1e-12 * max(1, L)
    P = np.linalg.matrix_power(M, T)
    assert relerr(gu.ravel(), P.T @ (uT - tg.ravel())) < 1e-12
    h = 1e-6
    fd = np.zeros_like(w)
    for j in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[j] += h
        wm[j] -= h
        fd[j] = (dense_loss(wp)[0] - dense_loss(wm)[0]) / (2 * h)
    assert relerr(gw, fd) < 1e-6


# ------------------------------------------------------------ reductions
def test_reductions():
    rng = np.random.default_rng(9)
    u = rng.uniform(-1, 1, 10007)
    # sequential summation error bound: n * eps * sum |terms|
    bound = u.size * 2.0 ** -53
    assert abs(oracle.total(u) - math.fsum(u)) <= bound * math.fsum(np.abs(u))
    assert abs(oracle.sumsq(u) - math.fsum(u * u)) <= bound * math.fsum(u * u)
    assert oracle.total(u[:1]) == u[0]

"""Pins of the variable-coefficient oracle (u_{t+1}[x] = sum_o c_o[x] u_t(x+o),
the per-point-coefficient form of the paper's Section 1 sweep) against facts
that do not come from its own code:

* dense brute force: a matrix built point by point from the definition,
  raised to the power T (FP64 and exact integers mod 2^32);
* a constant coefficient field reduces to the constant-weight oracle, which
  is pinned on its own (tests/test_oracle_pins.py);
* rows summing to one keep a constant field constant (periodic and Dirichlet
  with the same boundary value);
* a coefficient field that is a per-point scale s[x] times constant weights
  gives u_{t+1} = s * (A u_t) with A the constant-weight step;
* the adjoint against the dense model's exact gradient and central finite
  differences (the loss is quadratic in u0 and a polynomial in c).
A transposed index (c_o[x] read as c_o[x + o]), a dropped term or a wrong
boundary rule fails at least one of them.
"""

import itertools

import numpy as np
import pytest

import oracle
from synth import BOX, DIRICHLET, PERIODIC, STAR, npoints, uniform01, uniform_u16

from test_oracle_pins import SMALL_SHAPES, ref_offsets, relerr


def dense_vc(d, r, pattern, shape, c, bkind, bval, dtype=float):
    """(M, b) with u_{t+1} = M u_t + b for the coefficient field c, built from
    the definition: row x has c_o[x] in the column of x + o."""
    N = int(np.prod(shape))
    M = np.zeros((N, N), dtype=dtype)
    b = np.zeros(N, dtype=dtype)
    offs = ref_offsets(d, r, pattern)
    cf = np.asarray(c).reshape(len(offs), N)
    for lin, x in enumerate(itertools.product(*[range(s) for s in shape])):
        for j, o in enumerate(offs):
            coef = cf[j, lin] if dtype is float else int(cf[j, lin])
            y = [x[a] + o[a] for a in range(d)]
            if any(y[a] < 0 or y[a] >= shape[a] for a in range(d)):
                if bkind == DIRICHLET:
                    b[lin] += coef * (bval if dtype is float else int(bval))
                    continue
                y = [y[a] % shape[a] for a in range(d)]
            M[lin, int(np.ravel_multi_index(y, shape))] += coef
    return M, b


def coef_field(d, r, pattern, shape, seed, lo=-0.3, hi=0.6):
    N = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, npoints(d, r, pattern) * N)).reshape((-1,) + tuple(shape))


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_vc_dense_bruteforce_f64(d, r, pattern, bkind):
    if d == 3 and r == 2 and pattern == BOX:
        pytest.skip("125-point box on a 3D toy grid adds nothing to the r = 1 and 2D cases")
    for shape in SMALL_SHAPES[d]:
        c = coef_field(d, r, pattern, shape, 11 + d + r)
        u0 = uniform01(3, int(np.prod(shape))).reshape(shape)
        M, b = dense_vc(d, r, pattern, shape, c, bkind, 0.7)
        T = 5
        u = u0.ravel()
        for _ in range(T):
            u = M @ u + b
        got = oracle.run_vc(d, r, pattern, shape, c, bkind, 0.7, u0, T)
        assert relerr(got.ravel(), u) <= 1e-13


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pattern", [STAR, BOX])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_vc_dense_bruteforce_int(d, pattern, bkind):
    for shape in SMALL_SHAPES[d]:
        N = int(np.prod(shape))
        np_ = npoints(d, 1, pattern)
        c = (uniform_u16(21 + d, np_ * N) % 9 - 3).reshape((-1,) + tuple(shape))
        u0 = uniform_u16(22, N).reshape(shape)
        M, b = dense_vc(d, 1, pattern, shape, c, bkind, 5, dtype=object)
        T = 6
        u = [int(v) for v in u0.ravel()]
        for _ in range(T):
            u = [(sum(M[i, j] * u[j] for j in range(N)) + b[i]) % (1 << 32) for i in range(N)]
        exp = np.array(u, dtype=np.int64).astype(np.uint32).view(np.int32)
        got = oracle.run_vc_int(d, 1, pattern, shape, c, bkind, 5, u0, T)
        np.testing.assert_array_equal(got.ravel(), exp)


@pytest.mark.parametrize("d,shape", [(1, (50,)), (2, (13, 17)), (3, (6, 7, 9))])
@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_vc_constant_field_is_constant_weight_sweep(d, shape, bkind):
    for r, pattern in ((1, STAR), (1, BOX), (2, STAR)):
        w = list(uniform01(31 + r + pattern, npoints(d, r, pattern)) - 0.2)
        c = np.stack([np.full(shape, wj) for wj in w])
        u0 = uniform01(32, int(np.prod(shape))).reshape(shape)
        got = oracle.run_vc(d, r, pattern, shape, c, bkind, 0.4, u0, 7)
        ref = oracle.run(d, r, pattern, shape, w, bkind, 0.4, u0, 7)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("bkind", [DIRICHLET, PERIODIC])
def test_vc_rows_summing_to_one_keep_constants(bkind):
    shape = (23, 31)
    c = coef_field(2, 1, BOX, shape, 41, 0.0, 1.0)
    c = c / c.sum(axis=0, keepdims=True)
    u0 = np.full(shape, 0.625)
    got = oracle.run_vc(2, 1, BOX, shape, c, bkind, 0.625, u0, 20)
    assert np.max(np.abs(got - 0.625)) <= 1e-14


def test_vc_point_scaling_of_constant_weights():
    """c_o[x] = s[x] w_o: each step is the constant-weight step scaled by s."""
    shape = (17, 19)
    w = [0.5, 0.1, 0.15, 0.05, 0.2]
    s = 0.5 + uniform01(51, shape[0] * shape[1]).reshape(shape)
    c = np.stack([s * wj for wj in w])
    u0 = uniform01(52, shape[0] * shape[1]).reshape(shape)
    u = u0.copy()
    for _ in range(6):
        u = s * oracle.run(2, 1, STAR, shape, w, PERIODIC, 0.0, u, 1)
    got = oracle.run_vc(2, 1, STAR, shape, c, PERIODIC, 0.0, u0, 6)
    assert relerr(got, u) <= 1e-13


@pytest.mark.parametrize("d,shape", [(1, (11,)), (2, (5, 6)), (3, (3, 4, 4))])
@pytest.mark.parametrize("bkind,bval", [(PERIODIC, 0.0), (DIRICHLET, 0.3)])
def test_vc_adjoint_against_dense_and_fd(d, shape, bkind, bval):
    r, pattern = 1, STAR
    N = int(np.prod(shape))
    c = coef_field(d, r, pattern, shape, 61 + d, 0.0, 0.4)
    u0 = uniform01(62, N).reshape(shape)
    tg = uniform01(63, N).reshape(shape)
    T = 4
    loss, gu, gc = oracle.adjoint_vc(d, r, pattern, shape, c, bkind, bval, u0, tg, T)

    def dense_loss(cf, u_init):
        M, b = dense_vc(d, r, pattern, shape, cf, bkind, bval)
        u = u_init.ravel()
        for _ in range(T):
            u = M @ u + b
        return 0.5 * float(np.sum((u - tg.ravel()) ** 2)), M, b

    L, M, b = dense_loss(c, u0)
    assert abs(loss - L) <= 1e-12 * abs(L)
    # d loss / d u0 = (M^T)^T (u_T - target) exactly
    us = [u0.ravel()]
    for _ in range(T):
        us.append(M @ us[-1] + b)
    lam = us[-1] - tg.ravel()
    lam_t = lam.copy()
    for _ in range(T):
        lam_t = M.T @ lam_t
    assert relerr(gu.ravel(), lam_t) <= 1e-12
    # d loss / d c by central differences on a few coefficients (the loss is a
    # polynomial of degree 2T in c: h = 1e-5 leaves an O(h^2) error)
    rng = np.random.default_rng(d)
    h = 1e-5
    flat = c.reshape(-1)
    for idx in rng.choice(flat.size, size=6, replace=False):
        cp = flat.copy(); cm = flat.copy()
        cp[idx] += h; cm[idx] -= h
        fd = (dense_loss(cp.reshape(c.shape), u0)[0] - dense_loss(cm.reshape(c.shape), u0)[0]) / (2 * h)
        assert abs(fd - gc.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, gc.reshape(-1)[idx])

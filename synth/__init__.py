"""Seeded synthetic inputs for the iterated stencil sweep.

This module is shared by the tests, ``bench.py`` and ``__graft_entry__.smoke``.
It holds only input generation: the counter-based random stream, grid shapes,
stencil weights and initial fields of the workloads.  It performs none of the
stencil arithmetic, and it imports neither the oracle nor the CUDA package.

Random stream
-------------
``mix64(x)`` is the SplitMix64 output function (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014):
``z = x + 0x9E3779B97F4A7C15; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
z = (z ^ (z >> 27)) * 0x94D049BB133111EB; z ^ (z >> 31)`` in 64-bit wraparound.
Element ``i`` of stream ``seed`` is ``mix64(seed ^ (i * 0x9E3779B97F4A7C15))``.
``uniform01`` keeps its top 53 bits (``>> 11``) times 2**-53, so it lies in
[0, 1) and is exact in FP64.

Workloads
---------
The paper's experiments (Section 4.1, Table 1) run the 1D3P, 1D5P, 2D5P, 2D9P,
3D7P and 3D27P Jacobi stencils on synthetic grids; it gives no coefficients,
boundary rule or initial data.  The recipes below fix those (the coefficients
and sizes of the five workloads C1..C5 used throughout this repository).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STAR, BOX = 0, 1
DIRICHLET, PERIODIC = 0, 1


def mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wraparound arithmetic)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def raw64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Elements start..start+count-1 of stream ``seed`` as uint64."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed) ^ (idx * GAMMA))


def uniform01(seed: int, count: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """FP64 uniforms in [0, 1) from stream ``seed`` (53-bit, exact in FP64)."""
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        out[s:e] = (raw64(seed, e - s, start + s) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return out


def uniform_u16(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [0, 65535] (top 16 bits of the stream), as int32."""
    return (raw64(seed, count, start) >> np.uint64(48)).astype(np.int32)


# ----------------------------------------------------------------------------
# Stencil descriptions (compact weight order)
#   box : (2r+1)^d weights, offsets (o_0..o_{d-1}) in [-r, r]^d lexicographic,
#         innermost (last, unit-stride) dimension fastest;
#   star: 1 + 2dr weights: [centre, axis 0: -r..-1, +1..+r, axis 1: ..., ...],
#         axis 0 being the outermost dimension.
# ----------------------------------------------------------------------------

def npoints(d: int, r: int, pattern: int) -> int:
    return (2 * r + 1) ** d if pattern == BOX else 1 + 2 * d * r


def star_weights(d: int, r: int, centre: float, neighbour: float) -> list:
    return [centre] + [neighbour] * (2 * d * r)


def box_weights(d: int, r: int, value: float) -> list:
    return [value] * ((2 * r + 1) ** d)


@dataclass
class Problem:
    """One stencil problem: geometry, coefficients, boundary and step count."""
    name: str
    d: int
    r: int
    pattern: int
    shape: tuple
    weights: list
    bkind: int = DIRICHLET
    bval: float = 0.0
    T: int = 1
    seed: int = 1000
    extra: dict = field(default_factory=dict)

    @property
    def npts(self) -> int:
        return int(np.prod(self.shape))


# C1: 1D 3-point Jacobi heat stencil, FP64, N=65536, Dirichlet 0, T=100.
def c1_1d3p(n: int = 65536, T: int = 100) -> Problem:
    return Problem("1d3p", 1, 1, STAR, (n,), [0.5, 0.25, 0.25], DIRICHLET, 0.0, T, 1001)


def c1_1d3p_int(n: int = 65536, T: int = 100) -> Problem:
    return Problem("1d3p_int", 1, 1, STAR, (n,), [2.0, 1.0, 1.0], DIRICHLET, 0.0, T, 1001)


# C2: 2D 5-point star and 9-point box, 8192^2, Dirichlet 0, T=64.
def c2_2d5p(ny: int = 8192, nx: int = 8192, T: int = 64) -> Problem:
    return Problem("2d5p", 2, 1, STAR, (ny, nx), star_weights(2, 1, 0.5, 0.125), DIRICHLET, 0.0, T, 1002)


def c2_2d9p(ny: int = 8192, nx: int = 8192, T: int = 64) -> Problem:
    return Problem("2d9p", 2, 1, BOX, (ny, nx), box_weights(2, 1, 1.0 / 9.0), DIRICHLET, 0.0, T, 1002)


# C3: 3D 7-point star and 27-point box, 512^3, Dirichlet 0, T=32.
def c3_3d7p(n: int = 512, T: int = 32) -> Problem:
    return Problem("3d7p", 3, 1, STAR, (n, n, n), star_weights(3, 1, 0.4, 0.1), DIRICHLET, 0.0, T, 1003)


def c3_3d27p(n: int = 512, T: int = 32) -> Problem:
    return Problem("3d27p", 3, 1, BOX, (n, n, n), box_weights(3, 1, 1.0 / 27.0), DIRICHLET, 0.0, T, 1003)


# C5: differentiation workload, 3D 7-point star, periodic 256^3, T=64.
def c5_adjoint(n: int = 256, T: int = 64) -> Problem:
    return Problem("3d7p_adj", 3, 1, STAR, (n, n, n), star_weights(3, 1, 0.4, 0.1), PERIODIC, 0.0, T, 1005,
                   extra={"target_seed": 1007, "ckpt_every": 8})


# ----------------------------------------------------------------------------
# Initial fields
# ----------------------------------------------------------------------------

def u0_uniform(p: Problem, dtype=np.float64) -> np.ndarray:
    return uniform01(p.seed, p.npts).reshape(p.shape).astype(dtype)


def u0_int(p: Problem) -> np.ndarray:
    return uniform_u16(p.seed, p.npts).reshape(p.shape)


def sine_mode_1d(n: int, k: int) -> np.ndarray:
    """sin(pi k (i+1) / (n+1)) for i = 0..n-1: the discrete Dirichlet sine mode."""
    i = np.arange(n, dtype=np.float64)
    return np.sin(math.pi * k * (i + 1.0) / (n + 1.0))


def c3_modes(p: Problem, count: int = 8):
    """The 8 seeded sine modes of the 3D workload: list of (amplitude, (k0, k1, k2))."""
    raw = uniform01(p.seed + 10, 4 * count)
    modes = []
    for m in range(count):
        a = 0.9 * raw[4 * m]
        ks = tuple(1 + int(raw[4 * m + 1 + j] * 16.0) for j in range(3))
        modes.append((float(a), ks))
    return modes


def u0_modes_plus_noise(p: Problem, dtype=np.float32, noise: float = 0.1) -> np.ndarray:
    """Sum of the seeded Dirichlet sine modes plus noise * uniform01 (3D workload)."""
    shape = p.shape
    out = (noise * uniform01(p.seed, p.npts)).astype(np.float64).reshape(shape)
    for a, ks in c3_modes(p):
        v = [sine_mode_1d(shape[j], ks[j]) for j in range(3)]
        out += a * (v[0][:, None, None] * v[1][None, :, None] * v[2][None, None, :])
    return out.astype(dtype)


# ----------------------------------------------------------------------------
# C4: batched 2D 9-point box, periodic, 256 grids of uneven size and step count
# ----------------------------------------------------------------------------

def c4_batch(count: int = 256, lo: int = 64, hi: int = 2048, tlo: int = 8, thi: int = 128, seed: int = 1004):
    """Descriptors of the batched workload.

    Side lengths are exp(U(ln lo, ln hi)) rounded, independently per axis; T is
    uniform in [tlo, thi]; weights are 9 uniforms normalised in FP64 to sum 1.
    Returns a list of Problem (2D, r=1, BOX, periodic).
    """
    raw = uniform01(seed + 1, count * 12)
    probs = []
    for g in range(count):
        base = 12 * g
        ny = int(round(math.exp(math.log(lo) + raw[base] * (math.log(hi) - math.log(lo)))))
        nx = int(round(math.exp(math.log(lo) + raw[base + 1] * (math.log(hi) - math.log(lo)))))
        T = tlo + min(thi - tlo, int(raw[base + 2] * (thi - tlo + 1)))
        w = np.array(raw[base + 3: base + 12], dtype=np.float64)
        w = w / w.sum()
        probs.append(Problem(f"batch{g}", 2, 1, BOX, (ny, nx), [float(x) for x in w], PERIODIC, 0.0, T,
                             seed + 100 + g))
    return probs


def f32_weights(w) -> list:
    """Weights as the FP32 values a single-precision run uses, widened to FP64."""
    return [float(np.float32(x)) for x in w]

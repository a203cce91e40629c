"""Writes tests/golden/oracle_regression.json from the oracle alone.

The paper prints no worked numeric example (its result figures are absent and
its tables hold speedup ratios only), so the stored values here are
regression fixtures: outputs of the pinned oracle on small seeded cases, kept
so that any later change to the oracle's arithmetic shows up as a diff.
Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synth import BOX, DIRICHLET, PERIODIC, STAR, uniform01, uniform_u16  # noqa: E402

CASES = [
    # name, d, r, pattern, shape, weights, bkind, bval, T, int_mode, seed
    ("1d3p_int", 1, 1, STAR, [1001], [2, 1, 1], DIRICHLET, 0, 37, True, 1001),
    ("2d5p_f64", 2, 1, STAR, [37, 53], [0.5, 0.125, 0.125, 0.125, 0.125], DIRICHLET, 0.0, 11, False, 1002),
    ("2d9p_int_periodic", 2, 1, BOX, [23, 41], [1, 2, 3, 4, 5, 6, 7, 8, 9], PERIODIC, 0, 9, True, 1004),
    ("3d7p_f64", 3, 1, STAR, [9, 11, 13], [0.4, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1], DIRICHLET, 0.25, 5, False, 1003),
    ("2d_r2_box_int", 2, 2, BOX, [17, 19], list(range(-12, 13)), DIRICHLET, 7, 4, True, 1006),
]


def compute(case):
    name, d, r, pat, shape, w, bk, bv, T, is_int, seed = case
    n = int(np.prod(shape))
    if is_int:
        u0 = uniform_u16(seed, n).reshape(shape)
        out = oracle.run_int(d, r, pat, shape, [float(x) for x in w], bk, bv, u0, T)
        raw = out.astype(np.int32).tobytes()
        sample = [int(v) for v in out.ravel()[:: max(1, n // 8)]]
    else:
        u0 = uniform01(seed, n).reshape(shape)
        out = oracle.run(d, r, pat, shape, w, bk, bv, u0, T)
        raw = out.astype(np.float64).tobytes()
        sample = [float(v).hex() for v in out.ravel()[:: max(1, n // 8)]]
    return {"name": name, "d": d, "r": r, "pattern": pat, "shape": shape, "weights": w, "bkind": bk,
            "bval": bv, "T": T, "int": is_int, "seed": seed, "sha256": hashlib.sha256(raw).hexdigest(),
            "sample_stride": max(1, n // 8), "sample": sample}


if __name__ == "__main__":
    data = {"note": "outputs of the pinned FP64/uint32 oracle; inputs from synth (seeded)",
            "cases": [compute(c) for c in CASES]}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(data, f, indent=1)
    print("wrote", len(CASES), "cases")

"""The oracle reproduces its stored regression fixtures bit for bit."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_regression_fixtures():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        stored = json.load(f)["cases"]
    assert len(stored) == len(make_golden.CASES)
    for case, ref in zip(make_golden.CASES, stored):
        got = make_golden.compute(case)
        assert got["sha256"] == ref["sha256"], ref["name"]
        assert got["sample"] == ref["sample"], ref["name"]

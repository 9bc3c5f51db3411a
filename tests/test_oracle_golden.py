"""The oracle against its stored regression values (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle alone; the paper prints
no worked example). Tolerances cover rounding-order changes only."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_stored_regression_values():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        ref = json.load(f)
    got = make_golden.compute()
    for key in ("mhat", "mhat_dag", "dhop_e", "clover_odd", "trace_samples"):
        a, b = np.array(got[key]), np.array(ref[key])
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max()), key
    assert np.allclose(got["clover_logdet"], ref["clover_logdet"], rtol=1e-12, atol=1e-12)
    assert abs(got["cg_solution_norm"] - ref["cg_solution_norm"]) <= 1e-9 * ref["cg_solution_norm"]

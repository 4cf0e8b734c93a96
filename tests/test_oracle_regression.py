"""Regression pin of the oracle itself: its outputs on five small fixed cases
(the plain step, two iterations, the Jacobi solver, the grasper, connected
tissue) must match tests/golden/oracle_regression.json, written by
tests/golden/make_oracle_regression.py from the oracle. A change to the
oracle's arithmetic then fails here until the file is rewritten, and the
commit that rewrites it names the passage of the paper that justifies it.
The bound (1e-9 of the 5 mm cell) allows for a last-bit difference of the
host's libm, nothing more."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("name", sorted(_golden().keys()))
def test_oracle_matches_its_regression_values(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(HERE, "golden", "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    got = mod.run(mod.CASES[name])
    want = _golden()[name]
    tol = 1e-9 * 5e-3
    assert got["sample_ids"] == want["sample_ids"]
    assert got["contacts"] == want["contacts"]
    np.testing.assert_allclose(got["rewards"], want["rewards"], rtol=0, atol=tol)
    np.testing.assert_allclose(got["tool"], want["tool"], rtol=0, atol=0)
    np.testing.assert_allclose(got["x_sample"], want["x_sample"], rtol=0, atol=tol)
    np.testing.assert_allclose(got["v_sample"], want["v_sample"], rtol=0, atol=tol * 600)
    assert abs(got["x_abs_sum"] - want["x_abs_sum"]) <= tol * len(want["sample_ids"]) * 100

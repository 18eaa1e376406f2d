"""The oracle reproduces its stored output for a few small fixed-seed
iterations (tests/golden/oracle_small_iterations.json, written by
tests/golden/make_golden.py from the oracle alone): a change to the oracle's
arithmetic, or a host platform on which it computes differently, shows up
here.  Jump counts must match exactly, floating-point values to 1e-12."""

import json
import os

import numpy as np
import pytest

import oracle
from tests.golden.make_golden import cases

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_small_iterations.json")
STORED = json.load(open(GOLDEN))["cases"]


@pytest.mark.parametrize("name", sorted(STORED))
def test_oracle_matches_stored_iteration(name):
    prob, it = cases()[name]
    g = STORED[name]
    r = oracle.iteration(prob, np.array(g["x0"]), np.array(g["U_in"]), g["it"], want_counts=True)
    np.testing.assert_array_equal(r["counts"], np.array(g["counts"]))
    np.testing.assert_allclose(r["S"], g["S"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["U"], g["U"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r["diag"], g["diag"], rtol=1e-12, atol=1e-13)

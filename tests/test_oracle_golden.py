"""Regression pin: the oracle's outputs on a small fixed workload match the
stored fixture written by tests/golden/make_golden.py (oracle only)."""
import json
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_fixture():
    with open(os.path.join(HERE, "golden", "oracle_tiny.json")) as f:
        ref = json.load(f)
    got = compute()
    assert got.keys() == ref.keys()
    for k in ref:
        np.testing.assert_allclose(np.asarray(got[k], float), np.asarray(ref[k], float), rtol=1e-9, atol=1e-15,
                                   err_msg=k)

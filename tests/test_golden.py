"""The oracle reproduces its frozen outputs in tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py, which imports only oracle/ and synthetic/:
a regression freeze of the oracle, not a pin (the pins are in tests/test_oracle_*.py)."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_matches_frozen_values():
    with open(os.path.join(HERE, "oracle_regression.json")) as fh:
        stored = json.load(fh)["values"]
    fresh = _maker().compute()
    assert set(fresh) == set(stored)
    for key, want in stored.items():
        np.testing.assert_allclose(np.asarray(fresh[key]), np.asarray(want), rtol=1e-11, atol=1e-12, err_msg=key)

"""The FP64 oracle against its own recorded outputs (tests/golden/
oracle_regression.json, written by tests/golden/make_oracle_regression.py).

This is a regression record, not a pin. A failure means the oracle's arithmetic
changed. If the change is intended, regenerate the record with the script, and
name in the commit message the passage of the paper, or the reading of it, that
justifies the change. Floating-point entries compare to 1e-12 relative, which
allows for last-bit differences between libm versions. Counts compare exactly."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _script():
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(GOLDEN, "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


SCRIPT = _script()
RECORD = json.load(open(os.path.join(GOLDEN, "oracle_regression.json")))
CASES = SCRIPT.cases()


def test_record_covers_every_case():
    assert set(RECORD) == set(CASES)


@pytest.mark.parametrize("name", sorted(RECORD))
def test_oracle_matches_its_record(name):
    rec = RECORD[name]
    got = np.asarray(CASES[name][1](), dtype=np.float64)
    want = np.asarray(rec["values"], dtype=np.float64).reshape(rec["shape"])
    assert got.shape == want.shape
    if name.endswith("_stats"):
        np.testing.assert_array_equal(got, want)
    else:
        scale = float(np.max(np.abs(want))) if want.size else 0.0
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * scale)

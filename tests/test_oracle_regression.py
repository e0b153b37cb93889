"""The oracle's output against its stored regression record (tests/golden/oracle_regression.json,
written by tests/golden/make_oracle_regression.py from the oracle alone; no GPU).

Not a pin: the pins are in test_oracle_pins.py.  This makes any change of the oracle's arithmetic
visible; a commit that regenerates the record must name the passage or reading that justifies it.
Counts are exact; Γ and WP agree to 1e-12 (libm may differ in the last bits across platforms)."""
import json
import os

import numpy as np

from tests.golden.make_oracle_regression import compute

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_regression_record():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        rec = json.load(f)
    assert len(rec["cases"]) == 3
    for case in rec["cases"]:
        now = compute(case)
        assert np.array_equal(np.asarray(now["counts"]), np.asarray(case["counts"]))
        for k in ("gamma", "wp"):
            a, b = np.asarray(now[k]), np.asarray(case[k])
            scale = np.abs(b).max(axis=1, keepdims=True)
            assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(b), 1e-6 * scale)), (case["mesh"], k)

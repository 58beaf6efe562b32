"""The oracle against its stored results on one small seeded case
(tests/golden/oracle_anchor.json, written by tests/golden/make_oracle_anchor.py).

This is a regression anchor, not a pin: the pins against the paper and the mathematics
are the other tests/test_oracle_*.py. It makes any change to the oracle's arithmetic
visible. The bar is 1e-12 relative to each array's largest value, which allows a
different libm or compiler (the oracle is built without FMA contraction) and nothing
more. The accept/reject trace must be exact.
"""
import json
import os
import sys

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_its_anchor(O):
    sys.path.insert(0, GOLDEN)
    try:
        import make_oracle_anchor as mk
    finally:
        sys.path.remove(GOLDEN)
    want = json.load(open(os.path.join(GOLDEN, "oracle_anchor.json")))
    assert want["case"] == mk.CASE
    got = mk.compute(O)
    assert got["lm_accepted"] == want["lm_accepted"]
    assert abs(got["lm_f_final"] - want["lm_f_final"]) <= 1e-12 * abs(want["lm_f_final"])
    for k in ("forward", "jvp", "vjp_lambda", "vjp_mu", "lm_lambda", "lm_mu"):
        a, b = np.asarray(got[k]), np.asarray(want[k])
        assert a.shape == b.shape, k
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), k

"""Writes oracle_anchor.json: the oracle's forward model, JVP, adjoint and a three-step LM
run on one small seeded case (12 x 12 grid, 6 angles, two banks of 7 detectors, 3
triangular sub-rays).

It calls only the oracle. The file is a regression anchor: it pins the oracle to its
own earlier results, not to the paper (the pins in tests/test_oracle_*.py do that). A
change to the oracle's arithmetic that moves these values is deliberate, and the commit
that rewrites the file names the passage of the paper that justifies the change.

    python tests/golden/make_oracle_anchor.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASE = dict(n=12, n_angles=6, n_det=14, n_sub=3, collimator=1, seed=2604)


def inputs():
    rs = np.random.default_rng(CASE["seed"])
    n = CASE["n"]
    lam = rs.uniform(0.0, 1.5, (n, n))
    mu = rs.uniform(0.0, 0.15, (n, n))
    dl = rs.standard_normal((n, n))
    dm = 0.01 * rs.standard_normal((n, n))
    r = rs.standard_normal((CASE["n_angles"], CASE["n_det"]))
    return lam, mu, dl, dm, r


def compute(O):
    c = CASE
    g = O.geom(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"], collimator=c["collimator"])
    lam, mu, dl, dm, r = inputs()
    y = O.forward(g, lam, mu)
    gl, gm = O.vjp(g, lam, mu, r)
    l0, m0 = O.initial_guess(g, y)
    lo, mo, rep = O.lm(g, O.default_params(max_iters=3, cg_max_iters=5), y, l0, m0)
    return {"forward": y.ravel().tolist(), "jvp": O.jvp(g, lam, mu, dl, dm).ravel().tolist(),
            "vjp_lambda": gl.ravel().tolist(), "vjp_mu": gm.ravel().tolist(),
            "lm_lambda": lo.ravel().tolist(), "lm_mu": mo.ravel().tolist(),
            "lm_f_final": rep["f_final"], "lm_accepted": list(rep["acc"])}


if __name__ == "__main__":
    from oracle import oracle as O
    O.build()
    out = {"case": CASE, **compute(O)}
    with open(os.path.join(HERE, "oracle_anchor.json"), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")

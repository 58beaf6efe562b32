"""Writes lm_single128.npz and lm_single128.json: the oracle's full reconstruction of the
single-request workload (128 x 128 grid, 9 x 9 rods r = 5, 360 angles x 182 detectors in
two banks x 5 triangular sub-rays, Poisson noise at 1e5 counts, 20 LM iterations with CG
capped at 30 steps), and how far the oracle itself moves when only its rounding changes.

It calls only the oracle (and the seeded input generators, which hold none of the
method's arithmetic).  The data y are the oracle's forward model of the phantom with
Poisson noise; the file stores the Poisson counts, so y is rebuilt bitwise as
counts * ymax / C, exactly as the noise generator forms it.

Variants (same algorithm, inputs changed only as stated):
  * rounding: the adjoint's scatter summed in another order (1, 7 and 90 angle chunks
    instead of 32), and the data changed by a relative 1e-14 (two seeded sign patterns);
  * single-precision level: the data changed by a relative 1e-7 (two seeded sign
    patterns), the size of the rounding a float ray sum carries.
Each variant's distance to the base run measures how far the oracle itself moves at this
configuration: finite-precision CG over 30 steps on these damped normal equations (the
lagged TV weights reach 1/eps = 1e3 in flat regions) amplifies rounding, so an
implementation with other rounding cannot be expected to land closer to the base run than
the variants of its own rounding level do.

    python tests/golden/make_lm_single128.py        # about 60 minutes on 8 cores
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASE = dict(n=128, n_lat=9, radius=5.0, n_angles=360, n_det=182, n_sub=5, collimator=1,
            counts=1e5, phantom_seed=1100, noise_seed=2100, max_iters=20, cg_max_iters=30,
            cg_rel_tol=1e-6)
CHUNKS = (1, 7, 90)
PERTURB = ((1e-14, 31), (1e-14, 32), (1e-7, 41), (1e-7, 42))


def inputs(O):
    """Phantom, Poisson counts, ymax and the data y = counts * ymax / C."""
    from paper_2604_26745_gb300 import synth
    c = CASE
    ph = synth.lattice_phantom(c["n"], c["n_lat"], radius=c["radius"], seed=c["phantom_seed"])
    g = O.geom(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"], collimator=c["collimator"])
    y_clean = O.forward(g, ph.lam, ph.mu)
    ymax = float(y_clean.max())
    counts = synth.rng(c["noise_seed"]).poisson(np.clip(c["counts"] * y_clean / ymax, 0.0, None))
    y = counts.astype(np.float64) * ymax / c["counts"]
    assert np.array_equal(y, synth.poisson_noise(y_clean, c["counts"], c["noise_seed"]))
    return g, ph, counts.astype(np.int32), ymax, y


def solve(O, g, y):
    c = CASE
    pr = O.default_params(max_iters=c["max_iters"], cg_max_iters=c["cg_max_iters"], cg_rel_tol=c["cg_rel_tol"])
    l0, m0 = O.initial_guess(g, y)
    t0 = time.perf_counter()
    lam, mu, rep = O.lm(g, pr, y, l0, m0)
    return lam, mu, rep, time.perf_counter() - t0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stats(lam, mu, rep, base, ph):
    bl, bm = base
    return {"rel_l2_u_vs_base": rel(np.concatenate([lam.ravel(), mu.ravel()]),
                                    np.concatenate([bl.ravel(), bm.ravel()])),
            "rel_l2_lambda_vs_base": rel(lam, bl), "rel_l2_mu_vs_base": rel(mu, bm),
            "rel_err_truth_lambda": rel(lam, ph.lam), "rel_err_truth_mu": rel(mu, ph.mu),
            "f_final": rep["f_final"], "accepted": rep["acc"]}


def main():
    from oracle import oracle as O
    O.build()
    g, ph, counts, ymax, y = inputs(O)
    O.set_vjp_chunks(32)
    lam, mu, rep, dt = solve(O, g, y)
    l0, m0 = O.initial_guess(g, y)
    out = {"case": CASE, "threads": O.num_threads(), "seconds_base": dt,
           "base": {"f0": rep["f0"], "f_final": rep["f_final"], "accepted": rep["acc"], "f": rep["f"],
                    "nu": rep["nu"], "rho": rep["rho"], "cg_iters": rep["cg_iters"],
                    "rel_err_truth_lambda": rel(lam, ph.lam), "rel_err_truth_mu": rel(mu, ph.mu),
                    "initial_rel_err_truth_lambda": rel(l0, ph.lam),
                    "initial_rel_err_truth_mu": rel(m0, ph.mu)},
           "variants": {}}
    print("base", dt, out["base"]["rel_err_truth_lambda"], out["base"]["rel_err_truth_mu"], flush=True)
    for ch in CHUNKS:
        O.set_vjp_chunks(ch)
        vl, vm, vr, _ = solve(O, g, y)
        out["variants"][f"vjp_chunks_{ch}"] = stats(vl, vm, vr, (lam, mu), ph)
        print(ch, out["variants"][f"vjp_chunks_{ch}"]["rel_l2_u_vs_base"], flush=True)
    O.set_vjp_chunks(32)
    for eps, s in PERTURB:
        sign = np.where(np.random.default_rng(s).random(y.shape) < 0.5, -1.0, 1.0)
        vl, vm, vr, _ = solve(O, g, y * (1.0 + eps * sign))
        key = f"y_rel_{eps:.0e}_seed{s}"
        out["variants"][key] = stats(vl, vm, vr, (lam, mu), ph)
        print(key, out["variants"][key]["rel_l2_u_vs_base"], flush=True)
    rnd = [d["rel_l2_u_vs_base"] for k, d in out["variants"].items() if "1e-07" not in k]
    f32 = [d["rel_l2_u_vs_base"] for k, d in out["variants"].items() if "1e-07" in k]
    out["spread_max_rel_l2_u"] = max(rnd)
    out["spread_median_rel_l2_u"] = float(np.median(rnd))
    out["spread_f32_level_max_rel_l2_u"] = max(f32)
    np.savez_compressed(os.path.join(HERE, "lm_single128.npz"), counts=counts, ymax=np.float64(ymax),
                        lam=lam, mu=mu)
    with open(os.path.join(HERE, "lm_single128.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()

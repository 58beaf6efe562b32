"""Writes stress512.npz and stress512.json: the oracle's reconstructions of the first items
of the precision-stress workload (512 x 512 grid, 17 x 17 rods r = 10 with rod
attenuation ~ U(0.05, 0.12), 720 angles x 182 detectors in two banks x 9 triangular
sub-rays, Poisson noise at 1e6 counts, 10 LM iterations with CG capped at 30 steps).

It calls only the oracle (and the seeded input generators, which hold none of the
method's arithmetic).  Item i uses phantom seed 1500 + i and noise seed 2500 + i; its data
are the oracle's forward model with Poisson noise, stored as the counts, so y is rebuilt
bitwise as counts * ymax / C.  The reconstructions are stored in float32 (they are
compared with GPU results at the 1e-3 level; float32 keeps 6e-8).

    python tests/golden/make_stress512.py [items]     # about 20 minutes per item on 8 cores
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASE = dict(n=512, n_lat=17, radius=10.0, mu_rod=(0.05, 0.12), n_angles=720, n_det=182, n_sub=9, collimator=1,
            counts=1e6, phantom_seed0=1500, noise_seed0=2500, max_iters=10, cg_max_iters=30, cg_rel_tol=1e-10)


def inputs(O, i):
    from paper_2604_26745_gb300 import synth
    c = CASE
    ph = synth.lattice_phantom(c["n"], c["n_lat"], radius=c["radius"], seed=c["phantom_seed0"] + i,
                               mu_rod=c["mu_rod"])
    g = O.geom(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"], collimator=c["collimator"])
    y_clean = O.forward(g, ph.lam, ph.mu)
    ymax = float(y_clean.max())
    counts = synth.rng(c["noise_seed0"] + i).poisson(np.clip(c["counts"] * y_clean / ymax, 0.0, None))
    y = counts.astype(np.float64) * ymax / c["counts"]
    assert np.array_equal(y, synth.poisson_noise(y_clean, c["counts"], c["noise_seed0"] + i))
    return g, ph, counts.astype(np.int32), ymax, y


def main(items: int):
    from oracle import oracle as O
    O.build()
    c = CASE
    arrays, meta = {}, {"case": {k: list(v) if isinstance(v, tuple) else v for k, v in c.items()},
                        "threads": O.num_threads(), "items": []}
    for i in range(items):
        g, ph, counts, ymax, y = inputs(O, i)
        pr = O.default_params(max_iters=c["max_iters"], cg_max_iters=c["cg_max_iters"], cg_rel_tol=c["cg_rel_tol"],
                              mu_max=0.25)
        l0, m0 = O.initial_guess(g, y, mu_max=0.25)
        t0 = time.perf_counter()
        lam, mu, rep = O.lm(g, pr, y, l0, m0)
        dt = time.perf_counter() - t0
        arrays[f"counts{i}"] = counts
        arrays[f"ymax{i}"] = np.float64(ymax)
        arrays[f"lam{i}"] = lam.astype(np.float32)
        arrays[f"mu{i}"] = mu.astype(np.float32)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        meta["items"].append({"item": i, "seconds": dt, "f0": rep["f0"], "f_final": rep["f_final"],
                              "accepted": rep["acc"], "rel_err_truth_lambda": rel(lam, ph.lam),
                              "rel_err_truth_mu": rel(mu, ph.mu)})
        print(i, dt, meta["items"][-1]["rel_err_truth_lambda"], flush=True)
    np.savez_compressed(os.path.join(HERE, "stress512.npz"), **arrays)
    with open(os.path.join(HERE, "stress512.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)

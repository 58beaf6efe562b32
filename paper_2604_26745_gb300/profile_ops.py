"""Run each hot-path operator once on a named workload (for profilers such as ncu).

  python -m paper_2604_26745_gb300.profile_ops [--config single128|plain64|stress512] [--op all|forward|jvp|vjp|lm]

The single-request workload is 128 x 128, 360 angles x 182 detectors x 5 triangular
sub-rays (FP32 with Kahan sums); plain64 is 64 x 64, 90 x 91 x 1 in FP64; stress512 is
512 x 512, 720 x 182 x 9 (FP32 Kahan)."""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import build, pget as P, synth

CONFIGS = {
    "single128": dict(n=128, n_lat=9, radius=5.0, n_angles=360, n_det=182, n_sub=5, prec=P.PGET_F32_KAHAN),
    "plain64": dict(n=64, n_lat=9, radius=3.0, n_angles=90, n_det=91, n_sub=1, prec=P.PGET_F64),
    "stress512": dict(n=512, n_lat=17, radius=10.0, n_angles=720, n_det=182, n_sub=9, prec=P.PGET_F32_KAHAN),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="single128", choices=sorted(CONFIGS))
    ap.add_argument("--op", default="all", choices=["all", "forward", "jvp", "vjp", "lm"])
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args()
    build.build()
    c = CONFIGS[a.config]
    dt = P.dtype_of(c["prec"])
    ph = synth.lattice_phantom(c["n"], c["n_lat"], radius=c["radius"], seed=1)
    g = P.geometry(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"])
    t = lambda x: torch.tensor(x, dtype=dt, device="cuda")
    lam, mu = t(ph.lam), t(ph.mu)
    rs = np.random.default_rng(0)
    dl, dm = t(rs.standard_normal(ph.lam.shape)), t(0.01 * rs.standard_normal(ph.lam.shape))
    with P.Context(0) as ctx:
        y = P.pget_forward(ctx, g, c["prec"], lam, mu)
        r = t(rs.standard_normal(tuple(y.shape)))
        for _ in range(a.repeat):
            if a.op in ("all", "forward"):
                P.pget_forward(ctx, g, c["prec"], lam, mu, y)
            if a.op in ("all", "jvp"):
                P.pget_jvp(ctx, g, c["prec"], lam, mu, dl, dm)
            if a.op in ("all", "vjp"):
                P.pget_vjp(ctx, g, c["prec"], lam, mu, r)
            if a.op == "lm":
                p = P.default_params(max_iters=2, cg_max_iters=5, precision=c["prec"])
                l0, m0 = P.pget_initial_guess(ctx, g, p, y)
                P.pget_lm_solve(ctx, g, p, y, l0, m0)
        torch.cuda.synchronize()
    print("profile_ops done", a.config, a.op)


if __name__ == "__main__":
    main()

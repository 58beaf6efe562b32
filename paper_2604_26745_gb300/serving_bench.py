"""Serving benchmark: a stream of reconstruction requests of mixed sizes through the
continuous-admission path (pget_submit / pget_poll), against the same requests solved one
at a time through the single-request path (pget_initial_guess + pget_lm_solve).

  python -m paper_2604_26745_gb300.serving_bench [--requests 64] [--rate 50] [--seed 4242]
         [--iters 15] [--cg 30] [--inflight 8] [--saturate] [--rates 50,3]

Requests follow the mixed serving workload: exponential inter-arrival gaps at the given
rate; per request N in {96, 128, 192, 256}, lattice in {9, 10, 17}, angles in {180, 360},
182 detectors, 3..7 triangular sub-rays, counts 10^U(4,6); FP32 rays with Kahan sums and
FP64 scalars.  Data are generated before timing (GPU FP64 forward + Poisson noise).

Both arms are timed warm (workspaces and captured graphs exist, as in a long-running
server): the single-request arm solves every request once untimed, then once timed; the
serving arm replays the whole stream once untimed, then once timed.  --rates serves the same
requests at each listed arrival rate in turn (the seeded stream draws the same sizes at
every rate; only the gaps scale), against one single-request arm.  Prints one JSON
line per rate: serving recon/s (requests / time from the first arrival to the last completion),
single-request recon/s (requests / sum of the per-request solve times), p50/p99 latency
(completion - arrival), and the largest relative L2 difference between a serving result
and the same request solved alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

import numpy as np
import torch

from . import build, pget as P, synth


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--seed", type=int, default=4242)
    ap.add_argument("--iters", type=int, default=15)
    ap.add_argument("--cg", type=int, default=30)
    ap.add_argument("--inflight", type=int, default=8)
    ap.add_argument("--saturate", action="store_true", help="all requests arrive at t = 0")
    ap.add_argument("--rates", default="", help="comma-separated arrival rates, one serving run each")
    return ap.parse_args()


def make_requests(ctx, stream):
    reqs = []
    for rq in stream:
        g = P.geometry(rq.n, rq.n_angles, rq.n_det, n_sub=rq.n_sub, collimator=1)
        ph = synth.lattice_phantom(rq.n, rq.n_lat, seed=rq.phantom_seed)
        y_clean = P.pget_forward(ctx, g, P.PGET_F64, torch.tensor(ph.lam, device="cuda"),
                                 torch.tensor(ph.mu, device="cuda"))
        y = synth.poisson_noise(y_clean.cpu().numpy(), rq.counts, rq.noise_seed)
        reqs.append((rq, g, torch.tensor(y, dtype=torch.float32, device="cuda")))
    return reqs


def single_arm(ctx, reqs, p):
    times, outs = [], []
    for timed in (False, True):
        for rq, g, y in reqs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam, mu = P.pget_initial_guess(ctx, g, p, y)
            P.pget_lm_solve(ctx, g, p, y, lam, mu)
            torch.cuda.synchronize()
            if timed:
                times.append(time.perf_counter() - t0)
                outs.append(torch.cat([lam.ravel(), mu.ravel()]).double())
    return times, outs


def serving_arm(ctx, reqs, p, saturate: bool):
    outs = [None] * len(reqs)
    lat = [0.0] * len(reqs)
    bufs = [(torch.empty((g.n, g.n), device="cuda"), torch.empty((g.n, g.n), device="cuda")) for _, g, _ in reqs]
    t_first = t_last = 0.0
    for timed in (False, True):
        pending = list(range(len(reqs)))
        inflight = {}
        t0 = time.perf_counter()
        done_at = {}
        while pending or inflight:
            now = time.perf_counter() - t0
            progressed = False
            while pending:
                k = pending[0]
                arr = 0.0 if saturate else reqs[k][0].arrival_s
                if arr > now:
                    break
                try:
                    t = P.pget_submit(ctx, reqs[k][1], p, reqs[k][2])
                except P.PgetError as e:
                    if e.status != P.PGET_EAGAIN:
                        raise
                    break
                inflight[t] = k
                pending.pop(0)
                progressed = True
            for t, k in list(inflight.items()):
                done, _ = P.pget_poll(ctx, t, bufs[k][0], bufs[k][1])
                if done:
                    done_at[k] = time.perf_counter() - t0
                    del inflight[t]
                    progressed = True
            if not progressed:
                time.sleep(0.0002)
        if timed:
            arrivals = [0.0 if saturate else rq.arrival_s for rq, _, _ in reqs]
            for k in range(len(reqs)):
                lat[k] = done_at[k] - arrivals[k]
                outs[k] = torch.cat([bufs[k][0].ravel(), bufs[k][1].ravel()]).double()
            t_first, t_last = min(arrivals), max(done_at.values())
    return t_last - t_first, lat, outs


def main():
    a = _args()
    os.environ["PGET_MAX_INFLIGHT"] = str(a.inflight)
    build.build()
    rates = [float(x) for x in a.rates.split(",") if x] or [a.rate]
    stream = synth.serving_stream(a.requests, rates[0], a.seed)
    p = P.default_params(max_iters=a.iters, cg_max_iters=a.cg, cg_rel_tol=1e-6, precision=P.PGET_F32_KAHAN)
    with P.Context(0) as ctx:
        reqs = make_requests(ctx, stream)
        times, alone = single_arm(ctx, reqs, p)
    single = len(reqs) / sum(times)
    for rate in rates:
        st = synth.serving_stream(a.requests, rate, a.seed)  # same sizes and seeds, scaled gaps
        reqs_r = [(rq, g, y) for (_, g, y), rq in zip(reqs, st)]
        with P.Context(0) as sctx:
            span, lat, served = serving_arm(sctx, reqs_r, p, a.saturate)
        diff = max(float(torch.linalg.norm(s_ - r) / torch.linalg.norm(r)) for s_, r in zip(served, alone))
        lat_ms = sorted(x * 1e3 for x in lat)
        line = {
            "metric": "serving recon/s", "value": round(len(reqs) / span, 3), "unit": "recon/s",
            "single_request_recon_s": round(single, 3), "speedup_vs_single": round(len(reqs) / span / single, 3),
            "latency_ms": {"p50": round(statistics.median(lat_ms), 1),
                           "p99": round(lat_ms[min(len(lat_ms) - 1, int(np.ceil(0.99 * len(lat_ms))) - 1)], 1)},
            "single_request_ms": {"p50": round(statistics.median(times) * 1e3, 1), "max": round(max(times) * 1e3, 1)},
            "max_rel_l2_diff_vs_alone": diff,
            "config": {"requests": len(reqs), "rate_hz": None if a.saturate else rate, "seed": a.seed,
                       "arrival_span_s": round(max(rq.arrival_s for rq in st), 2),
                       "lm_iters": a.iters, "cg_max": a.cg, "max_inflight": a.inflight, "precision": "f32-kahan",
                       "sizes": sorted({rq.n for rq, _, _ in reqs}), "data": "synthetic"},
        }
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

"""Throughput and precision of the hot path on the other standard workloads (the
single-request LM is bench.py, the mixed request stream is serving_bench.py).

  python -m paper_2604_26745_gb300.config_bench --config plain64|diff256|stress512 [--count K]

plain64    plain LM in FP64: 64 x 64, 9 x 9 rods r = 3, 90 angles x 91 detectors x 1 ray,
           Poisson 1e4, 10 LM iterations, CG <= 50 (tol 1e-10); K reconstructions
           (phantom seeds 1000+i, noise 2000+i): recon/s and p50/p99 latency.
diff256    differentiation: K pairs (lambda, mu) on 256 x 256 (17 x 17 rods r = 5),
           360 x 182 x 5: gradient of 1/2 |A(lambda, mu) - y|^2 through the autograd
           wrapper (pairs/s, FP32-Kahan and FP64) and the memory the recompute saves.
stress512  precision stress: K reconstructions on 512 x 512 (17 x 17 rods r = 10, rod
           mu ~ U(0.05, 0.12)), 720 x 182 x 9, Poisson 1e6, 10 LM iterations, CG <= 30,
           box mu <= 0.25, in FP32, FP32-Kahan and FP64: recon/s per precision and, per
           result, the relative L2 distance of the FP32 and FP32-Kahan sinogram, gradient and
           final reconstruction from the FP64 GPU path on the same input; for the items the
           oracle has reconstructed (--oracle, default tests/golden/stress512), the data are
           the oracle's and every precision's reconstruction is compared with the oracle's.

ops128     the three ray operators alone on the single-request geometry (128 x 128, 360 x
           182 x 5, FP32-Kahan): forward, JVP and adjoint, K launches each after one
           warm-up: average device time per launch and in-grid samples of distinct rays
           per second.  --op forward|jvp|vjp|all restricts the launches (also the small,
           named case for kernel profilers).
ops512     the same on the precision-stress geometry (512 x 512, 720 x 182 x 9).
ops256     the same on the differentiation geometry (256 x 256, 360 x 182 x 5).
ops64      the same on the plain-LM geometry (64 x 64, 90 x 91 x 1) in FP64.

Prints one JSON line per configuration.  Timing: CUDA events on the current stream around
each reconstruction or launch (after one untimed warm-up), data resident in HBM.
"""
from __future__ import annotations

import argparse
import json
import os
import math
import statistics

import numpy as np
import torch

from . import build, pget as P, synth


def _rel(a, b) -> float:
    a = a.double().ravel()
    b = b.double().ravel()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def _timed_solve(ctx, g, p, y):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    lam, mu = P.pget_initial_guess(ctx, g, p, y)
    rep = P.pget_lm_solve(ctx, g, p, y, lam, mu)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b), lam, mu, rep


def plain64(k: int) -> dict:
    g = P.geometry(64, 90, 91, n_sub=1)
    p = P.default_params(max_iters=10, cg_max_iters=50, cg_rel_tol=1e-10, precision=P.PGET_F64)
    ms = []
    with P.Context(0) as ctx:
        ys = []
        for i in range(k):
            ph = synth.lattice_phantom(64, 9, radius=3.0, seed=1000 + i)
            yc = P.pget_forward(ctx, g, P.PGET_F64, torch.tensor(ph.lam, device="cuda"),
                                torch.tensor(ph.mu, device="cuda"))
            ys.append(torch.tensor(synth.poisson_noise(yc.cpu().numpy(), 1e4, 2000 + i), device="cuda"))
        _timed_solve(ctx, g, p, ys[0])  # warm-up: workspace and captured graph
        for y in ys:
            ms.append(_timed_solve(ctx, g, p, y)[0])
    return {"config": "plain LM FP64: 64x64, 9x9 rods r=3, 90 x 91 x 1, Poisson 1e4, 10 LM x CG<=50",
            "reconstructions": k, "recon_per_s": round(1e3 * k / sum(ms), 2),
            "latency_ms": {"p50": round(statistics.median(ms), 2), "p99": round(_pct(ms, 0.99), 2)}}


def diff256(k: int) -> dict:
    from . import autograd as AG
    n, na, nd, S = 256, 360, 182, 5
    g = P.geometry(n, na, nd, n_sub=S)
    pairs = [synth.lattice_phantom(n, 17, radius=5.0, seed=1200 + i) for i in range(k)]
    out = {"config": "differentiation: 256x256, 17x17 rods r=5, 360 x 182 x 5", "pairs": k}
    for name, dt in (("f32_kahan", torch.float32), ("f64", torch.float64)):
        L = torch.tensor(np.stack([p.lam for p in pairs]), dtype=dt, device="cuda", requires_grad=True)
        M = torch.tensor(np.stack([p.mu for p in pairs]), dtype=dt, device="cuda", requires_grad=True)
        y = torch.zeros((k, na, nd), dtype=dt, device="cuda")
        AG.data_loss(L[:1], M[:1], y[:1], g).backward()  # warm-up
        L.grad = None
        M.grad = None
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        AG.data_loss(L, M, y, g).backward()
        b.record()
        torch.cuda.synchronize()
        out[f"{name}_pairs_per_s"] = round(1e3 * k / a.elapsed_time(b), 2)
    # what recomputing the attenuation prefixes saves: storing exp(-E_j) and the prefix
    # sum per in-grid sample (8 bytes in FP32) for every ray of one pair
    samples = _in_grid_samples(n, na, nd, S)
    out["recompute_saves_bytes_per_pair"] = 8 * samples
    return out


def samples_per_launch(g: dict) -> dict:
    """Ray samples one walk launch processes, counted on the host from the geometry (dict
    with n, n_angles, n_det, n_sub; triangular sub-rays): in-grid samples (bilinear base
    pixel inside [-1, n-1]^2) of every sub-ray, and of the distinct rays the kernels trace
    (sub-rays of neighbouring detectors that lie on one line are one ray)."""
    n, na, nd, S = g["n"], g["n_angles"], g["n_det"], g["n_sub"]
    nbk = 2 if nd == 182 else 1
    nb = nd // nbk
    r = n / math.sqrt(2.0)
    p = 2 * r / nb
    T = math.ceil(2 * r)
    c = 0.5 * (n - 1)
    t = -r + (np.arange(T) + 0.5)
    u = np.array([(k - (S - 1) / 2) * 2 * p / (S + 1) for k in range(S)])
    total_sub, total_distinct = 0, 0
    for a in range(na):
        for b in range(nbk):
            psi = 2 * math.pi * a / na + b * math.pi
            ct, st = math.cos(psi), math.sin(psi)
            s_all = (((np.arange(nb) - 0.5 * (nb - 1) + 0.5 * b) * p)[:, None] + u[None, :]).ravel()
            s_dist = np.unique(np.round(s_all / p * 2 * (S + 1)) * p / (2 * (S + 1)))
            for arr, sub in ((s_all, True), (s_dist, False)):
                fx = -arr[:, None] * st + t[None, :] * ct + c
                fy = arr[:, None] * ct + t[None, :] * st + c
                ok = (np.floor(fx) >= -1) & (np.floor(fx) <= n - 1) & (np.floor(fy) >= -1) & (np.floor(fy) <= n - 1)
                if sub:
                    total_sub += int(ok.sum())
                else:
                    total_distinct += int(ok.sum())
    return {"sub_ray_samples": total_sub, "distinct_ray_samples": total_distinct}


def _in_grid_samples(n, na, nd, S) -> int:
    """In-grid samples of all sub-rays of one pass (host count from the geometry)."""
    nbk = 2 if nd == 182 else 1
    nb = nd // nbk
    r = n / math.sqrt(2.0)
    p = 2 * r / nb
    T = math.ceil(2 * r)
    c = 0.5 * (n - 1)
    t = -r + (np.arange(T) + 0.5)
    u = np.array([(k - (S - 1) / 2) * 2 * p / (S + 1) for k in range(S)])
    tot = 0
    for a in range(na):
        for b in range(nbk):
            psi = 2 * math.pi * a / na + b * math.pi
            ct, st = math.cos(psi), math.sin(psi)
            s = (((np.arange(nb) - 0.5 * (nb - 1) + 0.5 * b) * p)[:, None] + u[None, :]).ravel()
            fx = np.floor(-s[:, None] * st + t[None, :] * ct + c)
            fy = np.floor(s[:, None] * ct + t[None, :] * st + c)
            tot += int(((fx >= -1) & (fx <= n - 1) & (fy >= -1) & (fy <= n - 1)).sum())
    return tot


def _stored_oracle(path: str):
    """The oracle's stored reconstructions of the first precision-stress items, if present
    (written by tests/golden/make_stress512.py, which calls only the oracle)."""
    if not path or not os.path.exists(path + ".npz"):
        return None
    z = np.load(path + ".npz")
    with open(path + ".json") as fh:
        meta = json.load(fh)
    return z, meta


def stress512(k: int, oracle_path: str = "") -> dict:
    n, na, nd, S = 512, 720, 182, 9
    g = P.geometry(n, na, nd, n_sub=S)
    stored = _stored_oracle(oracle_path)
    n_stored = len(stored[1]["items"]) if stored else 0
    precs = (("f32", P.PGET_F32), ("f32_kahan", P.PGET_F32_KAHAN), ("f64", P.PGET_F64))
    res = {name: [] for name, _ in precs}
    ms = {name: [] for name, _ in precs}
    per = []
    with P.Context(0) as ctx:
        for i in range(k):
            ph = synth.lattice_phantom(n, 17, radius=10.0, seed=1500 + i, mu_rod=(0.05, 0.12))
            lam64 = torch.tensor(ph.lam, device="cuda")
            mu64 = torch.tensor(ph.mu, device="cuda")
            yc = P.pget_forward(ctx, g, P.PGET_F64, lam64, mu64)
            if i < n_stored:  # the oracle's data for this item (its forward model, stored counts)
                z, meta = stored
                y_or = z[f"counts{i}"].astype(np.float64) * float(z[f"ymax{i}"]) / meta["case"]["counts"]
            y64 = torch.tensor(synth.poisson_noise(yc.cpu().numpy(), 1e6, 2500 + i), device="cuda")
            if i < n_stored:
                y64 = torch.tensor(y_or, device="cuda")
            r64 = (yc - y64).contiguous()
            ops = {}
            for name, prec in precs:
                dt = P.dtype_of(prec)
                lam, mu, r = lam64.to(dt), mu64.to(dt), r64.to(dt)
                sino = P.pget_forward(ctx, g, prec, lam, mu)
                gl, gm = P.pget_vjp(ctx, g, prec, lam, mu, r)
                ops[name] = (sino, torch.cat([gl.ravel(), gm.ravel()]))
                p = P.default_params(max_iters=10, cg_max_iters=30, cg_rel_tol=1e-6 if dt == torch.float32 else 1e-10,
                                     mu_max=0.25, precision=prec)
                y = y64.to(dt)
                if i == 0:
                    _timed_solve(ctx, g, p, y)  # warm-up per precision
                t, l_, m_, rep = _timed_solve(ctx, g, p, y)
                ms[name].append(t)
                res[name].append(torch.cat([l_.ravel(), m_.ravel()]))
            item = {"seed": 1500 + i}
            for name in ("f32", "f32_kahan"):
                item[name] = {"sinogram": _rel(ops[name][0], ops["f64"][0]),
                              "gradient": _rel(ops[name][1], ops["f64"][1]),
                              "reconstruction": _rel(res[name][-1], res["f64"][-1])}
            if i < n_stored:  # each GPU reconstruction against the oracle's, same data
                z, meta = stored
                u_or = torch.tensor(np.concatenate([z[f"lam{i}"].ravel(), z[f"mu{i}"].ravel()]).astype(np.float64),
                                    device="cuda")
                item["vs_oracle"] = {name: _rel(res[name][-1], u_or) for name, _ in precs}
                item["oracle_rel_err_truth"] = {"lambda": meta["items"][i]["rel_err_truth_lambda"],
                                                "mu": meta["items"][i]["rel_err_truth_mu"]}
            per.append(item)
    return {"config": "precision stress: 512x512, 17x17 rods r=10, rod mu ~ U(0.05,0.12), 720 x 182 x 9, "
                      "Poisson 1e6, 10 LM x CG<=30, box mu <= 0.25",
            "oracle_items": n_stored,
            "reconstructions": k,
            "recon_per_s": {name: round(1e3 * len(v) / sum(v), 3) for name, v in ms.items()},
            "rel_l2_vs_f64_gpu": per}


OPS = {"ops128": dict(n=128, n_lat=9, radius=5.0, n_angles=360, n_det=182, n_sub=5),
       "ops512": dict(n=512, n_lat=17, radius=10.0, n_angles=720, n_det=182, n_sub=9),
       "ops256": dict(n=256, n_lat=17, radius=5.0, n_angles=360, n_det=182, n_sub=5),
       "ops64": dict(n=64, n_lat=9, radius=3.0, n_angles=90, n_det=91, n_sub=1, precision=0)}


def ops(k: int, name: str, op: str = "all", prec: int | None = None) -> dict:
    c = OPS[name]
    prec = c.get("precision", P.PGET_F32_KAHAN) if prec is None else prec
    dt = P.dtype_of(prec)
    ph = synth.lattice_phantom(c["n"], c["n_lat"], radius=c["radius"], seed=1)
    g = P.geometry(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"])
    t = lambda x: torch.tensor(x, dtype=dt, device="cuda")
    lam, mu = t(ph.lam), t(ph.mu)
    rs = np.random.default_rng(0)
    dl, dm = t(rs.standard_normal(ph.lam.shape)), t(0.01 * rs.standard_normal(ph.lam.shape))
    samples = samples_per_launch(c)["distinct_ray_samples"]
    out = {"config": f"operators: {c['n']}x{c['n']}, {c['n_angles']} x {c['n_det']} x {c['n_sub']}",
           "precision": prec, "launches": k}
    with P.Context(0) as ctx:
        y = P.pget_forward(ctx, g, prec, lam, mu)
        r = t(rs.standard_normal(tuple(y.shape)))
        calls = {"forward": lambda: P.pget_forward(ctx, g, prec, lam, mu, y),
                 "jvp": lambda: P.pget_jvp(ctx, g, prec, lam, mu, dl, dm),
                 "vjp": lambda: P.pget_vjp(ctx, g, prec, lam, mu, r)}
        for nm, fn in calls.items():
            if op not in ("all", nm):
                continue
            fn()  # warm-up
            P.pget_profile_enable(ctx, True)
            for _ in range(k):
                fn()
            torch.cuda.synchronize()
            prof = P.pget_profile_read(ctx)
            P.pget_profile_enable(ctx, False)
            P.pget_operator_status(ctx)
            out[nm] = {kk: {"avg_us": round(1e3 * v["total_ms"] / v["launches"], 2), "launches": v["launches"]}
                       for kk, v in prof.items() if v["launches"]}
            walk = out[nm].get("walk_" + nm)
            if walk:
                walk["distinct_ray_samples_per_s"] = round(samples / (walk["avg_us"] * 1e-6), 1)
    out["distinct_ray_samples_per_launch"] = samples
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", required=True, choices=["plain64", "diff256", "stress512", *OPS])
    ap.add_argument("--count", type=int, default=0)
    ap.add_argument("--op", default="all", choices=["all", "forward", "jvp", "vjp"])
    ap.add_argument("--oracle", default=os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                     "tests", "golden", "stress512"),
                    help="stored oracle reconstructions of the first stress512 items (prefix of .npz/.json)")
    a = ap.parse_args()
    build.build()
    if a.config in OPS:
        print(json.dumps(ops(a.count or 20, a.config, a.op)), flush=True)
        return
    if a.config == "stress512":
        print(json.dumps(stress512(a.count or 4, a.oracle)), flush=True)
        return
    fn, k0 = {"plain64": (plain64, 16), "diff256": (diff256, 32)}[a.config]
    print(json.dumps(fn(a.count or k0)), flush=True)


if __name__ == "__main__":
    main()

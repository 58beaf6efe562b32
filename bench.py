"""Benchmark: Levenberg-Marquardt PGET reconstructions per second on GB300.

Workload (one "step" = one full reconstruction through the C ABI):
  128 x 128 grid, 9 x 9 rod lattice (pitch 14, r = 5 px), lambda ~ U(0.5, 1.5) per rod with
  10% of rods non-emitting, mu = 0.08 px^-1 in rods / 0.01 elsewhere; 360 angles over
  360 degrees x 182 detectors (two opposed banks of 91) x 5 triangular sub-rays; Poisson
  noise at 1e5 counts in the brightest bin; initial guess + 20 LM iterations with CG
  capped at 30 steps; FP32 ray sums with Kahan compensation, FP64 CG scalars.
Every step reconstructs a different seeded phantom; data are generated before timing and
stay resident in HBM.  L2 is flushed (256 MB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pget|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank reconstructs its own
requests (weak scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=128, n_lat=9, radius=5.0, n_angles=360, n_det=182, n_sub=5, collimator=1,
                counts=1e5, max_iters=20, cg_max_iters=30)
WORKLOAD_NAME = ("single-request LM: 128x128 grid, 9x9 rods r=5, 360 angles x 182 det (2 banks) "
                 "x 5 triangular sub-rays, Poisson 1e5, 20 LM x 30 CG, FP32-Kahan rays / FP64 scalars")
METRIC = "recon/s"
# precisions whose reconstruction of the oracle-stored case is compared with the oracle
PRECISIONS_CHECKED = (("f32_kahan", 2), ("mixed", 3), ("f64", 0))
SUB = (16, 16)

# DRAM bytes (read + write) and shared-memory wavefronts (all, and those from bank
# conflicts) per launch of the dominant kernel from one ncu capture of the adjoint walk on
# this workload, valid only for the kernel code it was taken on: reported while the device
# code of csrc/walk.cu (the part before its host section) and csrc/kernels.cuh, without
# comments, blank lines and includes, hash to these values; null otherwise.
TRAFFIC = {"walk_vjp": {"bytes": 3036416 + 33065728, "smem_wavefronts": 41371717, "smem_conflicts": 14797675,
                        "walk.cu": "0217d75420bb33a71616afaea2fa0963289773a5c05e4db921509f354eeca477",
                        "kernels.cuh": "96cb443f5a2135cf26f2465870fa9ed91417abbaf763465a89b14aeb64a58982"}}


def _device_code_hash(path: str, split: str | None = None) -> str:
    import hashlib
    import re
    with open(path) as fh:
        src = fh.read()
    if split:
        src = src.split(split)[0]
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    lines = [ln.strip() for ln in src.split("\n") if ln.strip() and not ln.strip().startswith("#include")]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def captured_traffic(kernel: str):
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    csrc = os.path.join(ROOT, "paper_2604_26745_gb300", "csrc")
    if _device_code_hash(os.path.join(csrc, "walk.cu"), "static int smem_pitch(") != t["walk.cu"]:
        return None
    if _device_code_hash(os.path.join(csrc, "kernels.cuh")) != t["kernels.cuh"]:
        return None
    return t


def workload_config(world: int) -> dict:
    """The config object of both arms' JSON lines: the workload and its sizes."""
    return {"workload": WORKLOAD_NAME, "parallelism": f"replicas x{world}",
            "l2": "flushed between timed steps (256 MB write)", **dict(WORKLOAD)}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pget", choices=["pget", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dist-timeout", type=float, default=300.0,
                    help="seconds a collective waits for the other ranks before it fails")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def init_dist(backend: str, timeout_s: float, **kw):
    """The process group of a multi-rank run, with a bounded timeout: a rank that dies or
    never arrives makes the others' next collective fail after timeout_s instead of
    hanging.  Ranks leave only between steps, with none of their kernels in flight."""
    import datetime

    import torch.distributed as dist
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s), **kw)
    return dist


def rank_request_ids(rank: int, world: int, per_rank: int) -> list:
    """Phantom seeds of the requests one rank reconstructs (disjoint across ranks)."""
    return [rank * per_rank + k for k in range(per_rank)]


def make_problem(P, ctx, torch, seed: int, device: str):
    from paper_2604_26745_gb300 import synth
    W = WORKLOAD
    ph = synth.lattice_phantom(W["n"], W["n_lat"], radius=W["radius"], seed=1100 + seed)
    g = P.geometry(W["n"], W["n_angles"], W["n_det"], n_sub=W["n_sub"], collimator=W["collimator"])
    lam = torch.tensor(ph.lam, dtype=torch.float64, device=device)
    mu = torch.tensor(ph.mu, dtype=torch.float64, device=device)
    y_clean = P.pget_forward(ctx, g, P.PGET_F64, lam, mu)
    y = synth.poisson_noise(y_clean.cpu().numpy(), W["counts"], 2100 + seed)
    return g, ph, y


def cpu_baseline(y, g_dims) -> dict:
    """The FP64 oracle as it stands, on this host's cores: one LM iteration (of 20) of one
    reconstruction of the same workload on all cores, recon/s scaled by 20 iterations; and
    one forward, one JVP and one adjoint pass on a single thread, scaled by the passes of
    one reconstruction."""
    from oracle import oracle as O
    import numpy as np
    W = WORKLOAD
    go = O.geom(W["n"], W["n_angles"], W["n_det"], n_sub=W["n_sub"], collimator=W["collimator"])
    pr = O.default_params(max_iters=1, cg_max_iters=W["cg_max_iters"], cg_rel_tol=1e-6)
    t0 = time.perf_counter()
    l0, m0 = O.initial_guess(go, y)
    O.lm(go, pr, y, l0, m0)
    dt = time.perf_counter() - t0
    per_recon = dt * W["max_iters"]
    out = {"value": 1.0 / per_recon, "unit": METRIC, "cores": O.num_threads(), "kind": "oracle",
           "sample": f"initial guess + 1 of {W['max_iters']} LM iterations (30 CG steps) of one "
                     f"reconstruction, {dt:.2f} s, scaled x{W['max_iters']}"}
    # single thread: per pass, then the passes of one reconstruction (initial guess: 2
    # forward; per iteration: gradient adjoint, 30 CG steps of JVP + adjoint, the trial's
    # JVP and forward), vector work neglected
    O.set_num_threads(1)
    try:
        r = np.asarray(y) - O.forward(go, l0, m0)
        t0 = time.perf_counter()
        O.forward(go, l0, m0)
        t_f = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.jvp(go, l0, m0, l0, m0)
        t_j = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.vjp(go, l0, m0, r)
        t_v = time.perf_counter() - t0
    finally:
        O.set_num_threads(0)
    it, cg = W["max_iters"], W["cg_max_iters"]
    n_f, n_j, n_v = 2 + it, 1 + it * (cg + 1), 1 + it * (cg + 1)
    t1 = n_f * t_f + n_j * t_j + n_v * t_v
    out["single_thread"] = {"value": 1.0 / t1, "unit": METRIC, "cores": 1, "kind": "oracle",
                            "sample": f"1 forward ({t_f:.2f} s), 1 JVP ({t_j:.2f} s), 1 adjoint ({t_v:.2f} s) "
                                      f"on one thread, scaled by the {n_f} + {n_j} + {n_v} passes of one "
                                      f"reconstruction"}
    return out


def accuracy_vs_oracle(P, ctx, torch, dev: str) -> dict | None:
    """GPU reconstructions of the oracle's stored single-request case (the same workload,
    phantom seed 1100, data from the oracle's forward model with the stored Poisson
    counts) against the oracle's own FP64 reconstruction, and the oracle's spread under
    changes of its rounding alone (both written by tests/golden/make_lm_single128.py)."""
    import numpy as np
    from paper_2604_26745_gb300 import synth
    base = os.path.join(ROOT, "tests", "golden", "lm_single128")
    if not (os.path.exists(base + ".npz") and os.path.exists(base + ".json")):
        return None
    z = np.load(base + ".npz")
    with open(base + ".json") as fh:
        meta = json.load(fh)
    c = meta["case"]
    y = z["counts"].astype(np.float64) * float(z["ymax"]) / c["counts"]
    ref = np.concatenate([z["lam"].ravel(), z["mu"].ravel()])
    ph = synth.lattice_phantom(c["n"], c["n_lat"], radius=c["radius"], seed=c["phantom_seed"])
    g = P.geometry(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"], collimator=c["collimator"])
    out = {"case": "oracle-stored single request (phantom seed 1100), " + WORKLOAD_NAME,
           "oracle_self_spread_rel_l2_max": meta["spread_max_rel_l2_u"],
           "oracle_self_spread_rel_l2_median": meta["spread_median_rel_l2_u"],
           "oracle_rel_err_truth_lambda": meta["base"]["rel_err_truth_lambda"],
           "oracle_rel_err_truth_mu": meta["base"]["rel_err_truth_mu"],
           "initial_rel_err_truth_mu": meta["base"]["initial_rel_err_truth_mu"],
           "oracle_accepted": meta["base"]["accepted"]}
    for name, prec in PRECISIONS_CHECKED:
        p = P.default_params(max_iters=c["max_iters"], cg_max_iters=c["cg_max_iters"], cg_rel_tol=c["cg_rel_tol"],
                             precision=prec)
        dt = P.dtype_of(prec)
        yd = torch.tensor(y, dtype=dt, device=dev)
        lam, mu = P.pget_initial_guess(ctx, g, p, yd)
        rep = P.pget_lm_solve(ctx, g, p, yd, lam, mu)
        u = np.concatenate([lam.double().cpu().numpy().ravel(), mu.double().cpu().numpy().ravel()])
        out[f"gpu_{name}_vs_oracle_rel_l2"] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
        out[f"gpu_{name}_rel_err_truth_mu"] = float(np.linalg.norm(mu.double().cpu().numpy() - ph.mu)
                                                   / np.linalg.norm(ph.mu))
        out[f"gpu_{name}_accepted"] = rep["acc"]
    return out


# ------------------------------------------------------------------ reference
def run_reference(args, rank: int):
    """The CPU oracle timed as the reference arm: every step is one LM iteration of one
    reconstruction of the same workload (bounded sample), reported as recon/s."""
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    from paper_2604_26745_gb300 import synth
    W = WORKLOAD
    go = O.geom(W["n"], W["n_angles"], W["n_det"], n_sub=W["n_sub"], collimator=W["collimator"])
    ph = synth.lattice_phantom(W["n"], W["n_lat"], radius=W["radius"], seed=1100)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), W["counts"], 2100)
    pr = O.default_params(max_iters=1, cg_max_iters=W["cg_max_iters"], cg_rel_tol=1e-6)
    l0, m0 = O.initial_guess(go, y)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.lm(go, pr, y, l0, m0)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    per_iter = sum(times) / len(times)
    value = 1.0 / (per_iter * W["max_iters"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"each step = 1 of {W['max_iters']} LM iterations of one reconstruction; "
                                       f"recon/s = 1 / ({W['max_iters']} x mean step time)"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- product
def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    import numpy as np
    import torch
    from paper_2604_26745_gb300 import build, pget as P
    build.build()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = None
    if world > 1:
        dist = init_dist("nccl" if torch.cuda.is_available() else "gloo", args.dist_timeout)
    W = WORKLOAD
    ctx = P.Context(local)
    prec = P.PGET_F32_KAHAN
    p = P.default_params(max_iters=W["max_iters"], cg_max_iters=W["cg_max_iters"], cg_rel_tol=1e-6,
                         precision=prec)
    nsteps = args.warmup + args.steps
    probs = []
    for k in rank_request_ids(rank, world, nsteps):
        g, ph, y = make_problem(P, ctx, torch, k, dev)
        probs.append((g, ph, torch.tensor(y, dtype=torch.float32, device=dev)))
    lam = torch.empty((W["n"], W["n"]), dtype=torch.float32, device=dev)
    mu = torch.empty_like(lam)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reps = []
    # warm-up (untimed)
    for k in range(args.warmup):
        g, ph, yd = probs[k]
        l0, m0 = P.pget_initial_guess(ctx, g, p, yd)
        P.pget_lm_solve(ctx, g, p, yd, l0, m0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    P.pget_profile_enable(ctx, False)  # the timed region runs the plain graph (no event nodes)
    launches0 = P.pget_launch_count()
    torch.cuda.synchronize()
    for i in range(args.steps):
        g, ph, yd = probs[args.warmup + i]
        flush.fill_(float(i))  # between timed steps, outside the events
        ev[i][0].record(stream)
        l0, m0 = P.pget_initial_guess(ctx, g, p, yd)
        reps.append(P.pget_lm_solve(ctx, g, p, yd, l0, m0))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = P.pget_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        total_s = float(t.item())
    value = world * args.steps / total_s

    # per-kernel device times: a separate, untimed pass over the same steps with CUDA events
    # recorded around every hot kernel on its launching stream (they become event nodes of
    # the captured graph; the headline above runs without them)
    P.pget_profile_enable(ctx, True)
    prof_ms = []
    for i in range(args.steps):
        g, ph, yd = probs[args.warmup + i]
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        l0, m0 = P.pget_initial_guess(ctx, g, p, yd)
        P.pget_lm_solve(ctx, g, p, yd, l0, m0)
        b.record(stream)
        prof_ms.append((a, b))
    torch.cuda.synchronize()
    prof = P.pget_profile_read(ctx)
    P.pget_profile_enable(ctx, False)
    prof_step_ms = [a.elapsed_time(b) for a, b in prof_ms]

    # end to end through the host-buffer entry point (pinned buffers, copies inside)
    e2e = None
    if not args.no_e2e:
        yh = [probs[args.warmup + i][2].cpu().pin_memory() for i in range(args.steps)]
        lh = torch.empty((W["n"], W["n"]), dtype=torch.float32).pin_memory()
        mh = torch.empty_like(lh).pin_memory()
        g = probs[0][0]
        P.pget_lm_solve_host(ctx, g, p, yh[0], lh, mh, True)  # warm
        torch.cuda.synchronize()
        ee = []
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P.pget_lm_solve_host(ctx, g, p, yh[i], lh, mh, True)
            ee.append(time.perf_counter() - t0)
        e_total = sum(ee)
        if dist:
            t = torch.tensor([e_total], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_total = float(t.item())
        e2e = {"value": world * args.steps / e_total, "unit": METRIC,
               "h2d_bytes_per_step": int(yh[0].numel() * 4), "d2h_bytes_per_step": int(2 * lh.numel() * 4),
               "timing": "host wall clock around pget_lm_solve_host (which synchronises)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # accuracy: the reconstruction of the oracle-stored case against the oracle's own, and
    # the first timed reconstruction against its phantom
    g, ph, yd = probs[args.warmup]
    acc = accuracy_vs_oracle(P, ctx, torch, dev) or {"oracle_case": "tests/golden/lm_single128.* missing"}
    l0, m0 = P.pget_initial_guess(ctx, g, p, yd)
    P.pget_lm_solve(ctx, g, p, yd, l0, m0)
    acc["first_timed_rel_err_truth_lambda"] = float(np.linalg.norm(l0.double().cpu().numpy() - ph.lam)
                                                    / np.linalg.norm(ph.lam))
    acc["first_timed_rel_err_truth_mu"] = float(np.linalg.norm(m0.double().cpu().numpy() - ph.mu)
                                                / np.linalg.norm(ph.mu))
    acc["first_timed_f0"], acc["first_timed_f_final"] = reps[0]["f0"], reps[0]["f_final"]
    acc["first_timed_accepted"] = reps[0]["accepted"]

    # roofline of the dominant kernel: algorithmic on-chip bytes per launch / measured time
    from paper_2604_26745_gb300.config_bench import samples_per_launch
    counts = samples_per_launch(dict(n=W["n"], n_angles=W["n_angles"], n_det=W["n_det"], n_sub=W["n_sub"]))
    bytes_per_sample = {"walk_forward": 32, "walk_jvp": 64, "walk_vjp": 64}
    dom = max(prof, key=lambda k: prof[k]["total_ms"])
    kern = {}
    sm_mhz = clk.get("sm_mhz") or 1432.0
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    smem_peak = n_sm * 128 * sm_mhz * 1e6 / 1e9  # GB/s: SMs x 128 B/clk at the sampled clock
    for k, v in prof.items():
        if v["launches"] == 0:
            continue
        avg_ms = v["total_ms"] / v["launches"]
        d = {"launches": v["launches"], "total_ms": round(v["total_ms"], 3), "avg_us": round(avg_ms * 1e3, 2),
             "share_of_step": round(v["total_ms"] / (sum(prof_step_ms)), 4)}
        if k in bytes_per_sample:
            d["achieved_gbs"] = bytes_per_sample[k] * counts["distinct_ray_samples"] / (avg_ms * 1e-3) / 1e9
        kern[k] = d
    dk = dom if dom in bytes_per_sample else max((k for k in kern if k in bytes_per_sample),
                                                 key=lambda k: kern[k]["total_ms"])
    achieved = kern[dk]["achieved_gbs"]
    cap = captured_traffic(dk)
    traffic = cap["bytes"] if cap else None
    smem_pipe = None
    if cap and "smem_wavefronts" in cap:
        wb = 128 * cap["smem_wavefronts"]
        got = wb / (kern[dk]["avg_us"] * 1e-6) / 1e9
        smem_pipe = {"wavefront_bytes": wb, "conflict_wavefronts": cap["smem_conflicts"],
                     "achieved_gbs": round(got, 1), "frac": round(got / smem_peak, 4),
                     "note": "ncu shared-memory wavefronts x 128 B per launch (bank conflicts included) over the "
                             "live launch time, against the same peak: the traffic the pipe actually serves"}
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm_peak = float(json.load(fh)["hbm_gbs"])
        if traffic:
            got = traffic / (kern[dk]["avg_us"] * 1e-6) / 1e9
            hbm = {"achieved_gbs": round(got, 1), "peak_gbs": hbm_peak, "frac": round(got / hbm_peak, 4),
                   "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
                   "note": "DRAM bytes of the captured kernel / its live launch time; the path is not HBM-bound"}
    except (OSError, KeyError, ValueError):
        pass
    roof = {"kernel": dk, "bound": "smem", "achieved": round(achieved, 1), "peak": round(smem_peak, 1),
            "unit": "GB/s", "frac": round(achieved / smem_peak, 4), "traffic": traffic,
            "traffic_unit": "DRAM bytes read + written per launch (ncu)", "hbm": hbm, "smem_pipe": smem_pipe,
            "peak_source": f"derived: {n_sm} SMs x 128 B/clk shared-memory bandwidth x median sampled SM clock",
            "timing": "average launch time from CUDA events on the launching stream, in an untimed pass "
                      "over the same steps (the headline pass runs without events)",
            "algorithmic_bytes_per_launch": bytes_per_sample[dk] * counts["distinct_ray_samples"],
            "units_per_launch": counts["distinct_ray_samples"],
            "unit_desc": "in-grid samples of distinct rays (sub-rays sharing a line are one ray)"}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(sum(step_ms) / len(step_ms), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(world),
        "latency_ms": {"p50": round(statistics.median(step_ms), 3),
                       "p99": round(sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)], 3)},
        "accuracy": acc,
        "roofline": roof, "kernels": kern, "gpu_launches": int(launches),
        "profiled_pass_ms_per_step": round(sum(prof_step_ms) / len(prof_step_ms), 3),
        "clocks": clk, "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(probs[args.warmup][2].cpu().double().numpy(), None)
        except Exception as ex:  # reported, never fatal
            line["cpu_baseline"] = {"error": str(ex)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Serving path (pget_submit / pget_poll): continuous admission of reconstructions of
uneven sizes into in-flight slots whose work overlaps on the GPU.

- every result in a mix of concurrent requests equals the same request solved alone
  (bitwise: the kernels are deterministic and slots share no state);
- admission: PGET_EAGAIN when all slots are busy or the memory budget is held by
  in-flight requests, PGET_ENOMEM when a request can never fit;
- unknown tickets, double polls and cancellation are reported, never fatal.
"""
import time

import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

MIX = [  # (n, n_lat, n_angles, n_sub, counts)
    (48, 4, 60, 3, 1e4),
    (64, 5, 90, 5, 1e5),
    (40, 4, 45, 4, 1e6),
    (56, 5, 72, 7, 3e4),
    (48, 4, 60, 3, 2e5),
]


def _request(P, torch, k, prec=2):
    n, nl, na, S, counts = MIX[k % len(MIX)]
    g = P.geometry(n, na, 182, n_sub=S)
    ph = synth.lattice_phantom(n, nl, radius=2.0, seed=300 + k)
    with P.Context(0) as c:
        y_clean = P.pget_forward(c, g, P.PGET_F64, torch.tensor(ph.lam, device="cuda"),
                                 torch.tensor(ph.mu, device="cuda"))
    y = synth.poisson_noise(y_clean.cpu().numpy(), counts, 400 + k)
    return g, torch.tensor(y, dtype=P.dtype_of(prec), device="cuda")


def _wait(P, ctx, ticket, lam, mu, timeout=120.0):
    t0 = time.time()
    while True:
        done, rep = P.pget_poll(ctx, ticket, lam, mu)
        if done:
            return rep
        assert time.time() - t0 < timeout
        time.sleep(0.001)


def test_mixed_results_equal_alone(P, torch):
    p = P.default_params(max_iters=4, cg_max_iters=10, precision=P.PGET_F32_KAHAN)
    reqs = [_request(P, torch, k) for k in range(len(MIX))]
    alone = []
    with P.Context(0) as c:
        for g, y in reqs:
            lam, mu = P.pget_initial_guess(c, g, p, y)
            rep = P.pget_lm_solve(c, g, p, y, lam, mu)
            alone.append((lam.clone(), mu.clone(), rep["f"]))
    with P.Context(0) as ctx:
        tickets = [P.pget_submit(ctx, g, p, y) for g, y in reqs]
        assert P.pget_inflight(ctx) == len(reqs)
        outs = []
        for t, (g, y) in zip(tickets, reqs):
            lam = torch.empty((g.n, g.n), device="cuda")
            mu = torch.empty_like(lam)
            rep = _wait(P, ctx, t, lam, mu)
            outs.append((lam, mu, rep["f"]))
        assert P.pget_inflight(ctx) == 0
    for (la, ma, fa), (lb, mb, fb) in zip(alone, outs):
        assert torch.equal(la, lb) and torch.equal(ma, mb) and fa == fb


def test_continuous_admission_and_slot_reuse(P, torch, monkeypatch):
    """Two slots, six requests: the third waits (EAGAIN) until a poll frees a slot; the
    order of completion does not change any result."""
    monkeypatch.setenv("PGET_MAX_INFLIGHT", "2")
    p = P.default_params(max_iters=3, cg_max_iters=8, precision=P.PGET_F32_KAHAN)
    reqs = [_request(P, torch, k) for k in range(6)]
    ref = []
    with P.Context(0) as c:
        for g, y in reqs:
            lam, mu = P.pget_initial_guess(c, g, p, y)
            P.pget_lm_solve(c, g, p, y, lam, mu)
            ref.append(lam.clone())
    with P.Context(0) as ctx:
        pending, results, saw_eagain = {}, {}, False
        nxt = 0
        while len(results) < len(reqs):
            while nxt < len(reqs):
                g, y = reqs[nxt]
                try:
                    pending[P.pget_submit(ctx, g, p, y)] = nxt
                    nxt += 1
                except P.PgetError as e:
                    assert e.status == P.PGET_EAGAIN
                    saw_eagain = True
                    break
            for t, k in list(pending.items()):
                g, _ = reqs[k]
                lam = torch.empty((g.n, g.n), device="cuda")
                done, rep = P.pget_poll(ctx, t, lam, None)
                if done:
                    results[k] = lam
                    del pending[t]
        assert saw_eagain
    for k in range(len(reqs)):
        assert torch.equal(results[k], ref[k])


def test_memory_budget_admission(P, torch):
    p = P.default_params(max_iters=2, cg_max_iters=5, precision=P.PGET_F32_KAHAN)
    g, y = _request(P, torch, 1)
    with P.Context(0, mem_budget_bytes=1 << 20) as tiny:
        with pytest.raises(P.PgetError) as e:
            P.pget_submit(tiny, g, p, y)
        assert e.value.status == P.PGET_ENOMEM
    # a budget that holds one request of this size but not two
    with P.Context(0) as probe:
        t = P.pget_submit(probe, g, p, y)
        _wait(P, probe, t, None, None)
    with P.Context(0, mem_budget_bytes=60 << 20) as ctx:
        t1 = P.pget_submit(ctx, g, p, y)
        g2, y2 = _request(P, torch, 3)  # a different geometry needs its own workspace
        try:
            t2 = P.pget_submit(ctx, g2, p, y2)
            second = True
        except P.PgetError as e:
            assert e.value.status == P.PGET_EAGAIN
            second = False
        _wait(P, ctx, t1, None, None)
        if second:
            _wait(P, ctx, t2, None, None)
        else:  # admitted once the first request has been collected
            t2 = P.pget_submit(ctx, g2, p, y2)
            _wait(P, ctx, t2, None, None)


def test_tickets_and_cancel(P, torch):
    p = P.default_params(max_iters=2, cg_max_iters=5, precision=P.PGET_F32_KAHAN)
    g, y = _request(P, torch, 0)
    with P.Context(0) as ctx:
        with pytest.raises(P.PgetError) as e:
            P.pget_poll(ctx, 12345)
        assert e.value.status == P.PGET_ENOTFOUND
        t = P.pget_submit(ctx, g, p, y)
        P.pget_cancel(ctx, t)
        assert P.pget_inflight(ctx) == 0
        with pytest.raises(P.PgetError) as e:
            P.pget_poll(ctx, t)
        assert e.value.status == P.PGET_ENOTFOUND
        t = P.pget_submit(ctx, g, p, y)
        _wait(P, ctx, t, None, None)
        with pytest.raises(P.PgetError) as e:  # already collected
            P.pget_poll(ctx, t)
        assert e.value.status == P.PGET_ENOTFOUND
        with pytest.raises(P.PgetError) as e:
            P.pget_submit(ctx, P.geometry(1, 10, 91), p, y)
        assert e.value.status == P.PGET_EINVAL


def test_serving_with_the_method_options(P, torch):
    """Requests that use the optional parts of the method at once (gradient-projection
    inner solver, linear bound, geometry priors, alpha continuation, depth tables of
    Eq. (5)), mixed with a plain request, equal the same requests solved alone, bitwise;
    the depth tables are copied at submission (the caller's arrays are overwritten with NaN
    right after it)."""
    n, na, S = 40, 45, 3
    T = P.geometry_info(P.geometry(n, na, 182, n_sub=S))["n_samples"]
    jj = np.arange(T) / (T - 1)
    mask = torch.tensor(np.clip(synth.lattice_phantom(n, 4, radius=3.0, seed=5, zero_frac=0.0, mu_rod=1.0,
                                                      mu_bg=0.0).mu, 0.0, 1.0), dtype=torch.float32, device="cuda")
    opts = [dict(), dict(inner_solver=1, lin_constraint=1, lin_slope=14.0, lin_offset=0.0),
            dict(geo_mask=mask, geo_alpha_lambda=2.0, geo_alpha_mu=20.0, geo_mu_water=0.01, alpha_decay=5.0,
                 alpha_decay_iters=2, lin_constraint=1, lin_slope=20.0, lin_offset=0.05)]
    reqs = []
    for k, o in enumerate(opts):
        depth = dict(depth_w=list(0.7 + 0.3 * jj), depth_c=list(1.0 + 0.5 * (1.0 - jj) ** 2)) if k else {}
        g = P.geometry(n, na, 182, n_sub=S, **depth)
        ph = synth.lattice_phantom(n, 4, radius=2.0, seed=500 + k)
        with P.Context(0) as c:
            yc = P.pget_forward(c, g, P.PGET_F64, torch.tensor(ph.lam, device="cuda"), torch.tensor(ph.mu, device="cuda"))
        y = torch.tensor(synth.poisson_noise(yc.cpu().numpy(), 1e5, 600 + k), dtype=torch.float32, device="cuda")
        p = P.default_params(max_iters=4, cg_max_iters=8, precision=P.PGET_F32_KAHAN, **o)
        reqs.append((g, p, y))
    alone = []
    with P.Context(0) as c:
        for g, p, y in reqs:
            lam, mu = P.pget_initial_guess(c, g, p, y)
            rep = P.pget_lm_solve(c, g, p, y, lam, mu)
            alone.append((lam.clone(), mu.clone(), rep["f"]))
    with P.Context(0) as ctx:
        tickets = []
        for g, p, y in reqs:
            tickets.append(P.pget_submit(ctx, g, p, y))
            for tab in getattr(g, "_keep", []):  # the caller's tables are spoilt once submitted
                for i in range(len(tab)):
                    tab[i] = float("nan")
        outs = []
        for t, (g, p, y) in zip(tickets, reqs):
            lam = torch.empty((g.n, g.n), device="cuda")
            mu = torch.empty_like(lam)
            rep = _wait(P, ctx, t, lam, mu)
            outs.append((lam, mu, rep["f"]))
    for (la, ma, fa), (lb, mb, fb) in zip(alone, outs):
        assert torch.equal(la, lb) and torch.equal(ma, mb) and fa == fb

"""Safeguarded acceleration (Prop. conv_check, Alg. 2) on the GPU against the oracle.

- pget_lm_trial equals the oracle's trial (step, model and actual decrease, rho,
  acceptance, nu_0) in FP64 to rounding and in FP32-Kahan to single precision (CG <= 6
  steps: the stable regime where the iteration is a smooth function of its input);
- pget_proposal_check equals the oracle's check on the same step for the truth, a random
  perturbation, half the LM step and the LM step itself (same decisions, FP64 values to
  rounding);
- the driver of Alg. 2: without proposals it reproduces pget_lm_solve; proposing the
  truth near the solution is accepted in the first iteration; random proposals are never
  accepted and leave the plain LM iterates unchanged.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

N, NA, ND, S = 24, 30, 182, 3


def _setup(O, P, torch, seed=21, noise=1e4):
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=seed)
    go = O.geom(N, NA, ND, n_sub=S)
    y = O.forward(go, ph.lam, ph.mu)
    if noise:
        y = synth.poisson_noise(y, noise, seed + 1)
    return ph, go, P.geometry(N, NA, ND, n_sub=S), y


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("seed", [21, 25])  # first trial rejected (no model decrease) / accepted
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 2e-4)])
def test_trial_matches_oracle(O, P, torch, prec, tol, seed):
    ph, go, g, y = _setup(O, P, torch, seed=seed)
    pr = O.default_params(cg_max_iters=6)
    l0, m0 = O.initial_guess(go, y)
    so, to = O.lm_trial(go, pr, y, l0, m0)
    dt = P.dtype_of(prec)
    p = P.default_params(cg_max_iters=6, cg_rel_tol=1e-10, precision=prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    with P.Context(0) as c:
        s, tr = P.pget_lm_trial(c, g, p, t(y), t(l0), t(m0), 0.0)
    assert _rel(s.double().cpu().numpy(), so) <= tol
    for k in ("f", "pred", "ared", "rho", "nu0"):
        if np.isfinite(to[k]):
            assert abs(tr[k] - to[k]) <= tol * max(1.0, abs(to[k])), (k, tr[k], to[k])
        else:
            assert tr[k] == to[k], k
    assert tr["accept"] == to["accept"] and tr["cg_iters"] == to["cg_iters"]


def test_check_matches_oracle(O, P, torch):
    ph, go, g, y = _setup(O, P, torch, seed=23, noise=None)
    pr = O.default_params(cg_max_iters=6)
    rs = np.random.default_rng(5)
    lk = np.clip(ph.lam + 0.05 * rs.standard_normal(ph.lam.shape), 0, pr.lambda_max)
    mk = np.clip(ph.mu + 0.005 * rs.standard_normal(ph.mu.shape), 0, pr.mu_max)
    so, to = O.lm_trial(go, pr, y, lk, mk, 1e2)
    props = {"truth": (ph.lam, ph.mu),
             "noise": (lk + rs.uniform(-1, 1, lk.shape), mk + rs.uniform(-0.1, 0.1, mk.shape)),
             "half": (lk + 0.5 * so[0], mk + 0.5 * so[1]),
             "step": (lk + so[0], mk + so[1])}
    p = P.default_params(cg_max_iters=6, cg_rel_tol=1e-10, precision=0)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    seen = set()
    with P.Context(0) as c:
        for name, (pl, pm) in props.items():
            co = O.check_proposal(go, pr, y, lk, mk, so, pl, pm)
            cg = P.pget_proposal_check(c, g, p, t(y), t(lk), t(mk), t(so), t(pl), t(pm))
            assert cg["accept"] == co["accept"], name
            for k in ("f", "pred_step", "pred_prop", "ared_prop"):
                assert abs(cg[k] - co[k]) <= 1e-9 * max(1.0, abs(co[k])), (name, k)
            if np.isfinite(co["rho_prop"]):
                assert abs(cg["rho_prop"] - co["rho_prop"]) <= 1e-8, name
            else:
                assert cg["rho_prop"] == co["rho_prop"]
            seen.add((name, bool(co["accept"])))
    assert ("truth", True) in seen and ("noise", False) in seen


def test_driver(O, P, torch):
    from paper_2604_26745_gb300.accelerated import accelerated_solve
    ph, go, g, y = _setup(O, P, torch, seed=25, noise=None)
    p = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0)
    yd = torch.tensor(y, device="cuda")
    with P.Context(0) as c:
        l0, m0 = P.pget_initial_guess(c, g, p, yd)
        # no proposals: the plain LM solve
        la, ma, h = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), None)
        lb, mb = l0.clone(), m0.clone()
        rep = P.pget_lm_solve(c, g, p, yd, lb, mb)
        assert [x["took"] == "step" for x in h] == [bool(a) for a in rep["acc"]]
        assert float((la - lb).abs().max()) <= 1e-12 and float((ma - mb).abs().max()) <= 1e-12
        # the truth, proposed near the solution, is taken at once
        truth = torch.stack([torch.tensor(ph.lam, device="cuda"), torch.tensor(ph.mu, device="cuda")])
        gen1 = torch.Generator("cuda").manual_seed(1)
        near = truth + 0.02 * torch.randn(truth.shape, generator=gen1, device="cuda", dtype=truth.dtype)
        lt, mt, ht = accelerated_solve(c, g, p, yd, near[0].clone(), near[1].clone(),
                                       lambda u, s, k: truth if k == 0 else None)
        assert ht[0]["took"] == "proposal"
        # random proposals are never taken and do not change the LM iterates
        gen = torch.Generator("cuda").manual_seed(2)
        junk = lambda u, s, k: u + torch.rand(u.shape, generator=gen, device="cuda", dtype=u.dtype)
        lj, mj, hj = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), junk)
        assert all(x["took"] != "proposal" for x in hj)
        assert torch.equal(lj, la) and torch.equal(mj, ma)


def test_alpha_continuation_matches_oracle(O, P, torch):
    """Sec. 3.1's alpha / 5^k (halted after K iterations) in pget_lm_solve against the
    oracle LM with the same continuation (FP64, CG <= 6: the stable regime), and the Alg. 2
    driver without proposals against pget_lm_solve."""
    from paper_2604_26745_gb300.accelerated import accelerated_solve
    ph, go, g, y = _setup(O, P, torch, seed=27)
    pr = O.default_params(max_iters=5, cg_max_iters=6, alpha_decay=5.0, alpha_decay_iters=3)
    l0, m0 = O.initial_guess(go, y)
    lo, mo, ro = O.lm(go, pr, y, l0, m0)
    p = P.default_params(max_iters=5, cg_max_iters=6, cg_rel_tol=1e-10, precision=0, alpha_decay=5.0,
                         alpha_decay_iters=3)
    t = lambda a: torch.tensor(a, device="cuda")
    with P.Context(0) as c:
        lam, mu = t(l0), t(m0)
        rep = P.pget_lm_solve(c, g, p, t(y), lam, mu)
        la, ma, h = accelerated_solve(c, g, p, t(y), t(l0), t(m0), None)
    assert rep["acc"] == ro["acc"] and sum(ro["acc"]) >= 3
    assert _rel(lam.cpu().numpy(), lo) <= 1e-10 and _rel(mu.cpu().numpy(), mo) <= 1e-10
    for k in range(5):
        assert abs(rep["f"][k] - ro["f"][k]) <= 1e-10 * abs(ro["f"][k])
    assert [x["took"] == "step" for x in h] == [bool(a) for a in rep["acc"]]
    assert float((la - lam).abs().max()) <= 1e-12 and float((ma - mu).abs().max()) <= 1e-12
    # continuation off reproduces the fixed-alpha solve bitwise
    with P.Context(0) as c:
        outs = []
        for dec, K in ((1.0, 3), (5.0, 0)):
            pp = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0,
                                  alpha_decay=dec, alpha_decay_iters=K)
            lam, mu = t(l0), t(m0)
            P.pget_lm_solve(c, g, pp, t(y), lam, mu)
            outs.append((lam, mu))
        lam, mu = t(l0), t(m0)
        P.pget_lm_solve(c, g, P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0),
                        t(y), lam, mu)
    for a, b in outs:
        assert torch.equal(a, lam) and torch.equal(b, mu)


def test_driver_with_the_conv_proposal(O, P, torch):
    """Alg. 2 with the convolutional proposal operator of Sec. 3.3 (untrained): with all
    weights zero it proposes u itself (s~ = 0, no model decrease) and the scheme is the
    plain LM bitwise; with random weights every proposal it takes passed the check
    (rho(s~) > eta and m_k(s~) <= m_k(s_k))."""
    from paper_2604_26745_gb300.accelerated import accelerated_solve
    from paper_2604_26745_gb300.proposals import ConvProposal, as_proposal
    ph, go, g, y = _setup(O, P, torch, seed=25)
    p = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0)
    yd = torch.tensor(y, device="cuda")
    with P.Context(0) as c:
        l0, m0 = P.pget_initial_guess(c, g, p, yd)
        lb, mb, hb = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), None)
        zero = ConvProposal().cuda().double()
        for q in zero.parameters():
            torch.nn.init.zeros_(q)
        lz, mz, hz = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), as_proposal(zero))
        torch.manual_seed(0)
        net = ConvProposal().cuda().double()
        ln, mn, hn = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), as_proposal(net))
    assert all(x["took"] != "proposal" and x["check"] is not None for x in hz)
    assert torch.equal(lz, lb) and torch.equal(mz, mb)
    for x in hn:
        assert x["check"] is not None
        if x["took"] == "proposal":
            assert x["check"]["rho_prop"] > p.eta and x["check"]["pred_prop"] >= x["check"]["pred_step"]
    assert (ln >= 0).all() and (mn >= 0).all()


@pytest.mark.parametrize("case", ["truth", "noise", "none", "continuation"])
def test_step_with_proposal_matches_oracle(O, P, torch, case):
    """pget_lm_step_with_proposal (Alg. 2 after the trial, in the library): the check, the
    next iterate (P(u~), P(u + s) or u) and the clamped damping equal the oracle's check
    and projection on the same trial, FP64."""
    ph, go, g, y = _setup(O, P, torch, seed=23, noise=None)
    kw = dict(alpha_decay=5.0, alpha_decay_iters=3) if case == "continuation" else {}
    k = 2 if case == "continuation" else 0
    pr = O.params_at(O.default_params(cg_max_iters=6, **kw), k)
    rs = np.random.default_rng(5)
    lk = np.clip(ph.lam + 0.05 * rs.standard_normal(ph.lam.shape), 0, pr.lambda_max)
    mk = np.clip(ph.mu + 0.005 * rs.standard_normal(ph.mu.shape), 0, pr.mu_max)
    so, to = O.lm_trial(go, pr, y, lk, mk, 1e2)
    prop = {"truth": (ph.lam, ph.mu), "noise": (lk + rs.uniform(-1, 1, lk.shape), mk + rs.uniform(-0.1, 0.1, mk.shape)),
            "none": None, "continuation": (ph.lam, ph.mu)}[case]
    co = O.check_proposal(go, pr, y, lk, mk, so, *prop) if prop else None
    if co and co["accept"]:
        want = O.project(pr, *prop)
    elif to["accept"]:
        want = O.project(pr, lk + so[0], mk + so[1])
    else:
        want = (lk, mk)
    p = P.default_params(cg_max_iters=6, cg_rel_tol=1e-10, precision=0, **kw)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lam, mu = t(lk), t(mk)
    with P.Context(0) as c:
        pk = P.pget_params_at(p, k)
        assert abs(pk.alpha_lambda - pr.alpha_lambda) <= 1e-15 * pr.alpha_lambda
        s, tr = P.pget_lm_trial(c, g, pk, t(y), lam, mu, 1e2)
        st = P.pget_lm_step_with_proposal(c, g, p, k, t(y), lam, mu, s, tr, 7.0,
                                          *(t(a) for a in prop) if prop else (None, None))
    assert tr["accept"] == to["accept"]
    assert (st["check"] is None) == (co is None)
    if co:
        assert st["check"]["accept"] == co["accept"]
    assert st["took"] == ("proposal" if co and co["accept"] else ("step" if to["accept"] else "none"))
    assert _rel(lam.cpu().numpy(), want[0]) <= 1e-10 and _rel(mu.cpu().numpy(), want[1]) <= 1e-10
    assert st["nu_next"] == min(max(tr["nu_next"], p.nu_min * 7.0), p.nu_max * 7.0)
    if case == "truth":
        assert st["took"] == "proposal"

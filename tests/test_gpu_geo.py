"""Geometry priors of Eq. (6) (P1 lambda = (1 - M) lambda, P2 mu = (1 - M)(mu - mu_water)) on
the GPU against the oracle: the LM solve (FP64 to 1e-10, FP32-Kahan to 1e-4, CG <= 6 steps,
alone and with the alpha continuation, which scales these weights too), the CG solve, and
a mask of ones giving the prior-free solve bitwise."""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

N, NA, ND, S = 24, 30, 182, 3


def _setup(O, seed=31):
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=seed)
    go = O.geom(N, NA, ND, n_sub=S)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e4, seed + 1)
    mask = np.clip(synth.lattice_phantom(N, 3, radius=3.0, seed=seed, zero_frac=0.0, mu_rod=1.0, mu_bg=0.0).mu,
                   0.0, 1.0)
    return ph, go, y, mask


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("decay", [1.0, 5.0])
def test_lm_with_geometry_priors_matches_oracle(O, P, torch, prec, tol, decay):
    ph, go, y, mask = _setup(O)
    kw = dict(max_iters=4, cg_max_iters=6, geo_alpha_lambda=2.0, geo_alpha_mu=20.0, geo_mu_water=0.01,
              alpha_decay=decay, alpha_decay_iters=2)
    l0, m0 = O.initial_guess(go, y)
    lo, mo, ro = O.lm(go, O.default_params(geo_mask=mask, **kw), y, l0, m0)
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    p = P.default_params(precision=prec, cg_rel_tol=1e-10 if prec == 0 else 1e-6, geo_mask=t(mask), **kw)
    g = P.geometry(N, NA, ND, n_sub=S)
    with P.Context(0) as c:
        lam, mu = t(l0), t(m0)
        rep = P.pget_lm_solve(c, g, p, t(y), lam, mu)
    assert rep["acc"] == ro["acc"] and sum(ro["acc"]) >= 2
    assert _rel(lam.double().cpu().numpy(), lo) <= tol and _rel(mu.double().cpu().numpy(), mo) <= tol
    assert abs(rep["f_final"] - ro["f_final"]) <= tol * abs(ro["f_final"])


def test_cg_with_geometry_priors_matches_oracle(O, P, torch):
    ph, go, y, mask = _setup(O, seed=33)
    pr = O.default_params(cg_max_iters=8, geo_mask=mask, geo_alpha_lambda=0.5, geo_alpha_mu=5.0, geo_mu_water=0.01)
    lam, mu = ph.lam + 0.05, ph.mu
    Wl, Wm = O.reg_weights(lam, pr.tv_eps), O.reg_weights(mu, pr.tv_eps)
    b = np.random.default_rng(4).standard_normal((2, N, N))
    xo, it = O.cg(go, pr, lam, mu, Wl, Wm, 0.3, b)
    t = lambda a: torch.tensor(a, device="cuda")
    p = P.default_params(cg_max_iters=8, cg_rel_tol=1e-10, precision=0, geo_mask=t(mask), geo_alpha_lambda=0.5,
                         geo_alpha_mu=5.0, geo_mu_water=0.01)
    with P.Context(0) as c:
        x, itg = P.pget_cg_solve(c, P.geometry(N, NA, ND, n_sub=S), p, t(lam), t(mu), 0.3, t(b))
    assert itg == it and _rel(x.cpu().numpy(), xo) <= 1e-10


def test_mask_of_ones_is_the_prior_free_solve(O, P, torch):
    ph, go, y, mask = _setup(O, seed=35)
    l0, m0 = O.initial_guess(go, y)
    t = lambda a: torch.tensor(a, device="cuda")
    g = P.geometry(N, NA, ND, n_sub=S)
    outs = []
    with P.Context(0) as c:
        for geo in (None, np.ones_like(mask)):
            kw = {} if geo is None else dict(geo_mask=t(geo), geo_alpha_lambda=3.0, geo_alpha_mu=3.0,
                                              geo_mu_water=0.01)
            p = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0, **kw)
            lam, mu = t(l0), t(m0)
            P.pget_lm_solve(c, g, p, t(y), lam, mu)
            outs.append((lam, mu))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])

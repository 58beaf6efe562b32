"""Pins of the oracle's safeguarded acceleration check (Prop. conv_check and Alg. 2 of
Sec. 3.1) and of the single LM trial it is built on.

- the trial at (u_0, nu_0) is the first iteration of the (separately pinned) LM solver:
  same step, model decrease, actual decrease, rho, acceptance and damping update;
- a proposal equal to u + s_k reproduces the LM step's own rho (exact special case);
- closed form: A is linear in lambda for fixed mu and the quadratic prior is quadratic,
  so for a lambda-only proposal the Gauss-Newton model is exact and rho = 1;
- the model comparison: half the LM step has rho > eta but a larger model value than the
  full step (the undamped model keeps decreasing past the damped step), so it is
  rejected; a wrong direction of the comparison accepts it;
- proposals: the truth is accepted near the solution on noiseless data, a large random
  perturbation and the zero step are rejected, and a proposal outside the box is
  evaluated at its projection.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _case(O, n=16, na=12, nd=91, S=1, seed=3, noise=None):
    g = O.geom(n, na, nd, n_sub=S)
    ph = synth.lattice_phantom(n, 2, radius=2.0, seed=seed)
    y = O.forward(g, ph.lam, ph.mu)
    if noise:
        y = synth.poisson_noise(y, noise, seed + 100)
    return g, ph, y


@pytest.mark.parametrize("seed,S", [(3, 1), (4, 3)])
def test_trial_is_the_first_lm_iteration(O, seed, S):
    g, ph, y = _case(O, S=S, seed=seed, noise=1e4)
    pr = O.default_params(max_iters=1, cg_max_iters=6)
    l0, m0 = O.initial_guess(g, y)
    s, t = O.lm_trial(g, pr, y, l0, m0, 0.0)
    l1, m1, rep = O.lm(g, pr, y, l0, m0)
    assert t["nu0"] == rep["nu0"] and t["f"] == rep["f0"]
    for k in ("pred", "ared", "rho"):
        assert t[k] == rep[k][0]
    assert t["accept"] == rep["acc"][0] and t["nu_next"] == rep["nu"][0]
    if t["accept"]:
        assert np.array_equal(l0 + s[0], l1) and np.array_equal(m0 + s[1], m1)
    # an explicit damping is used as given
    s2, t2 = O.lm_trial(g, pr, y, l0, m0, 10 * rep["nu0"])
    assert t2["nu0"] == 0.0 and np.linalg.norm(s2) < np.linalg.norm(s)


def test_proposal_equal_to_the_lm_step(O):
    g, ph, y = _case(O, noise=1e4)
    pr = O.default_params(max_iters=1, cg_max_iters=6)
    l0, m0 = O.initial_guess(g, y)
    s, t = O.lm_trial(g, pr, y, l0, m0)
    c = O.check_proposal(g, pr, y, l0, m0, s, l0 + s[0], m0 + s[1])
    assert c["pred_step"] == t["pred"] and c["f"] == t["f"]
    assert abs(c["pred_prop"] - t["pred"]) <= 1e-12 * abs(t["pred"])
    assert abs(c["rho_prop"] - t["rho"]) <= 1e-9
    assert c["accept"] == t["accept"]
    # the threshold is rho > eta, strictly: eta just above / below this proposal's rho
    for d, want in ((1e-6, False), (-1e-6, True)):
        pe = O.default_params(max_iters=1, cg_max_iters=6, eta=c["rho_prop"] + d)
        assert O.check_proposal(g, pe, y, l0, m0, s, l0 + s[0], m0 + s[1])["accept"] == want


def test_lambda_only_proposal_with_quadratic_prior_has_rho_one(O):
    g, ph, y = _case(O, seed=5, noise=1e4)
    pr = O.default_params(tv_eps=0.0, alpha_lambda=0.05, alpha_mu=0.05)
    l0, m0 = O.initial_guess(g, y)
    s, _ = O.lm_trial(g, pr, y, l0, m0)
    rs = np.random.default_rng(9)
    for scale in (1e-3, 0.1, 0.4):
        pl = np.clip(l0 + scale * rs.standard_normal(l0.shape), 0.0, pr.lambda_max)
        c = O.check_proposal(g, pr, y, l0, m0, s, pl, m0)
        if c["pred_prop"] > 0:
            assert abs(c["rho_prop"] - 1.0) <= 1e-8, (scale, c)
        else:  # no predicted decrease: exactly the actual change, with the opposite sign
            assert abs(c["ared_prop"] - c["pred_prop"]) <= 1e-9 * abs(c["pred_prop"])
        assert abs(c["ared_prop"] - c["pred_prop"]) <= 1e-9 * max(1.0, abs(c["pred_prop"]))


def test_half_step_is_rejected_by_the_model_comparison(O):
    g, ph, y = _case(O, seed=6, noise=1e4)
    pr = O.default_params(cg_max_iters=8)
    l0, m0 = O.initial_guess(g, y)
    s, t = O.lm_trial(g, pr, y, l0, m0)
    c = O.check_proposal(g, pr, y, l0, m0, s, l0 + 0.5 * s[0], m0 + 0.5 * s[1])
    assert c["rho_prop"] > pr.eta  # the half step alone would pass the rho test
    assert c["pred_prop"] < c["pred_step"]  # but m_k(s/2) > m_k(s_k)
    assert not c["accept"]


def test_truth_accepted_noise_and_zero_rejected(O):
    g, ph, y = _case(O, seed=7)  # noiseless data
    pr = O.default_params(cg_max_iters=8)
    rs = np.random.default_rng(11)
    lk = np.clip(ph.lam + 0.05 * rs.standard_normal(ph.lam.shape), 0.0, pr.lambda_max)
    mk = np.clip(ph.mu + 0.005 * rs.standard_normal(ph.mu.shape), 0.0, pr.mu_max)
    s, t = O.lm_trial(g, pr, y, lk, mk, 1e3)  # heavily damped LM step
    truth = O.check_proposal(g, pr, y, lk, mk, s, ph.lam, ph.mu)
    assert truth["accept"] and truth["rho_prop"] > 0.5
    noise = O.check_proposal(g, pr, y, lk, mk, s, lk + rs.uniform(-1, 1, lk.shape),
                             mk + rs.uniform(-0.1, 0.1, mk.shape))
    assert not noise["accept"] and noise["ared_prop"] < 0
    zero = O.check_proposal(g, pr, y, lk, mk, s, lk, mk)
    assert zero["pred_prop"] == 0.0 and zero["rho_prop"] == -np.inf and not zero["accept"]


def test_proposal_outside_the_box_is_projected(O):
    g, ph, y = _case(O, seed=8, noise=1e5)
    pr = O.default_params()
    l0, m0 = O.initial_guess(g, y)
    s, _ = O.lm_trial(g, pr, y, l0, m0)
    rs = np.random.default_rng(12)
    pl = l0 + rs.uniform(-3, 3, l0.shape)
    pm = m0 + rs.uniform(-0.5, 0.5, m0.shape)
    a = O.check_proposal(g, pr, y, l0, m0, s, pl, pm)
    b = O.check_proposal(g, pr, y, l0, m0, s, np.clip(pl, 0, pr.lambda_max), np.clip(pm, 0, pr.mu_max))
    assert a == b


def _chain_trials(O, g, y, l0, m0, alpha, decay, K, iters, cg):
    """The LM with continuation rebuilt from single (pinned) trials: iteration k uses
    alpha / decay^min(k, K) with the damping carried over."""
    lam, mu = np.clip(l0, 0, 2.0), np.clip(m0, 0, 0.2)
    nu, nu0, out = 0.0, None, []
    for k in range(iters):
        sc = decay ** -min(k, K)
        pk = O.default_params(cg_max_iters=cg, alpha_lambda=alpha * sc, alpha_mu=alpha * sc)
        s, t = O.lm_trial(g, pk, y, lam, mu, nu)
        if nu0 is None:
            nu0 = nu = t["nu0"]
        if t["accept"]:
            lam, mu = lam + s[0], mu + s[1]
        nu = min(max(t["nu_next"], 1e-12 * nu0), 1e12 * nu0)
        out.append((t, nu))
    return lam, mu, out


def test_alpha_continuation_is_a_chain_of_trials(O):
    """Sec. 3.1: alpha^(k) = alpha / 5^k, halted after K iterations; each iteration's f and
    gradient use alpha^(k).  The LM with continuation equals the chain of single trials
    with those weights, iteration by iteration (pred, ared, rho, acceptance, damping)."""
    g, ph, y = _case(O, seed=9, noise=1e4)
    l0, m0 = O.initial_guess(g, y)
    for K in (2, 4):
        pr = O.default_params(max_iters=6, cg_max_iters=6, alpha_decay=5.0, alpha_decay_iters=K)
        lam, mu, rep = O.lm(g, pr, y, l0, m0)
        lc, mc, chain = _chain_trials(O, g, y, l0, m0, 1e-2, 5.0, K, 6, 6)
        for k, (t, nu) in enumerate(chain):
            for key in ("pred", "ared", "rho"):
                assert abs(t[key] - rep[key][k]) <= 1e-9 * max(1.0, abs(rep[key][k])), (K, k, key)
            assert t["accept"] == rep["acc"][k] and abs(nu - rep["nu"][k]) <= 1e-12 * rep["nu"][k]
        assert np.abs(lc - lam).max() <= 1e-12 and np.abs(mc - mu).max() <= 1e-12
        assert sum(rep["acc"]) >= 3  # the chain exercises accepted steps


def test_alpha_continuation_off_is_the_plain_lm(O):
    g, ph, y = _case(O, seed=10, noise=1e4)
    l0, m0 = O.initial_guess(g, y)
    base = O.lm(g, O.default_params(max_iters=4, cg_max_iters=6), y, l0, m0)
    for dec, K in ((1.0, 5), (5.0, 0), (0.0, 3)):
        got = O.lm(g, O.default_params(max_iters=4, cg_max_iters=6, alpha_decay=dec, alpha_decay_iters=K),
                   y, l0, m0)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]) and got[2] == base[2]

"""Pins of the oracle's geometry priors (Eq. (6)): alpha_1 |P1 lambda|^2 + alpha_2 |P2 mu|^2
with P1 lambda = (1 - M) lambda and P2 mu = (1 - M)(mu - mu_water), M the mask of
potential rod locations.

- M = 1 everywhere switches the priors off: the LM is bitwise the plain one;
- value, gradient and Hessian agree: with the quadratic smoothness prior as well, the
  objective is exactly quadratic along lambda (A is linear in lambda), so every
  lambda-only proposal has actual = predicted decrease; for mixed steps their ratio
  tends to 1 as the step shrinks;
- CG on the normal equations with the priors equals a dense solve whose matrix is built
  column by column from the JVP, the adjoint, the smoothness prior and the diagonal
  Hessian 2 alpha (1 - M)^2;
- on noisy data the priors pull the emission outside the rod locations toward zero and
  the attenuation there toward water.
"""
import numpy as np

from paper_2604_26745_gb300 import synth


def _case(O, seed=3, n=16):
    g = O.geom(n, 12, 91, n_sub=1)
    ph = synth.lattice_phantom(n, 2, radius=2.0, seed=seed)
    y = synth.poisson_noise(O.forward(g, ph.lam, ph.mu), 1e3, seed + 50)
    mask = np.clip(synth.lattice_phantom(n, 2, radius=3.0, seed=seed, zero_frac=0.0, mu_rod=1.0,
                                         mu_bg=0.0).mu, 0.0, 1.0)  # rod disks, dilated by a pixel
    return g, ph, y, mask


def test_full_mask_is_the_plain_lm(O):
    g, ph, y, mask = _case(O)
    l0, m0 = O.initial_guess(g, y)
    base = O.lm(g, O.default_params(max_iters=3, cg_max_iters=6), y, l0, m0)
    got = O.lm(g, O.default_params(max_iters=3, cg_max_iters=6, geo_mask=np.ones_like(mask), geo_alpha_lambda=5.0,
                                   geo_alpha_mu=5.0, geo_mu_water=0.01), y, l0, m0)
    assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]) and got[2] == base[2]


def test_quadratic_along_lambda_rho_is_one(O):
    g, ph, y, mask = _case(O, seed=4)
    pr = O.default_params(tv_eps=0.0, geo_mask=mask, geo_alpha_lambda=0.3, geo_alpha_mu=0.7, geo_mu_water=0.01)
    l0, m0 = O.initial_guess(g, y)
    s, _ = O.lm_trial(g, pr, y, l0, m0)
    rs = np.random.default_rng(1)
    for scale in (1e-2, 0.2):
        pl = np.clip(l0 + scale * rs.standard_normal(l0.shape), 0.0, pr.lambda_max)
        c = O.check_proposal(g, pr, y, l0, m0, s, pl, m0)
        assert abs(c["ared_prop"] - c["pred_prop"]) <= 1e-9 * max(1.0, abs(c["pred_prop"])), (scale, c)
    # the prior term alone is not negligible here
    c0 = O.check_proposal(g, O.default_params(tv_eps=0.0), y, l0, m0, s, pl, m0)
    assert abs(c0["ared_prop"] - c["ared_prop"]) > 1e-3 * abs(c["ared_prop"])


def test_small_steps_rho_tends_to_one(O):
    g, ph, y, mask = _case(O, seed=5)
    pr = O.default_params(geo_mask=mask, geo_alpha_lambda=0.5, geo_alpha_mu=50.0, geo_mu_water=0.01)
    l0, m0 = O.initial_guess(g, y)
    s, _ = O.lm_trial(g, pr, y, l0, m0)
    rs = np.random.default_rng(2)
    d = (rs.standard_normal(l0.shape), 0.1 * rs.standard_normal(m0.shape))
    gaps = []
    for eps in (1e-2, 1e-3, 1e-4):
        c = O.check_proposal(g, pr, y, l0, m0, s, np.clip(l0 + eps * d[0], 0, 2), np.clip(m0 + eps * d[1], 0, 0.2))
        gaps.append(abs(c["ared_prop"] / c["pred_prop"] - 1.0))  # the sign of the step is free
    assert gaps[-1] <= 1e-3 and gaps[0] > 10 * gaps[-1]


def test_cg_matches_dense_solve_with_priors(O):
    g, ph, y, _ = _case(O, seed=6, n=8)
    n = 8
    mask = synth.disk_image(n, 2.3, 1.0)  # zeros, ones and fractional edge values
    assert (mask == 0).any() and (mask == 1).any() and ((mask > 0) & (mask < 1)).any()
    pr = O.default_params(tv_eps=0.0, cg_max_iters=2000, cg_rel_tol=1e-14, geo_mask=mask, geo_alpha_lambda=0.2,
                          geo_alpha_mu=3.0, geo_mu_water=0.01)
    lam, mu = ph.lam + 0.1, ph.mu
    Wl = O.reg_weights(lam, pr.tv_eps)
    Wm = O.reg_weights(mu, pr.tv_eps)
    np_ = n * n
    cols = []
    for k in range(2 * np_):
        e = np.zeros(2 * np_)
        e[k] = 1.0
        jv = O.jvp(g, lam, mu, e[:np_].reshape(n, n), e[np_:].reshape(n, n))
        gl, gm = O.vjp(g, lam, mu, jv)
        col = np.concatenate([gl.ravel(), gm.ravel()])
        col[:np_] += O.reg_apply(Wl, e[:np_].reshape(n, n), pr.alpha_lambda).ravel()
        col[np_:] += O.reg_apply(Wm, e[np_:].reshape(n, n), pr.alpha_mu).ravel()
        cols.append(col)
    H = np.array(cols).T
    om2 = (1.0 - mask.ravel()) ** 2
    H += np.diag(np.concatenate([2 * pr.geo_alpha_lambda * om2, 2 * pr.geo_alpha_mu * om2]))
    nu = 0.05
    H += nu * np.eye(2 * np_)
    b = np.random.default_rng(3).standard_normal(2 * np_)
    x, it = O.cg(g, pr, lam, mu, Wl, Wm, nu, b)
    xd = np.linalg.solve(H, b)
    assert np.linalg.norm(x.ravel() - xd) <= 1e-8 * np.linalg.norm(xd)


def test_priors_pull_outside_the_rods(O):
    g, ph, y, mask = _case(O, seed=7)
    l0, m0 = O.initial_guess(g, y)
    out = 1.0 - mask
    plain = O.lm(g, O.default_params(max_iters=6, cg_max_iters=10), y, l0, m0)
    geo = O.lm(g, O.default_params(max_iters=6, cg_max_iters=10, geo_mask=mask, geo_alpha_lambda=10.0,
                                   geo_alpha_mu=10.0, geo_mu_water=0.01), y, l0, m0)
    assert np.linalg.norm(out * geo[0]) < 0.7 * np.linalg.norm(out * plain[0])
    assert np.linalg.norm(out * (geo[1] - 0.01)) < np.linalg.norm(out * (plain[1] - 0.01))

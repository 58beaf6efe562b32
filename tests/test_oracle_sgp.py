"""Pins of the oracle's gradient-projection inner solver (Sec. 2.2: the box-constrained
LM subproblem solved by scaled gradient projection; identity scaling here).

The subproblem is the convex quadratic program
    min_s q(s) = <g, s> + 1/2 s^T A s,  A = J^T J + H + nu I,  subject to  u + s in the box.
Pins, on an 8 x 8 problem whose A is built column by column from the JVP, the adjoint and
the prior (independently of the solver):
- the result equals scipy's bounded quasi-Newton solution of the same QP (library
  special case) and satisfies the KKT conditions;
- with bounds far away it is the unconstrained Newton step -A^{-1} g (the dense solve);
- q decreases monotonically along the iterations and every iterate is feasible;
- on an LM problem with many active bounds the solver reaches a lower model value than
  CG followed by projection, and the LM with it decreases f monotonically.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _dense(O, n=8, seed=6, tv_eps=0.0, nu=0.05):
    g = O.geom(n, 12, 91, n_sub=1)
    ph = synth.lattice_phantom(n, 2, radius=1.5, seed=seed)
    pr = O.default_params(tv_eps=tv_eps)
    lam, mu = ph.lam + 0.02, ph.mu
    Wl, Wm = O.reg_weights(lam, pr.tv_eps), O.reg_weights(mu, pr.tv_eps)
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
        cols.append(col + nu * e)
    A = np.array(cols).T
    A = 0.5 * (A + A.T)
    return g, pr, lam, mu, Wl, Wm, nu, A


def _q(A, gvec, s):
    return gvec @ s + 0.5 * s @ A @ s


def _bounds(lam, mu, lmax, mmax):
    u = np.concatenate([lam.ravel(), mu.ravel()])
    hi = np.concatenate([np.full(lam.size, lmax), np.full(mu.size, mmax)])
    return u, -u, hi - u


def test_matches_scipy_bounded_qp_and_kkt(O):
    scipy_opt = pytest.importorskip("scipy.optimize")
    g, pr, lam, mu, Wl, Wm, nu, A = _dense(O)
    gvec = np.random.default_rng(1).standard_normal(A.shape[0]) * 5.0
    pr.cg_max_iters, pr.cg_rel_tol = 20000, 1e-13
    s, it = O.sgp(g, pr, lam, mu, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
    s = s.ravel()
    u, lo, hi = _bounds(lam, mu, pr.lambda_max, pr.mu_max)
    res = scipy_opt.minimize(lambda x: _q(A, gvec, x), np.zeros_like(gvec), jac=lambda x: gvec + A @ x,
                             bounds=list(zip(lo, hi)), method="L-BFGS-B",
                             options=dict(ftol=1e-15, gtol=1e-12, maxiter=20000))
    assert np.all(s >= lo - 1e-12) and np.all(s <= hi + 1e-12)
    assert np.abs(s - res.x).max() <= 1e-5 * max(1.0, np.abs(res.x).max())
    assert _q(A, gvec, s) <= _q(A, gvec, res.x) + 1e-9 * abs(_q(A, gvec, res.x))
    # KKT with the gradient rebuilt from the dense matrix
    gq = gvec + A @ s
    act_lo, act_hi = np.isclose(s, lo, atol=1e-10), np.isclose(s, hi, atol=1e-10)
    free = ~(act_lo | act_hi)
    assert np.abs(gq[free]).max() <= 1e-6 * np.abs(gvec).max()
    assert np.all(gq[act_lo] >= -1e-6 * np.abs(gvec).max()) and np.all(gq[act_hi] <= 1e-6 * np.abs(gvec).max())
    assert act_lo.any()  # bounds are active in this case


def test_far_bounds_give_the_newton_step(O):
    g, pr, lam, mu, Wl, Wm, nu, A = _dense(O, seed=7)
    gvec = np.random.default_rng(2).standard_normal(A.shape[0]) * 1e-3
    pr.cg_max_iters, pr.cg_rel_tol = 20000, 1e-13
    pr.lambda_max, pr.mu_max = 1e6, 1e6
    lam2, mu2 = lam + 10.0, mu + 10.0  # far from both bounds
    s, it = O.sgp(g, pr, lam2, mu2, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
    # A at the shifted point: rebuild (the Jacobian depends on u)
    _, _, _, _, _, _, _, A2 = _dense_at(O, g, pr, lam2, mu2, Wl, Wm, nu)
    xd = -np.linalg.solve(A2, gvec)
    assert np.linalg.norm(s.ravel() - xd) <= 1e-7 * np.linalg.norm(xd)


def _dense_at(O, g, pr, lam, mu, Wl, Wm, nu):
    n = lam.shape[0]
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
        cols.append(col + nu * e)
    A = np.array(cols).T
    return g, pr, lam, mu, Wl, Wm, nu, 0.5 * (A + A.T)


def test_monotone_and_feasible(O):
    g, pr, lam, mu, Wl, Wm, nu, A = _dense(O, seed=8)
    gvec = np.random.default_rng(3).standard_normal(A.shape[0]) * 5.0
    u, lo, hi = _bounds(lam, mu, pr.lambda_max, pr.mu_max)
    pr.cg_rel_tol = 0.0
    qs = []
    for k in range(1, 25):
        pr.cg_max_iters = k
        s, it = O.sgp(g, pr, lam, mu, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
        s = s.ravel()
        assert np.all(s >= lo - 1e-12) and np.all(s <= hi + 1e-12)
        qs.append(_q(A, gvec, s))
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(qs[:-1], qs[1:])) and qs[-1] < qs[0]


def test_lm_with_gradient_projection(O):
    g = O.geom(16, 12, 91, n_sub=1)
    ph = synth.lattice_phantom(16, 2, radius=2.0, seed=1)
    y = synth.poisson_noise(O.forward(g, ph.lam, ph.mu), 1e4, 5)
    l0, m0 = O.initial_guess(g, y)
    rep_cg = O.lm(g, O.default_params(max_iters=6, cg_max_iters=20), y, l0, m0)[2]
    lam, mu, rep = O.lm(g, O.default_params(max_iters=6, cg_max_iters=20, inner_solver=1), y, l0, m0)
    f = [rep["f0"]] + rep["f"]
    assert all(b <= a for a, b in zip(f[:-1], f[1:])) and sum(rep["acc"]) >= 4
    assert rep["pred"][0] > rep_cg["pred"][0]  # the constrained model decrease is larger
    assert (lam >= 0).all() and (lam <= 2.0).all() and (mu >= 0).all() and (mu <= 0.2).all()

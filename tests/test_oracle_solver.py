"""Pins of the oracle's regulariser, CG and Levenberg-Marquardt iteration (Sec. 2.2, 3.1).

- the quadratic prior's Hessian equals the 5-point graph Laplacian built independently;
- the smoothed-TV gradient against finite differences of its value, and the frozen-weight
  quadratic model majorises the value (concavity of the square root);
- CG run to a 1e-14 residual equals a dense Cholesky solve of the damped normal equations;
- the first LM step equals the damped least-squares problem of Eq. (9) solved by lstsq;
- the objective never increases over LM iterates and accepted steps satisfy rho > eta
  (the monotone decrease of the convergence proposition, Sec. 3.1);
- rho -> 1 as the step shrinks (nu large);
- on noiseless data the error against the truth decreases.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _graph_laplacian(n):
    """Dense 5-point graph Laplacian of an n x n grid with a zero-flux boundary."""
    L = np.zeros((n * n, n * n))
    for iy in range(n):
        for ix in range(n):
            i = iy * n + ix
            for dy, dx in ((0, 1), (1, 0), (0, -1), (-1, 0)):
                jy, jx = iy + dy, ix + dx
                if 0 <= jy < n and 0 <= jx < n:
                    L[i, i] += 1.0
                    L[i, jy * n + jx] -= 1.0
    return L


def test_quadratic_prior_is_graph_laplacian(O):
    n, alpha = 6, 0.3
    W = O.reg_weights(np.zeros((n, n)), -1.0)
    assert np.all(W == 1.0)
    H = np.zeros((n * n, n * n))
    for i in range(n * n):
        e = np.zeros(n * n)
        e[i] = 1.0
        H[:, i] = O.reg_apply(W, e.reshape(n, n), alpha).ravel()
    np.testing.assert_allclose(H, alpha * _graph_laplacian(n), atol=1e-15)
    u = np.random.default_rng(0).standard_normal((n, n))
    # value alpha/2 |grad u|^2 = alpha/2 u^T L u
    v = O.reg_value(u, alpha, -1.0)
    assert abs(v - 0.5 * alpha * u.ravel() @ _graph_laplacian(n) @ u.ravel()) < 1e-12 * abs(v)


def test_tv_gradient_and_majoriser(O):
    n, alpha, eps = 10, 0.02, 1e-2
    ph = synth.lattice_phantom(n, 2, seed=3)
    u = ph.lam + 0.01 * np.random.default_rng(1).standard_normal((n, n))
    W = O.reg_weights(u, eps)
    grad = O.reg_apply(W, u, alpha)
    d = np.random.default_rng(2).standard_normal((n, n))
    h = 1e-5
    fd = (O.reg_value(u + h * d, alpha, eps) - O.reg_value(u - h * d, alpha, eps)) / (2 * h)
    assert abs(fd - np.sum(grad * d)) <= 1e-6 * abs(fd)
    # R(u + s) <= R(u) + <grad, s> + 1/2 s^T H s, H = alpha grad^T W grad (frozen at u)
    R0 = O.reg_value(u, alpha, eps)
    for k in range(5):
        s = np.random.default_rng(10 + k).standard_normal((n, n)) * 10.0 ** (-k)
        Hs = O.reg_apply(W, s, alpha)
        model = R0 + np.sum(grad * s) + 0.5 * np.sum(s * Hs)
        assert O.reg_value(u + s, alpha, eps) <= model + 1e-12 * abs(model)
    # symmetric positive semi-definite
    s1, s2 = d, np.random.default_rng(5).standard_normal((n, n))
    assert abs(np.sum(O.reg_apply(W, s1, alpha) * s2) - np.sum(s1 * O.reg_apply(W, s2, alpha))) < 1e-12
    assert np.sum(s1 * O.reg_apply(W, s1, alpha)) >= 0


def _dense(O, g, lam, mu):
    N = g.n
    npx = N * N
    J = np.zeros((g.n_angles * g.n_det, 2 * npx))
    for i in range(2 * npx):
        e = np.zeros(2 * npx)
        e[i] = 1.0
        J[:, i] = O.jvp(g, lam, mu, e[:npx].reshape(N, N), e[npx:].reshape(N, N)).ravel()
    return J


def test_cg_equals_dense_cholesky(O):
    N = 8
    g = O.geom(N, 8, 91, n_sub=3)
    ph = synth.lattice_phantom(N, 2, seed=9)
    pr = O.default_params(alpha_lambda=0.05, alpha_mu=0.2, tv_eps=-1.0,
                          cg_max_iters=2000, cg_rel_tol=1e-14)
    Wl = O.reg_weights(ph.lam, -1.0)
    Wm = O.reg_weights(ph.mu, -1.0)
    nu = 0.37
    b = np.random.default_rng(3).standard_normal(2 * N * N)
    x, it = O.cg(g, pr, ph.lam, ph.mu, Wl, Wm, nu, b)
    assert 2 * N * N <= it < 2000
    J = _dense(O, g, ph.lam, ph.mu)
    Lg = _graph_laplacian(N)
    H = np.block([[0.05 * Lg, np.zeros_like(Lg)], [np.zeros_like(Lg), 0.2 * Lg]])
    A = J.T @ J + H + nu * np.eye(2 * N * N)
    c = np.linalg.cholesky(A)
    xd = np.linalg.solve(c.T, np.linalg.solve(c, b))
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_first_lm_step_is_damped_least_squares(O):
    """With the prior switched off and a box that never binds, the first LM trial step
    solves min |J s + r|^2 + nu |s|^2 (Eq. (9)); its model decrease and the step's
    objective then fix rho.  Checked through m_k(0) - m_k(s) recomputed densely."""
    N = 6
    g = O.geom(N, 6, 91, n_sub=1)
    ph = synth.lattice_phantom(N, 2, seed=12)
    lam, mu = ph.lam + 0.2, ph.mu + 0.02
    y = O.forward(g, lam * 1.05, mu * 0.95)
    pr = O.default_params(alpha_lambda=0.0, alpha_mu=0.0, tv_eps=-1.0, lambda_max=1e9,
                          mu_max=1e9, max_iters=1, cg_max_iters=4 * N * N, cg_rel_tol=0.0)
    lam1, mu1, rep = O.lm(g, pr, y, lam, mu)
    J = _dense(O, g, lam, mu)
    r = (O.forward(g, lam, mu) - y).ravel()
    nu = rep["nu0"]
    A = np.vstack([J, np.sqrt(nu) * np.eye(2 * N * N)])
    s = np.linalg.lstsq(A, -np.concatenate([r, np.zeros(2 * N * N)]), rcond=None)[0]
    pred = -(J @ s) @ r - 0.5 * np.sum((J @ s) ** 2)
    assert abs(rep["pred"][0] - pred) <= 1e-8 * abs(pred)
    if rep["acc"][0]:
        got = np.concatenate([(lam1 - lam).ravel(), (mu1 - mu).ravel()])
        assert np.linalg.norm(got - s) <= 1e-8 * np.linalg.norm(s)
    # nu_0 from its definition: nu0_scale |J g|^2 / |g|^2, g = J^T r
    gr = J.T @ r
    assert abs(nu - 1e-3 * np.sum((J @ gr) ** 2) / np.sum(gr ** 2)) <= 1e-10 * nu


def _c1_like(O, N=24, Na=30, counts=None, seed=0):
    g = O.geom(N, Na, 91, n_sub=1)
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=1000 + seed)
    y = O.forward(g, ph.lam, ph.mu)
    if counts:
        y = synth.poisson_noise(y, counts, 2000 + seed)
    return g, ph, y


def test_lm_objective_monotone_and_acceptance(O):
    g, ph, y = _c1_like(O, counts=1e4)
    pr = O.default_params(max_iters=8, cg_max_iters=20)
    lam0, mu0 = O.initial_guess(g, y)
    lam, mu, rep = O.lm(g, pr, y, lam0, mu0)
    f = [rep["f0"]] + rep["f"]
    assert all(b <= a for a, b in zip(f[:-1], f[1:]))
    for k in range(rep["iters_run"]):
        if rep["acc"][k]:
            assert rep["rho"][k] > pr.eta
            assert rep["ared"][k] > pr.eta * rep["pred"][k] > 0
            assert f[k + 1] < f[k]
        else:
            assert f[k + 1] == f[k]
    assert rep["accepted"] >= 4
    assert rep["f_final"] < 0.5 * rep["f0"]
    # box respected
    assert lam.min() >= 0 and lam.max() <= pr.lambda_max
    assert mu.min() >= 0 and mu.max() <= pr.mu_max


def test_damping_schedule(O):
    """nu (beta_k of Eq. (9)) follows the trust-region update that Thm. 3.1 assumes
    (Nocedal-Wright Alg. 4.1 in LM form): 4x when rho < 1/4, halved when rho > 3/4.
    A far-off attenuation guess with a small nu_0 makes the first steps overshoot,
    so both branches occur."""
    g = O.geom(24, 30, 91, n_sub=1)
    ph = synth.lattice_phantom(24, 3, radius=2.0, seed=1000, mu_rod=0.15)
    y = synth.poisson_noise(O.forward(g, ph.lam, ph.mu), 1e4, 2000)
    lam0, mu0 = O.initial_guess(g, y, mu_init=0.2)
    pr = O.default_params(max_iters=8, cg_max_iters=200, nu0_scale=1e-5, tv_eps=-1.0,
                          alpha_lambda=1e-6, alpha_mu=1e-6)
    _, _, rep = O.lm(g, pr, y, lam0, mu0)
    nus = [rep["nu0"]] + rep["nu"]
    saw_up = saw_down = False
    for k in range(rep["iters_run"]):
        rho = rep["rho"][k]
        want = nus[k] * (4.0 if rho < 0.25 else (0.5 if rho > 0.75 else 1.0))
        assert abs(nus[k + 1] - want) <= 1e-15 * want
        saw_up |= bool(rho < 0.25)
        saw_down |= bool(rho > 0.75)
    assert saw_up and saw_down
    f = [rep["f0"]] + rep["f"]
    assert all(b <= a for a, b in zip(f[:-1], f[1:]))


def test_rho_tends_to_one_for_small_steps(O):
    g, ph, y = _c1_like(O, N=16, Na=16)
    lam0, mu0 = O.initial_guess(g, y)
    rhos = []
    for scale in (1e2, 1e4, 1e6):
        pr = O.default_params(max_iters=1, cg_max_iters=10, nu0_scale=scale)
        _, _, rep = O.lm(g, pr, y, lam0, mu0)
        rhos.append(rep["rho"][0])
    assert abs(rhos[-1] - 1.0) < 1e-3
    assert abs(rhos[-1] - 1.0) < abs(rhos[0] - 1.0)


def test_initial_guess_matches_total_counts(O):
    g, ph, y = _c1_like(O, N=16, Na=12)
    lam0, mu0 = O.initial_guess(g, y, mu_init=0.01)
    assert np.all(mu0 == 0.01) and np.ptp(lam0) == 0.0
    assert abs(O.forward(g, lam0, mu0).sum() - y.sum()) <= 1e-12 * y.sum()


def test_lm_reduces_error_on_noiseless_data(O):
    g, ph, y = _c1_like(O, N=24, Na=30)
    pr = O.default_params(alpha_lambda=1e-6, alpha_mu=1e-6, max_iters=10, cg_max_iters=30)
    lam0, mu0 = O.initial_guess(g, y)
    e0 = np.linalg.norm(lam0 - ph.lam) / np.linalg.norm(ph.lam)
    lam, mu, rep = O.lm(g, pr, y, lam0, mu0)
    e1 = np.linalg.norm(lam - ph.lam) / np.linalg.norm(ph.lam)
    assert e1 < 0.5 * e0
    m0 = np.linalg.norm(mu0 - ph.mu) / np.linalg.norm(ph.mu)
    m1 = np.linalg.norm(mu - ph.mu) / np.linalg.norm(ph.mu)
    assert m1 < m0

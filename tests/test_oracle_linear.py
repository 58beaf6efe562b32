"""Pins of the oracle's constraint set with the linear bound (Sec. 2.2: box bounds combined
with a linear bound that excludes strongly emitting pixels of low attenuation), read as
the per-pixel half-plane lambda <= k mu + b (k, b >= 0) intersected with the box.

- The projection equals an independent construction: the box clipped by the half-plane
  (Sutherland-Hodgman), then the nearest point of the polygon found by an inside test and
  the nearest points of all its edges, on points in every region around the polygon and
  for slopes and offsets that cut off one corner, two corners, a strip (k = 0), or
  nothing;
- it is feasible, idempotent and firmly non-expansive; without the bound it is the clamp;
- an LM whose bound never binds inside the box is bitwise the box-only LM (CG and
  gradient projection); with a binding bound every iterate is feasible and f decreases;
- the gradient-projection step with the bound solves the constrained quadratic program:
  it is a fixed point of the projected gradient map and agrees with scipy's SLSQP on a
  dense 8 x 8 problem.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

LMAX, MMAX = 2.0, 0.2


def _polygon(k, b):
    """Counter-clockwise vertices (lambda, mu) of the box clipped by lambda - k mu <= b."""
    box = [(0.0, 0.0), (LMAX, 0.0), (LMAX, MMAX), (0.0, MMAX)]
    f = lambda p: p[0] - k * p[1] - b
    out = []  # consecutive duplicates (a corner on the line) are dropped below
    for i in range(4):
        p, q = box[i], box[(i + 1) % 4]
        if f(q) <= 0:
            if f(p) > 0:
                t = f(p) / (f(p) - f(q))
                out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
            out.append(q)
        elif f(p) <= 0:
            t = f(p) / (f(p) - f(q))
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    uniq = [v for i, v in enumerate(out) if v != out[i - 1]]
    return [np.array(v) for v in uniq]


def _nearest(poly, z):
    edges = [(poly[i], poly[(i + 1) % len(poly)]) for i in range(len(poly))]
    cross = lambda a, c: a[0] * c[1] - a[1] * c[0]
    if all(cross(q - p, z - p) >= 0 for p, q in edges):
        return z
    best, bd = None, np.inf
    for p, q in edges:
        e = q - p
        t = np.clip(np.dot(z - p, e) / np.dot(e, e), 0.0, 1.0)
        c = p + t * e
        d = np.dot(z - c, z - c)
        if d < bd:
            best, bd = c, d
    return best


CASES = [(10.0, 0.0), (10.0, 0.3), (0.0, 1.2), (25.0, 0.5), (4.0, 1.9), (3.0, 2.5)]


@pytest.mark.parametrize("k,b", CASES)
def test_projection_matches_polygon_construction(O, k, b):
    pr = O.default_params(lin_constraint=1, lin_slope=k, lin_offset=b)
    rs = np.random.default_rng(int(10 * k + 100 * b))
    zl = rs.uniform(-1.0, 3.5, 3000)
    zm = rs.uniform(-0.3, 0.5, 3000)
    pl, pm = O.project(pr, zl, zm)
    poly = _polygon(k, b)
    ref = np.array([_nearest(poly, np.array([a, c])) for a, c in zip(zl, zm)])
    assert np.abs(pl - ref[:, 0]).max() <= 1e-12 and np.abs(pm - ref[:, 1]).max() <= 1e-12
    if b < LMAX:  # the bound cuts the box: some points land on the line
        assert np.sum(np.abs(pl - k * pm - b) < 1e-12) > 100


def test_projection_properties(O):
    pr = O.default_params(lin_constraint=1, lin_slope=10.0, lin_offset=0.3)
    rs = np.random.default_rng(5)
    zl, zm = rs.uniform(-1, 3, 2000), rs.uniform(-0.3, 0.5, 2000)
    pl, pm = O.project(pr, zl, zm)
    assert (pl >= 0).all() and (pl <= LMAX).all() and (pm >= 0).all() and (pm <= MMAX).all()
    assert (pl - 10.0 * pm - 0.3 <= 1e-12).all()
    ql, qm = O.project(pr, pl, pm)
    assert np.abs(ql - pl).max() <= 1e-14 and np.abs(qm - pm).max() <= 1e-14
    # firm non-expansiveness on pairs of points
    wl, wm = rs.uniform(-1, 3, 2000), rs.uniform(-0.3, 0.5, 2000)
    xl, xm = O.project(pr, wl, wm)
    lhs = (pl - xl) * (zl - wl) + (pm - xm) * (zm - wm)
    rhs = (pl - xl) ** 2 + (pm - xm) ** 2
    assert (lhs >= rhs - 1e-12).all()
    off = O.default_params()
    cl, cm = O.project(off, zl, zm)
    assert np.array_equal(cl, np.clip(zl, 0, LMAX)) and np.array_equal(cm, np.clip(zm, 0, MMAX))


def _case(O, seed=3, n=16):
    g = O.geom(n, 12, 91, n_sub=1)
    ph = synth.lattice_phantom(n, 2, radius=2.0, seed=seed)
    y = synth.poisson_noise(O.forward(g, ph.lam, ph.mu), 1e3, seed + 50)
    return g, ph, y


@pytest.mark.parametrize("solver", [0, 1])
def test_bound_outside_the_box_is_the_box_lm(O, solver):
    g, ph, y = _case(O)
    l0, m0 = O.initial_guess(g, y)
    kw = dict(max_iters=4, cg_max_iters=8, inner_solver=solver)
    base = O.lm(g, O.default_params(**kw), y, l0, m0)
    got = O.lm(g, O.default_params(lin_constraint=1, lin_slope=3.0, lin_offset=2.0, **kw), y, l0, m0)
    assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]) and got[2] == base[2]


@pytest.mark.parametrize("solver", [0, 1])
def test_binding_bound_feasible_and_monotone(O, solver):
    g, ph, y = _case(O, seed=4)
    l0, m0 = O.initial_guess(g, y)
    kw = dict(max_iters=6, cg_max_iters=10, inner_solver=solver)
    k, b = 8.0, 0.05
    base = O.lm(g, O.default_params(**kw), y, l0, m0)
    assert (base[0] - k * base[1] - b > 1e-3).any()  # the box-only result violates the bound
    pr = O.default_params(lin_constraint=1, lin_slope=k, lin_offset=b, **kw)
    lam, mu, rep = O.lm(g, pr, y, l0, m0)
    assert (lam - k * mu - b <= 1e-12).all() and (lam >= 0).all() and (mu >= 0).all()
    f = [rep["f0"]] + rep["f"]
    assert all(c <= a for a, c in zip(f[:-1], f[1:])) and sum(rep["acc"]) >= 3
    # the start violates the bound; the LM starts from its projection
    assert (l0 - k * m0 - b > 1e-3).any()
    pl0, pm0 = O.project(pr, l0, m0)
    f_start = O.lm(g, O.default_params(lin_constraint=1, lin_slope=k, lin_offset=b, max_iters=0), y, pl0, pm0)[2]
    assert abs(rep["f0"] - f_start["f0"]) <= 1e-12 * abs(f_start["f0"])


def _dense(O, k, b, n=8, seed=6, nu=0.05):
    """Dense A = J^T J + H + nu I at a point satisfying lambda <= k mu + b."""
    g = O.geom(n, 12, 91, n_sub=1)
    ph = synth.lattice_phantom(n, 2, radius=1.5, seed=seed)
    pr = O.default_params(tv_eps=0.0)
    lam, mu = np.minimum(ph.lam + 0.02, k * ph.mu + b), ph.mu
    Wl, Wm = O.reg_weights(lam, pr.tv_eps), O.reg_weights(mu, pr.tv_eps)
    np_ = n * n
    cols = []
    for c in range(2 * np_):
        e = np.zeros(2 * np_)
        e[c] = 1.0
        jv = O.jvp(g, lam, mu, e[:np_].reshape(n, n), e[np_:].reshape(n, n))
        gl, gm = O.vjp(g, lam, mu, jv)
        col = np.concatenate([gl.ravel(), gm.ravel()])
        col[:np_] += O.reg_apply(Wl, e[:np_].reshape(n, n), pr.alpha_lambda).ravel()
        col[np_:] += O.reg_apply(Wm, e[np_:].reshape(n, n), pr.alpha_mu).ravel()
        cols.append(col + nu * e)
    A = np.array(cols).T
    return g, lam, mu, Wl, Wm, nu, 0.5 * (A + A.T)


def test_gradient_projection_solves_the_constrained_qp(O):
    scipy_opt = pytest.importorskip("scipy.optimize")
    k, b = 6.0, 0.02
    g, lam, mu, Wl, Wm, nu, A = _dense(O, k, b)
    np_ = lam.size
    gvec = np.random.default_rng(1).standard_normal(2 * np_) * 5.0
    pr = O.default_params(tv_eps=0.0, cg_max_iters=20000, cg_rel_tol=1e-13, lin_constraint=1, lin_slope=k,
                          lin_offset=b)
    s, it = O.sgp(g, pr, lam, mu, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
    assert it < pr.cg_max_iters  # ended by the projected-gradient test, not by the cap
    s = s.ravel()
    u = np.concatenate([lam.ravel(), mu.ravel()])
    x = u + s
    assert (x[:np_] - k * x[np_:] - b <= 1e-12).all() and (x >= -1e-15).all()
    # first-order optimality: s is a fixed point of the projected gradient map
    gq = gvec + A @ s
    tau = 1e-2 / np.linalg.norm(A, 2)
    pl, pm = O.project(pr, x[:np_] - tau * gq[:np_], x[np_:] - tau * gq[np_:])
    assert np.abs(np.concatenate([pl, pm]) - x).max() <= 1e-9 * max(1.0, np.abs(x).max())
    # a general-purpose solver on the same program
    q = lambda v: gvec @ v + 0.5 * v @ A @ v
    G = np.zeros((np_, 2 * np_))
    G[np.arange(np_), np.arange(np_)] = -1.0
    G[np.arange(np_), np_ + np.arange(np_)] = k
    cons = [{"type": "ineq", "fun": lambda v: G @ (u + v) + b, "jac": lambda v: G}]
    bnds = list(zip(-u, np.concatenate([np.full(np_, LMAX), np.full(np_, MMAX)]) - u))
    res = scipy_opt.minimize(q, np.zeros_like(u), jac=lambda v: gvec + A @ v, bounds=bnds, constraints=cons,
                             method="SLSQP", options=dict(ftol=1e-15, maxiter=2000))
    assert q(s) <= q(res.x) + 1e-9 * abs(q(res.x))
    assert np.abs(s - res.x).max() <= 1e-5 * max(1.0, np.abs(res.x).max())
    # the bound is active somewhere, so the answer is not the box-only one
    sb, _ = O.sgp(g, O.default_params(tv_eps=0.0, cg_max_iters=20000, cg_rel_tol=1e-13), lam, mu, Wl, Wm, nu,
                  gvec.reshape(2, *lam.shape))
    assert np.abs(sb.ravel() - s).max() > 1e-3


def test_stopping_rule_is_the_projected_gradient(O):
    """The solver stops at the first iterate whose unit-step projected gradient
    |P(u + s - grad q(s)) - u - s| is at most cg_rel_tol times its value at s = 0."""
    k, b = 6.0, 0.02
    g, lam, mu, Wl, Wm, nu, A = _dense(O, k, b)
    np_ = lam.size
    gvec = np.random.default_rng(2).standard_normal(2 * np_) * 5.0
    u = np.concatenate([lam.ravel(), mu.ravel()])
    tol = 1e-4
    kw = dict(tv_eps=0.0, cg_rel_tol=tol, lin_constraint=1, lin_slope=k, lin_offset=b)

    def pg(s):
        x, gq = u + s, gvec + A @ s
        pl, pm = O.project(O.default_params(**kw), x[:np_] - gq[:np_], x[np_:] - gq[np_:])
        return np.linalg.norm(np.concatenate([pl, pm]) - x)

    s, it = O.sgp(g, O.default_params(cg_max_iters=20000, **kw), lam, mu, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
    assert 1 < it < 20000 and pg(s.ravel()) <= tol * pg(np.zeros_like(u))
    s1, it1 = O.sgp(g, O.default_params(cg_max_iters=it - 1, **kw), lam, mu, Wl, Wm, nu, gvec.reshape(2, *lam.shape))
    assert it1 == it - 1 and pg(s1.ravel()) > tol * pg(np.zeros_like(u))

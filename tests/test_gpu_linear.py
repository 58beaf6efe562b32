"""The linear bound of the constraint set (Sec. 2.2, lambda <= k mu + b per pixel with the
box) on the GPU against the oracle:

- pget_project equals the oracle's projection on points around the polygon for bounds
  that cut one corner, two corners, a strip (k = 0) or nothing (FP64 to rounding, FP32
  to single precision), and leaves the box-only clamp bitwise unchanged without a bound;
- the LM with CG + projection and with gradient projection equals the oracle (FP64
  1e-10, same accept/reject trace; FP32-Kahan 1e-4 with CG), every iterate feasible;
- a bound that never binds inside the box gives the box-only solve bitwise;
- the Alg. 2 driver without proposals reproduces pget_lm_solve under the bound, and a
  proposal outside the polygon that the oracle's Alg. 2 step takes is taken and lands on
  its projection.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

N, NA, ND, S = 24, 30, 182, 3
K, B = 8.0, 0.05


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("k,b", [(10.0, 0.0), (10.0, 0.3), (0.0, 1.2), (25.0, 0.5), (3.0, 2.5)])
@pytest.mark.parametrize("prec", [0, 1])
def test_projection_matches_oracle(O, P, torch, k, b, prec):
    rs = np.random.default_rng(3)
    zl, zm = rs.uniform(-1.0, 3.5, (64, 64)), rs.uniform(-0.3, 0.5, (64, 64))
    pl, pm = O.project(O.default_params(lin_constraint=1, lin_slope=k, lin_offset=b), zl, zm)
    dt = P.dtype_of(prec)
    p = P.default_params(precision=prec, lin_constraint=1, lin_slope=k, lin_offset=b)
    with P.Context(0) as c:
        gl = torch.tensor(zl, dtype=dt, device="cuda")
        gm = torch.tensor(zm, dtype=dt, device="cuda")
        P.pget_project(c, p, gl, gm)
        torch.cuda.synchronize()
        # without the bound: the clamp, bitwise
        bl = torch.tensor(zl, dtype=dt, device="cuda")
        bm = torch.tensor(zm, dtype=dt, device="cuda")
        P.pget_project(c, P.default_params(precision=prec), bl, bm)
        assert torch.equal(bl, torch.tensor(zl, dtype=dt, device="cuda").clamp(0, 2.0))
        assert torch.equal(bm, torch.tensor(zm, dtype=dt, device="cuda").clamp(0, 0.2))
    tol = 1e-14 if prec == 0 else 2e-6
    assert np.abs(gl.double().cpu().numpy() - pl).max() <= tol
    assert np.abs(gm.double().cpu().numpy() - pm).max() <= tol


def _setup(O, seed=51):
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=seed)
    go = O.geom(N, NA, ND, n_sub=S)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e4, seed + 1)
    return ph, go, y


@pytest.mark.parametrize("solver,prec,tol", [(0, 0, 1e-10), (1, 0, 1e-10), (0, 2, 1e-4)])
def test_lm_with_linear_bound_matches_oracle(O, P, torch, solver, prec, tol):
    ph, go, y = _setup(O)
    # CG + projection rejects its first trials under a binding bound (the projection onto
    # the slanted edge distorts the CG step until nu has grown); six iterations accept two
    kw = dict(max_iters=6, cg_max_iters=6, inner_solver=solver, lin_constraint=1, lin_slope=K, lin_offset=B)
    l0, m0 = O.initial_guess(go, y)
    assert (l0 - K * m0 - B > 1e-3).any()  # the start violates the bound
    lo, mo, ro = O.lm(go, O.default_params(**kw), y, l0, m0)
    base = O.lm(go, O.default_params(max_iters=6, cg_max_iters=6, inner_solver=solver), y, l0, m0)
    assert (base[0] - K * base[1] - B > 1e-3).any()  # the bound binds on the result
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    p = P.default_params(precision=prec, cg_rel_tol=1e-10 if prec == 0 else 1e-6, **kw)
    with P.Context(0) as c:
        lam, mu = t(l0), t(m0)
        rep = P.pget_lm_solve(c, P.geometry(N, NA, ND, n_sub=S), p, t(y), lam, mu)
    assert rep["acc"] == ro["acc"] and sum(ro["acc"]) >= 2
    assert _rel(lam.double().cpu().numpy(), lo) <= tol and _rel(mu.double().cpu().numpy(), mo) <= tol
    assert abs(rep["f_final"] - ro["f_final"]) <= tol * abs(ro["f_final"])
    lh, mh = lam.double().cpu().numpy(), mu.double().cpu().numpy()
    slack = 1e-12 if prec == 0 else 1e-6
    assert (lh - K * mh - B <= slack).all() and (lh >= 0).all() and (mh >= 0).all()


@pytest.mark.parametrize("solver", [0, 1])
def test_bound_outside_the_box_is_the_box_solve(O, P, torch, solver):
    ph, go, y = _setup(O, seed=53)
    l0, m0 = O.initial_guess(go, y)
    t = lambda a: torch.tensor(a, device="cuda")
    g = P.geometry(N, NA, ND, n_sub=S)
    outs = []
    with P.Context(0) as c:
        for kw in ({}, dict(lin_constraint=1, lin_slope=3.0, lin_offset=2.0)):
            p = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0, inner_solver=solver,
                                 **kw)
            lam, mu = t(l0), t(m0)
            P.pget_lm_solve(c, g, p, t(y), lam, mu)
            outs.append((lam, mu))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_driver_under_the_bound(O, P, torch):
    from paper_2604_26745_gb300.accelerated import accelerated_solve
    ph, go, y = _setup(O, seed=55)
    p = P.default_params(max_iters=3, cg_max_iters=6, cg_rel_tol=1e-10, precision=0, lin_constraint=1,
                         lin_slope=K, lin_offset=B)
    yd = torch.tensor(y, device="cuda")
    g = P.geometry(N, NA, ND, n_sub=S)
    with P.Context(0) as c:
        l0, m0 = P.pget_initial_guess(c, g, p, yd)
        la, ma, h = accelerated_solve(c, g, p, yd, l0.clone(), m0.clone(), None)
        lb, mb = l0.clone(), m0.clone()
        rep = P.pget_lm_solve(c, g, p, yd, lb, mb)
        assert [x["took"] == "step" for x in h] == [bool(a) for a in rep["acc"]]
        assert float((la - lb).abs().max()) <= 1e-12 and float((ma - mb).abs().max()) <= 1e-12
    # a proposal outside the polygon (the truth, whose brightest rods violate a tighter
    # bound), made near it from noiseless data: the oracle's Alg. 2 step takes it, and so
    # must the Alg. 2 driver, landing on its projection
    k2, b2 = 14.0, 0.0
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=57)
    go = O.geom(N, NA, ND, n_sub=S)
    y = O.forward(go, ph.lam, ph.mu)
    pr = O.default_params(max_iters=1, cg_max_iters=6, lin_constraint=1, lin_slope=k2, lin_offset=b2)
    rs = np.random.default_rng(1)
    nl, nm = O.project(pr, ph.lam + 0.02 * rs.standard_normal(ph.lam.shape),
                       ph.mu + 0.002 * rs.standard_normal(ph.mu.shape))
    so, _ = O.lm_trial(go, pr, y, nl, nm)
    co = O.check_proposal(go, pr, y, nl, nm, so, ph.lam, ph.mu)
    assert co["accept"] and (ph.lam - k2 * ph.mu - b2 > 1e-3).any()
    p2 = P.default_params(max_iters=1, cg_max_iters=6, cg_rel_tol=1e-10, precision=0, lin_constraint=1,
                          lin_slope=k2, lin_offset=b2)
    t = lambda a: torch.tensor(a, device="cuda")
    truth = torch.stack([t(ph.lam), t(ph.mu)])
    with P.Context(0) as c:
        lt, mt, ht = accelerated_solve(c, g, p2, t(y), t(nl), t(nm), lambda u, s, k: truth, iters=1)
    assert ht[0]["took"] == "proposal"
    pl, pm = O.project(pr, ph.lam, ph.mu)
    assert np.abs(lt.cpu().numpy() - pl).max() <= 1e-14 and np.abs(mt.cpu().numpy() - pm).max() <= 1e-14

"""Depth factors of Eq. (5) on the GPU (y = h sum_j w_j lambda_j exp(-c_j E_j) per sub-ray,
tables over the sample index j) against the oracle, through the C ABI:

- forward, JVP and VJP with random tables on small ragged geometries (one or two banks,
  box and triangular collimators, odd n) at the operator tolerances of the plain model;
- the hand-worked point emitter (FP64, to rounding);
- tables of ones give the plain kernels' results to rounding;
- the LM with tables equals the oracle (FP64 1e-10, same accept/reject trace);
- pget_geometry_info reports the oracle's samples per ray; the allocation-free forward
  rejects tables.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 1e-12), 2: (1e-6, 2e-6), 1: (2e-6, 5e-6)}

CASES = {
    # name: (n, n_angles, n_det, n_sub, collimator, n_lat)
    "two_banks_s5": (40, 36, 182, 5, 1, 4),
    "box_even_s4": (36, 20, 182, 4, 0, 3),
    "odd_n_s3": (27, 17, 91, 3, 1, 3),
}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _tables(O, go, seed):
    T = O.geom_info(go)["T"]
    rs = np.random.default_rng(seed)
    return rs.uniform(0.5, 1.5, T), rs.uniform(1.0, 2.0, T)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 2, 1])
def test_operators_with_depth_tables(ctx, O, P, torch, case, prec):
    n, na, nd, S, col, nl = CASES[case]
    ph = synth.lattice_phantom(n, nl, seed=200 + n, jitter=0.7)
    rs = np.random.default_rng(n)
    lam, mu = ph.lam, ph.mu
    dl, dm = rs.standard_normal((n, n)), 0.01 * rs.standard_normal((n, n))
    w, c = _tables(O, O.geom(n, na, nd, n_sub=S, collimator=col), n)
    go = O.geom(n, na, nd, n_sub=S, collimator=col, depth_w=w, depth_c=c)
    gg = P.geometry(n, na, nd, n_sub=S, collimator=col, depth_w=w, depth_c=c)
    assert P.geometry_info(gg)["n_samples"] == O.geom_info(go)["T"] == len(w)
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol_y, tol_g = TOL[prec]
    y = P.pget_forward(ctx, gg, prec, t(lam), t(mu))
    yo = O.forward(go, lam, mu)
    assert rel(y.cpu().numpy(), yo) <= tol_y
    assert rel(yo, O.forward(O.geom(n, na, nd, n_sub=S, collimator=col), lam, mu)) > 1e-2  # tables matter
    dy = P.pget_jvp(ctx, gg, prec, t(lam), t(mu), t(dl), t(dm))
    assert rel(dy.cpu().numpy(), O.jvp(go, lam, mu, dl, dm)) <= tol_y
    r = np.random.default_rng(7).standard_normal((na, nd))
    gl, gm = P.pget_vjp(ctx, gg, prec, t(lam), t(mu), t(r))
    ol, om = O.vjp(go, lam, mu, r)
    assert rel(gl.cpu().numpy(), ol) <= tol_g
    assert rel(gm.cpu().numpy(), om) <= tol_g


def test_point_emitter_by_hand(ctx, O, P, torch):
    T = 6
    w, c = 1.0 + 0.1 * np.arange(T), 1.0 + 0.2 * np.arange(T)
    gg = P.geometry(4, 1, 2, n_sub=1, n_banks=1, fov_radius=3.0, det_pitch=1.0, depth_w=w, depth_c=c)
    lam = np.zeros((4, 4))
    lam[1, 2] = 0.9
    mu = np.full((4, 4), 0.07)
    t = lambda a: torch.tensor(a, device="cuda")
    y = P.pget_forward(ctx, gg, 0, t(lam), t(mu)).cpu().numpy()
    expect = w[3] * 0.9 * np.exp(-c[3] * 1.5 * 0.07)
    assert abs(y[0, 0] - expect) <= 1e-15 and abs(y[0, 1]) <= 1e-15
    gl, gm = P.pget_vjp(ctx, gg, 0, t(lam), t(mu), t(np.array([[1.0, 0.0]])))
    gm = gm.cpu().numpy()
    assert abs(gm[1, 2] + 0.5 * c[3] * expect) <= 1e-15 and abs(gm[1, 3] + c[3] * expect) <= 1e-15
    assert abs(gl.cpu().numpy()[1, 2] - expect / 0.9) <= 1e-15


@pytest.mark.parametrize("prec,tol", [(0, 1e-14), (2, 1e-6)])
def test_tables_of_ones_are_the_plain_model(ctx, O, P, torch, prec, tol):
    """To rounding, not bitwise: the depth kernels multiply by w_j = 1 where the plain
    kernels let the compiler fuse the product into the next addition."""
    n, na, nd, S, col, nl = CASES["two_banks_s5"]
    ph = synth.lattice_phantom(n, nl, seed=9)
    T = O.geom_info(O.geom(n, na, nd, n_sub=S))["T"]
    g1 = P.geometry(n, na, nd, n_sub=S, collimator=col, depth_w=np.ones(T), depth_c=np.ones(T))
    g0 = P.geometry(n, na, nd, n_sub=S, collimator=col)
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    lam, mu = t(ph.lam), t(ph.mu)
    d = t(np.random.default_rng(1).standard_normal((n, n)))
    r = t(np.random.default_rng(2).standard_normal((na, nd)))
    c = lambda x: x.double().cpu().numpy()
    assert rel(c(P.pget_forward(ctx, g1, prec, lam, mu)), c(P.pget_forward(ctx, g0, prec, lam, mu))) <= tol
    assert rel(c(P.pget_jvp(ctx, g1, prec, lam, mu, d, 0.01 * d)), c(P.pget_jvp(ctx, g0, prec, lam, mu, d, 0.01 * d))) <= tol
    for a, b in zip(P.pget_vjp(ctx, g1, prec, lam, mu, r), P.pget_vjp(ctx, g0, prec, lam, mu, r)):
        assert rel(c(a), c(b)) <= 10 * tol


def test_lm_with_depth_tables_matches_oracle(O, P, torch):
    N, NA, ND, S = 24, 30, 182, 3
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=63)
    T = O.geom_info(O.geom(N, NA, ND, n_sub=S))["T"]
    jj = np.arange(T) / (T - 1)  # j = T - 1 is nearest the detector
    w, c = 0.7 + 0.3 * jj, 1.0 + 0.5 * (1.0 - jj) ** 2  # sensitivity and path factor vs distance
    go = O.geom(N, NA, ND, n_sub=S, depth_w=w, depth_c=c)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e4, 64)
    l0, m0 = O.initial_guess(go, y)
    kw = dict(max_iters=6, cg_max_iters=6)
    lo, mo, ro = O.lm(go, O.default_params(**kw), y, l0, m0)
    t = lambda a: torch.tensor(a, device="cuda")
    p = P.default_params(precision=0, cg_rel_tol=1e-10, **kw)
    with P.Context(0) as cx:
        lam, mu = t(l0), t(m0)
        rep = P.pget_lm_solve(cx, P.geometry(N, NA, ND, n_sub=S, depth_w=w, depth_c=c), p, t(y), lam, mu)
    assert rep["acc"] == ro["acc"] and sum(ro["acc"]) >= 2
    assert rel(lam.cpu().numpy(), lo) <= 1e-10 and rel(mu.cpu().numpy(), mo) <= 1e-10
    assert abs(rep["f_final"] - ro["f_final"]) <= 1e-10 * abs(ro["f_final"])


def test_noalloc_rejects_tables(O, P, torch):
    T = O.geom_info(O.geom(16, 8, 91))["T"]
    gg = P.geometry(16, 8, 91, depth_w=np.ones(T))
    lam = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    y = torch.empty((8, 91), dtype=torch.float64, device="cuda")
    assert P.pget_forward_noalloc(gg, 0, lam, lam, y) == 1  # PGET_EINVAL

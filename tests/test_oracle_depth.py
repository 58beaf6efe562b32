"""Pins of the oracle's depth factors of Eq. (5): y = h sum_j w_j lambda_j exp(-c_j E_j)
per sub-ray, with w_j the emission weight (the distance-dependent part of the detector
response r_{m,n}) and c_j >= 1 the vertical-opening correction c_{m,n} of the attenuation,
both tables over the sample index j of the rays.

- A point emitter on an axis-aligned ray through pixel centres, worked by hand: forward
  value and both adjoint gradients (the prefix Q_i carries c_j, the half self-term c_i/2);
- c = c0 everywhere is the plain model with mu scaled by c0 (forward, JVP, VJP);
- w = w0 everywhere scales forward, JVP and VJP by w0;
- tables of ones give the plain model bitwise;
- with general tables the JVP matches central differences and the VJP is its adjoint.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _hand_geom(O, **kw):
    # n = 4, one angle (phi = 0: rays along +x), one bank of two detectors at pitch 1 and
    # r = 3: detector 0 is the line y = row 1, and sample j sits on the centre of column
    # j - 1 (j = 1..4), so bilinear sampling picks single pixels
    return O.geom(4, 1, 2, n_sub=1, n_banks=1, fov_radius=3.0, det_pitch=1.0, **kw)


def test_point_emitter_by_hand(O):
    T = 6
    w = 1.0 + 0.1 * np.arange(T)
    c = 1.0 + 0.2 * np.arange(T)
    g = _hand_geom(O, depth_w=w, depth_c=c)
    assert O.geom_info(g)["T"] == T
    mu0, lam0 = 0.07, 0.9
    lam = np.zeros((4, 4))
    lam[1, 2] = lam0                       # sample j = 3
    mu = np.full((4, 4), mu0)
    y = O.forward(g, lam, mu)
    E3 = 0.5 * mu0 + mu0                   # half its own step, then sample j = 4
    expect = w[3] * lam0 * np.exp(-c[3] * E3)
    assert abs(y[0, 0] - expect) <= 1e-15 and abs(y[0, 1]) <= 1e-15
    r = np.array([[1.0, 0.0]])
    gl, gm = O.vjp(g, lam, mu, r)
    t3 = w[3] * lam0 * np.exp(-c[3] * E3)  # the only emitting sample
    assert abs(gl[1, 2] - w[3] * np.exp(-c[3] * E3)) <= 1e-15
    assert abs(gm[1, 2] + 0.5 * c[3] * t3) <= 1e-15   # its own half step
    assert abs(gm[1, 3] + c[3] * t3) <= 1e-15         # a pixel nearer the detector
    assert abs(gm[1, 1]) <= 1e-15 and abs(gm[1, 0]) <= 1e-15  # behind the emitter
    assert np.abs(gm[[0, 2, 3]]).max() == 0.0


def _case(O, seed=3, n=12, **tables):
    g = O.geom(n, 10, 91, n_sub=3, **tables)
    ph = synth.lattice_phantom(n, 2, radius=1.5, seed=seed)
    rs = np.random.default_rng(seed)
    lam, mu = ph.lam + 0.1, ph.mu + 0.02
    dl, dm = rs.standard_normal(lam.shape), 0.05 * rs.standard_normal(mu.shape)
    r = rs.standard_normal((10, 91))
    return g, lam, mu, dl, dm, r


def test_constant_c_is_scaled_attenuation(O):
    T = O.geom_info(O.geom(12, 10, 91, n_sub=3))["T"]
    c0 = 1.7
    g, lam, mu, dl, dm, r = _case(O, depth_c=np.full(T, c0))
    g0 = O.geom(12, 10, 91, n_sub=3)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(O.forward(g, lam, mu), O.forward(g0, lam, c0 * mu)) <= 1e-13
    assert rel(O.jvp(g, lam, mu, dl, dm), O.jvp(g0, lam, c0 * mu, dl, c0 * dm)) <= 1e-12
    gl, gm = O.vjp(g, lam, mu, r)
    gl0, gm0 = O.vjp(g0, lam, c0 * mu, r)
    assert rel(gl, gl0) <= 1e-12 and rel(gm, c0 * gm0) <= 1e-12


def test_constant_w_scales(O):
    T = O.geom_info(O.geom(12, 10, 91, n_sub=3))["T"]
    w0 = 0.6
    g, lam, mu, dl, dm, r = _case(O, depth_w=np.full(T, w0))
    g0 = O.geom(12, 10, 91, n_sub=3)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(O.forward(g, lam, mu), w0 * O.forward(g0, lam, mu)) <= 1e-13
    assert rel(O.jvp(g, lam, mu, dl, dm), w0 * O.jvp(g0, lam, mu, dl, dm)) <= 1e-12
    gl, gm = O.vjp(g, lam, mu, r)
    gl0, gm0 = O.vjp(g0, lam, mu, r)
    assert rel(gl, w0 * gl0) <= 1e-12 and rel(gm, w0 * gm0) <= 1e-12


def test_tables_of_ones_are_the_plain_model(O):
    T = O.geom_info(O.geom(12, 10, 91, n_sub=3))["T"]
    g, lam, mu, dl, dm, r = _case(O, depth_w=np.ones(T), depth_c=np.ones(T))
    g0 = O.geom(12, 10, 91, n_sub=3)
    assert np.array_equal(O.forward(g, lam, mu), O.forward(g0, lam, mu))
    assert np.array_equal(O.jvp(g, lam, mu, dl, dm), O.jvp(g0, lam, mu, dl, dm))
    for a, b in zip(O.vjp(g, lam, mu, r), O.vjp(g0, lam, mu, r)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", [4, 5])
def test_derivatives_with_tables(O, seed):
    T = O.geom_info(O.geom(12, 10, 91, n_sub=3))["T"]
    rs = np.random.default_rng(seed)
    w, c = rs.uniform(0.5, 1.5, T), rs.uniform(1.0, 2.0, T)
    g, lam, mu, dl, dm, r = _case(O, seed=seed, depth_w=w, depth_c=c)
    jv = O.jvp(g, lam, mu, dl, dm)
    e = 1e-4
    fd = (O.forward(g, lam + e * dl, mu + e * dm) - O.forward(g, lam - e * dl, mu - e * dm)) / (2 * e)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(jv).max()
    gl, gm = O.vjp(g, lam, mu, r)
    lhs, rhs = float(np.sum(jv * r)), float(np.sum(gl * dl) + np.sum(gm * dm))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(jv) * np.linalg.norm(r)
    # the tables change the model (they are not ignored)
    g0 = O.geom(12, 10, 91, n_sub=3)
    assert np.abs(O.forward(g, lam, mu) - O.forward(g0, lam, mu)).max() > 1e-3

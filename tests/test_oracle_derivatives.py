"""Pins of the oracle's Jacobian products (Sec. 2.1, Eq. (2)) and their adjoint.

- the emission part of the derivative equals the forward model itself (Eq. (2), first line);
- central finite differences of the forward model (h = 1e-3, FP64);
- the adjoint identity <J x, y> = <x, J^T y> (the F'* of Sec. 3.1);
- a brute-force dense J on an 8 x 8 grid, columns from JVPs and rows from VJPs;
- the gradient of 1/2 |A(u) - y|^2 against finite differences;
- the attenuation part of the JVP converging to the derivative of the concentric-disk
  closed form;
- the Lipschitz bound of the derivative that Sec. 2.1 proves (a loose bound: a weak pin).
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _case(O, N=16, Na=12, n_det=91, S=3, seed=7):
    g = O.geom(N, Na, n_det, n_sub=S)
    ph = synth.lattice_phantom(N, 3, seed=seed, jitter=0.5)
    rs = np.random.default_rng(seed)
    dl = rs.standard_normal((N, N))
    dm = 0.01 * rs.standard_normal((N, N))
    return g, ph.lam, ph.mu, dl, dm


def test_jvp_emission_part_is_forward(O):
    g, lam, mu, dl, _ = _case(O)
    dy = O.jvp(g, lam, mu, dl, np.zeros_like(dl))
    np.testing.assert_allclose(dy, O.forward(g, dl, mu), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n_det,S", [(91, 1), (182, 5)])
def test_jvp_matches_central_differences(O, n_det, S):
    g, lam, mu, dl, dm = _case(O, n_det=n_det, S=S)
    eps = 1e-3
    # lambda part: F is linear in lambda, the difference quotient is exact up to rounding
    fd_l = (O.forward(g, lam + eps * dl, mu) - O.forward(g, lam - eps * dl, mu)) / (2 * eps)
    jl = O.jvp(g, lam, mu, dl, np.zeros_like(dm))
    assert np.abs(fd_l - jl).max() <= 1e-10 * np.abs(jl).max()
    # mu part: second-order accurate central difference
    fd_m = (O.forward(g, lam, mu + eps * dm) - O.forward(g, lam, mu - eps * dm)) / (2 * eps)
    jm = O.jvp(g, lam, mu, np.zeros_like(dl), dm)
    assert np.linalg.norm(fd_m - jm) <= 1e-6 * np.linalg.norm(jm)
    # the mu part lowers the reading where dm > 0 everywhere (Eq. (2), second line)
    jpos = O.jvp(g, lam, mu, np.zeros_like(dl), np.abs(dm))
    assert np.all(jpos <= 1e-15)


def test_adjoint_identity(O):
    g, lam, mu, dl, dm = _case(O, N=20, Na=15, n_det=182, S=5)
    r = np.random.default_rng(11).standard_normal((g.n_angles, g.n_det))
    Jx = O.jvp(g, lam, mu, dl, dm)
    gl, gm = O.vjp(g, lam, mu, r)
    lhs = float(np.sum(Jx * r))
    rhs = float(np.sum(dl * gl) + np.sum(dm * gm))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jx) * np.linalg.norm(r) * 10


def test_dense_jacobian_8x8(O):
    """Columns J e_i from JVPs and rows J^T e_j from VJPs give the same dense matrix."""
    N, Na, S = 8, 8, 3
    g = O.geom(N, Na, 91, n_sub=S)
    ph = synth.lattice_phantom(N, 2, seed=5, jitter=0.5)
    lam, mu = ph.lam, ph.mu
    npx = N * N
    M = Na * 91
    Jc = np.zeros((M, 2 * npx))
    for i in range(2 * npx):
        e = np.zeros(2 * npx)
        e[i] = 1.0
        Jc[:, i] = O.jvp(g, lam, mu, e[:npx].reshape(N, N), e[npx:].reshape(N, N)).ravel()
    Jr = np.zeros((M, 2 * npx))
    for j in range(M):
        r = np.zeros(M)
        r[j] = 1.0
        gl, gm = O.vjp(g, lam, mu, r.reshape(Na, 91))
        Jr[j] = np.concatenate([gl.ravel(), gm.ravel()])
    scale = np.abs(Jc).max()
    assert np.abs(Jc - Jr).max() <= 1e-12 * scale
    # rank: enough rays to see every pixel of both maps
    assert np.linalg.matrix_rank(Jc, tol=1e-9 * scale) == 2 * npx


def test_gradient_of_data_term_matches_fd(O):
    g, lam, mu, dl, dm = _case(O, N=12, Na=10, S=3)
    y = O.forward(g, lam * 0.9 + 0.05, mu * 1.1)
    def f(l, m):
        r = O.forward(g, l, m) - y
        return 0.5 * float(np.sum(r * r))
    r = O.forward(g, lam, mu) - y
    gl, gm = O.vjp(g, lam, mu, r)
    eps = 1e-4
    d_fd = (f(lam + eps * dl, mu + eps * dm) - f(lam - eps * dl, mu - eps * dm)) / (2 * eps)
    d_an = float(np.sum(gl * dl) + np.sum(gm * dm))
    assert abs(d_fd - d_an) <= 1e-7 * abs(d_an)


def _closed_disk_dmu(s, lam0, mu0, Re, Ra):
    """d/dmu0 of the concentric-disk projection y(s) = 2 lam0/mu0 exp(-mu0 La) sinh(mu0 Le)
    (Eq. (1) for an emitting disk of radius Re inside an attenuating disk of radius Ra,
    Lx = sqrt(Rx^2 - s^2)), differentiated by hand:
    dy/dmu0 = 2 lam0/mu0 exp(-mu0 La) [Le cosh(mu0 Le) - (1/mu0 + La) sinh(mu0 Le)]."""
    Le = np.sqrt(np.clip(Re ** 2 - s ** 2, 0, None))
    La = np.sqrt(np.clip(Ra ** 2 - s ** 2, 0, None))
    val = 2 * lam0 / mu0 * np.exp(-mu0 * La) * (Le * np.cosh(mu0 * Le) - (1 / mu0 + La) * np.sinh(mu0 * Le))
    return np.where(Le > 0, val, 0.0)


def test_attenuation_derivative_converges_to_the_closed_form(O):
    """The μ-part of the JVP (Eq. (2)) against mathematics directly. With μ = μ0 χ, the
    indicator of the attenuating disk, the direction δμ = χ (δλ = 0) is d/dμ0, and the
    closed form's derivative is exact. The oracle's JVP must converge to it as the grid
    is refined, like the forward model."""
    errs = []
    for N in (64, 128, 256):
        g = O.geom(N, 8, 91, n_sub=5, collimator=1)
        p = O.geom_info(g)["pitch"]
        Re, Ra, mu0 = 19.5 * p, 25.5 * p, 4.0 / N  # edges half-way between detector centres
        lam = synth.disk_image(N, Re, 1.0, supersample=8)
        chi = synth.disk_image(N, Ra, 1.0, supersample=8)
        u = np.array([(k - 2) * 2 * p / 6 for k in range(5)])  # triangular sub-rays, S = 5
        w = 1 - np.abs(u) / p
        w = w / w.sum()
        sd = (np.arange(91) - 45) * p
        dyc = sum(w[k] * _closed_disk_dmu(sd + u[k], 1.0, mu0, Re, Ra) for k in range(5))
        dy = O.jvp(g, lam, mu0 * chi, np.zeros((N, N)), chi)
        assert np.all(dyc <= 0.0)  # more attenuation never raises a reading
        errs.append(np.linalg.norm(dy - dyc[None]) / (np.linalg.norm(dyc) * np.sqrt(8)))
    # measured 8.8e-3, 2.8e-3, 9.0e-4: a factor of about 3 per doubling of N
    assert errs[0] <= 1.5e-2 and errs[-1] <= 1.5e-3, errs
    for a, b in zip(errs[:-1], errs[1:]):
        assert a / b >= 2.2, errs


def test_closed_form_derivative_by_differences():
    """The hand derivative above against central differences of the closed form itself
    (no oracle involved), so a slip in the derivative cannot pass as a pin."""
    s = np.linspace(-10.5, 10.5, 15)
    for mu0 in (0.02, 0.05, 0.3):
        h = 1e-6 * mu0
        y = lambda m: 2 / m * np.exp(-m * np.sqrt(np.clip(11.0 ** 2 - s ** 2, 0, None))) * np.sinh(
            m * np.sqrt(np.clip(8.0 ** 2 - s ** 2, 0, None)))
        fd = (y(mu0 + h) - y(mu0 - h)) / (2 * h)
        np.testing.assert_allclose(_closed_disk_dmu(s, 1.0, mu0, 8.0, 11.0), fd, rtol=1e-6, atol=1e-7)


def test_lipschitz_bound_of_the_derivative(O):
    """The Lipschitz lemma of Sec. 2.1 bounds ‖DF(u1) − DF(u2)‖ by
    2 sqrt(π r)(1 + C_λ)(‖λ1 − λ2‖ + ‖μ1 − μ2‖), with C_λ = sqrt(2r)·max λ.

    The left side is the discrete operator norm of the JVP difference: power iteration
    with the VJPs, data weighted by ds dθ = p · 2π/N_a per bin, pixel area 1. The bound
    holds with a ratio of about 0.01. This weak pin catches only gross errors of scale in
    the derivative; the other pins do the fine work."""
    import math
    N, Na = 24, 24
    g = O.geom(N, Na, 91, n_sub=1)
    info = O.geom_info(g)
    r, wbin = info["radius"], info["pitch"] * 2 * math.pi / Na
    rs = np.random.default_rng(0)
    ph = synth.lattice_phantom(N, 3, seed=5)
    l1, m1 = ph.lam, ph.mu
    for scale in (1e-1, 1e-2):
        dl, dm = scale * rs.uniform(0, 1, (N, N)), 0.1 * scale * rs.uniform(0, 1, (N, N))
        l2, m2 = l1 + dl, m1 + dm

        def op(x):
            a, b = x[:N * N].reshape(N, N), x[N * N:].reshape(N, N)
            return O.jvp(g, l1, m1, a, b) - O.jvp(g, l2, m2, a, b)

        def op_t(y):
            a1, b1 = O.vjp(g, l1, m1, y)
            a2, b2 = O.vjp(g, l2, m2, y)
            return np.concatenate([(a1 - a2).ravel(), (b1 - b2).ravel()])

        x = rs.standard_normal(2 * N * N)
        x /= np.linalg.norm(x)
        for _ in range(40):
            x = op_t(wbin * op(x))
            nx = np.linalg.norm(x)
            x /= nx
        lhs = math.sqrt(nx)
        c_lam = math.sqrt(2 * r) * max(l1.max(), l2.max())
        rhs = 2 * math.sqrt(math.pi * r) * (1 + c_lam) * (np.linalg.norm(dl) + np.linalg.norm(dm))
        assert 0 < lhs <= rhs, (scale, lhs, rhs)

"""Pins of the oracle's Jacobian products (Sec. 2.1, Eq. (2)) and their adjoint.

- the emission part of the derivative equals the forward model itself (Eq. (2), first line);
- central finite differences of the forward model (h = 1e-3, FP64);
- the adjoint identity <J x, y> = <x, J^T y> (the F'* of Sec. 3.1);
- a brute-force dense J on an 8 x 8 grid, columns from JVPs and rows from VJPs;
- the gradient of 1/2 |A(u) - y|^2 against finite differences.
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

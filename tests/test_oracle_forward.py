"""Pins of the oracle's forward model (Sec. 2.1, Eq. (1) and its discrete form Eq. (5)).

Nothing here compares the oracle with itself: closed forms of the attenuated ray
transform for disks, rays worked by hand from the definition, exact symmetries of the
geometry, and linearity in the emission map that Eq. (1) states.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth


def _closed_disk(s, lam0, mu0, Re, Ra):
    """Attenuated projection of an emitting disk (radius Re, value lam0) inside a
    concentric attenuating disk (radius Ra >= Re, value mu0), from Eq. (1):
    y(s) = 2 lam0/mu0 exp(-mu0 La) sinh(mu0 Le), Lx = sqrt(Rx^2 - s^2);
    mu0 = 0 gives the plain Radon transform 2 lam0 Le."""
    Le = np.sqrt(np.clip(Re ** 2 - s ** 2, 0, None))
    La = np.sqrt(np.clip(Ra ** 2 - s ** 2, 0, None))
    if mu0 == 0:
        return 2 * lam0 * Le
    return np.where(Le > 0, 2 * lam0 / mu0 * np.exp(-mu0 * La) * np.sinh(mu0 * Le), 0.0)


def _subrays(S, p, triangular=True):
    if triangular:
        u = np.array([(k - (S - 1) / 2) * 2 * p / (S + 1) for k in range(S)])
        w = 1 - np.abs(u) / p
    else:
        u = np.array([(k - (S - 1) / 2) * p / S for k in range(S)])
        w = np.ones(S)
    return u, w / w.sum()


def _disk_case(O, N, S, supersample, mu_scale=4.0, step=0.0, n_angles=8):
    g = O.geom(N, n_angles, 91, n_sub=S, collimator=1, step=step)
    p = O.geom_info(g)["pitch"]
    # disk edges half-way between detector centres, so no ray grazes an edge
    Re, Ra, mu0 = 19.5 * p, 25.5 * p, mu_scale / N
    lam = synth.disk_image(N, Re, 1.0, supersample=supersample)
    mu = synth.disk_image(N, Ra, mu0, supersample=supersample)
    u, w = _subrays(S, p)
    sd = (np.arange(91) - 45) * p
    yc = sum(w[k] * _closed_disk(sd + u[k], 1.0, mu0, Re, Ra) for k in range(S))
    yc0 = sum(w[k] * _closed_disk(sd + u[k], 1.0, 0.0, Re, Ra) for k in range(S))
    y = O.forward(g, lam, mu)
    y0 = O.forward(g, lam, np.zeros_like(mu))
    err = np.linalg.norm(y - yc[None]) / (np.linalg.norm(yc) * np.sqrt(n_angles))
    err0 = np.linalg.norm(y0 - yc0[None]) / (np.linalg.norm(yc0) * np.sqrt(n_angles))
    return err, err0, y


@pytest.mark.parametrize("S", [1, 5])
def test_closed_form_disk_converges(O, S):
    """Discretisation error against the closed form falls with N (area-fraction disks)."""
    errs, errs0 = [], []
    for N in (64, 128, 256):
        e, e0, _ = _disk_case(O, N, S, supersample=8)
        errs.append(e)
        errs0.append(e0)
    assert errs[0] <= 2e-2 and errs0[0] <= 2e-2
    assert errs[-1] <= 2e-3 and errs0[-1] <= 2e-3
    for a, b in zip(errs[:-1], errs[1:]):
        assert a / b >= 1.8
    for a, b in zip(errs0[:-1], errs0[1:]):
        assert a / b >= 1.8


def test_closed_form_point_evaluated_disk(O):
    """Point-evaluated (not rasterised) disks: looser, still convergent."""
    errs = [_disk_case(O, N, 5, supersample=1)[0] for N in (64, 128, 256)]
    assert errs[0] <= 3e-2 and errs[-1] <= 5e-3
    assert errs[0] / errs[1] >= 1.7 and errs[1] / errs[2] >= 1.7


def test_closed_form_equal_radii_and_step(O):
    """R_a = R_e gives lam0/mu0 (1 - exp(-2 mu0 L)); a half-pixel step h = 1/2 (which
    pins the factor h in both sums) agrees with the same closed form."""
    N, S = 128, 3
    for step in (0.0, 0.5):
        g = O.geom(N, 4, 91, n_sub=S, collimator=1, step=step)
        p = O.geom_info(g)["pitch"]
        R, mu0 = 19.25 * p, 3.0 / N  # sub-rays lie on multiples of p/2: no ray grazes the edge
        lam = synth.disk_image(N, R, 2.0, supersample=8)
        mu = synth.disk_image(N, R, mu0, supersample=8)
        u, w = _subrays(S, p)
        sd = (np.arange(91) - 45) * p
        L = lambda s: np.sqrt(np.clip(R ** 2 - s ** 2, 0, None))
        yc = sum(w[k] * 2.0 / mu0 * (1 - np.exp(-2 * mu0 * L(sd + u[k]))) for k in range(S))
        y = O.forward(g, lam, mu)
        err = np.linalg.norm(y - yc[None]) / (np.linalg.norm(yc) * 2)
        assert err < 6e-3, (step, err)


def test_centred_disk_rotation_invariance(O):
    """A centred disk pair projects the same at every angle (row spread small)."""
    _, _, y = _disk_case(O, 128, 5, supersample=8, n_angles=16)
    spread = np.abs(y - y.mean(axis=0, keepdims=True)).max() / np.abs(y).max()
    assert spread < 5e-3


def test_hand_worked_rays(O):
    """3x3 grid, r_Omega = 3/2, h = 1: the 3 samples of the central ray sit on pixel
    centres, so lambda_j, mu_j are pixel values and Eq. (1) can be summed by hand with
    E_j = h (mu_j / 2 + sum of the samples nearer the detector)."""
    lam = np.zeros((3, 3))
    mu = np.zeros((3, 3))
    lam[1] = [1.0, 2.0, 3.0]
    mu[1] = [0.1, 0.2, 0.3]
    lam[:, 1] += [4.0, 0.0, 5.0]
    mu[:, 1] += [0.05, 0.0, 0.25]
    # angles 0, pi/2, pi, 3pi/2 with one detector at s = 0
    g = O.geom(3, 4, 1, n_sub=1, det_pitch=1.0, fov_radius=1.5, step=1.0)
    y = O.forward(g, lam, mu)[:, 0]
    # phi = 0: ray along +x through row 1, detector at +x:
    #   x=+1: lambda 3, E = 0.15;  x=0: lambda 2, E = 0.3 + 0.1;  x=-1: lambda 1, E = 0.5 + 0.05
    y0 = 3 * np.exp(-0.15) + 2 * np.exp(-0.4) + 1 * np.exp(-0.55)
    # phi = pi/2: ray along +y through column 1 (values 4, 2, 5 bottom to top;
    # mu 0.05, 0.2, 0.25), detector at +y:
    y1 = 5 * np.exp(-0.125) + 2 * np.exp(-0.25 - 0.1) + 4 * np.exp(-0.45 - 0.025)
    # phi = pi: ray along -x, detector at -x
    y2 = 1 * np.exp(-0.05) + 2 * np.exp(-0.1 - 0.1) + 3 * np.exp(-0.3 - 0.15)
    # phi = 3 pi / 2: ray along -y, detector at -y
    y3 = 4 * np.exp(-0.025) + 2 * np.exp(-0.05 - 0.1) + 5 * np.exp(-0.25 - 0.125)
    np.testing.assert_allclose(y, [y0, y1, y2, y3], rtol=1e-14)


def test_hand_worked_subrays_and_banks(O):
    """Sub-ray weights 1:2:1 (S = 3, triangular) and bank B looking the other way with
    a half-pitch shift, on hand-placed rays through pixel centres."""
    n = 5
    lam = np.arange(25, dtype=float).reshape(5, 5) / 10
    mu = np.zeros((5, 5))
    # pitch 2 with S = 3 gives sub-ray offsets -1, 0, +1 (spacing 2p/(S+1) = 1);
    # angle 0: ray along +x at height s, i.e. row 2 + s; plain Radon sum of that row.
    g = O.geom(n, 1, 1, n_sub=3, det_pitch=2.0, fov_radius=2.5, step=1.0)
    y = O.forward(g, lam, mu)[0, 0]
    rows = lam.sum(axis=1)
    assert abs(y - (rows[1] + 2 * rows[2] + rows[3]) / 4) < 1e-13
    # two banks of one detector, pitch 2, S = 1: bank A at s = 0 (row 2, along +x),
    # bank B along -x at own offset +1 (p / 2), i.e. image height -1 (row 1)
    g2 = O.geom(n, 1, 2, n_banks=2, n_sub=1, det_pitch=2.0, fov_radius=2.5, step=1.0)
    y2 = O.forward(g2, lam, mu)[0]
    np.testing.assert_allclose(y2, [rows[2], rows[1]], rtol=1e-14)


def test_zero_emission_and_linearity(O):
    N = 32
    g = O.geom(N, 12, 91, n_sub=3)
    ph = synth.lattice_phantom(N, 4, seed=1)
    ph2 = synth.lattice_phantom(N, 4, seed=2)
    assert np.all(O.forward(g, np.zeros((N, N)), ph.mu) == 0.0)
    # Eq. (1) is linear in lambda for fixed mu
    y1 = O.forward(g, ph.lam, ph.mu)
    y2 = O.forward(g, ph2.lam, ph.mu)
    y12 = O.forward(g, 2.0 * ph.lam - 0.5 * ph2.lam, ph.mu)
    np.testing.assert_allclose(y12, 2.0 * y1 - 0.5 * y2, rtol=1e-12, atol=1e-12 * np.abs(y1).max())
    # attenuation only lowers the reading (mu >= 0)
    y0 = O.forward(g, ph.lam, np.zeros((N, N)))
    assert np.all(y1 <= y0 + 1e-12)


def test_bank_b_is_bank_a_on_rotated_maps(O):
    """Without the half-pitch interleave, bank B at phi sees the 180-degree rotated
    maps exactly as bank A does (it looks along phi + pi)."""
    N = 24
    ph = synth.lattice_phantom(N, 3, seed=3, jitter=1.0)
    g = O.geom(N, 10, 182, n_sub=3, interleave=0)
    y = O.forward(g, ph.lam, ph.mu)
    yr = O.forward(g, np.rot90(ph.lam, 2), np.rot90(ph.mu, 2))
    np.testing.assert_allclose(y[:, 91:], yr[:, :91], rtol=1e-11, atol=1e-12)


def test_rot90_permutes_angles(O):
    """Rotating both maps by 90 degrees (grid onto grid) shifts sinogram rows by N_a / 4."""
    N, Na = 20, 16
    ph = synth.lattice_phantom(N, 3, seed=4, jitter=1.0)
    g = O.geom(N, Na, 182, n_sub=5)
    y = O.forward(g, ph.lam, ph.mu)
    yr = O.forward(g, np.rot90(ph.lam), np.rot90(ph.mu))
    np.testing.assert_allclose(yr, np.roll(y, -Na // 4, axis=0), rtol=1e-11, atol=1e-12)


def test_geometry_defaults(O):
    g = O.geom(128, 360, 182, n_sub=5)
    info = O.geom_info(g)
    assert info["T"] == 182 and info["n_banks"] == 2
    assert abs(info["radius"] - 128 / np.sqrt(2)) < 1e-12
    assert abs(info["pitch"] - 2 * info["radius"] / 91) < 1e-12
    with pytest.raises(ValueError):
        O.geom_info(O.geom(1, 10, 91))
    with pytest.raises(ValueError):
        O.geom_info(O.geom(16, 10, 91, n_sub=0))

"""Data from a twice finer grid (Sec. 4: phantoms generated at twice the resolution to
avoid the inverse crime).

CPU: the fine geometry doubles lengths and keeps the scanner; the fine lattice has the
same rods; and, pinned on the oracle against the closed-form attenuated projection of a
disk pair (Eq. (1)), y = 1/2 A_2n(lambda, mu / 2) is data for the n-grid problem that is
closer to the exact projection than the n-grid model itself (the unit conversion is
right: a wrong factor would be off by tens of percent).  GPU: project_fine equals that
oracle computation.
"""
import math

import numpy as np
import pytest

from paper_2604_26745_gb300 import finegrid, pget as P, synth


def _closed_disk(s, lam0, mu0, Re, Ra):
    """Emitting disk (Re, lam0) inside a concentric attenuating disk (Ra, mu0), Eq. (1):
    2 lam0 / mu0 exp(-mu0 La) sinh(mu0 Le), Lx = sqrt(Rx^2 - s^2)."""
    Le = np.sqrt(np.clip(Re ** 2 - s ** 2, 0, None))
    La = np.sqrt(np.clip(Ra ** 2 - s ** 2, 0, None))
    return np.where(Le > 0, 2 * lam0 / mu0 * np.exp(-mu0 * La) * np.sinh(mu0 * Le), 0.0)


def test_fine_geometry_doubles_lengths():
    g = P.geometry(64, 90, 182, n_sub=5, collimator=1)
    f = finegrid.fine_geometry(g)
    r = 64 / math.sqrt(2.0)
    assert (f.n, f.n_angles, f.n_det, f.n_sub, f.collimator, f.n_banks) == (128, 90, 182, 5, 1, 2)
    assert f.fov_radius == pytest.approx(2 * r) and f.det_pitch == pytest.approx(2 * (2 * r / 91))
    assert f.step == 1.0
    g2 = P.geometry(50, 30, 91, n_sub=3, step=0.5, fov_radius=40.0, det_pitch=0.9)
    f2 = finegrid.fine_geometry(g2)
    assert (f2.n, f2.n_banks, f2.step, f2.fov_radius, f2.det_pitch) == (100, 1, 0.5, 80.0, 1.8)


def test_fine_lattice_has_the_same_rods():
    c = synth.lattice_phantom(64, 9, radius=3.0, seed=5)
    f = finegrid.fine_lattice_phantom(64, 9, radius=3.0, seed=5)
    assert f.lam.shape == (128, 128) and np.array_equal(c.rod_lambda, f.rod_lambda)
    down = f.lam.reshape(64, 2, 64, 2).mean(axis=(1, 3))
    assert np.abs(down - c.lam).max() <= 0.05 and abs(down.sum() - c.lam.sum()) <= 5e-3 * c.lam.sum()


def _fine_oracle(O, N, S, n_angles, lam_f, mu_f):
    """1/2 A_2N(lambda, mu/2) with the oracle, the fine geometry written out here."""
    r = N / math.sqrt(2.0)
    p = 2 * r / 91
    gf = O.geom(2 * N, n_angles, 91, n_sub=S, collimator=1, fov_radius=2 * r, det_pitch=2 * p)
    return 0.5 * O.forward(gf, lam_f, 0.5 * mu_f)


def test_fine_data_is_closer_to_the_closed_form(O):
    N, S, na = 64, 5, 8
    g = O.geom(N, na, 91, n_sub=S, collimator=1)
    p = O.geom_info(g)["pitch"]
    Re, Ra, mu0 = 19.5 * p, 25.5 * p, 4.0 / N
    u = np.array([(k - (S - 1) / 2) * 2 * p / (S + 1) for k in range(S)])
    w = 1 - np.abs(u) / p
    w = w / w.sum()
    sd = (np.arange(91) - 45) * p
    yc = sum(w[k] * _closed_disk(sd + u[k], 1.0, mu0, Re, Ra) for k in range(S))
    coarse = O.forward(g, synth.disk_image(N, Re, 1.0), synth.disk_image(N, Ra, mu0))
    fine = _fine_oracle(O, N, S, na, synth.disk_image(2 * N, 2 * Re, 1.0), synth.disk_image(2 * N, 2 * Ra, mu0))
    err = lambda y: np.linalg.norm(y - yc[None]) / (np.linalg.norm(yc) * np.sqrt(na))
    ec, ef = err(coarse), err(fine)
    assert ef <= 5e-3 and ef * 1.8 <= ec, (ec, ef)


@pytest.mark.gpu
def test_project_fine_matches_oracle(O, torch):
    N, S, na = 48, 3, 30
    g = P.geometry(N, na, 91, n_sub=S)
    f = finegrid.fine_lattice_phantom(N, 4, radius=2.0, seed=8)
    ref = _fine_oracle(O, N, S, na, f.lam, f.mu)
    with P.Context(0) as c:
        y = finegrid.project_fine(c, g, P.PGET_F64, torch.tensor(f.lam, device="cuda"),
                                  torch.tensor(f.mu, device="cuda"))
    assert y.shape == (na, 91)
    assert float(np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()) <= 1e-12

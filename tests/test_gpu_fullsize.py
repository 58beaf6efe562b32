"""Operators at the benchmark's full size (128 x 128, 360 angles x 182 detectors x 5
triangular sub-rays, FP32 with Kahan sums) against the FP64 oracle, element by element
over the whole sinogram / gradient (the oracle computes these in about a second)."""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec,tol_y,tol_g", [(2, 1e-6, 2e-6), (0, 1e-12, 1e-12)])
def test_single_request_size_operators(ctx, O, P, torch, prec, tol_y, tol_g):
    n, na, nd, S = 128, 360, 182, 5
    go = O.geom(n, na, nd, n_sub=S)
    g = P.geometry(n, na, nd, n_sub=S)
    ph = synth.lattice_phantom(n, 9, radius=5.0, seed=1100)
    rs = np.random.default_rng(3)
    dl, dm = rs.standard_normal((n, n)), 0.01 * rs.standard_normal((n, n))
    r = rs.standard_normal((na, nd))
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    y = P.pget_forward(ctx, g, prec, t(ph.lam), t(ph.mu)).cpu().numpy()
    assert rel(y, O.forward(go, ph.lam, ph.mu)) <= tol_y
    dy = P.pget_jvp(ctx, g, prec, t(ph.lam), t(ph.mu), t(dl), t(dm)).cpu().numpy()
    assert rel(dy, O.jvp(go, ph.lam, ph.mu, dl, dm)) <= tol_y
    gl, gm = P.pget_vjp(ctx, g, prec, t(ph.lam), t(ph.mu), t(r))
    ol, om = O.vjp(go, ph.lam, ph.mu, r)
    assert rel(gl.cpu().numpy(), ol) <= tol_g
    assert rel(gm.cpu().numpy(), om) <= tol_g

"""Precision stress geometry (512 x 512, 720 angles x 182 detectors x 9 triangular
sub-rays, 17 x 17 rods r = 10 with rod mu ~ U(0.05, 0.12)): the forward sinogram and the
adjoint gradient of every precision mode against the FP64 oracle on the same input,
element by element (max-norm relative).  The measured errors are printed (-s).

Bars: FP64 to rounding; FP32 with Kahan-compensated ray sums below 1e-6 / 2e-6; plain FP32
below 5e-6 / 1e-5, and Kahan must be at least 2x closer to the oracle than plain FP32 on
the sinogram (compensation removes the sum-along-the-ray error; the exp2 of an FP32
attenuation remains).
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


def _mx(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def test_stress512_operators_against_oracle(O, P, torch):
    n, na, nd, S = 512, 720, 182, 9
    ph = synth.lattice_phantom(n, 17, radius=10.0, seed=1500, mu_rod=(0.05, 0.12))
    go = O.geom(n, na, nd, n_sub=S)
    y_ref = O.forward(go, ph.lam, ph.mu)
    y_obs = synth.poisson_noise(y_ref, 1e6, 2500)
    r = y_ref - y_obs
    gl_ref, gm_ref = O.vjp(go, ph.lam, ph.mu, r)
    g = P.geometry(n, na, nd, n_sub=S)
    errs = {}
    with P.Context(0) as ctx:
        for name, prec in (("f64", P.PGET_F64), ("f32_kahan", P.PGET_F32_KAHAN), ("f32", P.PGET_F32)):
            dt = P.dtype_of(prec)
            lam = torch.tensor(ph.lam, dtype=dt, device="cuda")
            mu = torch.tensor(ph.mu, dtype=dt, device="cuda")
            y = P.pget_forward(ctx, g, prec, lam, mu).double().cpu().numpy()
            gl, gm = P.pget_vjp(ctx, g, prec, lam, mu, torch.tensor(r, dtype=dt, device="cuda"))
            errs[name] = (_mx(y, y_ref), max(_mx(gl.double().cpu().numpy(), gl_ref),
                                             _mx(gm.double().cpu().numpy(), gm_ref)))
    print("stress512 max-norm relative error vs oracle (sinogram, gradient):", errs)
    assert errs["f64"][0] <= 1e-12 and errs["f64"][1] <= 1e-11
    assert errs["f32_kahan"][0] <= 1e-6 and errs["f32_kahan"][1] <= 2e-6
    assert errs["f32"][0] <= 5e-6 and errs["f32"][1] <= 1e-5
    assert errs["f32_kahan"][0] * 2 <= errs["f32"][0]

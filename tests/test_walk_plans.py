"""Host-side launch plans of the ray walks (pget_walk_plans, no GPU).

The adjoint's phase-coloured row buffers rest on one geometric claim: the rays of slots t
and t + K (K the phase count the geometry needs) never touch the same pixel of a view, so
each buffer is written by one ray per pixel.  The tests check that claim by brute force,
enumerating every sample of every ray of sampled views with positions built here from the
geometry's definition (slot lattice, canonical frame), and check that it fails with one
phase fewer, so that the brute force can see a conflict at all.
"""
import math

import numpy as np
import pytest

from paper_2604_26745_gb300 import pget as P


def _views(n, n_angles, n_det, S, collimator=1):
    """Per view (bank, angle): canonical-frame origin, ray step and slot step (pixel index
    units), slot count, in the library's slot order (lattice index over the gcd step)."""
    nbanks = 2 if n_det == 182 else 1
    nb = n_det // nbanks
    h, r = 1.0, n / math.sqrt(2.0)
    p = 2 * r / nb
    c = 0.5 * (n - 1)
    sigma = p / (2 * (S + 1)) if collimator == 1 else p / (2 * S)
    out = []
    for b in range(nbanks):
        ms = []
        for d in range(nb):
            for k in range(S):
                a = 2 * d - nb + 1 + b
                ms.append(a * (S + 1) + 2 * (2 * k - S + 1) if collimator == 1 else a * S + (2 * k - S + 1))
        mn, mx = min(ms), max(ms)
        g = 0
        for m in ms:
            g = math.gcd(g, m - mn)
        g = g or 1
        ns = (mx - mn) // g + 1
        for a in range(n_angles):
            psi = 2 * math.pi * a / n_angles + b * math.pi
            ct, st = math.cos(psi), math.sin(psi)
            s0, t0, ds = mn * sigma, -r + 0.5 * h, g * sigma
            px, py = -s0 * st + t0 * ct + c, s0 * ct + t0 * st + c
            Dx, Dy, Rx, Ry = h * ct, h * st, -ds * st, ds * ct
            if abs(ct) > abs(st):
                px, py, Dx, Dy, Rx, Ry = py, px, Dy, Dx, Ry, Rx
            if Dy < 0:
                py, Dy, Ry = (n - 1) - py, -Dy, -Ry
            out.append((a, px, py, Dx, Dy, Rx, Ry, ns))
    return out, math.ceil(2 * r / h)


def _phase_conflicts(n, n_angles, n_det, S, K, angles, collimator=1):
    """Pixels touched by two different rays of one phase (slot mod K), over the views of
    the given angles: every in-grid sample (base pixel in [-1, n - 1]^2) touches the four
    pixels of its bilinear cell."""
    views, T = _views(n, n_angles, n_det, S, collimator)
    j = np.arange(T, dtype=np.float64)
    bad = 0
    for (a, px, py, Dx, Dy, Rx, Ry, ns) in views:
        if a not in angles:
            continue
        per_phase = [[] for _ in range(K)]
        for t in range(ns):
            X = px + t * Rx + j * Dx
            Y = py + t * Ry + j * Dy
            ix, iy = np.floor(X).astype(np.int64), np.floor(Y).astype(np.int64)
            ok = (ix >= -1) & (ix <= n - 1) & (iy >= -1) & (iy <= n - 1)
            ix, iy = ix[ok], iy[ok]
            W = n + 3
            keys = np.concatenate([(iy + 1) * W + ix + 1, (iy + 1) * W + ix + 2,
                                   (iy + 2) * W + ix + 1, (iy + 2) * W + ix + 2])
            per_phase[t % K].append(np.unique(keys))
        for ks in per_phase:
            if ks:
                allk = np.concatenate(ks)
                bad += len(allk) - len(np.unique(allk))
    return bad


GEOS = [  # (n, n_angles, n_det, n_sub, collimator)
    (128, 360, 182, 5, 1),   # single-request workload
    (64, 90, 91, 1, 1),      # plain LM workload
    (256, 360, 182, 5, 1),   # differentiation workload
    (40, 36, 182, 5, 1),
    (27, 17, 91, 3, 1),
    (96, 90, 182, 7, 1),
]


@pytest.mark.parametrize("geo", GEOS)
@pytest.mark.parametrize("prec", [P.PGET_F32_KAHAN, P.PGET_F64])
def test_adjoint_phases_never_share_a_pixel(geo, prec):
    n, na, nd, S, coll = geo
    g = P.geometry(n, na, nd, n_sub=S, collimator=coll)
    info = P.geometry_info(g)
    views, T = _views(n, na, nd, S, coll)
    assert info["n_samples"] == T and info["max_slots"] == max(v[-1] for v in views)
    pl = P.walk_plans(g, prec)
    K = pl["phases_needed"]
    assert K > 0 and pl["adjoint_phases"] in (0, K)
    step = max(1, na // 24)
    angles = set(range(0, na, step)) | {na // 8, na // 4 - 1, 3 * na // 8}  # near 45 degrees too
    assert _phase_conflicts(n, na, nd, S, K, angles, coll) == 0


def test_one_phase_fewer_conflicts():
    """The brute force sees conflicts when the phase count is too small (here one fewer than
    the single-request geometry needs)."""
    g = P.geometry(128, 360, 182, n_sub=5)
    K = P.walk_plans(g, P.PGET_F32_KAHAN)["phases_needed"]
    assert K > 1
    assert _phase_conflicts(128, 360, 182, 5, K - 1, set(range(0, 360, 15))) > 0


@pytest.mark.parametrize("geo", GEOS + [(24, 8, 182, 10, 1), (36, 20, 182, 4, 0), (512, 720, 182, 9, 1)])
@pytest.mark.parametrize("prec", [P.PGET_F32, P.PGET_F32_KAHAN, P.PGET_F64, P.PGET_MIXED])
def test_plans_fit_their_budgets(geo, prec):
    n, na, nd, S, coll = geo
    g = P.geometry(n, na, nd, n_sub=S, collimator=coll)
    pl = P.walk_plans(g, prec)
    assert pl["threads"] % 32 == 0 and pl["threads"] >= P.geometry_info(g)["max_slots"]
    for op, kb in (("forward", 64), ("jvp", 72), ("vjp", 72)):
        q = pl[op]
        assert 1 <= q["rows_per_chunk"] <= n + 1
        assert q["chunks"] == -(-(n + 1) // q["rows_per_chunk"])
        assert 0 < q["smem_bytes"] <= kb * 1024 or q["rows_per_chunk"] == 1
    assert pl["adjoint_phases"] in (0, pl["phases_needed"]) and pl["adjoint_phases"] <= 16


def test_walk_plans_refuses_bad_input():
    g = P.geometry(32, 10, 91)
    with pytest.raises(ValueError):
        P.walk_plans(g, 7)

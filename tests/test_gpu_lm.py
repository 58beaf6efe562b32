"""GPU parity of the CG solve (Eq. (9)) and the LM iteration (Sec. 2.2, 3.1) against the
FP64 oracle on identical seeded inputs (noisy data drawn once on the host)."""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


def rel2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem(O, n, na, nd, S, n_lat, radius, counts, seed):
    go = O.geom(n, na, nd, n_sub=S)
    ph = synth.lattice_phantom(n, n_lat, radius=radius, seed=1000 + seed)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), counts, 2000 + seed)
    return go, ph, y


@pytest.mark.parametrize("prec", [0, 2])
def test_cg_parity(ctx, O, P, torch, prec):
    """Before CG converges its iterates are a smooth function of the data, so the GPU
    and oracle trajectories agree to rounding (10 steps).  Run to a 1e-10 residual both
    land on the same solution within the conditioning of the system; past that point
    CG iterates chase rounding noise (a 1e-15 change of the right-hand side moves the
    oracle's own 25-step iterate by ~1e-7), so no tighter comparison is meaningful."""
    n, na, nd, S = 24, 24, 182, 3
    go, ph, y = _problem(O, n, na, nd, S, 3, 2.0, 1e4, 1)
    g = P.geometry(n, na, nd, n_sub=S)
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    b = np.random.default_rng(5).standard_normal(2 * n * n)
    for its, nu, tol_cg, tol in ((10, 0.5, 1e-14, 1e-9 if prec == 0 else 2e-4),
                                 (600, 50.0, 1e-9, 1e-6 if prec == 0 else 2e-3)):
        pr = O.default_params(cg_max_iters=its, cg_rel_tol=tol_cg)
        Wl = O.reg_weights(ph.lam, pr.tv_eps)
        Wm = O.reg_weights(ph.mu, pr.tv_eps)
        x_ref, it_ref = O.cg(go, pr, ph.lam, ph.mu, Wl, Wm, nu, b)
        p = P.default_params(cg_max_iters=its, cg_rel_tol=tol_cg if prec == 0 else 1e-6, precision=prec)
        x, it = P.pget_cg_solve(ctx, g, p, t(ph.lam), t(ph.mu), nu, t(b))
        if its == 10:
            assert it == it_ref == 10
        else:
            assert it < its and it_ref < its
            if prec == 0:
                assert abs(it - it_ref) <= 5
        assert rel2(x.cpu().numpy(), x_ref) <= tol, (its, rel2(x.cpu().numpy(), x_ref))


def test_initial_guess_parity(ctx, O, P, torch):
    go, ph, y = _problem(O, 32, 30, 91, 1, 4, 2.0, 1e4, 2)
    l0, m0 = O.initial_guess(go, y, mu_init=0.01)
    g = P.geometry(32, 30, 91)
    p = P.default_params(precision=0)
    lam, mu = P.pget_initial_guess(ctx, g, p, torch.tensor(y, device="cuda"), 0.01)
    assert abs(lam[0, 0].item() - l0[0, 0]) <= 1e-12 * l0[0, 0]
    assert torch.all(mu == 0.01)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4), (1, 3e-4)])
def test_lm_parity_stable_regime(ctx, O, P, torch, prec, tol):
    """Six LM iterations with 8 CG steps each: in this regime the iteration is a smooth
    function of its inputs (the oracle moves by 1e-14 under a 1e-15 change of the data),
    so the GPU must reproduce the oracle's accept/reject pattern, objective trace and
    iterate to rounding."""
    n, na, nd, S = 32, 30, 182, 3
    go, ph, y = _problem(O, n, na, nd, S, 4, 2.5, 1e4, 3)
    pr = O.default_params(max_iters=6, cg_max_iters=8, cg_rel_tol=1e-10)
    l0, m0 = O.initial_guess(go, y)
    lr, mr, rep_ref = O.lm(go, pr, y, l0, m0)
    g = P.geometry(n, na, nd, n_sub=S)
    p = P.default_params(max_iters=6, cg_max_iters=8, cg_rel_tol=1e-10, precision=prec)
    dt = P.dtype_of(prec)
    lam = torch.tensor(l0, dtype=dt, device="cuda")
    mu = torch.tensor(m0, dtype=dt, device="cuda")
    rep = P.pget_lm_solve(ctx, g, p, torch.tensor(y, dtype=dt, device="cuda"), lam, mu)
    assert rep["acc"] == rep_ref["acc"] and sum(rep["acc"]) >= 2
    assert rel2(lam.cpu().numpy(), lr) <= tol
    assert rel2(mu.cpu().numpy(), mr) <= tol
    np.testing.assert_allclose(rep["f"], rep_ref["f"], rtol=max(tol, 1e-12))
    np.testing.assert_allclose(rep["nu"], rep_ref["nu"], rtol=max(tol, 1e-12))
    assert rep["cg_iters"] == rep_ref["cg_iters"]


def _c1(O):
    n = 64
    go = O.geom(n, 90, 91, n_sub=1)
    ph = synth.lattice_phantom(n, 9, radius=3.0, seed=1000)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e4, 2000)
    return n, go, ph, y


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-4)])
def test_lm_c1_geometry_stable_regime(ctx, O, P, torch, prec, tol):
    """The full plain-LM configuration (64 x 64, 9 x 9 rods r = 3, 90 angles x 91
    detectors, one sub-ray, Poisson 1e4, 10 LM iterations, TV prior alpha 1e-2) with CG
    capped at 8 steps, where the iteration is a smooth function of its inputs."""
    n, go, ph, y = _c1(O)
    pr = O.default_params(max_iters=10, cg_max_iters=8, cg_rel_tol=1e-10)
    l0, m0 = O.initial_guess(go, y)
    lr, mr, rep_ref = O.lm(go, pr, y, l0, m0)
    g = P.geometry(n, 90, 91, n_sub=1)
    p = P.default_params(max_iters=10, cg_max_iters=8, cg_rel_tol=1e-10, precision=prec)
    dt = P.dtype_of(prec)
    lam = torch.tensor(l0, dtype=dt, device="cuda")
    mu = torch.tensor(m0, dtype=dt, device="cuda")
    rep = P.pget_lm_solve(ctx, g, p, torch.tensor(y, dtype=dt, device="cuda"), lam, mu)
    assert rep["acc"] == rep_ref["acc"]
    assert rel2(lam.cpu().numpy(), lr) <= tol
    assert rel2(mu.cpu().numpy(), mr) <= tol
    np.testing.assert_allclose(rep["f"], rep_ref["f"], rtol=max(tol, 1e-12))


def test_lm_c1_statistical(ctx, O, P, torch):
    """The plain-LM configuration with its own CG cap of 50 steps.  There the finite-
    precision iteration is chaotic: the oracle run with a different summation order of its
    adjoint, or with the data changed by 1e-14, lands up to ~1e-2 away (measured).  No
    implementation with different rounding can match it pointwise, so the GPU result is
    required to (a) make the same accept/reject decisions, (b) reach the same objective
    within 3x the spread of those oracle variants, (c) improve on the initial guess as
    much as they do, and (d) be bitwise reproducible from run to run."""
    n, go, ph, y = _c1(O)
    pr = O.default_params(max_iters=10, cg_max_iters=50, cg_rel_tol=1e-10)
    l0, m0 = O.initial_guess(go, y)
    variants = []
    for chunks, eps in ((32, 0.0), (7, 0.0), (13, 0.0), (32, 1e-14)):
        O.set_vjp_chunks(chunks)
        yv = y * (1 + eps * np.random.default_rng(5).standard_normal(y.shape))
        variants.append(O.lm(go, pr, yv, l0, m0))
    O.set_vjp_chunks(32)
    ref = variants[0][2]
    f_spread = max(abs(v[2]["f_final"] - ref["f_final"]) for v in variants[1:])
    g = P.geometry(n, 90, 91, n_sub=1)
    p = P.default_params(max_iters=10, cg_max_iters=50, cg_rel_tol=1e-10, precision=P.PGET_F64)
    outs = []
    for _ in range(2):
        lam = torch.tensor(l0, device="cuda")
        mu = torch.tensor(m0, device="cuda")
        rep = P.pget_lm_solve(ctx, g, p, torch.tensor(y, device="cuda"), lam, mu)
        outs.append((lam.cpu().numpy(), mu.cpu().numpy(), rep))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    lam, mu, rep = outs[0]
    assert all(rep["acc"] == v[2]["acc"] for v in variants)
    assert abs(rep["f_final"] - ref["f_final"]) <= 3 * f_spread + 1e-9 * ref["f_final"]
    e_l = [rel2(v[0], ph.lam) for v in variants]
    e_m = [rel2(v[1], ph.mu) for v in variants]
    assert min(e_l) - 0.01 <= rel2(lam, ph.lam) <= max(e_l) + 0.01
    assert min(e_m) - 0.02 <= rel2(mu, ph.mu) <= max(e_m) + 0.02
    assert rel2(lam, variants[0][0]) < 0.05 and rel2(mu, variants[0][1]) < 0.05


def test_lm_c2_geometry_stable_regime(ctx, O, P, torch):
    """Single-request geometry (128 x 128, 360 angles x 182 detectors x 5 triangular
    sub-rays, Poisson 1e5) in the FP32-Kahan path against the FP64 oracle: three LM
    iterations with CG capped at 8 steps (stable regime); bar 1e-4 relative L2."""
    n = 128
    go = O.geom(n, 360, 182, n_sub=5)
    ph = synth.lattice_phantom(n, 9, radius=5.0, seed=1100)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e5, 2100)
    pr = O.default_params(max_iters=3, cg_max_iters=8, cg_rel_tol=1e-6)
    l0, m0 = O.initial_guess(go, y)
    lr, mr, rep_ref = O.lm(go, pr, y, l0, m0)
    g = P.geometry(n, 360, 182, n_sub=5)
    p = P.default_params(max_iters=3, cg_max_iters=8, cg_rel_tol=1e-6, precision=P.PGET_F32_KAHAN)
    lam = torch.tensor(l0, dtype=torch.float32, device="cuda")
    mu = torch.tensor(m0, dtype=torch.float32, device="cuda")
    rep = P.pget_lm_solve(ctx, g, p, torch.tensor(y, dtype=torch.float32, device="cuda"), lam, mu)
    assert rep["acc"] == rep_ref["acc"]
    assert rel2(lam.cpu().numpy(), lr) <= 1e-4
    assert rel2(mu.cpu().numpy(), mr) <= 1e-4


def test_graph_replay_matches_direct_launches(ctx, O, P, torch, monkeypatch):
    """The LM body runs as a captured CUDA graph by default; replays and the direct
    (graph-free) launch sequence must give bitwise-identical results."""
    n, na, nd, S = 48, 60, 182, 5
    go, ph, y = _problem(O, n, na, nd, S, 5, 2.5, 1e5, 7)
    g = P.geometry(n, na, nd, n_sub=S)
    p = P.default_params(max_iters=4, cg_max_iters=10, precision=P.PGET_F32_KAHAN)
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    outs = []
    for no_graph in ("0", "0", "1"):
        monkeypatch.setenv("PGET_NO_GRAPH", no_graph)
        lam, mu = P.pget_initial_guess(ctx, g, p, yd)
        rep = P.pget_lm_solve(ctx, g, p, yd, lam, mu)
        outs.append((lam.clone(), mu.clone(), rep["f"]))
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1]) and o[2] == outs[0][2]


def _single128(P, torch):
    """The oracle-stored single-request case (128^2, 360 x 182 x 5, Poisson 1e5, 20 LM x
    CG <= 30): data rebuilt bitwise from the stored counts, the oracle's reconstruction and
    its measured spreads (tests/golden/make_lm_single128.py)."""
    import json
    import os
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lm_single128")
    z = np.load(base + ".npz")
    with open(base + ".json") as fh:
        meta = json.load(fh)
    c = meta["case"]
    y = z["counts"].astype(np.float64) * float(z["ymax"]) / c["counts"]
    g = P.geometry(c["n"], c["n_angles"], c["n_det"], n_sub=c["n_sub"], collimator=c["collimator"])
    ref = np.concatenate([z["lam"].ravel(), z["mu"].ravel()])
    return c, meta, y, g, ref


def _solve_c2(ctx, P, torch, g, c, prec, y):
    p = P.default_params(max_iters=c["max_iters"], cg_max_iters=c["cg_max_iters"], cg_rel_tol=c["cg_rel_tol"],
                         precision=prec)
    yd = torch.tensor(y, dtype=P.dtype_of(prec), device="cuda")
    lam, mu = P.pget_initial_guess(ctx, g, p, yd)
    rep = P.pget_lm_solve(ctx, g, p, yd, lam, mu)
    return np.concatenate([lam.double().cpu().numpy().ravel(), mu.double().cpu().numpy().ravel()]), rep


def test_lm_single_request_configuration_fp64_vs_oracle(ctx, P, torch):
    """The benchmark's configuration in full (20 LM iterations, CG <= 30) in FP64 against the
    oracle's own reconstruction of the same data.  At this configuration rounding alone moves
    the result: the oracle's variants (other summation orders, relative 1e-14 changes of the
    data) lie 1.7e-6 to 7.7e-5 from it, and the GPU's own result moves by 1e-4 to 1e-3
    under relative 1e-14 changes of the data.  The bar: the same accept/reject trace as the
    oracle, and a distance within twice the larger of the two measured rounding spreads."""
    c, meta, y, g, ref = _single128(P, torch)
    u, rep = _solve_c2(ctx, P, torch, g, c, 0, y)
    assert rep["acc"] == meta["base"]["accepted"], (rep["acc"], meta["base"]["accepted"])
    own = []
    for s in (31, 32):  # the oracle's perturbation seeds
        sign = np.where(np.random.default_rng(s).random(y.shape) < 0.5, -1.0, 1.0)
        up, rp = _solve_c2(ctx, P, torch, g, c, 0, y * (1.0 + 1e-14 * sign))
        assert rp["acc"] == rep["acc"]
        own.append(rel2(up, u))
    bar = 2.0 * max(meta["spread_max_rel_l2_u"], max(own))
    d = rel2(u, ref)
    assert d <= bar, (d, bar, own)


@pytest.mark.parametrize("prec", [2, 3])
def test_lm_single_request_configuration_float_regression(ctx, P, torch, prec):
    """The same configuration with the float Jacobian products of CG (PGET_F32_KAHAN, and
    PGET_MIXED with its double objective).  At iteration 2 the model decrease of the
    projected CG step is a small difference of terms of ~1e5 (+781 in FP64, negative with
    float products, whose adjoint is the transpose of their JVP only to ~2e-9): the step is
    rejected and the trajectory departs, ending ~5.7 % from the oracle with a ~5 % higher
    objective.  This is reported, not a parity claim; the bars guard against regressions:
    distance <= 0.1, final objective within 10 % of the oracle's."""
    c, meta, y, g, ref = _single128(P, torch)
    u, rep = _solve_c2(ctx, P, torch, g, c, prec, y)
    assert rel2(u, ref) <= 0.1
    assert rep["f_final"] <= 1.1 * meta["base"]["f_final"]
    assert rep["acc"][0] == meta["base"]["accepted"][0] == 1

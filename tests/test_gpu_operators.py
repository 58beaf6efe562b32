"""GPU parity of the operators (forward, JVP, VJP, prior) against the FP64 oracle, called
through the C ABI on identical seeded inputs.

Tolerances (relative, max-norm over the output unless stated):
  PGET_F64        1e-12  (same arithmetic as the oracle up to rounding order and exp)
  PGET_F32_KAHAN  sinogram and JVP 1e-6, gradient 2e-6: float exp(-E) carries |E| 2^-24
                  relative error (E up to ~10 here), positions are exact (32.32 fixed point);
                  measured at most 1.6e-7 / 1.2e-7 / 3.4e-7 over these cases and the full
                  128^2 geometry
  PGET_F32        sinogram and JVP 2e-6, gradient 5e-6 (uncompensated float sums of ~200
                  terms; measured at most 4.3e-7)
  PGET_MIXED  the FP32-Kahan bars: the same ray kernels on double inputs rounded
                  to float, outputs widened to double
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 1e-12), 2: (1e-6, 2e-6), 1: (2e-6, 5e-6), 3: (1e-6, 2e-6)}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    # name: (n, n_angles, n_det, n_sub, collimator, n_lat)
    "c1_like": (32, 30, 91, 1, 1, 4),
    "two_banks_s5": (40, 36, 182, 5, 1, 4),
    "box_even_s4": (36, 20, 182, 4, 0, 3),
    "odd_n_s3": (27, 17, 91, 3, 1, 3),
    # 1009 lattice slots per view (910 on a sub-ray): more than 896 threads, so the
    # 64-register instantiation runs
    "many_rays_s10": (24, 8, 182, 10, 1, 3),
}


def _inputs(n, n_lat, seed):
    ph = synth.lattice_phantom(n, n_lat, seed=seed, jitter=0.7)
    rs = np.random.default_rng(seed)
    return ph.lam, ph.mu, rs.standard_normal((n, n)), 0.01 * rs.standard_normal((n, n))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 2, 1, 3])
def test_forward_jvp_vjp_parity(ctx, O, P, torch, case, prec):
    n, na, nd, S, col, nl = CASES[case]
    lam, mu, dl, dm = _inputs(n, nl, 100 + n)
    go = O.geom(n, na, nd, n_sub=S, collimator=col)
    gg = P.geometry(n, na, nd, n_sub=S, collimator=col)
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol_y, tol_g = TOL[prec]
    y = P.pget_forward(ctx, gg, prec, t(lam), t(mu))
    assert rel(y.cpu().numpy(), O.forward(go, lam, mu)) <= tol_y
    dy = P.pget_jvp(ctx, gg, prec, t(lam), t(mu), t(dl), t(dm))
    assert rel(dy.cpu().numpy(), O.jvp(go, lam, mu, dl, dm)) <= tol_y
    r = np.random.default_rng(7).standard_normal((na, nd))
    gl, gm = P.pget_vjp(ctx, gg, prec, t(lam), t(mu), t(r))
    ol, om = O.vjp(go, lam, mu, r)
    assert rel(gl.cpu().numpy(), ol) <= tol_g
    assert rel(gm.cpu().numpy(), om) <= tol_g


def test_adjoint_identity_gpu(ctx, P, torch):
    n, na, nd = 48, 40, 182
    lam, mu, dl, dm = _inputs(n, 5, 3)
    g = P.geometry(n, na, nd, n_sub=5)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    r = np.random.default_rng(9).standard_normal((na, nd))
    Jx = P.pget_jvp(ctx, g, 0, t(lam), t(mu), t(dl), t(dm)).cpu().numpy()
    gl, gm = P.pget_vjp(ctx, g, 0, t(lam), t(mu), t(r))
    lhs = float(np.sum(Jx * r))
    rhs = float(np.sum(dl * gl.cpu().numpy()) + np.sum(dm * gm.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jx) * np.linalg.norm(r) * 10


def test_vjp_deterministic(ctx, P, torch):
    n, na, nd = 64, 45, 182
    lam, mu, _, _ = _inputs(n, 6, 5)
    g = P.geometry(n, na, nd, n_sub=5)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    r = t(np.random.default_rng(2).standard_normal((na, nd)))
    a1 = [x.clone() for x in P.pget_vjp(ctx, g, 2, t(lam), t(mu), r)]
    a2 = P.pget_vjp(ctx, g, 2, t(lam), t(mu), r)
    assert torch.equal(a1[0], a2[0]) and torch.equal(a1[1], a2[1])


# Runs in a child process on a library built with -DPGET_TUNING (the only build that reads
# the shared-memory budgets of the walk plans from the environment): forward, JVP and
# adjoint three times each at one budget, saved for the parent to compare.
_CHUNK_CHILD = r"""
import sys
import numpy as np
import torch
from paper_2604_26745_gb300 import pget as P, synth
P.load(sys.argv[1])
n, na, S = (int(x) for x in sys.argv[3:6])
ph = synth.lattice_phantom(n, 9, radius=3.0, seed=41)
g = P.geometry(n, na, 182, n_sub=S)
t = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
lam, mu = t(ph.lam), t(ph.mu)
rs = np.random.default_rng(42)
dl, dm = t(rs.standard_normal((n, n))), t(0.01 * rs.standard_normal((n, n)))
r = t(rs.standard_normal((na, 182)))
out = {}
with P.Context(0) as c:
    for k in range(3):
        gl, gm = P.pget_vjp(c, g, P.PGET_F32_KAHAN, lam, mu, r)
        y = P.pget_forward(c, g, P.PGET_F32_KAHAN, lam, mu)
        dy = P.pget_jvp(c, g, P.PGET_F32_KAHAN, lam, mu, dl, dm)
        for name, v in (("y", y), ("dy", dy), ("gl", gl), ("gm", gm)):
            out[f"{name}{k}"] = v.cpu().numpy()
np.savez(sys.argv[2], **out)
"""


@pytest.fixture(scope="module")
def tuning_lib(tmp_path_factory):
    from paper_2604_26745_gb300 import build
    d = tmp_path_factory.mktemp("tuning_build")
    return build.build(extra=["-DPGET_TUNING"], out=str(d / "libpget_tuning.so"), build_dir=str(d))


@pytest.mark.parametrize("geo", [(128, 360, 5), (96, 90, 7)])
def test_walks_independent_of_chunk_height(tuning_lib, tmp_path, geo):
    """The chunk height is a tuning choice (shared-memory budget): forward and JVP must be
    bitwise the same at every height (each ray sums in the same order), the adjoint the
    same up to rounding (carried rows split the per-pixel sums differently), and every
    operator bitwise reproducible at a fixed height.  A stencil column written by one
    thread and cleared by another would break the last two.  The budgets reach the plans
    only in a -DPGET_TUNING build, which the test builds and runs in child processes; an
    adjoint that stays bitwise equal at every budget means the budget did not take effect,
    and fails the test."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for kb in (72, 40, 100):
        env = dict(os.environ, PGET_SMEM_KB_FWD=str(kb), PGET_SMEM_KB_JVP=str(kb), PGET_SMEM_KB_VJP=str(kb),
                   PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
        f = tmp_path / f"kb{kb}.npz"
        subprocess.run([sys.executable, "-c", _CHUNK_CHILD, tuning_lib, str(f), *(str(x) for x in geo)],
                       env=env, cwd=root, check=True, timeout=600)
        res[kb] = dict(np.load(f))
    moved = False
    for kb, d in res.items():
        for name in ("y", "dy", "gl", "gm"):
            assert np.array_equal(d[name + "1"], d[name + "0"]) and np.array_equal(d[name + "2"], d[name + "0"]), \
                (kb, name)
        ref = res[72]
        assert np.array_equal(d["y0"], ref["y0"]) and np.array_equal(d["dy0"], ref["dy0"]), kb
        for name in ("gl0", "gm0"):
            assert float(np.abs(d[name] - ref[name]).max() / np.abs(ref[name]).max()) <= 1e-6, (kb, name)
            moved |= not np.array_equal(d[name], ref[name])
    assert moved, "the adjoint is bitwise equal at every budget: the chunk height did not change"


# Child process on the -DPGET_TUNING build: the adjoint three times at one geometry and
# precision, with the plan's phase count (PGET_VJP_DESIGN forces phase buffers or stencils).
_DESIGN_CHILD = r"""
import sys
import numpy as np
import torch
from paper_2604_26745_gb300 import pget as P, synth
P.load(sys.argv[1])
n, na, nd, S, prec = (int(x) for x in sys.argv[3:8])
ph = synth.lattice_phantom(n, 9 if n >= 64 else 4, radius=3.0, seed=43, jitter=0.7)
g = P.geometry(n, na, nd, n_sub=S)
dt = torch.float64 if prec in (0, 3) else torch.float32
t = lambda x: torch.tensor(x, dtype=dt, device="cuda")
lam, mu = t(ph.lam), t(ph.mu)
r = t(np.random.default_rng(44).standard_normal((na, nd)))
out = {"phases": np.int64(P.walk_plans(g, prec)["adjoint_phases"])}
with P.Context(0) as c:
    for k in range(3):
        gl, gm = P.pget_vjp(c, g, prec, lam, mu, r)
        out[f"gl{k}"], out[f"gm{k}"] = gl.cpu().numpy(), gm.cpu().numpy()
np.savez(sys.argv[2], **out)
"""


@pytest.mark.parametrize("geo", [(128, 360, 182, 5, 2), (64, 90, 91, 1, 0), (40, 36, 182, 5, 1),
                                 (96, 45, 182, 7, 2), (27, 17, 91, 3, 3)])
def test_adjoint_designs_agree(tuning_lib, tmp_path, geo):
    """The two accumulation schemes of the adjoint (phase-coloured row buffers and per-ray
    stencils) give the same gradient up to the order of the per-pixel sums, each bitwise
    reproducible: FP64 within 1e-12, the float walks within 1e-6 (max-norm relative)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for arm in ("phases", "stencil"):
        env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""),
                   PGET_VJP_DESIGN=arm)
        f = tmp_path / f"{arm}.npz"
        subprocess.run([sys.executable, "-c", _DESIGN_CHILD, tuning_lib, str(f), *(str(x) for x in geo)],
                       env=env, cwd=root, check=True, timeout=600)
        res[arm] = dict(np.load(f))
    assert int(res["phases"]["phases"]) > 0 and int(res["stencil"]["phases"]) == 0
    for d in res.values():
        for name in ("gl", "gm"):
            assert np.array_equal(d[name + "1"], d[name + "0"]) and np.array_equal(d[name + "2"], d[name + "0"])
    tol = 1e-12 if geo[-1] == 0 else 1e-6
    for name in ("gl0", "gm0"):
        a, b = res["phases"][name], res["stencil"][name]
        assert float(np.abs(a - b).max() / np.abs(b).max()) <= tol, name


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("eps", [1e-3, -1.0])
def test_prior_parity(ctx, O, P, torch, prec, eps):
    n = 45
    ph = synth.lattice_phantom(n, 4, seed=11)
    v = np.random.default_rng(4).standard_normal((n, n))
    dt = P.dtype_of(prec)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    out, val = P.pget_reg_apply(ctx, n, prec, 0.02, eps, t(ph.lam), t(v), want_value=True)
    W = O.reg_weights(ph.lam, eps)
    ref = O.reg_apply(W, v, 0.02)
    tol = 1e-12 if prec == 0 else 5e-5
    assert rel(out.cpu().numpy(), ref) <= tol
    assert abs(val - O.reg_value(ph.lam, 0.02, eps)) <= tol * abs(val)


def test_invalid_geometry_is_einval(ctx, P, torch):
    x = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PgetError) as e:
        P.pget_forward(ctx, P.geometry(1, 4, 91), 2, x, x, torch.zeros((4, 91), device="cuda"))
    assert e.value.status == P.PGET_EINVAL
    with pytest.raises(P.PgetError) as e:
        P.pget_forward(ctx, P.geometry(8, 4, 91, n_sub=0), 2, x, x, torch.zeros((4, 91), device="cuda"))
    assert e.value.status == P.PGET_EINVAL


@pytest.mark.parametrize("prec", [0, 2])
def test_batched_operators_equal_single_item_calls(ctx, P, torch, prec):
    """pget_forward_batch, pget_jvp_batch and pget_vjp_batch: item b of a batch equals the
    single-item call on item b, bitwise (one walk launch covers all items' views)."""
    n, na, nd, S, B = 40, 36, 182, 5, 5
    g = P.geometry(n, na, nd, n_sub=S)
    dt = P.dtype_of(prec)
    rs = np.random.default_rng(11)
    items = [_inputs(n, 4, 300 + b) for b in range(B)]
    t = lambda k: torch.tensor(np.stack([it[k] for it in items]), dtype=dt, device="cuda")
    L, M, DL, DM = t(0), t(1), t(2), t(3)
    R = torch.tensor(rs.standard_normal((B, na, nd)), dtype=dt, device="cuda")
    y = P.pget_forward_batch(ctx, g, prec, L, M)
    dy = P.pget_jvp_batch(ctx, g, prec, L, M, DL, DM)
    gl, gm = P.pget_vjp_batch(ctx, g, prec, L, M, R)
    for b in range(B):
        assert torch.equal(y[b], P.pget_forward(ctx, g, prec, L[b], M[b]))
        assert torch.equal(dy[b], P.pget_jvp(ctx, g, prec, L[b], M[b], DL[b], DM[b]))
        sl, sm = P.pget_vjp(ctx, g, prec, L[b], M[b], R[b])
        assert torch.equal(gl[b], sl) and torch.equal(gm[b], sm)


def test_batched_adjoint_in_several_chunks(ctx, P, torch):
    """At 256 x 256 (360 x 182 x 5) a chunk holds about ten items of adjoint partial
    images: twelve items run as two launches and still equal the single-item calls."""
    n, na, nd, S, B = 256, 360, 182, 5, 12
    g = P.geometry(n, na, nd, n_sub=S)
    ph = [synth.lattice_phantom(n, 17, radius=5.0, seed=1200 + b) for b in range(B)]
    L = torch.tensor(np.stack([p.lam for p in ph]), dtype=torch.float32, device="cuda")
    M = torch.tensor(np.stack([p.mu for p in ph]), dtype=torch.float32, device="cuda")
    R = torch.tensor(np.random.default_rng(3).standard_normal((B, na, nd)), dtype=torch.float32, device="cuda")
    gl, gm = P.pget_vjp_batch(ctx, g, 2, L, M, R)
    for b in (0, 9, 10, B - 1):
        sl, sm = P.pget_vjp(ctx, g, 2, L[b], M[b], R[b])
        assert torch.equal(gl[b], sl) and torch.equal(gm[b], sm), b

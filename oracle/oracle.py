"""ctypes wrapper around the plain FP64 CPU oracle (``pget_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product path (``paper_2604_26745_gb300``) never
imports this module and the oracle shares no code with the CUDA library.

Each wrapper mirrors one function of the C file; the C file's header lists what each
computes and which passage of the paper (arXiv 2604.26745) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pget_oracle.c")
_LIB = os.path.join(_HERE, "libpget_oracle.so")
_lock = threading.Lock()
_lib = None

TRACE = 256


class Geom(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("n_angles", C.c_int32),
        ("n_det", C.c_int32),
        ("n_banks", C.c_int32),
        ("n_sub", C.c_int32),
        ("collimator", C.c_int32),
        ("step", C.c_double),
        ("fov_radius", C.c_double),
        ("det_pitch", C.c_double),
        ("interleave", C.c_int32),
        ("depth_w", C.c_void_p),
        ("depth_c", C.c_void_p),
    ]


class Params(C.Structure):
    _fields_ = [
        ("alpha_lambda", C.c_double),
        ("alpha_mu", C.c_double),
        ("tv_eps", C.c_double),
        ("lambda_max", C.c_double),
        ("mu_max", C.c_double),
        ("max_iters", C.c_int32),
        ("cg_max_iters", C.c_int32),
        ("cg_rel_tol", C.c_double),
        ("nu0_scale", C.c_double),
        ("nu_up", C.c_double),
        ("nu_down", C.c_double),
        ("eta", C.c_double),
        ("rho_lo", C.c_double),
        ("rho_hi", C.c_double),
        ("nu_min", C.c_double),
        ("nu_max", C.c_double),
        ("alpha_decay_iters", C.c_int32),
        ("pad", C.c_int32),
        ("alpha_decay", C.c_double),
        ("geo_alpha_lambda", C.c_double),
        ("geo_alpha_mu", C.c_double),
        ("geo_mu_water", C.c_double),
        ("geo_mask", C.c_void_p),
        ("inner_solver", C.c_int32),
        ("lin_constraint", C.c_int32),
        ("lin_slope", C.c_double),
        ("lin_offset", C.c_double),
    ]


class Report(C.Structure):
    _fields_ = [
        ("iters_run", C.c_int32),
        ("accepted", C.c_int32),
        ("cg_iters_total", C.c_int32),
        ("status", C.c_int32),
        ("f0", C.c_double),
        ("f_final", C.c_double),
        ("nu0", C.c_double),
        ("nu_final", C.c_double),
        ("f", C.c_double * TRACE),
        ("rho", C.c_double * TRACE),
        ("nu", C.c_double * TRACE),
        ("pred", C.c_double * TRACE),
        ("ared", C.c_double * TRACE),
        ("acc", C.c_int32 * TRACE),
        ("cg_iters", C.c_int32 * TRACE),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                   "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        gp = C.POINTER(Geom)
        L.og_forward.argtypes = [gp, dp, dp, dp]
        L.og_jvp.argtypes = [gp, dp, dp, dp, dp, dp]
        L.og_vjp.argtypes = [gp, dp, dp, dp, dp, dp]
        L.og_reg_weights.argtypes = [C.c_int, C.c_double, dp, dp]
        L.og_reg_value.argtypes = [C.c_int, C.c_double, C.c_double, dp]
        L.og_reg_value.restype = C.c_double
        L.og_reg_apply.argtypes = [C.c_int, C.c_double, dp, dp, dp]
        L.og_cg.argtypes = [gp, C.POINTER(Params), dp, dp, dp, dp, C.c_double, dp, dp]
        L.og_sgp.argtypes = [gp, C.POINTER(Params), dp, dp, dp, dp, C.c_double, dp, dp]
        L.og_lm.argtypes = [gp, C.POINTER(Params), dp, dp, dp, C.POINTER(Report)]
        L.og_initial_guess.argtypes = [gp, dp, C.c_double, C.c_double, C.c_double, dp, dp]
        L.og_geom_info.argtypes = [gp, C.POINTER(C.c_int32), dp, dp, C.POINTER(C.c_int32)]
        L.og_num_threads.restype = C.c_int
        L.og_set_num_threads.argtypes = [C.c_int]
        L.og_set_vjp_chunks.argtypes = [C.c_int]
        L.og_lm_trial.argtypes = [gp, C.POINTER(Params), dp, dp, dp, C.c_double, dp, C.POINTER(Trial)]
        L.og_check_proposal.argtypes = [gp, C.POINTER(Params), dp, dp, dp, dp, dp, dp, C.POINTER(Check)]
        L.og_project.argtypes = [C.POINTER(Params), C.c_int, dp, dp]
        L.og_params_at_k.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(Params)]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def geom(n, n_angles, n_det, n_sub=1, collimator=1, n_banks=0, step=0.0, fov_radius=0.0,
         det_pitch=0.0, interleave=1, depth_w=None, depth_c=None) -> Geom:
    """Geometry; depth_w, depth_c (arrays of length T, the samples per ray) are the depth
    factors of Eq. (5): the emission weight and the attenuation factor of sample j."""
    g = Geom(n, n_angles, n_det, n_banks, n_sub, collimator, step, fov_radius, det_pitch, interleave)
    keep = []
    for name, tab in (("depth_w", depth_w), ("depth_c", depth_c)):
        if tab is not None:
            a = _f64(tab)
            setattr(g, name, a.ctypes.data)
            keep.append(a)
    g._keep = keep  # the tables must live as long as the geometry
    if keep:
        T = geom_info(g)["T"]
        for a in keep:
            if a.shape != (T,):
                raise ValueError(f"depth tables need {T} entries (one per ray sample)")
    return g


def geom_info(g: Geom):
    T = C.c_int32()
    p = C.c_double()
    r = C.c_double()
    nb = C.c_int32()
    if lib().og_geom_info(C.byref(g), C.byref(T), C.byref(p), C.byref(r), C.byref(nb)):
        raise ValueError("invalid geometry")
    return {"T": T.value, "pitch": p.value, "radius": r.value, "n_banks": nb.value}


def forward(g: Geom, lam, mu) -> np.ndarray:
    lam, mu = _f64(lam), _f64(mu)
    y = np.zeros((g.n_angles, g.n_det))
    if lib().og_forward(C.byref(g), _p(lam), _p(mu), _p(y)):
        raise ValueError("invalid geometry")
    return y


def jvp(g: Geom, lam, mu, dl, dm) -> np.ndarray:
    lam, mu, dl, dm = map(_f64, (lam, mu, dl, dm))
    dy = np.zeros((g.n_angles, g.n_det))
    if lib().og_jvp(C.byref(g), _p(lam), _p(mu), _p(dl), _p(dm), _p(dy)):
        raise ValueError("invalid geometry")
    return dy


def vjp(g: Geom, lam, mu, r):
    lam, mu, r = map(_f64, (lam, mu, r))
    gl = np.zeros((g.n, g.n))
    gm = np.zeros((g.n, g.n))
    if lib().og_vjp(C.byref(g), _p(lam), _p(mu), _p(r), _p(gl), _p(gm)):
        raise ValueError("invalid geometry")
    return gl, gm


def reg_weights(u, eps) -> np.ndarray:
    u = _f64(u)
    W = np.zeros_like(u)
    lib().og_reg_weights(u.shape[0], float(eps), _p(u), _p(W))
    return W


def reg_value(u, alpha, eps) -> float:
    u = _f64(u)
    return lib().og_reg_value(u.shape[0], float(alpha), float(eps), _p(u))


def reg_apply(W, v, alpha) -> np.ndarray:
    W, v = _f64(W), _f64(v)
    out = np.zeros_like(v)
    lib().og_reg_apply(v.shape[0], float(alpha), _p(W), _p(v), _p(out))
    return out


def default_params(**kw) -> Params:
    """Parameters; geo_mask (an [n, n] array) switches on the geometry priors of Eq. (6)
    with weights geo_alpha_lambda, geo_alpha_mu and water attenuation geo_mu_water;
    lin_constraint = 1 adds the per-pixel bound lambda <= lin_slope mu + lin_offset to the
    box (Sec. 2.2)."""
    d = dict(alpha_lambda=1e-2, alpha_mu=1e-2, tv_eps=1e-3, lambda_max=2.0, mu_max=0.2,
             max_iters=10, cg_max_iters=50, cg_rel_tol=1e-10, nu0_scale=1e-3, nu_up=4.0,
             nu_down=0.5, eta=1e-3, rho_lo=0.25, rho_hi=0.75, nu_min=1e-12, nu_max=1e12,
             alpha_decay=1.0, alpha_decay_iters=0, geo_alpha_lambda=0.0, geo_alpha_mu=0.0,
             geo_mu_water=0.0)
    mask = kw.pop("geo_mask", None)
    d.update(kw)
    pr = Params(**d)
    if mask is not None:
        m = _f64(mask)
        pr.geo_mask = m.ctypes.data
        pr._keep = m  # the array must live as long as the parameters
    return pr


def params_at(pr: Params, k: int) -> Params:
    """The parameters of LM iteration k under the continuation of Sec. 3.1."""
    out = Params()
    lib().og_params_at_k(C.byref(pr), int(k), C.byref(out))
    if hasattr(pr, "_keep"):
        out._keep = pr._keep
    return out


def project(pr: Params, lam, mu):
    """Euclidean projection of every pixel's (lambda, mu) onto the constraint set."""
    lam, mu = _f64(lam).copy(), _f64(mu).copy()
    lib().og_project(C.byref(pr), lam.size, _p(lam), _p(mu))
    return lam, mu


def cg(g: Geom, pr: Params, lam, mu, Wl, Wm, nu, b):
    lam, mu, Wl, Wm, b = map(_f64, (lam, mu, Wl, Wm, b))
    x = np.zeros_like(b)
    it = lib().og_cg(C.byref(g), C.byref(pr), _p(lam), _p(mu), _p(Wl), _p(Wm), float(nu),
                     _p(b), _p(x))
    if it < 0:
        raise ValueError("invalid geometry")
    return x, it


def sgp(g: Geom, pr: Params, lam, mu, Wl, Wm, nu, grad):
    """Gradient projection on the constrained LM subproblem: returns (s, iterations)."""
    lam, mu, Wl, Wm, grad = map(_f64, (lam, mu, Wl, Wm, grad))
    s = np.zeros_like(grad)
    it = lib().og_sgp(C.byref(g), C.byref(pr), _p(lam), _p(mu), _p(Wl), _p(Wm), float(nu), _p(grad), _p(s))
    if it < 0:
        raise ValueError("invalid geometry")
    return s, it


def lm(g: Geom, pr: Params, y, lam0, mu0):
    y = _f64(y)
    lam = _f64(lam0).copy()
    mu = _f64(mu0).copy()
    rep = Report()
    if lib().og_lm(C.byref(g), C.byref(pr), _p(y), _p(lam), _p(mu), C.byref(rep)):
        raise ValueError("invalid geometry")
    return lam, mu, report_dict(rep)


def report_dict(rep: Report) -> dict:
    k = min(rep.iters_run, TRACE)
    return {
        "iters_run": rep.iters_run,
        "accepted": rep.accepted,
        "cg_iters_total": rep.cg_iters_total,
        "f0": rep.f0,
        "f_final": rep.f_final,
        "nu0": rep.nu0,
        "nu_final": rep.nu_final,
        "f": list(rep.f[:k]),
        "rho": list(rep.rho[:k]),
        "nu": list(rep.nu[:k]),
        "pred": list(rep.pred[:k]),
        "ared": list(rep.ared[:k]),
        "acc": list(rep.acc[:k]),
        "cg_iters": list(rep.cg_iters[:k]),
    }


class Trial(C.Structure):
    _fields_ = [("f", C.c_double), ("pred", C.c_double), ("ared", C.c_double), ("rho", C.c_double),
                ("nu_next", C.c_double), ("nu0", C.c_double), ("accept", C.c_int32), ("cg_iters", C.c_int32)]


class Check(C.Structure):
    _fields_ = [("f", C.c_double), ("pred_step", C.c_double), ("pred_prop", C.c_double),
                ("ared_prop", C.c_double), ("rho_prop", C.c_double), ("accept", C.c_int32), ("pad", C.c_int32)]


def _fields(st) -> dict:
    return {k: getattr(st, k) for k, _ in st._fields_ if k != "pad"}


def lm_trial(g: Geom, pr: Params, y, lam, mu, nu=0.0):
    """One LM trial at the feasible point (lam, mu) with damping nu (<= 0: nu_0 at that
    point): returns the stacked step s_k = (s_lambda, s_mu) and the trial's scalars."""
    y, lam, mu = map(_f64, (y, lam, mu))
    s = np.zeros((2,) + lam.shape)
    t = Trial()
    if lib().og_lm_trial(C.byref(g), C.byref(pr), _p(y), _p(lam), _p(mu), float(nu), _p(s), C.byref(t)):
        raise ValueError("invalid geometry")
    return s, _fields(t)


def check_proposal(g: Geom, pr: Params, y, lam, mu, s_step, prop_lam, prop_mu) -> dict:
    """The safeguard of Alg. 2 for the proposal (prop_lam, prop_mu) at (lam, mu) with the
    LM step s_step (stacked, as returned by lm_trial)."""
    y, lam, mu, s_step, pl, pm = map(_f64, (y, lam, mu, s_step, prop_lam, prop_mu))
    c = Check()
    if lib().og_check_proposal(C.byref(g), C.byref(pr), _p(y), _p(lam), _p(mu), _p(s_step), _p(pl), _p(pm),
                               C.byref(c)):
        raise ValueError("invalid geometry")
    return _fields(c)


def initial_guess(g: Geom, y, mu_init=0.01, lambda_max=2.0, mu_max=0.2):
    y = _f64(y)
    lam = np.zeros((g.n, g.n))
    mu = np.zeros((g.n, g.n))
    if lib().og_initial_guess(C.byref(g), _p(y), float(mu_init), float(lambda_max),
                              float(mu_max), _p(lam), _p(mu)):
        raise ValueError("invalid geometry")
    return lam, mu


def set_vjp_chunks(c: int = 32) -> None:
    """Summation order of the VJP scatter (angle chunks, summed in order); the default 32
    is what every other result uses.  Only the rounding changes."""
    lib().og_set_vjp_chunks(int(c))


def num_threads() -> int:
    return lib().og_num_threads()


def set_num_threads(n: int = 0) -> None:
    """Threads of the oracle's OpenMP loops (n <= 0: the default); results do not change."""
    lib().og_set_num_threads(int(n))

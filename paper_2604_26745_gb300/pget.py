"""Thin ctypes binding of libpget.so (include/pget.h).  Argument marshalling only: every
step of the hot path runs in the library's CUDA kernels; torch supplies device memory
and streams.  There is no fallback: if the library is missing, load() raises."""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpget.so")

PGET_OK, PGET_EINVAL, PGET_ENOMEM, PGET_EAGAIN, PGET_ECUDA, PGET_ETIMEOUT, PGET_ENUMERIC, PGET_ENOTFOUND, PGET_EINTERNAL = range(9)
PGET_F64, PGET_F32, PGET_F32_KAHAN, PGET_MIXED = 0, 1, 2, 3
PGET_TRACE = 256

_DTYPE = {PGET_F64: torch.float64, PGET_F32: torch.float32, PGET_F32_KAHAN: torch.float32,
          PGET_MIXED: torch.float64}


class PgetError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pget status {status}: {msg}")
        self.status = status


class pget_geometry(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_angles", C.c_int32), ("n_det", C.c_int32),
                ("n_banks", C.c_int32), ("n_sub", C.c_int32), ("collimator", C.c_int32),
                ("step", C.c_double), ("fov_radius", C.c_double), ("det_pitch", C.c_double),
                ("depth_w", C.c_void_p), ("depth_c", C.c_void_p)]


class pget_lm_params(C.Structure):
    _fields_ = [("alpha_lambda", C.c_double), ("alpha_mu", C.c_double), ("tv_eps", C.c_double),
                ("lambda_max", C.c_double), ("mu_max", C.c_double), ("max_iters", C.c_int32),
                ("cg_max_iters", C.c_int32), ("cg_rel_tol", C.c_double), ("nu0_scale", C.c_double),
                ("nu_up", C.c_double), ("nu_down", C.c_double), ("eta", C.c_double),
                ("rho_lo", C.c_double), ("rho_hi", C.c_double), ("nu_min", C.c_double),
                ("nu_max", C.c_double), ("precision", C.c_int32), ("alpha_decay_iters", C.c_int32),
                ("alpha_decay", C.c_double), ("geo_alpha_lambda", C.c_double), ("geo_alpha_mu", C.c_double),
                ("geo_mu_water", C.c_double), ("geo_mask", C.c_void_p), ("inner_solver", C.c_int32),
                ("lin_constraint", C.c_int32), ("lin_slope", C.c_double), ("lin_offset", C.c_double)]


class pget_lm_report(C.Structure):
    _fields_ = [("iters_run", C.c_int32), ("accepted", C.c_int32), ("cg_iters_total", C.c_int32),
                ("status", C.c_int32), ("f0", C.c_double), ("f_final", C.c_double),
                ("nu0", C.c_double), ("nu_final", C.c_double),
                ("f", C.c_double * PGET_TRACE), ("rho", C.c_double * PGET_TRACE),
                ("nu", C.c_double * PGET_TRACE), ("pred", C.c_double * PGET_TRACE),
                ("ared", C.c_double * PGET_TRACE), ("acc", C.c_int32 * PGET_TRACE),
                ("cg_iters", C.c_int32 * PGET_TRACE), ("device_ms", C.c_double)]

    def to_dict(self) -> dict:
        k = min(self.iters_run, PGET_TRACE)
        return {"iters_run": self.iters_run, "accepted": self.accepted,
                "cg_iters_total": self.cg_iters_total, "status": self.status, "f0": self.f0,
                "f_final": self.f_final, "nu0": self.nu0, "nu_final": self.nu_final,
                "f": list(self.f[:k]), "rho": list(self.rho[:k]), "nu": list(self.nu[:k]),
                "pred": list(self.pred[:k]), "ared": list(self.ared[:k]),
                "acc": list(self.acc[:k]), "cg_iters": list(self.cg_iters[:k]),
                "device_ms": self.device_ms}


class pget_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


# exported symbols and their argument types
_vp = C.c_void_p
class pget_trial_report(C.Structure):
    _fields_ = [("f", C.c_double), ("pred", C.c_double), ("ared", C.c_double), ("rho", C.c_double),
                ("nu_next", C.c_double), ("nu0", C.c_double), ("accept", C.c_int32), ("cg_iters", C.c_int32)]


class pget_check_report(C.Structure):
    _fields_ = [("f", C.c_double), ("pred_step", C.c_double), ("pred_prop", C.c_double),
                ("ared_prop", C.c_double), ("rho_prop", C.c_double), ("accept", C.c_int32), ("pad", C.c_int32)]


class pget_step_report(C.Structure):
    _fields_ = [("check", pget_check_report), ("checked", C.c_int32), ("took", C.c_int32), ("nu_next", C.c_double)]


class pget_walk_plan_info(C.Structure):
    _fields_ = [("threads", C.c_int32), ("rows_per_chunk", C.c_int32 * 3), ("chunks", C.c_int32 * 3),
                ("smem_bytes", C.c_int32 * 3), ("adjoint_phases", C.c_int32), ("phases_needed", C.c_int32)]


def _fields(st) -> dict:
    return {k: getattr(st, k) for k, _ in st._fields_ if k != "pad"}


_SIGS = {
    "pget_create": ([C.POINTER(_vp), C.c_int, C.c_size_t], C.c_int),
    "pget_destroy": ([_vp], C.c_int),
    "pget_default_params": ([C.POINTER(pget_lm_params)], None),
    "pget_forward": ([_vp, C.POINTER(pget_geometry), C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "pget_jvp": ([_vp, C.POINTER(pget_geometry), C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "pget_vjp": ([_vp, C.POINTER(pget_geometry), C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "pget_operator_status": ([_vp, _vp], C.c_int),
    "pget_forward_batch": ([_vp, C.POINTER(pget_geometry), C.c_int32, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "pget_jvp_batch": ([_vp, C.POINTER(pget_geometry), C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "pget_vjp_batch": ([_vp, C.POINTER(pget_geometry), C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "pget_reg_apply": ([_vp, C.c_int32, C.c_int32, C.c_double, C.c_double, _vp, _vp, _vp,
                        C.POINTER(C.c_double), _vp], C.c_int),
    "pget_cg_solve": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp,
                       C.c_double, _vp, _vp, C.POINTER(C.c_int32), _vp], C.c_int),
    "pget_initial_guess": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), C.c_double,
                            _vp, _vp, _vp, _vp], C.c_int),
    "pget_lm_solve": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp, _vp,
                       C.POINTER(pget_lm_report), _vp], C.c_int),
    "pget_lm_trial": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp, _vp, C.c_double,
                       _vp, C.POINTER(pget_trial_report), _vp], C.c_int),
    "pget_proposal_check": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp, _vp, _vp,
                             _vp, _vp, C.POINTER(pget_check_report), _vp], C.c_int),
    "pget_project": ([_vp, C.POINTER(pget_lm_params), C.c_int32, _vp, _vp, _vp], C.c_int),
    "pget_lm_step_with_proposal": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), C.c_int32, _vp, _vp,
                                    _vp, _vp, C.POINTER(pget_trial_report), C.c_double, _vp, _vp,
                                    C.POINTER(pget_step_report), _vp], C.c_int),
    "pget_params_at": ([C.POINTER(pget_lm_params), C.c_int32, C.POINTER(pget_lm_params)], C.c_int),
    "pget_check_params": ([C.POINTER(pget_lm_params)], C.c_int),
    "pget_geometry_info": ([C.POINTER(pget_geometry), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32)], C.c_int),
    "pget_walk_plans": ([C.POINTER(pget_geometry), C.c_int32, C.POINTER(pget_walk_plan_info)], C.c_int),
    "pget_lm_solve_host": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp,
                            _vp, C.c_int32, C.POINTER(pget_lm_report), _vp], C.c_int),
    "pget_submit": ([_vp, C.POINTER(pget_geometry), C.POINTER(pget_lm_params), _vp, _vp, _vp,
                     C.POINTER(C.c_uint64)], C.c_int),
    "pget_poll": ([_vp, C.c_uint64, _vp, _vp, C.POINTER(pget_lm_report), C.POINTER(C.c_int)], C.c_int),
    "pget_cancel": ([_vp, C.c_uint64], C.c_int),
    "pget_inflight": ([_vp], C.c_int32),
    "pget_forward_noalloc": ([C.POINTER(pget_geometry), C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "pget_profile_enable": ([_vp, C.c_int32], C.c_int),
    "pget_profile_read": ([_vp, C.POINTER(pget_kernel_stat), C.c_int32], C.c_int32),
    "pget_launch_count": ([], C.c_longlong),
    "pget_last_error": ([_vp], C.c_char_p),
    "pget_version": ([], C.c_char_p),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpget.so; raises if it has not been built (no CPU or Python fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols() -> list:
    return sorted(_SIGS)


def _check(status: int, ctx=None):
    if status != PGET_OK:
        msg = load().pget_last_error(ctx).decode() if _lib is not None else ""
        raise PgetError(status, msg)


def _arr(t, precision, numel: int, device, name: str, host: bool = False):
    """Pointer of an array argument, after the checks a raw pointer cannot carry: a
    contiguous tensor on the right side (the context's CUDA device, or the host), with the
    precision's element size (8 bytes for PGET_F64, else 4) and at least numel elements.
    A mismatch raises here instead of reaching the kernels as an out-of-range pointer.
    precision None skips the element-size check (pget_poll: the request's precision)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if host:
        if t.is_cuda:
            raise ValueError(f"{name} must be a CPU tensor")
    else:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if device is not None and t.device.index != device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if precision is not None:
        want = 8 if precision in (PGET_F64, PGET_MIXED) else 4
        if not t.is_floating_point() or t.element_size() != want:
            raise ValueError(f"{name} is {t.dtype}; precision {precision} takes "
                             f"{'float64' if want == 8 else 'float32'}")
    if t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, {numel} needed")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def geometry(n: int, n_angles: int, n_det: int, n_sub: int = 1, collimator: int = 1,
             n_banks: int = 0, step: float = 0.0, fov_radius: float = 0.0,
             det_pitch: float = 0.0, depth_w=None, depth_c=None) -> pget_geometry:
    """Geometry; depth_w, depth_c (host sequences of T = geometry_info(...)["n_samples"]
    entries) are the depth factors of Eq. (5): emission weight and attenuation factor of
    sample j of every ray."""
    g = pget_geometry(n, n_angles, n_det, n_banks, n_sub, collimator, step, fov_radius, det_pitch)
    keep = []
    if depth_w is not None or depth_c is not None:
        T = geometry_info(g)["n_samples"]
        for name, tab in (("depth_w", depth_w), ("depth_c", depth_c)):
            if tab is None:
                continue
            a = (C.c_double * T)(*[float(v) for v in tab]) if len(tab) == T else None
            if a is None:
                raise ValueError(f"{name} needs {T} entries (one per ray sample)")
            setattr(g, name, C.cast(a, C.c_void_p).value)
            keep.append(a)
    g._keep = keep  # the host tables must live as long as the geometry
    return g


def geometry_info(g: pget_geometry) -> dict:
    """Derived sizes: samples per ray, banks, field-of-view radius, pitch, rays per view."""
    T, nb, ms = C.c_int32(), C.c_int32(), C.c_int32()
    r, p = C.c_double(), C.c_double()
    st = load().pget_geometry_info(C.byref(g), C.byref(T), C.byref(nb), C.byref(r), C.byref(p), C.byref(ms))
    if st == PGET_EINVAL:
        raise ValueError("invalid geometry: " + load().pget_last_error(None).decode())
    _check(st)
    return {"n_samples": T.value, "n_banks": nb.value, "fov_radius": r.value, "det_pitch": p.value,
            "max_slots": ms.value}


def walk_plans(g: pget_geometry, precision: int) -> dict:
    """Launch plans of the forward, JVP and adjoint walks (host only): threads per CTA,
    rows per chunk, chunks and shared memory per operator, adjoint phase count."""
    out = pget_walk_plan_info()
    st = load().pget_walk_plans(C.byref(g), int(precision), C.byref(out))
    if st == PGET_EINVAL:
        raise ValueError("invalid walk plan query: " + load().pget_last_error(None).decode())
    _check(st)
    ops = ("forward", "jvp", "vjp")
    return {"threads": out.threads, "adjoint_phases": out.adjoint_phases, "phases_needed": out.phases_needed,
            **{o: {"rows_per_chunk": out.rows_per_chunk[k], "chunks": out.chunks[k], "smem_bytes": out.smem_bytes[k]}
               for k, o in enumerate(ops)}}


def check_params(p: pget_lm_params) -> None:
    """Raise ValueError (with the library's message) if p would be refused by any call."""
    st = load().pget_check_params(C.byref(p))
    if st == PGET_EINVAL:
        raise ValueError("invalid parameters: " + load().pget_last_error(None).decode())
    _check(st)


def default_params(**kw) -> pget_lm_params:
    """Library defaults with overrides; geo_mask may be a CUDA tensor (kept alive with the
    parameters) for the geometry priors."""
    p = pget_lm_params()
    load().pget_default_params(C.byref(p))
    mask = kw.pop("geo_mask", None)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    if mask is not None:
        m = mask.contiguous()
        p.geo_mask = m.data_ptr()
        p._keep = m
    return p


def dtype_of(precision: int) -> torch.dtype:
    return _DTYPE[precision]


class Context:
    """Owns a pget_ctx (one device, its workspace and memory budget)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        L = load()
        h = _vp()
        _check(L.pget_create(C.byref(h), int(device), int(mem_budget_bytes)))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            load().pget_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------- entry points
def pget_forward(ctx: Context, g: pget_geometry, precision: int, lam, mu, y=None, stream=None):
    if y is None:
        y = torch.empty((g.n_angles, g.n_det), dtype=lam.dtype, device=lam.device)
    nn, M, d = g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_forward(ctx.h, C.byref(g), precision, _arr(lam, precision, nn, d, "lam"),
                               _arr(mu, precision, nn, d, "mu"), _arr(y, precision, M, d, "y"),
                               _stream(stream)), ctx.h)
    return y


def pget_jvp(ctx: Context, g: pget_geometry, precision: int, lam, mu, dlam, dmu, dy=None, stream=None):
    if dy is None:
        dy = torch.empty((g.n_angles, g.n_det), dtype=lam.dtype, device=lam.device)
    nn, M, d = g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_jvp(ctx.h, C.byref(g), precision, _arr(lam, precision, nn, d, "lam"),
                           _arr(mu, precision, nn, d, "mu"), _arr(dlam, precision, nn, d, "dlam"),
                           _arr(dmu, precision, nn, d, "dmu"), _arr(dy, precision, M, d, "dy"),
                           _stream(stream)), ctx.h)
    return dy


def pget_vjp(ctx: Context, g: pget_geometry, precision: int, lam, mu, r, glam=None, gmu=None,
             stream=None):
    if glam is None:
        glam = torch.empty_like(lam)
    if gmu is None:
        gmu = torch.empty_like(mu)
    nn, M, d = g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_vjp(ctx.h, C.byref(g), precision, _arr(lam, precision, nn, d, "lam"),
                           _arr(mu, precision, nn, d, "mu"), _arr(r, precision, M, d, "r"),
                           _arr(glam, precision, nn, d, "glam"), _arr(gmu, precision, nn, d, "gmu"),
                           _stream(stream)), ctx.h)
    return glam, gmu


def pget_forward_batch(ctx: Context, g: pget_geometry, precision: int, lam, mu, y=None, stream=None):
    """y[b] = A(lam[b], mu[b]) for lam, mu [B, n, n] in one call (see pget.h)."""
    B, nn, M, d = lam.shape[0], g.n * g.n, g.n_angles * g.n_det, ctx.device
    if y is None:
        y = torch.empty((B, g.n_angles, g.n_det), dtype=lam.dtype, device=lam.device)
    _check(load().pget_forward_batch(ctx.h, C.byref(g), precision, B, _arr(lam, precision, B * nn, d, "lam"),
                                     _arr(mu, precision, B * nn, d, "mu"), _arr(y, precision, B * M, d, "y"),
                                     _stream(stream)), ctx.h)
    return y


def pget_jvp_batch(ctx: Context, g: pget_geometry, precision: int, lam, mu, dlam, dmu, dy=None, stream=None):
    """dy[b] = J(lam[b], mu[b]) (dlam[b], dmu[b]) for [B, n, n] inputs in one call."""
    B, nn, M, d = lam.shape[0], g.n * g.n, g.n_angles * g.n_det, ctx.device
    if dy is None:
        dy = torch.empty((B, g.n_angles, g.n_det), dtype=lam.dtype, device=lam.device)
    _check(load().pget_jvp_batch(ctx.h, C.byref(g), precision, B, _arr(lam, precision, B * nn, d, "lam"),
                                 _arr(mu, precision, B * nn, d, "mu"), _arr(dlam, precision, B * nn, d, "dlam"),
                                 _arr(dmu, precision, B * nn, d, "dmu"), _arr(dy, precision, B * M, d, "dy"),
                                 _stream(stream)), ctx.h)
    return dy


def pget_vjp_batch(ctx: Context, g: pget_geometry, precision: int, lam, mu, r, glam=None, gmu=None, stream=None):
    """(glam[b], gmu[b]) = J(lam[b], mu[b])^T r[b] for [B, n, n] / [B, n_angles, n_det] inputs."""
    B, nn, M, d = lam.shape[0], g.n * g.n, g.n_angles * g.n_det, ctx.device
    glam = torch.empty_like(lam) if glam is None else glam
    gmu = torch.empty_like(mu) if gmu is None else gmu
    _check(load().pget_vjp_batch(ctx.h, C.byref(g), precision, B, _arr(lam, precision, B * nn, d, "lam"),
                                 _arr(mu, precision, B * nn, d, "mu"), _arr(r, precision, B * M, d, "r"),
                                 _arr(glam, precision, B * nn, d, "glam"), _arr(gmu, precision, B * nn, d, "gmu"),
                                 _stream(stream)), ctx.h)
    return glam, gmu


def pget_operator_status(ctx: Context, stream=None) -> None:
    """Waits for the stream and raises if a forward, JVP or adjoint call made since the
    last check met a device-side error (a chunk copy wait that ran out: PGET_ETIMEOUT)."""
    _check(load().pget_operator_status(ctx.h, _stream(stream)), ctx.h)


def pget_reg_apply(ctx: Context, n: int, precision: int, alpha: float, eps: float, u, v, out=None,
                   want_value: bool = False, stream=None):
    if out is None:
        out = torch.empty_like(v)
    val = C.c_double(0.0)
    nn, d = int(n) * int(n), ctx.device
    _check(load().pget_reg_apply(ctx.h, n, precision, alpha, eps, _arr(u, precision, nn, d, "u"),
                                 _arr(v, precision, nn, d, "v"), _arr(out, precision, nn, d, "out"),
                                 C.byref(val) if want_value else None, _stream(stream)), ctx.h)
    return (out, val.value) if want_value else out


def pget_cg_solve(ctx: Context, g: pget_geometry, p: pget_lm_params, lam, mu, nu: float, rhs, x=None,
                  stream=None):
    if x is None:
        x = torch.empty_like(rhs)
    it = C.c_int32(0)
    q, nn, d = p.precision, g.n * g.n, ctx.device
    _check(load().pget_cg_solve(ctx.h, C.byref(g), C.byref(p), _arr(lam, q, nn, d, "lam"),
                                _arr(mu, q, nn, d, "mu"), float(nu), _arr(rhs, q, 2 * nn, d, "rhs"),
                                _arr(x, q, 2 * nn, d, "x"), C.byref(it), _stream(stream)), ctx.h)
    return x, it.value


def pget_initial_guess(ctx: Context, g: pget_geometry, p: pget_lm_params, y, mu_init: float = 0.01,
                       stream=None):
    lam = torch.empty((g.n, g.n), dtype=y.dtype, device=y.device)
    mu = torch.empty_like(lam)
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_initial_guess(ctx.h, C.byref(g), C.byref(p), float(mu_init), _arr(y, q, M, d, "y"),
                                     _arr(lam, q, nn, d, "lam"), _arr(mu, q, nn, d, "mu"),
                                     _stream(stream)), ctx.h)
    return lam, mu


def pget_lm_trial(ctx: Context, g: pget_geometry, p: pget_lm_params, y, lam, mu, nu: float = 0.0, s_out=None,
                  stream=None):
    """One LM trial at (lam, mu) with damping nu (<= 0: nu_0 there); returns (s, report) with
    s the stacked step [2, n, n] (a new tensor unless s_out is given).  u is not changed."""
    if s_out is None:
        s_out = lam.new_empty((2,) + tuple(lam.shape))
    rep = pget_trial_report()
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_lm_trial(ctx.h, C.byref(g), C.byref(p), _arr(y, q, M, d, "y"), _arr(lam, q, nn, d, "lam"),
                                _arr(mu, q, nn, d, "mu"), float(nu), _arr(s_out, q, 2 * nn, d, "s_out"),
                                C.byref(rep), _stream(stream)), ctx.h)
    return s_out, _fields(rep)


def pget_proposal_check(ctx: Context, g: pget_geometry, p: pget_lm_params, y, lam, mu, s_step, prop_lam,
                        prop_mu, stream=None) -> dict:
    """The convergence check of Alg. 2 for the proposal (prop_lam, prop_mu)."""
    rep = pget_check_report()
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_proposal_check(ctx.h, C.byref(g), C.byref(p), _arr(y, q, M, d, "y"),
                                      _arr(lam, q, nn, d, "lam"), _arr(mu, q, nn, d, "mu"),
                                      _arr(s_step, q, 2 * nn, d, "s_step"), _arr(prop_lam, q, nn, d, "prop_lam"),
                                      _arr(prop_mu, q, nn, d, "prop_mu"), C.byref(rep), _stream(stream)), ctx.h)
    return _fields(rep)


TOOK = ("none", "step", "proposal")


def pget_lm_step_with_proposal(ctx: Context, g: pget_geometry, p: pget_lm_params, k: int, y, lam, mu, s_step,
                               trial: dict, nu0: float, prop_lam=None, prop_mu=None, stream=None) -> dict:
    """Alg. 2 after the LM trial of iteration k (see pget.h): checks the proposal (if
    given) and replaces (lam, mu) in place by the next iterate.  trial: the report
    pget_lm_trial returned.  Returns {"check": dict or None, "took": "none" | "step" |
    "proposal", "nu_next": the clamped damping of iteration k + 1}."""
    tr = pget_trial_report(**{f: trial[f] for f, _ in pget_trial_report._fields_})
    rep = pget_step_report()
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    if (prop_lam is None) != (prop_mu is None):
        raise ValueError("give both proposal images or neither")
    pl = None if prop_lam is None else _arr(prop_lam, q, nn, d, "prop_lam")
    pm = None if prop_mu is None else _arr(prop_mu, q, nn, d, "prop_mu")
    _check(load().pget_lm_step_with_proposal(ctx.h, C.byref(g), C.byref(p), int(k), _arr(y, q, M, d, "y"),
                                             _arr(lam, q, nn, d, "lam"), _arr(mu, q, nn, d, "mu"),
                                             _arr(s_step, q, 2 * nn, d, "s_step"), C.byref(tr), float(nu0), pl, pm,
                                             C.byref(rep), _stream(stream)), ctx.h)
    return {"check": _fields(rep.check) if rep.checked else None, "took": TOOK[rep.took], "nu_next": rep.nu_next}


def pget_params_at(p: pget_lm_params, k: int) -> pget_lm_params:
    """The parameters of LM iteration k under the continuation of Sec. 3.1."""
    out = pget_lm_params()
    _check(load().pget_params_at(C.byref(p), int(k), C.byref(out)))
    return out


def pget_project(ctx: Context, p: pget_lm_params, lam, mu, stream=None):
    """Project (lam, mu) in place onto the constraint set of p (box and optional linear
    bound); lam, mu: contiguous [n, n] CUDA tensors of the precision's dtype."""
    if lam.shape != mu.shape or lam.dim() != 2 or lam.shape[0] != lam.shape[1]:
        raise ValueError("lam and mu must be square images of one shape")
    if not (lam.is_contiguous() and mu.is_contiguous()):
        raise ValueError("lam and mu must be contiguous")
    q, nn, d = p.precision, lam.numel(), ctx.device
    _check(load().pget_project(ctx.h, C.byref(p), int(lam.shape[0]), _arr(lam, q, nn, d, "lam"),
                               _arr(mu, q, nn, d, "mu"), _stream(stream)), ctx.h)
    return lam, mu


def pget_lm_solve(ctx: Context, g: pget_geometry, p: pget_lm_params, y, lam, mu, stream=None):
    """Solve in place (lam, mu: initial guess in, result out); returns the report dict."""
    rep = pget_lm_report()
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_lm_solve(ctx.h, C.byref(g), C.byref(p), _arr(y, q, M, d, "y"), _arr(lam, q, nn, d, "lam"),
                                _arr(mu, q, nn, d, "mu"), C.byref(rep), _stream(stream)), ctx.h)
    return rep.to_dict()


def pget_lm_solve_host(ctx: Context, g: pget_geometry, p: pget_lm_params, y_host, lam_host,
                       mu_host, init_guess: bool = True, stream=None):
    """Host-buffer solve (y_host, lam_host, mu_host: CPU tensors, pinned for async copies)."""
    q, nn, M = p.precision, g.n * g.n, g.n_angles * g.n_det
    y_p = _arr(y_host, q, M, None, "y_host", host=True)
    lam_p = _arr(lam_host, q, nn, None, "lam_host", host=True)
    mu_p = _arr(mu_host, q, nn, None, "mu_host", host=True)
    rep = pget_lm_report()
    _check(load().pget_lm_solve_host(ctx.h, C.byref(g), C.byref(p), y_p, lam_p, mu_p, int(bool(init_guess)),
                                     C.byref(rep), _stream(stream)), ctx.h)
    return rep.to_dict()


def pget_submit(ctx: Context, g: pget_geometry, p: pget_lm_params, y, lam0=None, mu0=None) -> int:
    """Queue a reconstruction; returns its ticket.  Raises PgetError (status PGET_EAGAIN
    when no slot or memory is free right now)."""
    t = C.c_uint64(0)
    q, nn, M, d = p.precision, g.n * g.n, g.n_angles * g.n_det, ctx.device
    _check(load().pget_submit(ctx.h, C.byref(g), C.byref(p), _arr(y, q, M, d, "y"), _arr(lam0, q, nn, d, "lam0"),
                              _arr(mu0, q, nn, d, "mu0"), C.byref(t)), ctx.h)
    return t.value


def pget_poll(ctx: Context, ticket: int, lam_out=None, mu_out=None):
    """(done, report): report is None while the request still runs."""
    rep = pget_lm_report()
    done = C.c_int(0)
    d = ctx.device
    _check(load().pget_poll(ctx.h, C.c_uint64(ticket), _arr(lam_out, None, 0, d, "lam_out"),
                            _arr(mu_out, None, 0, d, "mu_out"), C.byref(rep), C.byref(done)), ctx.h)
    return bool(done.value), (rep.to_dict() if done.value else None)


def pget_cancel(ctx: Context, ticket: int):
    _check(load().pget_cancel(ctx.h, C.c_uint64(ticket)), ctx.h)


def pget_inflight(ctx: Context) -> int:
    return int(load().pget_inflight(ctx.h))


def pget_forward_noalloc(g: pget_geometry, precision: int, lam, mu, y, stream=None) -> int:
    """Forward projection without a context and without allocating (see pget.h); y must
    be preallocated.  Returns the pget status (no exception, no message)."""
    nn, M = g.n * g.n, g.n_angles * g.n_det
    return load().pget_forward_noalloc(C.byref(g), precision, _arr(lam, precision, nn, None, "lam"),
                                       _arr(mu, precision, nn, None, "mu"), _arr(y, precision, M, None, "y"),
                                       _stream(stream))


def pget_profile_enable(ctx: Context, enable: bool = True):
    _check(load().pget_profile_enable(ctx.h, int(bool(enable))), ctx.h)


def pget_profile_read(ctx: Context) -> dict:
    arr = (pget_kernel_stat * 8)()
    k = load().pget_profile_read(ctx.h, arr, 8)
    return {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms}
            for i in range(k)}


def pget_launch_count() -> int:
    return int(load().pget_launch_count())


def pget_version() -> str:
    return load().pget_version().decode()


def fov_radius(g: pget_geometry) -> float:
    return g.fov_radius if g.fov_radius > 0 else g.n / math.sqrt(2.0)

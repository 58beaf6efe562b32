"""Accelerated iteration scheme with checks (Alg. 2, Sec. 3.1) on the library's LM.

Every iteration computes the LM step s_k at u_k (pget_lm_trial), lets a proposal operator
G suggest u~ = G(u_k, s_k), and keeps u~ only if it passes the convergence check of
Prop. conv_check (pget_proposal_check): rho(s~) > eta and m_k(s~) <= m_k(s_k).
Otherwise the plain LM outcome stands: u_k + s_k if the trial was accepted, else u_k.
The damping follows the LM trial's own schedule (the paper leaves it open after an
accepted proposal; the LM step's rho drives it here, clamped as in a plain solve), and
the prior weights follow the continuation alpha / alpha_decay^min(k, alpha_decay_iters)
of Sec. 3.1 when p asks for it, as pget_lm_solve does.

G is any callable or torch.nn.Module taking (u, s, k) with u, s stacked [2, n, n] CUDA
tensors (lambda, mu) and k the iteration, returning a proposal of the same shape, or None
to skip the check in that iteration.  No trained model ships with the library; the
tests drive the scheme with synthetic proposals.
"""
from __future__ import annotations

import torch

from . import pget as P


def params_at(p: P.pget_lm_params, k: int) -> P.pget_lm_params:
    """The parameters of LM iteration k under the continuation (fixed when off)."""
    q = P.pget_lm_params.from_buffer_copy(p)
    if p.alpha_decay > 1.0 and p.alpha_decay_iters > 0:
        sc = p.alpha_decay ** -min(k, p.alpha_decay_iters)
        q.alpha_lambda = p.alpha_lambda * sc
        q.alpha_mu = p.alpha_mu * sc
        q.geo_alpha_lambda = p.geo_alpha_lambda * sc
        q.geo_alpha_mu = p.geo_alpha_mu * sc
    return q


def accelerated_solve(ctx: P.Context, g: P.pget_geometry, p: P.pget_lm_params, y: torch.Tensor,
                      lam: torch.Tensor, mu: torch.Tensor, G=None, iters: int | None = None,
                      state: dict | None = None):
    """Run Alg. 2 from (lam, mu) (projected onto the constraint set first); returns
    (lam, mu, history) with one dict per iteration (trial scalars, check scalars, which
    update was taken, and the checkpoint "state" after it).  Every projection runs in the
    library (pget_project).

    Checkpoint and resume: the solver's whole state after iteration k is the iterate
    (lam, mu) and the scalars {"k": k + 1, "nu": damping, "nu0": first damping}, the
    "state" of that iteration's history entry.  Called with such a state and that
    iterate, the solve continues at iteration state["k"] (the continuation schedule and the
    damping clamps included) and gives the same iterates, bitwise, as the uninterrupted
    solve; the iterate is not projected again, since the solve left it in the constraint
    set.  iters counts this call's iterations (default: up to p.max_iters in total)."""
    proj = lambda a, b: P.pget_project(ctx, p, a.contiguous().clone(), b.contiguous().clone())
    if state is None:
        k0, nu, nu0 = 0, 0.0, None
        lam, mu = proj(lam, mu)
    else:
        k0, nu, nu0 = int(state["k"]), float(state["nu"]), float(state["nu0"])
        if k0 < 0 or not nu0 > 0.0 or not nu > 0.0:
            raise ValueError("invalid checkpoint state")
        lam, mu = lam.contiguous().clone(), mu.contiguous().clone()
    iters = max(p.max_iters - k0, 0) if iters is None else iters
    s = lam.new_empty((2,) + tuple(lam.shape))
    history = []
    for k in range(k0, k0 + iters):
        pk = params_at(p, k)
        s, tr = P.pget_lm_trial(ctx, g, pk, y, lam, mu, nu, s_out=s)
        if nu0 is None:
            nu0 = nu = tr["nu0"]
        took, chk = ("step" if tr["accept"] else "none"), None
        if G is not None:
            prop = G(torch.stack([lam, mu]), s, k)
            if prop is not None:
                pl, pm = prop[0].contiguous(), prop[1].contiguous()
                chk = P.pget_proposal_check(ctx, g, pk, y, lam, mu, s, pl, pm)
                if chk["accept"]:
                    lam, mu = proj(pl, pm)
                    took = "proposal"
        if took == "step":
            lam, mu = proj(lam + s[0], mu + s[1])
        nu = min(max(tr["nu_next"], p.nu_min * nu0), p.nu_max * nu0)
        history.append({"k": k, "trial": tr, "check": chk, "took": took, "nu": nu,
                        "state": {"k": k + 1, "nu": nu, "nu0": nu0}})
    return lam, mu, history

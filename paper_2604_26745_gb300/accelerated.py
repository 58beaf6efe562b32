"""Accelerated iteration scheme with checks (Alg. 2, Sec. 3.1) on the library's LM.

Every iteration computes the LM step s_k at u_k (pget_lm_trial), lets a proposal operator
G suggest u~ = G(u_k, s_k), and hands both to pget_lm_step_with_proposal, which keeps u~
only if it passes the convergence check of Prop. conv_check (rho(s~) > eta and
m_k(s~) <= m_k(s_k)), else takes the plain LM outcome (u_k + s_k if the trial was
accepted, else u_k), and clamps the damping.  The damping follows the LM trial's own
schedule (the paper leaves it open after an accepted proposal; the LM step's rho drives it
here, clamped as in a plain solve), and the prior weights follow the continuation
alpha / alpha_decay^min(k, alpha_decay_iters) of Sec. 3.1 (pget_params_at) when p asks
for it, as pget_lm_solve does.  All of the method's arithmetic runs in the library; this
module only sequences the calls and the proposal operator.

G is any callable or torch.nn.Module taking (u, s, k) with u, s stacked [2, n, n] CUDA
tensors (lambda, mu) and k the iteration, returning a proposal of the same shape, or None
to skip the check in that iteration.  No trained model ships with the library; the
tests drive the scheme with synthetic proposals.
"""
from __future__ import annotations

import torch

from . import pget as P


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
        pk = P.pget_params_at(p, k)
        s, tr = P.pget_lm_trial(ctx, g, pk, y, lam, mu, nu, s_out=s)
        if nu0 is None:
            nu0 = nu = tr["nu0"]
        pl = pm = None
        if G is not None:
            prop = G(torch.stack([lam, mu]), s, k)
            if prop is not None:
                pl, pm = prop[0].contiguous(), prop[1].contiguous()
        # the check, the next iterate (in place) and the clamped damping, in the library
        st = P.pget_lm_step_with_proposal(ctx, g, p, k, y, lam, mu, s, tr, nu0, pl, pm)
        nu = st["nu_next"]
        history.append({"k": k, "trial": tr, "check": st["check"], "took": st["took"], "nu": nu,
                        "state": {"k": k + 1, "nu": nu, "nu0": nu0}})
    return lam, mu, history

"""Checkpoint and resume of the Alg. 2 driver (accelerated.accelerated_solve), on the CPU.

The Alg. 2 driver's state after iteration k is the iterate and the scalars (k + 1, ν, ν₀). A solve
stopped there and resumed from that checkpoint must give the uninterrupted solve's
iterates bitwise, with the same decisions and damping. The cases:
- the plain LM (no proposal);
- the α continuation running across the checkpoint;
- proposals, some of them taken;
- a binding linear bound, where the resumed iterate is not projected a second time.

The Alg. 2 driver's host logic runs unchanged. Only its library calls (parameters of
iteration k, trial, the step with the proposal check, projection) are served by the oracle
on CPU tensors; on the GPU the same calls go to the CUDA library.
"""
import numpy as np
import pytest
import torch

from paper_2604_26745_gb300 import accelerated, pget as P, synth

N, NA, ND, S = 16, 12, 182, 3


class _OracleCalls:
    pget_lm_params = P.pget_lm_params

    def __init__(self, O, go):
        self.O, self.go = O, go

    def _pr(self, p):
        pr = self.O.default_params()
        for name, _ in pr._fields_:
            if name not in ("pad", "geo_mask") and hasattr(p, name):
                setattr(pr, name, getattr(p, name))
        return pr

    def pget_project(self, ctx, p, lam, mu):
        a, b = self.O.project(self._pr(p), lam.numpy(), mu.numpy())
        return torch.from_numpy(a), torch.from_numpy(b)

    def pget_lm_trial(self, ctx, g, p, y, lam, mu, nu, s_out=None):
        s, tr = self.O.lm_trial(self.go, self._pr(p), y.numpy(), lam.numpy(), mu.numpy(), nu)
        return torch.from_numpy(s), tr

    def pget_params_at(self, p, k):
        q = P.pget_lm_params.from_buffer_copy(p)
        o = self.O.params_at(self._pr(p), k)
        for name in ("alpha_lambda", "alpha_mu", "geo_alpha_lambda", "geo_alpha_mu"):
            setattr(q, name, getattr(o, name))
        return q

    def pget_lm_step_with_proposal(self, ctx, g, p, k, y, lam, mu, s, tr, nu0, pl=None, pm=None):
        # Alg. 2 after the trial, with the oracle's check and projection: P(u~) if the
        # proposal passes, else P(u + s) if the trial was accepted, else u; the damping
        # clamped to [nu_min nu0, nu_max nu0]
        pr = self.O.params_at(self._pr(p), k)
        chk, took = None, ("step" if tr["accept"] else "none")
        if pl is not None:
            chk = self.O.check_proposal(self.go, pr, y.numpy(), lam.numpy(), mu.numpy(), s.numpy(),
                                        pl.numpy(), pm.numpy())
            if chk["accept"]:
                a, b = self.O.project(pr, pl.numpy(), pm.numpy())
                took = "proposal"
        if took == "step":
            a, b = self.O.project(pr, (lam + s[0]).numpy(), (mu + s[1]).numpy())
        if took != "none":
            lam.copy_(torch.from_numpy(a))
            mu.copy_(torch.from_numpy(b))
        nu = min(max(tr["nu_next"], p.nu_min * nu0), p.nu_max * nu0)
        return {"check": chk, "took": took, "nu_next": nu}


def _proposal(u, s, k):
    return u + 1.5 * s if k % 2 else None  # overshooting the LM step: taken only when it passes


CASES = {
    "plain": (dict(), None),
    "continuation": (dict(alpha_decay=5.0, alpha_decay_iters=6), None),
    "proposals": (dict(), _proposal),
    "linear_bound": (dict(lin_constraint=1, lin_slope=8.0, lin_offset=0.1), _proposal),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_resume_equals_uninterrupted(O, monkeypatch, case):
    kw, G = CASES[case]
    ph = synth.lattice_phantom(N, 3, radius=2.0, seed=41)
    go = O.geom(N, NA, ND, n_sub=S)
    y = synth.poisson_noise(O.forward(go, ph.lam, ph.mu), 1e4, 42)
    l0, m0 = O.initial_guess(go, y)
    monkeypatch.setattr(accelerated, "P", _OracleCalls(O, go))
    p = P.default_params(precision=0, max_iters=8, cg_max_iters=6, **kw)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    run = lambda lam, mu, **a: accelerated.accelerated_solve(None, None, p, t(y), lam, mu, G=G, **a)

    lam8, mu8, h8 = run(t(l0), t(m0))
    lam4, mu4, h4 = run(t(l0), t(m0), iters=4)
    assert not (torch.equal(lam4, t(l0)) and torch.equal(mu4, t(m0)))  # the checkpoint has moved
    lamr, mur, hr = run(lam4, mu4, state=h4[-1]["state"])
    assert [h["k"] for h in hr] == [4, 5, 6, 7]
    assert torch.equal(lamr, lam8) and torch.equal(mur, mu8)
    assert len(h4 + hr) == len(h8)
    for a, b in zip(h4 + hr, h8):
        assert a["took"] == b["took"] and a["nu"] == b["nu"] and a["state"] == b["state"]
    took = [h["took"] for h in hr]
    assert "step" in took or "proposal" in took  # the resumed part moves too
    if case in ("proposals", "linear_bound"):
        assert "proposal" in [h["took"] for h in h8]
    if "lin_constraint" in kw:
        l, m = lam8.numpy(), mu8.numpy()
        assert np.all(l <= kw["lin_slope"] * m + kw["lin_offset"] + 1e-12)


def test_invalid_checkpoint_is_refused(O, monkeypatch):
    go = O.geom(N, NA, ND, n_sub=S)
    monkeypatch.setattr(accelerated, "P", _OracleCalls(O, go))
    p = P.default_params(precision=0, max_iters=2)
    z = torch.zeros((N, N), dtype=torch.float64)
    for bad in ({"k": -1, "nu": 1.0, "nu0": 1.0}, {"k": 1, "nu": 0.0, "nu0": 1.0},
                {"k": 1, "nu": 1.0, "nu0": float("nan")}):
        with pytest.raises(ValueError):
            accelerated.accelerated_solve(None, None, p, z, z, z, state=bad)

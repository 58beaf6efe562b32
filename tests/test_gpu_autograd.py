"""Differentiation: the torch.autograd wrapper of the forward model against the FP64 oracle
gradient of 1/2 |A(lam, mu) - y|^2, central finite differences (h = 1e-3, FP64) in
both modes, and a batch of random (lam, mu) pairs from the lattice distribution at
the differentiation workload's geometry (256 x 256, 360 angles x 182 x 5 sub-rays)."""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def AG(P):
    from paper_2604_26745_gb300 import autograd
    return autograd


def _pair(n, n_lat, seed, radius=5.0):
    ph = synth.lattice_phantom(n, n_lat, radius=radius, seed=seed)
    return ph.lam, ph.mu


def test_backward_matches_oracle_gradient_256(AG, O, P, torch):
    n, na, nd, S = 256, 360, 182, 5
    g = P.geometry(n, na, nd, n_sub=S)
    go = O.geom(n, na, nd, n_sub=S)
    lam, mu = _pair(n, 17, 1200)
    l2, m2 = _pair(n, 17, 1201)
    y = O.forward(go, l2, m2)
    ol, om = O.vjp(go, lam, mu, O.forward(go, lam, mu) - y)  # oracle gradient of the loss
    for dt, tol in ((torch.float64, 1e-11), (torch.float32, 5e-5)):
        L = torch.tensor(lam, dtype=dt, device="cuda", requires_grad=True)
        M = torch.tensor(mu, dtype=dt, device="cuda", requires_grad=True)
        loss = AG.data_loss(L, M, torch.tensor(y, dtype=dt, device="cuda"), g)
        loss.backward()
        for got, ref in ((L.grad, ol), (M.grad, om)):
            err = float(np.abs(got.double().cpu().numpy() - ref).max() / np.abs(ref).max())
            assert err <= tol, (dt, err)


def test_reverse_and_forward_mode_match_central_differences(AG, P, torch):
    n, na, nd, S = 64, 90, 182, 5
    g = P.geometry(n, na, nd, n_sub=S)
    lam, mu = _pair(n, 5, 7, radius=3.0)
    rs = np.random.default_rng(8)
    L = torch.tensor(lam, device="cuda", requires_grad=True)
    M = torch.tensor(mu, device="cuda", requires_grad=True)
    y = torch.tensor(rs.standard_normal((na, nd)), device="cuda")
    dl = torch.tensor(rs.standard_normal((n, n)), device="cuda")
    dm = torch.tensor(0.01 * rs.standard_normal((n, n)), device="cuda")
    h = 1e-3
    f = lambda a, b: float(AG.data_loss(a, b, y, g))
    fd = (f(L.detach() + h * dl, M.detach() + h * dm) - f(L.detach() - h * dl, M.detach() - h * dm)) / (2 * h)
    AG.data_loss(L, M, y, g).backward()
    an = float((L.grad * dl).sum() + (M.grad * dm).sum())
    assert abs(fd - an) <= 1e-6 * abs(an)  # O(h^2) truncation of the central quotient
    # forward mode (dual numbers): directional derivative of the projection
    import torch.autograd.forward_ad as fwAD
    with fwAD.dual_level():
        yd = AG.project(fwAD.make_dual(L.detach(), dl), fwAD.make_dual(M.detach(), dm), g)
        jv = fwAD.unpack_dual(yd).tangent
    yp = AG.project(L.detach() + h * dl, M.detach() + h * dm, g)
    ym = AG.project(L.detach() - h * dl, M.detach() - h * dm, g)
    fdj = (yp - ym) / (2 * h)
    assert float((jv - fdj).norm() / fdj.norm()) <= 1e-6


def test_batch_of_pairs_256(AG, P, torch):
    """A batch of random (lam, mu) pairs: batched gradient equals per-item gradients."""
    n, na, nd, S = 256, 360, 182, 5
    g = P.geometry(n, na, nd, n_sub=S)
    B = 4
    pairs = [_pair(n, 17, 1200 + i) for i in range(B)]
    L = torch.tensor(np.stack([p[0] for p in pairs]), dtype=torch.float32, device="cuda", requires_grad=True)
    M = torch.tensor(np.stack([p[1] for p in pairs]), dtype=torch.float32, device="cuda", requires_grad=True)
    y = torch.zeros((B, na, nd), dtype=torch.float32, device="cuda")
    AG.data_loss(L, M, y, g).backward()
    for i in (0, B - 1):
        Li = L.detach()[i].clone().requires_grad_(True)
        Mi = M.detach()[i].clone().requires_grad_(True)
        AG.data_loss(Li, Mi, y[i], g).backward()
        assert torch.equal(Li.grad, L.grad[i]) and torch.equal(Mi.grad, M.grad[i])

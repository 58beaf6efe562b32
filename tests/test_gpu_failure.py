"""Failure path of the bounded device-side waits, without faulting the GPU.

The forward and JVP kernels receive their image chunks by TMA bulk copies that complete
on an mbarrier, and every wait on a barrier phase is bounded by device time.  The test
aid PGET_TEST_TX_EXTRA makes the first chunk of every walk expect 16 bytes that no copy
delivers, so that wait runs out (after PGET_TEST_WAIT_NS); the kernel records the error,
issues no further copies, still waits for the copies already issued, and returns.  The
host must report PGET_ETIMEOUT, and a new context on the same device must work normally.
"""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


def _problem(P, torch):
    g = P.geometry(48, 30, 91, n_sub=3)
    ph = synth.lattice_phantom(48, 4, radius=2.0, seed=77)
    with P.Context(0) as c:
        y = P.pget_forward(c, g, P.PGET_F64, torch.tensor(ph.lam, device="cuda"),
                           torch.tensor(ph.mu, device="cuda"))
    y = synth.poisson_noise(y.cpu().numpy(), 1e5, 78)
    return g, torch.tensor(y, dtype=torch.float32, device="cuda")


def _solve(P, ctx, g, y):
    p = P.default_params(max_iters=2, cg_max_iters=4, precision=P.PGET_F32_KAHAN)
    lam, mu = P.pget_initial_guess(ctx, g, p, y)
    P.pget_lm_solve(ctx, g, p, y, lam, mu)
    return lam, mu


def test_lost_chunk_copy_times_out_and_device_stays_usable(P, torch, monkeypatch):
    g, y = _problem(P, torch)
    with P.Context(0) as c:
        ref = _solve(P, c, g, y)
    monkeypatch.setenv("PGET_TEST_TX_EXTRA", "16")
    monkeypatch.setenv("PGET_TEST_WAIT_NS", "2000000")  # 2 ms per wait
    with P.Context(0) as c:
        with pytest.raises(P.PgetError) as e:
            _solve(P, c, g, y)
        assert e.value.status == P.PGET_ETIMEOUT
    monkeypatch.delenv("PGET_TEST_TX_EXTRA")
    monkeypatch.delenv("PGET_TEST_WAIT_NS")
    with P.Context(0) as c:
        got = _solve(P, c, g, y)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    assert np.isfinite(got[0].cpu().numpy()).all()


def test_operator_status_reports_a_lost_chunk_copy(P, torch, monkeypatch):
    """The asynchronous operator calls cannot wait for their kernels; the error word they
    leave is read by pget_operator_status, which reports the timed-out chunk copy."""
    g, y = _problem(P, torch)
    lam = torch.full((48, 48), 0.5, dtype=torch.float32, device="cuda")
    mu = torch.full((48, 48), 0.01, dtype=torch.float32, device="cuda")
    monkeypatch.setenv("PGET_TEST_TX_EXTRA", "16")
    monkeypatch.setenv("PGET_TEST_WAIT_NS", "2000000")
    with P.Context(0) as c:
        P.pget_forward(c, g, P.PGET_F32_KAHAN, lam, mu)
        with pytest.raises(P.PgetError) as e:
            P.pget_operator_status(c)
        assert e.value.status == P.PGET_ETIMEOUT
    monkeypatch.delenv("PGET_TEST_TX_EXTRA")
    monkeypatch.delenv("PGET_TEST_WAIT_NS")
    with P.Context(0) as c:
        P.pget_forward(c, g, P.PGET_F32_KAHAN, lam, mu)
        P.pget_operator_status(c)  # clean: no error

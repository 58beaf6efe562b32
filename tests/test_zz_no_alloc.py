"""The allocation-free forward entry point (pget_forward_noalloc) against the regular
one.  It is meant for callers that may not allocate device memory, so it keeps its
scratch in a fixed array inside the library; this file checks that two calls in a row
(the second reusing the first call's scratch) give the regular entry point's result, and
that a geometry needing more scratch than the array holds is refused.  Collected last."""
import numpy as np
import pytest

from paper_2604_26745_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(2, 0.0), (0, 0.0)])
def test_noalloc_forward_matches_context_forward(ctx, P, torch, prec, tol):
    n, na, nd, S = 128, 360, 182, 5
    g = P.geometry(n, na, nd, n_sub=S)
    dt = P.dtype_of(prec)
    for seed in (1, 2):  # two calls in a row, different inputs
        ph = synth.lattice_phantom(n, 9, radius=5.0, seed=seed)
        lam = torch.tensor(ph.lam, dtype=dt, device="cuda")
        mu = torch.tensor(ph.mu, dtype=dt, device="cuda")
        y_ref = P.pget_forward(ctx, g, prec, lam, mu)
        y = torch.full((na, nd), float("nan"), dtype=dt, device="cuda")
        assert P.pget_forward_noalloc(g, prec, lam, mu, y) == P.PGET_OK
        torch.cuda.synchronize()
        err = float((y - y_ref).abs().max() / y_ref.abs().max())
        assert err <= tol, err


def test_noalloc_small_geometry_and_limit(ctx, P, torch):
    g = P.geometry(40, 36, 182, n_sub=3)
    ph = synth.lattice_phantom(40, 4, seed=3)
    lam = torch.tensor(ph.lam, dtype=torch.float32, device="cuda")
    mu = torch.tensor(ph.mu, dtype=torch.float32, device="cuda")
    y = torch.empty((36, 182), dtype=torch.float32, device="cuda")
    for _ in range(2):
        assert P.pget_forward_noalloc(g, P.PGET_F32_KAHAN, lam, mu, y) == P.PGET_OK
        y_ref = P.pget_forward(ctx, g, P.PGET_F32_KAHAN, lam, mu)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref)
    big = P.geometry(1024, 720, 182, n_sub=5)
    z = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    yb = torch.zeros((720, 182), dtype=torch.float32, device="cuda")
    assert P.pget_forward_noalloc(big, P.PGET_F32_KAHAN, z, z, yb) == P.PGET_ENOMEM
    assert P.pget_forward_noalloc(P.geometry(1, 4, 91), P.PGET_F32, z, z, yb) == P.PGET_EINVAL


def test_noalloc_two_host_threads_different_geometries(ctx, P, torch):
    """Two host threads call the allocation-free forward at the same time with different
    geometries; the process-wide lock keeps their host tables and device scratch apart,
    so every result equals the context forward of its own geometry bitwise."""
    import threading
    cases = []
    for n, na, nd, S, seed in ((48, 60, 182, 3, 11), (40, 36, 91, 5, 12)):
        g = P.geometry(n, na, nd, n_sub=S)
        ph = synth.lattice_phantom(n, 4, seed=seed)
        lam = torch.tensor(ph.lam, dtype=torch.float32, device="cuda")
        mu = torch.tensor(ph.mu, dtype=torch.float32, device="cuda")
        cases.append((g, lam, mu, P.pget_forward(ctx, g, P.PGET_F32_KAHAN, lam, mu).clone()))
    torch.cuda.synchronize()
    bad = []

    def worker(i):
        g, lam, mu, ref = cases[i]
        s = torch.cuda.Stream()
        y = torch.empty_like(ref)
        for _ in range(20):
            st = P.pget_forward_noalloc(g, P.PGET_F32_KAHAN, lam, mu, y, s)
            if st != P.PGET_OK or not torch.equal(y, ref):
                bad.append((i, st))

    th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not bad, bad


def test_noalloc_refuses_stream_capture(ctx, P, torch):
    g = P.geometry(40, 36, 182, n_sub=3)
    lam = torch.zeros((40, 40), dtype=torch.float32, device="cuda")
    y = torch.zeros((36, 182), dtype=torch.float32, device="cuda")
    assert P.pget_forward_noalloc(g, P.PGET_F32, lam, lam, y) == P.PGET_OK  # first call: set-up
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        graph.capture_begin()
        st = P.pget_forward_noalloc(g, P.PGET_F32, lam, lam, y, s)
        graph.capture_end()
    assert st == P.PGET_EINVAL

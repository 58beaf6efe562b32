"""Multi-rank host logic of bench.py on CPU: two gloo ranks each time their own
(independent) requests, the job time is the max over ranks and the throughput counts
every rank's requests (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import time

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank "reconstructs" its own request ids with a rank-dependent cost
    ids = bench.rank_request_ids(rank, world, 8)
    t0 = time.perf_counter()
    time.sleep(0.05 * (rank + 1))
    elapsed = time.perf_counter() - t0
    t = torch.tensor([elapsed], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, ids, float(t.item()), elapsed))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ids0, tmax0, e0), (r1, ids1, tmax1, e1) = res
    assert tmax0 == tmax1 and abs(tmax0 - max(e0, e1)) < 1e-12
    assert not set(ids0) & set(ids1)  # independent work per rank
    assert len(ids0) == len(ids1) == 8


def _solve_request(k):
    """A small reconstruction keyed by the request id, as bench.py keys its problems
    (phantom seed 1100 + k, noise seed 2100 + k), solved by the oracle on the CPU."""
    from oracle import oracle as O
    from paper_2604_26745_gb300 import synth
    g = O.geom(16, 12, 182, n_sub=3)
    ph = synth.lattice_phantom(16, 3, radius=2.0, seed=1100 + k)
    y = synth.poisson_noise(O.forward(g, ph.lam, ph.mu), 1e4, 2100 + k)
    l0, m0 = O.initial_guess(g, y)
    lam, mu, rep = O.lm(g, O.default_params(max_iters=3, cg_max_iters=5), y, l0, m0)
    return lam, mu, rep["f_final"]


def _worker(rank, world, port, q):
    import time

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = bench.rank_request_ids(rank, world, 3)
    t0 = time.perf_counter()
    out = {k: _solve_request(k) for k in ids}
    elapsed = time.perf_counter() - t0
    t = torch.tensor([elapsed], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, ids, float(t.item()), {k: (v[0].tobytes(), v[1].tobytes(), v[2]) for k, v in out.items()}))
    dist.destroy_process_group()


def test_two_ranks_reconstruct_their_own_requests():
    """The data path of the replicas: each rank reconstructs its own request ids with no
    collective on the data; every result equals the same request solved in one process,
    bitwise, and together the ranks cover every request once."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][2] == res[1][2]  # the job time: max over ranks
    ids = res[0][1] + res[1][1]
    assert sorted(ids) == list(range(6))
    for _, _, _, out in res:
        for k, (lb, mb, f) in out.items():
            lam, mu, f1 = _solve_request(k)
            assert lb == lam.tobytes() and mb == mu.tobytes() and f == f1


def _leaver(rank, world, port, q, how):
    import time

    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    dist = bench.init_dist("gloo", 5.0, rank=rank, world_size=world)
    t = torch.ones(1)
    dist.all_reduce(t)  # one step together
    if rank == 1:
        if how == "stall":
            time.sleep(40.0)  # alive, but never joins another collective
        os._exit(0)  # leaves between steps, without a word to the others
    time.sleep(0.5)
    t0 = time.perf_counter()
    try:
        dist.all_reduce(t)
        q.put(("returned", time.perf_counter() - t0))
    except Exception as e:  # the failure the survivor must see
        q.put((type(e).__name__, time.perf_counter() - t0))
    q.close()
    q.join_thread()  # the report is written before the process ends
    os._exit(0)


@pytest.mark.parametrize("how", ["exit", "stall"])
def test_a_rank_that_leaves_fails_the_next_collective(how):
    """Failure detection on the host.

    Rank 1 leaves between steps, either by exiting or by stalling alive. Rank 0's next
    collective must end with an error instead of waiting for ever. An exit closes the
    connection at once. A stall is caught by the process group's timeout: 5 s here, set
    in the bench by --dist-timeout."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, q, how)) for r in range(2)]
    for p in procs:
        p.start()
    what, waited = q.get(timeout=120)
    procs[0].join(timeout=60)
    procs[1].kill()  # the stalled rank: this test's own child process
    procs[1].join(timeout=60)
    assert what != "returned", "the collective completed without the rank that left"
    assert waited < 30.0
    if how == "stall":
        assert waited >= 4.0  # ended by the timeout, not by a closed connection

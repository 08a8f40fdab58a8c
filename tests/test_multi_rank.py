"""Independent problems sharded across two ranks (gloo, CPU): every problem is
solved exactly once and the gathered results equal a single-process run."""
import os
import socket

import numpy as np
import pytest

from paper_2205_06619_gb300 import batch, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problems():
    rng = np.random.default_rng(3)
    out = []
    for q in range(7):
        m = int(rng.integers(4, 14)); n = int(rng.integers(4, 14)); r = int(rng.integers(1, 4))
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.85, seed=100 + q)
        out.append(dict(R=R, M=M, m=m, n=n, rank=r, sweeps=1, seed=q))
    return out


def _solve(probs):
    import oracle
    res = []
    for p in probs:
        o = oracle.factorize(p["R"], p["M"], p["rank"], sweeps=p["sweeps"], seed=p["seed"])
        res.append((o["U"], o["V"], float(o["f_hist"][-1]), os.getpid()))
    return res


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = batch.run_sharded(_problems(), _solve)
        if rank == 0:
            queue.put([(u.tolist(), v.tolist(), f, pid) for (u, v, f, pid) in out])
    finally:
        dist.destroy_process_group()


def test_partition_balances_and_covers():
    costs = [batch.problem_cost(m, n, r, 10) for (m, n, r) in
             [(100, 200, 3), (2000, 8000, 20), (500, 500, 5), (1000, 300, 7), (150, 150, 3), (1800, 7000, 19)]]
    shares = batch.partition(costs, 2)
    assert sorted(q for s in shares for q in s) == list(range(len(costs)))
    loads = [sum(costs[q] for q in s) for s in shares]
    assert max(loads) <= 0.75 * sum(loads)
    assert batch.partition(costs, 2) == shares          # deterministic


def test_two_rank_gloo_sharding_matches_single_process():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = queue.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = _solve(_problems())
    assert len(got) == len(ref)
    pids = set()
    for (u, v, f, pid), (ur, vr, fr, _) in zip(got, ref):
        assert np.array_equal(np.array(u), ur) and np.array_equal(np.array(v), vr) and f == fr
        pids.add(pid)
    assert len(pids) == 2                                   # both ranks did work

"""The N > 1 path of bench.py on the CPU: two gloo ranks take interleaved tau
points (each point of the cycle once) and report the whole-job time (max over
ranks) and useful flops (sum over ranks)."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, steps, n_tau, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        taus = [bench.tau_index(i, world, rank, n_tau) for i in range(steps)]
        t, f = bench.job_totals(1.0 + 0.5 * rank, 10.0 * (rank + 1), "cpu")
        q.put((rank, taus, t, f))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("steps,n_tau", [(7, 20), (10, 20), (3, 5)])
def test_two_ranks_shard_tau_points_and_reduce(steps, n_tau):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, steps, n_tau, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # global step g = 2 i + r walks the tau cycle once per n_tau steps
    seen = {}
    for rank, taus, _, _ in res:
        for i, j in enumerate(taus):
            seen[2 * i + rank] = j
    assert sorted(seen) == list(range(2 * steps))
    assert all(seen[g] == g % n_tau for g in seen)
    # every tau point of a full cycle is taken exactly once when the job
    # covers it
    if 2 * steps >= n_tau:
        assert sorted(seen[g] for g in range(n_tau)) == list(range(n_tau))
    for _, _, t, f in res:
        assert t == pytest.approx(1.5)   # max over ranks
        assert f == pytest.approx(30.0)  # sum over ranks


def test_single_process_totals_are_local():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_totals(2.0, 5.0, "cpu") == (2.0, 5.0)
    assert [bench.tau_index(i, 1, 0, 4) for i in range(6)] == [0, 1, 2, 3, 0, 1]

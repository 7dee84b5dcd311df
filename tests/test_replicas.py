"""Replica aggregation across ranks (gloo, world size 2, CPU)."""
import os
import socket

import pytest

from paper_2301_05726_gb300.replicas import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2301_05726_gb300.replicas import combine_step
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = combine_step(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_combine_step_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 300.0), (1, 15.0, 300.0)]  # slowest rank's time, total work


def test_combine_step_single_process():
    from paper_2301_05726_gb300.replicas import combine_step
    assert combine_step(3.0, 7.0) == (3.0, 7.0)


@pytest.mark.parametrize("n,world", [(256, 2), (256, 8), (5, 4), (0, 3)])
def test_shard_partitions_jobs(n, world):
    parts = [shard(n, r, world) for r in range(world)]
    flat = sorted(x for p in parts for x in p)
    assert flat == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1

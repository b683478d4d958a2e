"""The N > 1 path of bench.py on CPU: two gloo ranks each time their own
replicas; the job's time is the slowest rank's and its rate counts every
rank's work (weak scaling, no data-path collective)."""
from __future__ import annotations

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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    my_seconds = [2.0, 3.0][rank]
    slowest = bench.max_over_ranks(my_seconds)
    rate = bench.whole_job_rate(6e12, ws, slowest)
    q.put((rank, ws, r, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, slowest, rate in out:
        assert ws == 2 and r == rank
        assert slowest == 3.0                             # the slowest rank's time
        assert abs(rate - 6e12 * 2 / 3.0e9) < 1e-6         # every rank's flips over that time


def test_single_process_aggregation():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_rate(1e12, 1, 1.0) == 1000.0

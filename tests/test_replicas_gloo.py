"""The N > 1 path of bench.py (independent replicas) on CPU with gloo, world size 2.

Each rank times its own replica; the job's time is the maximum over ranks and
the job's rate is all units over that time.  No data-path collective exists."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.0 + rank          # rank 1 is the slower replica
    t = bench.max_over_ranks(local, dist, "cpu")
    rate = bench.whole_job_rate(8192, world, t)
    dist.barrier()
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate():
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
    assert [r[1] for r in res] == [2.0, 2.0]
    assert res[0][2] == res[1][2] == 2 * 8192 / 2.0


def test_single_rank_has_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0

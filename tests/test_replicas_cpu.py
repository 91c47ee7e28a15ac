"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU only).

The library runs one independent replica per GPU (columns and FISTA instances shard with
no exchange), so the only multi-process logic is the barrier, the max-over-ranks time and
the whole-job units; this test runs it with two gloo ranks.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (1 + r) seconds for (10 + r) units of work
    rate, t = bench.job_throughput(1.0 + rank, 10.0 + rank, dist, None)
    dist.barrier()
    q.put((rank, rate, t))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for _, rate, t in out:
        assert t == pytest.approx(2.0)          # the slowest rank's time
        assert rate == pytest.approx(21.0 / 2.0)  # all units over that time


def test_single_process_is_plain_ratio():
    import bench
    rate, t = bench.job_throughput(2.0, 8.0)
    assert rate == 4.0 and t == 2.0

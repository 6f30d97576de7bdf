"""The benchmark's multi-rank logic on CPU with two gloo ranks: each rank times its own replica,
the job time is the maximum over ranks, and the throughput counts every rank's nodes."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 250.0][rank]
    t = bench.max_over_ranks(local_ms)
    value = bench.job_throughput(1000, 10, world, t)
    q.put((rank, t, value, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    for rank, t, value, env in out:
        assert t == pytest.approx(250.0)
        assert value == pytest.approx(2 * 1000 * 10 / 0.25)
        assert env == (rank, 2, rank)


def test_single_process_identity():
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_throughput(10, 2, 1, 1000.0) == pytest.approx(20.0)

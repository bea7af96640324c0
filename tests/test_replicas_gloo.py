"""The multi-GPU form of the benchmark is N independent replicas (no data-path collective): the host logic that
turns the ranks' timed steps into one whole-job rate, run here as two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [120.0, 180.0][rank]            # the slower rank sets the time
        ms, value = bench.replica_rate(ms_local, 10, world, dist, "cpu")
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_rate_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p_ in procs:
        p_.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p_ in procs:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    for rank, ms, value in out:
        assert ms == 180.0
        assert value == pytest.approx(2 * 10 / 0.180)


def test_single_replica_rate():
    ms, value = bench.replica_rate(200.0, 10, 1, None, "cpu")
    assert ms == 200.0 and value == pytest.approx(50.0)

"""Host logic of bench.py's multi-GPU mode on CPU: two gloo ranks.

With N GPUs the bench runs N independent replicas of the workload (the path
is replicated, not sharded: no collective on the data path); the only
cross-rank operations are the barrier and the max over ranks of the timed
duration, from which the whole-job throughput is computed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slowest
        worst = bench.max_over_ranks(ms, world)
        dist.barrier()
        out[rank] = (worst, bench.replica_value(1_000_000, world, worst))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    worst, value = res[0]
    assert worst == 15.0
    assert value == pytest.approx(2 * 1_000_000 / 0.015 / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_value(268435456, 1, 100.0) == pytest.approx(2.68435456)

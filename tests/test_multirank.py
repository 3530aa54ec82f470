"""The multi-GPU path of the benchmark on CPU: two `gloo` ranks run the host
logic that bench.py runs on N GPUs (replicas with a max-over-ranks time and
summed iterations; the batched workload partitioned across ranks)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0, 30.0][rank]          # rank 1 is the slowest
        iters = [500, 700][rank]
        value, tmax, total = bench.aggregate_over_ranks(torch, dist, world, ms, iters, "cpu")
        shard = bench.batch_shard(list(range(256)), rank, world)
        out[rank] = (value, tmax, total, shard)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        value, tmax, total, _ = out[rank]
        assert tmax == 30.0 and total == 1200.0
        assert abs(value - 1200.0 / 0.030) < 1e-6
    shards = [out[r][3] for r in range(world)]
    assert sorted(shards[0] + shards[1]) == list(range(256))
    assert not set(shards[0]) & set(shards[1])


def test_single_rank_aggregation():
    value, tmax, total = bench.aggregate_over_ranks(torch, None, 1, 20.0, 400, "cpu")
    assert (value, tmax, total) == (400 / 0.020, 20.0, 400.0)
    assert bench.batch_shard(list(range(5)), 0, 1) == list(range(5))

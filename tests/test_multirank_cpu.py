"""The N-rank paths of the benchmark on CPU with the gloo backend, world
size 2: whole-job aggregation (max time, summed updates) of replicated
ranks, and the work-balanced sharding of batch instances across ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, upd = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1), "cpu")
    sizes = [5000, 200000, 12000, 7000, 150000, 9000, 60000]
    part = bench.shard_instances(sizes, world)[rank]
    got = [torch.zeros(len(sizes), dtype=torch.int64) for _ in range(world)]
    mine = torch.zeros(len(sizes), dtype=torch.int64)
    mine[part] = 1
    dist.all_gather(got, mine)
    out[rank] = (ms, upd, [int(x) for x in sum(got)])
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        ms, upd, cover = out[r]
        assert ms == 15.0 and upd == 3000.0          # slowest rank, all ranks' updates
        assert cover == [1] * 7                      # every instance on exactly one rank


def test_shard_balances_work():
    sizes = [5000, 200000, 12000, 7000, 150000, 9000, 60000, 100000]
    parts = bench.shard_instances(sizes, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert bench.shard_instances(sizes, 1) == [list(range(len(sizes)))]

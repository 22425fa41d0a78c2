"""Host logic of the multi-GPU replicas path, on CPU with two gloo ranks:
balanced and cost-based sharding, and the max-over-ranks timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2109_05496_gb300 import dist as pdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank
        mx = pdist.max_over_ranks(local_ms)
        mine = pdist.shard_by_cost(costs, world)[rank]
        start, stop = pdist.shard_range(len(costs), rank, world)
        dist.barrier()
        q.put((rank, mx, mine, (start, stop)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo():
    world = 2
    costs = [64 * 64, 1024 * 1024, 300 * 200, 512 * 700, 90 * 90, 1000 * 80, 256 * 256]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(r[1] == 15.0 for r in res)              # the max of 10 and 15 on every rank
    shards = [r[2] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) <= sum(costs) - min(loads) + 1   # no rank has more than the other's complement
    ranges = [r[3] for r in res]
    assert ranges == [(0, 4), (4, 7)]


def test_shard_helpers_single_process():
    assert pdist.shard_range(10, 0, 3) == (0, 4) and pdist.shard_range(10, 2, 3) == (7, 10)
    assert pdist.max_over_ranks(3.5) == 3.5
    assert pdist.weak_scaling_value(1e9, 1000.0, 4) == pytest.approx(4e9)
    with pytest.raises(ValueError):
        pdist.shard_range(5, 3, 3)

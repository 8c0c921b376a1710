"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2).

One process per GPU runs independent replicas (the single-field workload does
not shard without an all-to-all per iteration); the whole-job figure takes the
step time as the max over ranks.  Batched workloads spread items over ranks by
bytes with no collective on the data path.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 20.0][rank]
        ms, value = bench.aggregate_ranks(torch, dist, local_ms, 1_000_000_000, world)
        items = [100, 7, 50, 50, 3, 99, 1]
        mine = bench.shard_items(items, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, ms, value, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_disjoint_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, shards in res:
        assert ms == 20.0                          # the slower rank sets the step time
        assert value == pytest.approx(2 * 1e9 / 0.020 / 1e9)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(7))              # every item on exactly one rank
    loads = [sum([100, 7, 50, 50, 3, 99, 1][i] for i in s) for s in res[0][3]]
    assert max(loads) - min(loads) <= 100


def test_single_rank_aggregation_is_identity():
    ms, value = bench.aggregate_ranks(torch, None, 8.0, 4_000_000, 1)
    assert ms == 8.0 and value == pytest.approx(4e6 / 0.008 / 1e9)
    assert bench.shard_items([5, 4, 3], 0, 1) == [0, 1, 2]

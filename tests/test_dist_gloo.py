"""Multi-rank host logic on CPU: two gloo ranks split an ensemble and combine
their timings (max) and work (sum) the way bench.py does with N GPUs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2309_03543_gb300.dist import aggregate, shard


def test_shard_is_a_partition():
    items = list(range(23))
    parts = [shard(items, r, 4) for r in range(4)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard(items, 4, 4)


def test_aggregate_without_a_group_is_local():
    assert aggregate(1.5, 7.0) == (1.5, 7.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard(range(10), rank, world)
        t, u = aggregate(0.5 + rank, float(sum(mine)))
        out[rank] = (t, u, mine)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_and_work():
    world = 2
    port = _free_port()
    # the manager's server process is spawned too: forking a process that
    # already runs OpenMP or torch threads can deadlock the child
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5                  # slowest rank
    assert res[0][1] == res[1][1] == float(sum(range(10)))  # all the work
    assert sorted(res[0][2] + res[1][2]) == list(range(10))

"""Sharding of independent cases over ranks (host logic of the multi-GPU
path) and its reductions, with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

from paper_2002_04353_gb300 import inputs as I
from paper_2002_04353_gb300 import shard


def test_assign_cases_partitions_and_balances():
    counts = [c.mesh.n_nodes for c in I.batched_sweep()]
    for world in (1, 2, 3, 4, 8):
        shards = shard.assign_cases(counts, world)
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(len(counts)))
        loads = [sum(counts[k] for k in s) for s in shards]
        assert max(loads) - sum(counts) / world < max(counts)
        assert all(s == sorted(s) for s in shards)
    assert shard.assign_cases(counts, 4) == shard.assign_cases(counts, 4)  # deterministic
    assert shard.assign_cases([5, 5, 5], 2) == [[0, 2], [1]]  # ties go to the lower rank
    with pytest.raises(ValueError):
        shard.assign_cases(counts, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, counts, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard.assign_cases(counts, world)[rank]
    nodes = sum(counts[k] for k in mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t_max = shard.max_over_ranks(10.0 + rank, torch)
    n_sum = shard.sum_over_ranks(nodes, torch)
    dist.destroy_process_group()
    out.put((rank, gathered, t_max, n_sum))


def test_two_gloo_ranks_share_the_sweep():
    import torch.multiprocessing as mp
    counts = [c.mesh.n_nodes for c in I.batched_sweep()]
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, counts, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t_max, n_sum in res:
        assert sorted(k for s in gathered for k in s) == list(range(len(counts)))  # no case twice, none lost
        assert t_max == 10.0 + world - 1  # the slowest rank's time
        assert n_sum == sum(counts)
    assert res[0][1] == res[1][1]

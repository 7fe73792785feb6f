"""The multi-GPU work split: independent pairs per rank, no data-path collective.

Checked on the CPU with two gloo ranks: every rank derives the same assignment, the ranks'
shares are disjoint and cover the batch, the load is balanced, and the benchmark's timing
aggregation (max over ranks) and its per-rank seeds behave as the contract needs.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1709_06509_gb300 import shard, synth


def test_assign_is_a_balanced_partition():
    specs = synth.batch_specs(64)
    for world in (1, 2, 3, 8):
        owned = shard.assign(specs, world)
        flat = sorted(i for o in owned for i in o)
        assert flat == list(range(64))
        loads = [sum(shard.work(specs[i]) for i in o) for o in owned]
        assert max(loads) - min(loads) <= max(shard.work(s) for s in specs)
    with pytest.raises(ValueError):
        shard.assign(specs, 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = synth.batch_specs(16)
        mine = shard.assign(specs, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        # the benchmark's aggregation: the slowest rank's time
        t = torch.tensor([1.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        q.put((rank, gathered, float(t.item()), shard.seed_offset(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_split():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    g0, g1 = results[0][1], results[1][1]
    assert g0 == g1  # both ranks derived the same assignment
    assert sorted(g0[0] + g0[1]) == list(range(16)) and not set(g0[0]) & set(g0[1])
    assert results[0][2] == results[1][2] == 2.0
    assert results[0][3] != results[1][3]  # replicas draw different pairs

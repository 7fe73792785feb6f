"""Work split for several GPUs: independent stereo pairs, no data-path collective.

Each rank owns whole pairs (a pair never spans GPUs).  Pairs are assigned greedily, the
largest estimated work W*H*D first, to the rank with the least work so far (LPT
scheduling); ties go to the lowest rank, so every rank computes the same split.
"""
from __future__ import annotations


def work(spec) -> int:
    """Estimated work of a pair: pixels times labels."""
    _seed, W, H, D = spec
    return int(W) * int(H) * int(D)


def assign(specs, world: int) -> list[list[int]]:
    """Indices of `specs` owned by each of `world` ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(specs)), key=lambda i: (-work(specs[i]), i))
    load = [0] * world
    owned: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(i)
        load[r] += work(specs[i])
    return [sorted(o) for o in owned]


def seed_offset(rank: int) -> int:
    """Seed offset of a rank's replica of a fixed per-GPU workload (weak scaling)."""
    return 1_000_000 * rank

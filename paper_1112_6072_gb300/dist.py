"""Host logic for running the path on several GPUs, one process per GPU.

Jobs are independent (Algorithm PH, Step 3), so ranks never exchange data
while they compute; the only exchange is Step 4's sum.  Two ways to split
work, both without a data-path collective:

* independent batches: each rank evaluates its own seeded batch (weak
  scaling; the bench does this);
* one matrix's job queue dealt round-robin over ranks in queue order, so an
  LPT queue stays LPT across ranks (list scheduling over GPUs), then the
  ranks' per-matrix sums -- 256-bit residues -- are gathered and added on the
  host with carries.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np

MASK256 = (1 << 256) - 1


def shard_queue(queue, rank: int, world: int):
    """Queue positions rank, rank + world, ... of an ordered job queue."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    q = np.asarray(queue, dtype=np.uint32)
    return q[rank::world]


def batch_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's independent batch."""
    return int(base_seed) + int(rank)


def words_from_int(v: int):
    """A signed integer as four little-endian 64-bit words (mod 2^256)."""
    v &= MASK256
    return np.array([(v >> (64 * k)) & ((1 << 64) - 1) for k in range(4)], dtype=np.uint64)


def int_from_words(w, bits: int = 256) -> int:
    """Four words -> signed integer, sign-extended from bit bits-1."""
    v = 0
    for k in range(3, -1, -1):
        v = (v << 64) | int(w[k])
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


def combine_words(parts):
    """Sum of per-rank 256-bit residues with carries between words."""
    total = 0
    for w in parts:
        total = (total + int_from_words(w, 256)) & MASK256
    return words_from_int(total)


def gather_sum(local_words, group=None):
    """All ranks' word arrays (shape (..., 4), uint64) gathered and summed
    exactly on every rank.  A plain all_reduce of int64 words would drop the
    carries between words, so the words are gathered and added as integers."""
    import torch
    import torch.distributed as dist

    local = np.ascontiguousarray(local_words, dtype=np.uint64).reshape(-1, 4)
    t = torch.from_numpy(local.view(np.int64).copy())
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    out = np.zeros_like(local)
    for i in range(local.shape[0]):
        out[i] = combine_words([p.numpy().view(np.uint64)[i] for p in parts])
    return out


def max_over_ranks(value: float, group=None) -> float:
    """The slowest rank's time: the step time of the whole job."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

"""Lambda-batch sharding across ranks, one process per GPU.

The likelihood of one Lambda point does not depend on any other, so a batch of
world * K points splits into contiguous blocks of K rows, one block per rank, each
evaluated over the whole catalogue by that rank's own context.  The data path needs no
collective: each rank's outputs are final.  `gather_rows` collects the blocks back in
rank order for a caller that wants the whole batch in one place, and `max_over_ranks`
gives the job's time (the slowest rank) for throughput figures.  Works with any
torch.distributed backend (NCCL on GPUs, gloo on CPUs) or with no process group at all.
"""
from __future__ import annotations

import numpy as np


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def row_range(n_rows: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [a, b) of an n_rows batch owned by `rank`: contiguous, sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return n_rows * rank // world, n_rows * (rank + 1) // world


def rank_rows(lam_all, rank: int, world: int):
    """This rank's block of the global Lambda batch lam_all [world * K, 13]."""
    a, b = row_range(len(lam_all), rank, world)
    return lam_all[a:b]


def gather_rows(block, n_rows: int):
    """All ranks' blocks, concatenated in rank order (a tensor [n_rows, ...] on every rank).

    `block` is this rank's tensor of row_range(n_rows, rank, world) rows; blocks of
    unequal length are padded for the exchange and trimmed after it.
    """
    import torch
    dist = _dist()
    if dist is None:
        return block
    world, rank = dist.get_world_size(), dist.get_rank()
    sizes = [row_range(n_rows, r, world) for r in range(world)]
    width = max(b - a for a, b in sizes)
    if block.shape[0] != sizes[rank][1] - sizes[rank][0]:
        raise ValueError("block does not match this rank's rows")
    pad = torch.zeros((width,) + tuple(block.shape[1:]), dtype=block.dtype, device=block.device)
    pad[:block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, sizes)])


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    dist = _dist()
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def world_batch(K: int, world: int, make_batch) -> np.ndarray:
    """The global batch of world * K points (make_batch(n) draws n points)."""
    return np.asarray(make_batch(K * world))

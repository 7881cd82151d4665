"""Sharding across ranks, one process per GPU: by Lambda batch, or by events.

The likelihood of one Lambda point does not depend on any other, so a batch of
world * K points splits into contiguous blocks of K rows, one block per rank, each
evaluated over the whole catalogue by that rank's own context.  The data path needs no
collective: each rank's outputs are final.  `gather_rows` collects the blocks back in
rank order for a caller that wants the whole batch in one place, and `max_over_ranks`
gives the job's time (the slowest rank) for throughput figures.  Works with any
torch.distributed backend (NCCL on GPUs, gloo on CPUs) or with no process group at all.

Event sharding (for a catalogue too large for one device): each rank holds a share of
the events and of the found injections (with n_draw of the whole injection set) and
evaluates its parts with gwc_loglik_parts; `merge_parts` combines the shards exactly,
because the selection integral is a sum over injections, xi = sum_r xi_r:
    ln L = sum_r sum_events_r - N_det ln(sum_r xi_r)
    d ln L = sum_r d sum_events_r - N_det sum_r (xi_r / xi) d ln xi_r
`merge_parts_distributed` does the one exchange (an all_gather of K (5 + 2P) numbers,
on the GPU with NCCL) and the combination (gwc_merge_parts: a kernel for device rows, the
same FP64 arithmetic on the host for gloo's host rows).
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


def pack_parts(part, device=None):
    """One shard's gwc_loglik_parts outputs (a dict of tensors or arrays with keys
    sum_events, ln_xi, neff_sel, flags, n_events and, for the gradient, grad_events,
    grad_ln_xi) as the [K, 5 + 2P] FP64 rows that gwc_merge_parts reads, on `device`
    (default: where the part's tensors are; host for numpy arrays)."""
    import torch

    def t(x):
        x = x if isinstance(x, torch.Tensor) else torch.as_tensor(np.asarray(x))
        return x.to(dtype=torch.float64, device=device) if device is not None else x.to(torch.float64)
    se = t(part["sum_events"])
    if device is None:
        device = se.device
    K = int(se.shape[0])
    cols = [se[:, None], t(part["ln_xi"]).to(device)[:, None], t(part["neff_sel"]).to(device)[:, None],
            t(part["flags"]).to(device)[:, None],
            torch.full((K, 1), float(part["n_events"]), dtype=torch.float64, device=device)]
    if "grad_events" in part:
        cols += [t(part["grad_events"]).to(device).reshape(K, -1), t(part["grad_ln_xi"]).to(device).reshape(K, -1)]
    return torch.cat(cols, dim=1).contiguous()


def merge_packed(rows):
    """gwc_merge_parts on the packed rows [R, K, 5 + 2P] of R shards: a kernel on the
    current stream when rows is a CUDA tensor, the same FP64 arithmetic on the host for a
    CPU tensor.  Returns lnL_total, ln_xi, neff_sel, flags (and grad_total when P > 0) as
    tensors on the rows' device."""
    import ctypes
    import torch
    from . import _check, _stream_ptr, lib
    rows = rows.to(torch.float64).contiguous()
    R, K, W = (int(v) for v in rows.shape)
    P = (W - 5) // 2
    dev = rows.device
    out = {"lnL_total": torch.empty(K, dtype=torch.float64, device=dev),
           "ln_xi": torch.empty(K, dtype=torch.float64, device=dev),
           "neff_sel": torch.empty(K, dtype=torch.float64, device=dev),
           "flags": torch.empty(K, dtype=torch.int32, device=dev)}
    if P > 0:
        out["grad_total"] = torch.empty((K, P), dtype=torch.float64, device=dev)
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    _check(lib().gwc_merge_parts(R, K, P, p(rows), 1 if rows.is_cuda else 0, p(out["lnL_total"]),
                                 p(out["ln_xi"]), p(out["neff_sel"]), p(out["flags"]),
                                 p(out["grad_total"]) if P > 0 else None,
                                 _stream_ptr(None) if rows.is_cuda else None))
    return out


def merge_parts(parts):
    """Combine the gwc_loglik_parts outputs of every shard (a list of dicts, see
    pack_parts) into lnL_total, ln_xi, neff_sel, flags and grad_total (gwc_merge_parts, on
    the device of the first part's tensors)."""
    import torch
    first = pack_parts(parts[0])
    return merge_packed(torch.stack([first] + [pack_parts(q, first.device) for q in parts[1:]]))


def merge_parts_distributed(part):
    """merge_parts over all ranks of the process group: one all_gather of every rank's
    K (5 + 2P) numbers (P = 13, or 16 for the multi-peak model, taken from the
    gradients' width), then the same exact combination on every rank.  With NCCL the
    exchange and the combination stay on this rank's GPU; with gloo they run on the host."""
    import torch
    dist = _dist()
    if dist is None:
        return merge_parts([part])
    world = dist.get_world_size()
    on_gpu = dist.get_backend() == "nccl"
    device = torch.device("cuda", torch.cuda.current_device()) if on_gpu else torch.device("cpu")
    mine = pack_parts(part, device)
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine)
    return merge_packed(torch.stack(every))

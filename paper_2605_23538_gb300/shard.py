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
`merge_parts_distributed` does the one exchange (an all_gather of K (5 + 2P) numbers).
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


def merge_parts(parts):
    """Combine the gwc_loglik_parts outputs of every shard (a list of dicts of tensors or
    arrays with keys sum_events, ln_xi, neff_sel, flags, n_events and, for the gradient,
    grad_events, grad_ln_xi) into lnL_total, ln_xi, neff_sel, flags and grad_total."""
    def a(x):
        return np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x, dtype=np.float64)
    n_det = float(sum(int(p["n_events"]) for p in parts))
    lx = np.stack([a(p["ln_xi"]) for p in parts])               # [R, K]
    ns = np.stack([a(p["neff_sel"]) for p in parts])
    se = np.stack([a(p["sum_events"]) for p in parts])
    fl = np.bitwise_or.reduce(np.stack([np.asarray(a(p["flags"]), np.int64) for p in parts]), axis=0)
    M = np.max(lx, axis=0)
    fin = np.isfinite(M)
    w = np.where(fin[None, :] & np.isfinite(lx), np.exp(lx - np.where(fin, M, 0.0)[None, :]), 0.0)
    sw = w.sum(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ln_xi = np.where(fin & (sw > 0), M + np.log(sw), -np.inf)
        # sum of squared injection weights of shard r, in units of exp(2 M): w_r^2 / N_eff,r
        s2 = np.where(ns > 0, w * w / np.where(ns > 0, ns, 1.0), 0.0).sum(axis=0)
        neff = np.where(s2 > 0, sw * sw / s2, 0.0)
    # bits 0 (domain) and 1 (an event's N_eff) carry over; bit 3 (no injection weight) is
    # decided by the merged sum; a shard's own selection N_eff cut (bit 2) says nothing
    # about the merged one -- shards are built with neff_min_sel = 0 and a caller applies
    # its threshold to the merged neff_sel
    flags = (fl & ~np.int64(4 | 8)) | np.where(np.isfinite(ln_xi), 0, 8)
    dead = ~np.all(np.isfinite(se), axis=0)
    total = np.where((flags != 0) | dead, -np.inf, se.sum(axis=0) - n_det * ln_xi)
    out = {"lnL_total": total, "ln_xi": ln_xi, "neff_sel": neff, "flags": flags.astype(np.int32)}
    if all("grad_events" in p for p in parts):
        ge = np.stack([a(p["grad_events"]) for p in parts]).sum(axis=0)          # [K, 13]
        gx = np.stack([a(p["grad_ln_xi"]) for p in parts])                      # [R, K, 13]
        with np.errstate(divide="ignore", invalid="ignore"):
            q = np.where(sw > 0, w / np.where(sw > 0, sw, 1.0), 0.0)             # xi_r / xi
        grad = ge - n_det * np.einsum("rk,rki->ki", q, gx)
        out["grad_total"] = np.where(((flags != 0) | dead)[:, None], 0.0, grad)
    return out


def merge_parts_distributed(part):
    """merge_parts over all ranks of the process group: one all_gather of every rank's
    K (5 + 2P) numbers (P = 13, or 16 for the multi-peak model, taken from the
    gradients' width), then the same exact combination on every rank."""
    import torch
    dist = _dist()
    if dist is None:
        return merge_parts([part])
    world = dist.get_world_size()
    grad = "grad_events" in part

    def t(x):
        return torch.as_tensor(np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x,
                                          dtype=np.float64))
    K = int(t(part["ln_xi"]).shape[0])
    cols = [t(part["sum_events"])[:, None], t(part["ln_xi"])[:, None], t(part["neff_sel"])[:, None],
            t(part["flags"])[:, None], torch.full((K, 1), float(part["n_events"]), dtype=torch.float64)]
    P = 0
    if grad:
        ge, gx = t(part["grad_events"]).reshape(K, -1), t(part["grad_ln_xi"]).reshape(K, -1)
        P = ge.shape[1]
        cols += [ge, gx]
    mine = torch.cat(cols, dim=1)
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine)
    parts = []
    for m in every:
        m = m.numpy()
        p = {"sum_events": m[:, 0], "ln_xi": m[:, 1], "neff_sel": m[:, 2],
             "flags": m[:, 3].astype(np.int64), "n_events": int(m[0, 4])}
        if grad:
            p["grad_events"] = m[:, 5:5 + P]
            p["grad_ln_xi"] = m[:, 5 + P:5 + 2 * P]
        parts.append(p)
    return merge_parts(parts)

"""Splitting one absorption job over several ranks (one process per GPU).

Pressure-temperature levels are independent (every level is its own sum over the same
line list, Sec. 2.1 and Appendix A's one file per level), and so are the requests of a
batch. So a job shards with no exchange step: each rank keeps the whole line list and
computes a share of the levels (or of the requests), and the only collective is an
optional gather of the results for a caller that wants them in one place. Host logic
only; the computation on each rank is the library's.
"""
from __future__ import annotations

import numpy as np


def level_shards(n_levels: int, world: int, cost=None, mode: str = "interleaved") -> list[list[int]]:
    """The levels of each rank: every level exactly once, each rank's list ascending.

    mode "interleaved": rank r takes r, r + world, ... (neighbouring levels cost about
    the same, so this balances a smooth cost profile); "contiguous": consecutive blocks
    of near-equal size; "balanced": longest-processing-time-first on the given per-level
    costs (ties by level index, so the split is deterministic)."""
    if n_levels < 0 or world < 1:
        raise ValueError("need n_levels >= 0 and world >= 1")
    if mode == "interleaved":
        return [list(range(r, n_levels, world)) for r in range(world)]
    if mode == "contiguous":
        edges = [round(r * n_levels / world) for r in range(world + 1)]
        return [list(range(edges[r], edges[r + 1])) for r in range(world)]
    if mode == "balanced":
        c = np.ones(n_levels) if cost is None else np.asarray(cost, dtype=np.float64)
        if c.shape != (n_levels,):
            raise ValueError("one cost per level")
        load = [0.0] * world
        out = [[] for _ in range(world)]
        for lev in sorted(range(n_levels), key=lambda i: (-c[i], i)):
            r = min(range(world), key=lambda k: (load[k], k))
            out[r].append(lev)
            load[r] += c[lev]
        return [sorted(x) for x in out]
    raise ValueError(f"unknown mode {mode}")


def request_shards(n_req: int, world: int) -> list[list[int]]:
    """The requests of each rank for a batch: interleaved, every request exactly once."""
    return level_shards(n_req, world, mode="interleaved")


def gather_levels(local, levels: list[int], n_levels: int, dist, dst: int | None = 0):
    """Assemble [n_levels, npts] from each rank's [len(levels), npts] block (a torch
    tensor, rows in the order of `levels`). Every rank passes its own block and level
    list; the result (a tensor on the block's device) is returned on rank dst, or on
    every rank when dst is None; other ranks get None. With dist None (one rank) the
    block is returned in level order."""
    import torch
    if dist is None:
        out = torch.empty((n_levels,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
        out[torch.as_tensor(levels, dtype=torch.long, device=local.device)] = local
        return out
    world = dist.get_world_size()
    rank = dist.get_rank()
    dev = local.device
    # level lists of every rank (padded to a common length with -1)
    nmax_t = torch.tensor([len(levels)], dtype=torch.long, device=dev)
    dist.all_reduce(nmax_t, op=dist.ReduceOp.MAX)
    nmax = int(nmax_t.item())
    idx = torch.full((nmax,), -1, dtype=torch.long, device=dev)
    idx[:len(levels)] = torch.as_tensor(levels, dtype=torch.long, device=dev)
    all_idx = [torch.empty_like(idx) for _ in range(world)]
    dist.all_gather(all_idx, idx)
    blk = torch.zeros((nmax,) + tuple(local.shape[1:]), dtype=local.dtype, device=dev)
    blk[:len(levels)] = local
    all_blk = [torch.empty_like(blk) for _ in range(world)]
    dist.all_gather(all_blk, blk)
    if dst is not None and rank != dst:
        return None
    out = torch.empty((n_levels,) + tuple(local.shape[1:]), dtype=local.dtype, device=dev)
    seen = torch.zeros(n_levels, dtype=torch.long, device=dev)
    for ix, b in zip(all_idx, all_blk):
        keep = ix >= 0
        out[ix[keep]] = b[keep]
        seen[ix[keep]] += 1
    if not bool((seen == 1).all()):
        raise RuntimeError("the ranks' level lists do not cover every level exactly once")
    return out

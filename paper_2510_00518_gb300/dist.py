"""Sharding of the mode set across ranks (one process per GPU).

Under the relaxation-time approximation every mode's Γ is independent (paper, Introduction), so
the q points are split into contiguous blocks, one per rank, with no exchange while the rates
are computed.  κ is a sum over modes: each rank evaluates the contribution of its own modes
(the Γ of all other modes set to 0, which fc4_kappa skips) and one all-reduce of 9 doubles
assembles the total."""
from __future__ import annotations

import numpy as np


def shard_q(n_q: int, rank: int, world: int) -> np.ndarray:
    """Contiguous block of q indices of ``rank`` out of ``world`` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(n_q, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return np.arange(start, stop, dtype=np.int32)


def allreduce_kappa(partial, group=None):
    """Sum the per-rank κ contributions (a 3x3 or 9-element tensor) over ``group``."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial


def sharded_rates_kappa(engine, T: float, sigma_thz: float, channel_mask: int = 31, group=None):
    """Γ of this rank's q block and the total κ (all ranks call it; one all-reduce)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    qs = shard_q(engine.nq, rank, world)
    g, wp, cnt = engine.rates(T, sigma_thz, channel_mask, q_subset=qs)
    full = torch.zeros((5, engine.nq * engine.nb), dtype=torch.float64, device=g.device)
    if qs.size:
        full[:, int(qs[0]) * engine.nb:(int(qs[-1]) + 1) * engine.nb] = g
    kap = engine.kappa(T, full, channel_mask).reshape(-1).clone()
    return qs, g, allreduce_kappa(kap, group).view(3, 3)

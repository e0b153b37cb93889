"""Sharding of the mode set across ranks (one process per GPU).

Under the relaxation-time approximation every mode's Γ is independent (paper, Introduction), so
the q points are split into contiguous blocks, one per rank, with no exchange while the rates
are computed.  κ is a sum over modes: each rank evaluates the contribution of its own modes
(the Γ of all other modes set to 0, which fc4_kappa skips) and one all-reduce of 9 doubles
assembles the total.  With irreducible q-points the representatives are split the same way
and each rank spreads its own over their stars before its κ contribution."""
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


def sharded_rates_kappa_irreducible(engine, T: float, sigma_thz: float, rot=None,
                                    channel_mask: int = 31, time_reversal: bool = True,
                                    deg_tol: float = 1e-5, group=None):
    """The irreducible q-points split into contiguous blocks over the ranks: each rank computes
    the rates of its block (fixed σ), spreads them over the stars it owns (the other stars stay
    0 and fc4_kappa skips them) and adds its κ contribution in one all-reduce of 9 doubles.
    Returns (this rank's irreducible q, their Γ [5, n*nb], the total κ)."""
    import torch
    import torch.distributed as dist
    from .symmetry import expand_irreducible, irreducible_q
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    r = np.zeros((0, 3, 3), np.int32) if rot is None else rot
    rep, irr = irreducible_q(engine.mesh, r, time_reversal)
    pos = shard_q(irr.size, rank, world)
    mine = irr[pos]
    g, _, _ = engine.rates(T, sigma_thz, channel_mask, q_subset=mine)
    nb = engine.nb
    sub = np.zeros((5, irr.size * nb))
    if pos.size:
        sub[:, int(pos[0]) * nb:(int(pos[-1]) + 1) * nb] = g.cpu().numpy()
    full = expand_irreducible(engine.mesh, nb, rep, engine.get_modes()[0], sub, deg_tol)
    kap = engine.kappa(T, torch.from_numpy(full).to(g.device), channel_mask).reshape(-1).clone()
    return mine, g, allreduce_kappa(kap, group).view(3, 3)


def allreduce_grad(d3, d4, group=None):
    """Sum the per-rank gradients dL/dΦ3 [nc3, 27] and dL/dΦ4 [nc4, 81] over ``group`` (one
    all-reduce of nc3·27 + nc4·81 doubles; either may be None)."""
    import torch
    import torch.distributed as dist
    parts = [x for x in (d3, d4) if x is not None]
    if not parts or not (dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1):
        return d3, d4
    flat = torch.cat([x.reshape(-1) for x in parts])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    out, o = [], 0
    for x in (d3, d4):
        if x is None:
            out.append(None)
            continue
        out.append(flat[o:o + x.numel()].view_as(x))
        o += x.numel()
    return out[0], out[1]


def sharded_kappa_gradient(engine, T: float, sigma_thz: float, dL_dkappa, channel_mask: int = 31, group=None):
    """dL/dΦ3, dL/dΦ4 of L = Σ dL_dkappa κ with the modes sharded over the ranks: each rank runs
    the rates of its q block, the κ all-reduce, its share of the adjoint (dL/dΓ of its own modes
    through fc4_kappa_backward, then fc4_rates_backward), and one gradient all-reduce.  Returns
    (κ, dL/dΦ3, dL/dΦ4); every rank gets the totals."""
    import torch
    qs, g, kap = sharded_rates_kappa(engine, T, sigma_thz, channel_mask, group)
    nb = engine.nb
    full = torch.zeros((5, engine.nq * nb), dtype=torch.float64, device=g.device)
    if qs.size:
        full[:, int(qs[0]) * nb:(int(qs[-1]) + 1) * nb] = g
    dk = torch.as_tensor(dL_dkappa, dtype=torch.float64, device=g.device).reshape(3, 3)
    dg_full = engine.kappa_backward(T, full, dk, channel_mask)
    dg = dg_full[:, int(qs[0]) * nb:(int(qs[-1]) + 1) * nb].contiguous() if qs.size else dg_full[:, :0]
    if qs.size:
        engine.rates(T, sigma_thz, channel_mask, q_subset=qs)       # the subset the backward reads
        d3, d4 = engine.backward(dg)
    else:
        d3 = torch.zeros((engine.nc3, 27), dtype=torch.float64, device=g.device) if engine.nc3 else None
        d4 = torch.zeros((engine.nc4, 81), dtype=torch.float64, device=g.device) if engine.nc4 else None
    d3, d4 = allreduce_grad(d3, d4, group)
    return kap, d3, d4

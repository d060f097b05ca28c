"""Spin sharding across ranks (one process per GPU).

Spins are independent (the paper's spin-independence remark in Section
"Physical and Mathematical Background"), so a phantom splits into contiguous
spin ranges, one per rank, with the sequence replicated; the only exchange is
one sum of the per-rank signals at the end. Grouped phantoms split on group
boundaries, and then every group's signal lives on exactly one rank, so the
sum is a gather of disjoint rows.
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np


def shard_range(n: int, rank: int, world: int):
    """Contiguous [lo, hi) of n items for `rank` of `world` (sizes differ by <= 1)."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside world of {world}")
    return n * rank // world, n * (rank + 1) // world


def shard_phantom(phantom, rank: int, world: int):
    """The rank's part of a phantom. Ungrouped: a contiguous spin range.
    Grouped: a contiguous range of whole groups, returned with the offset of
    its first group (its signal rows are [g_lo, g_hi) of the full output)."""
    from .workloads import Phantom
    go = getattr(phantom, "group_offsets", None)
    fields = ("x", "y", "z", "pd", "t1", "t2", "dw")
    vel = getattr(phantom, "velocity", None)
    if go is None:
        lo, hi = shard_range(phantom.n, rank, world)
        part = Phantom(*(getattr(phantom, f)[lo:hi] for f in fields),
                       velocity=None if vel is None else vel[:, lo:hi])
        return part, (0, 1)
    g_lo, g_hi = shard_range(len(go) - 1, rank, world)
    s_lo, s_hi = int(go[g_lo]), int(go[g_hi])
    part = Phantom(*(getattr(phantom, f)[s_lo:s_hi] for f in fields),
                   group_offsets=np.asarray(go[g_lo:g_hi + 1]) - s_lo,
                   velocity=None if vel is None else vel[:, s_lo:s_hi])
    return part, (g_lo, g_hi)


def simulate_sharded(phantom, seq, simulate_shard: Callable, rank: int, world: int,
                     group=None, device: Optional[str] = None):
    """Simulate this rank's shard with ``simulate_shard(part, seq)`` (returns
    complex128 [groups_in_part, n_adc]) and combine across ranks with one
    torch.distributed all-reduce (sum). Every rank returns the full signal
    [n_groups, n_adc] as a numpy array."""
    import torch
    import torch.distributed as dist
    part, (g_lo, g_hi) = shard_phantom(phantom, rank, world)
    go = getattr(phantom, "group_offsets", None)
    n_groups = 1 if go is None else len(go) - 1
    n_adc = int(np.count_nonzero(seq.adc))
    full = np.zeros((n_groups, n_adc), dtype=np.complex128)
    if part.n > 0 and (go is None or g_hi > g_lo):
        full[g_lo:g_lo + (g_hi - g_lo if go is not None else 1)] = simulate_shard(part, seq)
    if world > 1:
        t = torch.from_numpy(full.view(np.float64).copy())
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        full = t.cpu().numpy().view(np.complex128).reshape(n_groups, n_adc)
    return full

"""Photon-range sharding across ranks (one process per GPU).

Photons are independent and each photon's random numbers depend only on
(seed, photon id), so a run of N photons splits into contiguous id ranges,
one per rank, with no exchange while transporting.  The only exchange is an
integer sum of the Q32.32 tallies, which is exact and order-independent, so
the merged tallies equal a single-process run bit for bit.
"""
from __future__ import annotations

import numpy as np


def photon_range(rank: int, world: int, n_total: int) -> tuple[int, int]:
    """(first photon id, count) of this rank: contiguous blocks, the
    remainder spread over the lowest ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, rem = divmod(int(n_total), int(world))
    count = base + (1 if rank < rem else 0)
    first = rank * base + min(rank, rem)
    return first, count


def allreduce_u64(arrays, dist, group=None):
    """Sum uint64 tally arrays over ranks in place (int64 two's-complement
    addition is the modular unsigned sum)."""
    import torch
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        t = torch.from_numpy(a.view(np.int64).copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.append(t.numpy().view(np.uint64).reshape(a.shape))
    return out


def max_over_ranks(value: float, dist, device="cpu", group=None) -> float:
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

"""Host logic for runs on several GPUs of one node.

Stars are independent problems: each rank advances its own subset with no
data-path exchange.  The collectives are the final gather of the per-star
FP64 totals (each star is owned by one rank) and the timing/accounting
reductions of the benchmark (max of the ranks' times, sum of their pairs).
"""
from __future__ import annotations

import numpy as np


def assign_stars(counts, world_size: int):
    """Longest-processing-time assignment of stars to ranks.

    counts: particles per star.  Stars are taken in order of decreasing count
    (ties by star index) and each goes to the rank with the least particles so
    far (ties by rank index).  Returns one sorted list of star ids per rank.
    """
    counts = np.asarray(counts, dtype=np.int64)
    order = sorted(range(len(counts)), key=lambda s: (-int(counts[s]), s))
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for s in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(s)
        load[r] += int(counts[s])
    return [sorted(x) for x in out]


def reduce_timing(t_ms: float, pairs: float, device=None):
    """(max over ranks of t_ms, sum over ranks of pairs) via torch.distributed."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_ms), float(pairs)
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    p = torch.tensor([pairs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def gather_star_totals(star_ids, totals, nstars: int, device=None) -> np.ndarray:
    """Per-star FP64 totals of all ranks, [nstars, 16] on every rank.

    star_ids: the global ids of this rank's stars; totals: their rows
    (sph_totals_per_star of this rank's context, in the same order).  Each
    star belongs to exactly one rank, so the exchange is a sum of arrays that
    are zero outside each rank's rows: exact, whatever the reduction order.
    """
    import torch
    import torch.distributed as dist

    out = np.zeros((nstars, 16), np.float64)
    out[np.asarray(star_ids, dtype=np.int64)] = np.asarray(totals, dtype=np.float64)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return out
    t = torch.from_numpy(out)
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()

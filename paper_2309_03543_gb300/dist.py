"""Host-side logic of multi-GPU runs: one rank per GPU, independent systems.

The corrector solves of independent systems (ensemble members, separate
corrector problems) share nothing, so ranks split the systems and never talk
during the solves.  The only collective is at the end: the slowest rank's
time and the total work, for the throughput of the whole job.
"""
from __future__ import annotations

import torch


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (disjoint, covering, sizes
    differing by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(items)[rank::world]


def aggregate(seconds: float, units: float, group=None, device=None):
    """(max seconds over ranks, sum of units over ranks).  Without an
    initialised process group the local values are returned."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, units
    t = torch.tensor([seconds, units], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    gathered = [torch.zeros_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(gathered, t, group=group)
    return max(float(g[0]) for g in gathered), sum(float(g[1]) for g in gathered)

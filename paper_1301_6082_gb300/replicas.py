"""Multi-GPU sharding by group range.  The 32-sample groups of one ensemble are independent
systems (the paper runs one system per workgroup, Sec. 3) whose random numbers are addressed
by their global group index, so an ensemble splits over ranks with no exchange at all: rank r
runs groups [group0, group0 + n) of the ensemble (pcpd_params.group0) and the ranks together
reproduce the one-GPU run of the whole ensemble bit for bit.  The only combination is an
exact integer sum of occupation counts plus, for timing, a maximum over ranks.  No collective
touches the data path."""
from __future__ import annotations

PHASE_GROUP = 4   # 32-sample groups per 128-sample phase group (the unit a shard must respect)


def shard_groups(total_groups: int, world: int, rank: int) -> tuple[int, int]:
    """(group0, n_groups) of rank `rank`'s share of an ensemble of `total_groups` 32-sample
    groups split over `world` ranks: contiguous runs of whole phase groups, as even as
    possible (a rank may get none when there are fewer phase groups than ranks)."""
    if total_groups <= 0 or world <= 0 or not 0 <= rank < world:
        raise ValueError("need total_groups > 0 and 0 <= rank < world")
    n_pg = -(-total_groups // PHASE_GROUP)
    a, b = rank * n_pg // world, (rank + 1) * n_pg // world
    g0 = PHASE_GROUP * a
    return g0, max(0, min(PHASE_GROUP * b, total_groups) - g0)


def weak_shard(groups_per_rank: int, rank: int) -> tuple[int, int]:
    """(group0, n_groups) when every rank runs the same number of groups of one ensemble of
    world * groups_per_rank groups (weak scaling): rank r holds groups
    [r * groups_per_rank, (r + 1) * groups_per_rank)."""
    if groups_per_rank % PHASE_GROUP:
        raise ValueError("groups_per_rank must be a multiple of 4 (whole phase groups)")
    return rank * groups_per_rank, groups_per_rank


def combine(dist, sums, maxes, device="cpu"):
    """All-reduce over ranks: integer sums (exact, int64) and maxima (float64).  With one
    process (dist is None) the inputs are returned unchanged."""
    import torch
    if dist is None:
        return [int(x) for x in sums], [float(x) for x in maxes]
    s = torch.tensor([int(x) for x in sums], dtype=torch.int64, device=device)
    m = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return [int(x) for x in s.tolist()], [float(x) for x in m.tolist()]

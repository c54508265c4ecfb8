"""Multi-GPU replicas.  Independent PCPD systems (the paper runs one system per workgroup,
Sec. 3) shard with no exchange at all: each rank simulates its own samples with its own
seed, and the only combination is an exact integer sum of occupation counts plus, for
timing, a maximum over ranks.  No collective touches the data path."""
from __future__ import annotations

SEED_STRIDE = 1_000_003


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: disjoint Philox keys for every rank."""
    return (base_seed + SEED_STRIDE * rank) % (1 << 64)


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

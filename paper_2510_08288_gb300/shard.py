"""Host-side multi-rank helpers: scenario sharding and replica bookkeeping.

The robust RG update is data parallel over scenarios: every candidate's
admissibility is an AND over scenarios and its min slack a MIN over them
(Eq. 5 reduced per row).  Splitting the N_sim scenarios into contiguous shards
across ranks therefore needs one exchange per search round: an all-reduce MIN
of the m per-candidate flags (AND on {0, 1}) and of the m min slacks.  The
shards use the global scenario indices, so the result does not depend on the
number of ranks.

Replicas (independent RG instances, one per rank) need no data exchange at
all; only the benchmark's timing uses a MAX all-reduce.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_scenarios: int, world: int, rank: int):
    """Contiguous [k0, k1) of the global scenario indices owned by `rank`."""
    if not (0 <= rank < world) or n_scenarios < world:
        raise ValueError("need 0 <= rank < world <= n_scenarios")
    base, extra = divmod(n_scenarios, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def replica_seed(seed: int, rank: int) -> int:
    """Seed of the independent RG instance a rank runs as a replica."""
    return int(seed) + 1000 * int(rank)


def allreduce_candidates(admissible, min_slack, group=None, device=None):
    """Combines per-shard candidate results: AND of the flags, MIN of the
    slacks, over all ranks of `group` (torch.distributed must be initialised).
    Returns numpy arrays (uint8 flags, float64 slacks)."""
    import torch
    import torch.distributed as dist
    a = torch.as_tensor(np.asarray(admissible, dtype=np.int32), device=device)
    s = torch.as_tensor(np.asarray(min_slack, dtype=np.float64), device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MIN, group=group)
    return a.cpu().numpy().astype(np.uint8), s.cpu().numpy()


def allreduce_max(value: float, group=None, device=None) -> float:
    """MAX over ranks of a scalar (the timed region of the slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

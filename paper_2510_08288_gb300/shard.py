"""Host-side multi-rank helpers: scenario sharding and replica bookkeeping.

The robust RG update is data parallel over scenarios: every candidate's
admissibility is an AND over scenarios and its min slack a MIN over them
(Eq. 5 reduced per row).  Splitting the N_sim scenarios into contiguous shards
across ranks therefore needs one exchange per search round: an all-reduce MIN
of the m per-candidate flags (AND on {0, 1}) and of the m min slacks.  The
shards use the global scenario indices (a handle's rrg_config.scenario_base),
so the result does not depend on the number of ranks.  sharded_search runs
the speculative bisection by rounds around that exchange, with the library's
rrg_bisect_plan / rrg_bisect_decide deciding each round.

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


def sharded_search(evaluate, n_bisect: int, m_max: int, combine=None):
    """Alg. 1 (joint predicate over every shard's scenarios) by rounds of the
    speculative bisection: rrg_bisect_plan lists the round's kappas,
    evaluate(kappas) -> (admissible[m], min_slack[m]) evaluates them on this
    caller's shard(s), combine (default: allreduce_candidates, AND / MIN over
    the ranks of the default group) makes them global, and rrg_bisect_decide
    walks Alg. 1's path.  Returns (kappa, flags, rounds); flags bit 0: no
    kappa was admissible (kappa = 0, hold)."""
    from paper_2510_08288_gb300 import rrg as R
    combine = combine or allreduce_candidates
    s = R.rrg_bisect_init(n_bisect)
    rounds = 0
    while not s.done:
        kap = R.rrg_bisect_plan(s, m_max)
        a, ms = evaluate(kap)
        a, _ = combine(a, ms)
        R.rrg_bisect_decide(s, a)
        rounds += 1
    return s.kappa_opt, (0 if s.any else 1), rounds

"""Host-side logic of the multi-GPU path: independent chains spread over
ranks (one process per GPU), and the whole-job reduction of a timed run.

A single chain does not shard (its pairs are visited in order), so ranks
only ever run independent problems: each rank sweeps its own chains and
the ranks meet once, after the timed region, to reduce the elapsed time
(maximum) and the work done (sum).  Nothing here touches a GPU; the
reduction runs over whatever backend the process group has (NCCL between
GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def chain_cost(n_sites: int, chi_max: int, d: int = 2) -> float:
    """Relative cost of sweeping one chain: n_sites pair updates whose
    contractions and splits grow like (d chi_max)^3."""
    return float(n_sites) * float(d * chi_max) ** 3


def shard_chains(costs: list, world: int, rank: int) -> list:
    """Indices of the chains that `rank` of `world` runs.

    Largest cost first, each chain to the rank with the least load so far
    (ties: lower chain index first, then lower rank), so every rank computes
    the same assignment without communicating; every chain lands on exactly
    one rank and the loads differ by at most the largest single cost."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    mine = []
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[k]
        if r == rank:
            mine.append(k)
    return sorted(mine)


def reduce_run(elapsed: float, work: float, launches: int, device=None) -> tuple:
    """Whole-job numbers of a timed region: (max elapsed over ranks, total
    work, total launches).  Without an initialised process group the local
    values are returned."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed), float(work), int(launches)
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    s = torch.tensor([work, float(launches)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t[0]), float(s[0]), int(round(float(s[1])))

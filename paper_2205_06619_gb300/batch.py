"""Independent problems across ranks (one process per GPU).

FastSTMF's row loop is sequential within a factorization, so one problem
never spans GPUs; many independent problems (a batch, or restarts of one
input) shard across ranks with no data-path collective.  ``partition`` is a
size-balanced greedy assignment (largest estimated cost first, each to the
least-loaded rank); ``run_sharded`` solves a rank's share with any solver and
gathers the results on rank 0 with one ``gather_object`` at the end.
"""
from __future__ import annotations


def problem_cost(m: int, n: int, rank: int, sweeps: int) -> float:
    """Work estimate of one problem: sweeps x rows x given entries x rank."""
    rows = min(m, n)
    return float(sweeps) * rows * m * n * max(rank, 1)


def partition(costs, world: int):
    """Indices of the problems each rank solves (deterministic)."""
    order = sorted(range(len(costs)), key=lambda q: (-costs[q], q))
    load = [0.0] * world
    shares = [[] for _ in range(world)]
    for q in order:
        w = min(range(world), key=lambda k: (load[k], k))
        shares[w].append(q)
        load[w] += costs[q]
    return [sorted(s) for s in shares]


def run_sharded(problems, solver, costs=None, group=None):
    """Solves ``problems`` across the ranks of the default (or given) process
    group.  ``solver(list_of_problems) -> list_of_results`` runs on each rank's
    share.  Returns the list of all results (in problem order) on rank 0 and
    None elsewhere.  Without an initialised process group it solves
    everything locally."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return solver(list(problems))
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if costs is None:
        costs = [problem_cost(p["m"], p["n"], p["rank"], p.get("sweeps", 1)) for p in problems]
    share = partition(costs, world)[rank]
    local = solver([problems[q] for q in share])
    mine = list(zip(share, local))
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = [None] * len(problems)
    for part in gathered:
        for q, res in part:
            out[q] = res
    return out

"""Sharding a batch of independent IDs across ranks (one process per GPU).

The batched workload is a set of independent problems (the off-diagonal blocks
of a hierarchical kernel matrix, the paper's future-work item on batching,
Sec. 6): they shard with no collective on the data path.  Each rank takes a
subset whose estimated cost is balanced against the others' (greedy longest
processing time: problems in decreasing cost, each to the least-loaded rank,
ties to the lower rank), runs it with id_batched, and the per-problem results
are gathered on rank 0 afterwards (outside the timed work).

The cost of a problem is the dominant term of the method's work, the sketch
2 m n (k + b) (Sec. 2.4), with the rank k unknown in advance: the caller passes
an estimate (the rank cap min(m, n) when nothing better is known).
"""
from __future__ import annotations


def problem_cost(m: int, n: int, k_est: int, b: int) -> float:
    """Sketch flops 2 m n (k + b) of a rank-k adaptive ID with block b."""
    return 2.0 * m * n * (k_est + b)


def assign(costs: list, world: int) -> list:
    """Greedy LPT assignment: a list of `world` index lists (each ascending) whose
    cost sums are balanced.  Deterministic: equal costs keep their index order,
    equal loads go to the lower rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def imbalance(costs: list, parts: list) -> float:
    """Largest rank load over the mean load (1.0 = perfect balance)."""
    loads = [sum(costs[i] for i in p) for p in parts]
    mean = sum(loads) / max(len(loads), 1)
    return max(loads) / mean if mean > 0 else 1.0


def gather_results(local: dict, world: int, rank: int):
    """{problem index: result} of every rank on rank 0 (None elsewhere), through
    torch.distributed's object gather on the default process group."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    out = [None] * world if rank == 0 else None
    dist.gather_object(local, out, dst=0)
    if rank != 0:
        return None
    merged = {}
    for part in out:
        for i, v in part.items():
            if i in merged:
                raise RuntimeError("problem %d was run by two ranks" % i)
            merged[i] = v
    return merged

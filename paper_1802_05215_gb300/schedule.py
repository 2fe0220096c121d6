"""Slice-to-rank assignment for multi-GPU runs (Sec. 2.6: slices are independent, so the first
level of parallelism maps groups of slices to processes).

Each rank owns a replica of the matrix, recomputes the bounds and the KPM density itself, and
solves its own slices; no data-path collective is needed.  Slices go to ranks by a greedy
longest-processing-time schedule on an estimated cost, eigenvalue count x filter degree (the
filter cost per Lanczos step grows with the degree, the number of steps with the count).
"""
from __future__ import annotations


def slice_costs(est_counts, degrees):
    return [max(float(c), 1.0) * max(int(d), 1) for c, d in zip(est_counts, degrees)]


def assign_slices(costs, world: int) -> list[list[int]]:
    """LPT: slices by decreasing cost, each to the currently least-loaded rank (ties to the
    lower rank).  Returns, per rank, its slice indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    owned: list[list[int]] = [[] for _ in range(world)]
    for s in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(s)
        load[r] += costs[s]
    return [sorted(o) for o in owned]

"""Sharding a batch of independent systems over ranks (one GPU per rank).

The systems of a batch share nothing, so a multi-GPU run splits them between
the ranks with no collective on the data path: every rank evaluates its own
systems, and only timing (the maximum over ranks) is reduced.  The split is a
greedy longest-processing-time assignment of estimated per-system costs; it is
deterministic, so every rank computes the same partition without
communicating.
"""
from __future__ import annotations

import math

from .se import choose_params


def system_costs(kernel: str, sizes, boxes=None, n_rhs: int = 1, tol: float = 2e-6,
                 prec: str = "fp32") -> list[float]:
    """Relative cost of each system: grid work (spreading and gather, N P^3 per
    right-hand side), FFTs (Mf^3 log Mf per right-hand side) and real-space
    pairs (N^2 4/3 pi rc^3 / L^3), with the parameters the library would choose."""
    out = []
    for s, n in enumerate(sizes):
        L = 1.0 if boxes is None else float(boxes[s][3])
        p = choose_params(kernel, int(n), L, tol=tol, prec=prec)
        mf = 2 * (p["M"] + p["P"])
        grid = n * p["P"] ** 3 * n_rhs
        fft = 6.0 * mf ** 3 * math.log2(mf) * n_rhs
        pairs = n * n * 4.18879 * p["rc"] ** 3 / L ** 3 * (1.0 + n_rhs / 4.0)
        out.append(0.1 * grid + 0.6 * fft + pairs)
    return out


def partition(costs, world: int) -> list[list[int]]:
    """Systems of each rank: largest cost first onto the least loaded rank (ties
    to the lowest rank); each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for s in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(s)
        load[r] += costs[s]
    return [sorted(p) for p in parts]

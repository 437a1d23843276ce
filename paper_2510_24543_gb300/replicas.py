"""Multi-GPU bookkeeping: one independent instance per GPU, no data-path collective.

The solver's unit of work is one ground-state problem on one grid; problems do
not exchange data, so N GPUs run N replicas (independent instances, e.g. the
points of a parameter scan) and the only collectives are the end-of-run
reductions of a few host scalars (max of the timed durations, sum of the
iterations).  These helpers are used by bench.py and tested with the gloo
backend on CPU.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple


def rank_workload(w, rank: int):
    """Rank r solves the same physics with seed + r (an independent start)."""
    return dataclasses.replace(w, seed=w.seed + rank)


def shard_instances(n_instances: int, rank: int, world: int) -> List[int]:
    """Round-robin assignment of instance indices to ranks (every instance
    exactly once; sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return list(range(rank, n_instances, world))


def combine(dist, elapsed_ms: float, iterations: float, device=None) -> Tuple[float, float]:
    """(max over ranks of elapsed_ms, sum over ranks of iterations).  `dist` is
    torch.distributed (initialised) or None for a single process."""
    if dist is None:
        return float(elapsed_ms), float(iterations)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(iterations)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def aggregate_rate(dist, elapsed_ms: float, iterations: float, device=None) -> float:
    """Whole-job iterations per second: all ranks' iterations over the slowest
    rank's time (weak scaling: fixed work per GPU)."""
    ms, it = combine(dist, elapsed_ms, iterations, device)
    return it / (ms * 1e-3)


def balance(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Greedy longest-first assignment of instances with the given costs to
    ranks (for scans mixing grid sizes); returns per-rank instance lists."""
    order = sorted(range(len(sizes)), key=lambda i: -sizes[i])
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += sizes[i]
    for lst in out:
        lst.sort()
    return out

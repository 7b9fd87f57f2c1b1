"""Sharding of independent films over ranks (one process per GPU).

Films of a field sweep are independent problems, so they shard with no data-path
collective: each rank advances its own subset as one batch, and only the small
per-film results (steps taken, <m>, max|dm/dt|) are gathered at the end.  A
single film does not shard (its transforms would need a global transpose) and
runs as independent replicas instead.

partition(grids, world)   films -> ranks, balancing the estimated cost: the FFT
                          work per step, N_pad log2 N_pad with N_pad the padded
                          cell count (longest-processing-time-first greedy).
gather(values, idx, n)    per-rank rows for films idx -> the full (n, ...) array
                          on every rank, ordered by film index.
max_over_ranks(x)         the slowest rank's time (the job's wall time).
"""
import math
from typing import List, Sequence

import numpy as np


def _pow2_at_least(v: int) -> int:
    p = 1
    while p < v:
        p *= 2
    return p


def film_cost(grid: Sequence[int]) -> float:
    nx, ny, nz = (int(g) for g in grid)
    px = 1 if nx == 1 else _pow2_at_least(2 * nx - 1)
    py = 1 if ny == 1 else _pow2_at_least(2 * ny - 1)
    npad = px * py * nz
    return npad * max(1.0, math.log2(npad))


def partition(grids: Sequence[Sequence[int]], world: int) -> List[List[int]]:
    """Film indices per rank; every film exactly once, costs balanced greedily."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(grids)), key=lambda i: -film_cost(grids[i]))
    loads = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += film_cost(grids[i])
    return [sorted(p) for p in parts]


def gather(values: np.ndarray, idx: Sequence[int], n: int, group=None) -> np.ndarray:
    """All ranks' rows (values[j] belongs to film idx[j]) -> the (n, ...) array of all films."""
    import torch
    import torch.distributed as dist
    values = np.asarray(values, dtype=np.float64)
    row = values.shape[1:] if values.ndim > 1 else ()
    if not dist.is_available() or not dist.is_initialized():
        out = np.zeros((n,) + row)
        out[list(idx)] = values
        return out
    payload = [None] * dist.get_world_size(group)
    dist.all_gather_object(payload, (list(idx), values.tolist()), group=group)
    out = np.zeros((n,) + row)
    for ids, vals in payload:
        if ids:
            out[ids] = np.asarray(vals, dtype=np.float64).reshape((len(ids),) + row)
    return out


def max_over_ranks(x: float, group=None, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

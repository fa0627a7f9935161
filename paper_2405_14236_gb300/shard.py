"""Host-side split of one batch of independent instances across ranks (one GPU per rank).

The batched interior-point solves of different instances share nothing, so a batch shards with
no collective on the data path: each rank solves a subset and the results are gathered on the
host afterwards.  The split balances a per-instance cost (the supernode count of its pattern,
or n) by longest-processing-time-first assignment.
"""
from __future__ import annotations

import numpy as np


def partition_by_cost(costs, world):
    """Indices of the instances each of `world` ranks takes: instances in decreasing cost, each to
    the rank with the least total so far (ties to the lower rank).  Every rank's total is within
    the largest single cost of every other rank's.  Each rank's indices are returned ascending."""
    costs = np.asarray(costs, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(local, indices, total, world):
    """Gathers per-instance result arrays (dict name -> array over this rank's instances, in the
    order of `indices`) into arrays over all `total` instances on every rank
    (torch.distributed.all_gather_object; world == 1 needs no process group)."""
    if world == 1:
        gathered = [(list(indices), {k: np.asarray(v) for k, v in local.items()})]
    else:
        import torch.distributed as dist
        gathered = [None] * world
        dist.all_gather_object(gathered, (list(indices), {k: np.asarray(v) for k, v in local.items()}))
    out = {}
    seen = np.zeros(total, bool)
    for idx, res in gathered:
        for k, v in res.items():
            if k not in out:
                out[k] = np.zeros(total, dtype=v.dtype)
            out[k][idx] = v
        seen[idx] = True
    if not seen.all():
        raise RuntimeError("gather_results: some instances were solved by no rank")
    return out

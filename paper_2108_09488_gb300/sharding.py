"""Host-side multi-rank logic: one process per GPU, no collective on the data path.

* Batched plumes are independent problems: ``shard_plumes`` assigns whole plumes to ranks
  (longest-processing-time first on an estimated cost, deterministic), each rank steps its own
  batch, and only the timing is combined.
* A single plume has no exchange-free decomposition here, so it runs as one replica per rank.

``aggregate`` combines per-rank work and time into the whole-job throughput: all ranks' units
divided by the slowest rank's time (max over ranks), using the caller's process group (NCCL on
GPUs, gloo on CPUs).
"""
from __future__ import annotations

import math


def plume_cost(plume):
    """Estimated pair work of one rate evaluation: particles x expected neighbours."""
    ratio = plume.support / plume.dx
    if plume.dim == 2:
        neigh = math.pi * ratio * ratio
    else:
        neigh = 4.0 / 3.0 * math.pi * ratio ** 3
    return plume.n * neigh


def shard_plumes(costs, world):
    """Assign plumes to ranks: largest cost first to the currently lightest rank (ties: lower
    plume index first, lower rank first).  Returns one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in out]


def aggregate(units, ms, group=None, device=None):
    """Whole-job throughput over ranks: (sum of units) / (max of times).  Returns
    (units per second, max ms, total units).  Without a process group: this rank's numbers."""
    import torch
    import torch.distributed as dist

    if group is None and not (dist.is_available() and dist.is_initialized()):
        return units / (ms * 1e-3), ms, units
    dev = device if device is not None else torch.device("cpu")
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item()), float(u.item())

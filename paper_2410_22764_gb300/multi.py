"""Host-side logic for runs over several GPUs (one process per GPU, torch.distributed).

The single-DFA path does not shard: every round needs every block id of the previous round, so
splitting one DFA's states over GPUs would exchange all of block[] every round.  Several GPUs
therefore run independent replicas (the benchmark's weak scaling).  Batches and served streams
are collections of independent DFAs, so they shard with no data-path collective: the DFAs are
assigned to ranks by a size-balanced greedy rule and only results are gathered.
"""
from __future__ import annotations

import numpy as np


def shard_batch(ns, ks, world: int) -> list[np.ndarray]:
    """Assign DFAs to ranks: largest work first (n * (k + 1)), each to the least loaded rank.
    Returns, per rank, the ascending indices of its DFAs."""
    ns = np.asarray(ns, dtype=np.int64)
    ks = np.asarray(ks, dtype=np.int64)
    work = ns * (ks + 1)
    order = np.argsort(-work, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(ns.size, dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += work[i]
    return [np.nonzero(owner == r)[0] for r in range(world)]


def aggregate(local_ms: float, local_units: float, dist=None, device=None):
    """Job-wide timing of a multi-rank run: the slowest rank's time and the units of all ranks.
    With no process group (one rank) the local values are returned."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_ms, local_units
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())

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


def member_subbatch(delta, accept, state_off, ks, idx):
    """The members `idx` (ascending) of a concatenated batch, as a concatenated batch of their
    own: (delta int32, accept uint32 bitmap, state_off int64, ks int32), the layout of the batch
    C ABI."""
    state_off = np.asarray(state_off, dtype=np.int64)
    ks = np.asarray(ks, dtype=np.int32)
    idx = np.asarray(idx, dtype=np.int64)
    ns = np.diff(state_off)
    doff = np.zeros(ks.size + 1, dtype=np.int64)
    doff[1:] = np.cumsum(ns * ks.astype(np.int64))
    sub_ns, sub_ks = ns[idx], ks[idx]
    sub_off = np.zeros(idx.size + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum(sub_ns)
    sub_delta = np.concatenate([delta[doff[i]: doff[i + 1]] for i in idx] +
                               [np.zeros(0, np.int32)]).astype(np.int32, copy=False)
    bits = np.unpackbits(np.ascontiguousarray(accept, dtype=np.uint32).view(np.uint8),
                         bitorder="little")
    sub_bits = np.concatenate([bits[state_off[i]: state_off[i + 1]] for i in idx] +
                              [np.zeros(0, np.uint8)])
    words = (int(sub_off[-1]) + 31) // 32
    buf = np.zeros(words * 4, dtype=np.uint8)
    packed = np.packbits(sub_bits, bitorder="little")
    buf[: packed.size] = packed
    return sub_delta, buf.view("<u4").astype(np.uint32), sub_off, sub_ks


def gpu_batch_runner(opt=None, device=None):
    """Runs one (sub-)batch through the batch C ABI (one persistent launch) on this rank's GPU;
    returns host (out_block int32 [states], per int32 [3, count] = nblocks, passes, status)."""
    def run(delta, accept, state_off, ks):
        import torch
        from . import dfamin
        dev = torch.device(device or "cuda")
        plan = dfamin.BatchPlan(state_off, ks, opt)
        try:
            dd = torch.from_numpy(np.ascontiguousarray(delta, np.int32)).to(dev)
            aa = torch.from_numpy(np.ascontiguousarray(accept, np.uint32).view(np.int32)).to(dev)
            out, per = plan.run(dd, aa)
            return out.cpu().numpy(), per.cpu().numpy()
        finally:
            plan.close()
    return run


def run_sharded_batch(delta, accept, state_off, ks, dist=None, runner=None, opt=None,
                      device=None, gather_labels: bool = True):
    """Minimize a batch of DFAs over all ranks of `dist` (torch.distributed, initialised; None =
    this process alone).  Every rank holds the batch description, takes its share by
    shard_batch, runs it with `runner` (default: the GPU batch launch on this rank's device) and
    the results are gathered on every rank's host: (out_block [states] or None when
    gather_labels is False, per [3, count] = nblocks, passes, status), in the batch's order.
    The only collective is that gather: no data-path exchange, the DFAs are independent."""
    state_off = np.asarray(state_off, dtype=np.int64)
    ks = np.asarray(ks, dtype=np.int32)
    count = ks.size
    on = dist is not None and dist.is_initialized()
    world = dist.get_world_size() if on else 1
    rank = dist.get_rank() if on else 0
    mine = shard_batch(np.diff(state_off), ks, world)[rank]
    run = runner or gpu_batch_runner(opt, device)
    if mine.size:
        out, per = run(*member_subbatch(delta, accept, state_off, ks, mine))
    else:
        out, per = np.zeros(0, np.int32), np.zeros((3, 0), np.int32)
    part = (mine, out if gather_labels else None, per)
    parts = [None] * world
    if on:
        dist.all_gather_object(parts, part)
    else:
        parts[0] = part
    per_all = np.zeros((3, count), dtype=np.int32)
    labels = np.empty(int(state_off[-1]), dtype=np.int32) if gather_labels else None
    for idx, o, p in parts:
        sub_off = np.zeros(idx.size + 1, dtype=np.int64)
        sub_off[1:] = np.cumsum(np.diff(state_off)[idx])
        for j, i in enumerate(idx):
            per_all[:, i] = p[:, j]
            if gather_labels:
                labels[state_off[i]: state_off[i + 1]] = o[sub_off[j]: sub_off[j + 1]]
    return labels, per_all

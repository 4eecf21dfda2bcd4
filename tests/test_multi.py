"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2410_22764_gb300 import inputs as I
from paper_2410_22764_gb300.multi import aggregate, shard_batch


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_batch_is_a_balanced_partition():
    ns, ks, _, _ = I.batch_sizes(4096, 1)
    for world in (1, 2, 3, 8):
        parts = shard_batch(ns, ks, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(ns.size))
        loads = [int((ns[p] * (ks[p] + 1)).sum()) for p in parts]
        biggest = int((ns * (ks + 1)).max())
        assert max(loads) - min(loads) <= biggest


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # timing aggregation: slowest rank, units of every rank
        ms, units = aggregate(10.0 + 5 * rank, 100.0 * (rank + 1), dist)
        # a sharded batch: each rank minimizes its share (CPU oracle stands in for the device),
        # results are gathered on every rank
        ns, ks, ps, seeds = I.batch_sizes(40, 3, n_lo=2, n_hi=400, k_lo=0, k_hi=4)
        mine = shard_batch(ns, ks, world)[rank]
        res = {}
        for i in mine:
            d = I.random_dfa(int(ns[i]), int(ks[i]), float(ps[i]), int(seeds[i]))
            b, nb, psn = oracle.moore(d.delta, d.accept, d.n, d.k)
            res[int(i)] = (b.tolist(), nb, psn)
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put((rank, ms, units, merged))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ns, ks, ps, seeds = I.batch_sizes(40, 3, n_lo=2, n_hi=400, k_lo=0, k_hi=4)
    for rank, ms, units, merged in out:
        assert ms == 15.0 and units == 300.0
        assert sorted(merged) == list(range(40))
        for i in range(40):
            d = I.random_dfa(int(ns[i]), int(ks[i]), float(ps[i]), int(seeds[i]))
            b, nb, psn = oracle.moore(d.delta, d.accept, d.n, d.k)
            assert merged[i] == (b.tolist(), nb, psn)


def test_aggregate_single_rank():
    assert aggregate(3.0, 7.0, None) == (3.0, 7.0)

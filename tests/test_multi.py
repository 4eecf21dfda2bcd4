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
from paper_2410_22764_gb300.multi import (aggregate, member_subbatch, run_sharded_batch,
                                          shard_batch)


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


def oracle_runner(delta, accept, state_off, ks):
    """Stands in for the GPU batch launch on CPU ranks: the same (out_block, per) contract,
    computed by the oracle member by member."""
    count = ks.size
    out = np.empty(int(state_off[-1]), np.int32)
    per = np.zeros((3, count), np.int32)
    for j in range(count):
        d = I.batch_member(delta, accept, state_off, ks, j)
        b, nb, psn = oracle.moore(d.delta, d.accept, d.n, d.k)
        out[state_off[j]: state_off[j + 1]] = b
        per[:, j] = (nb, psn, 0)
    return out, per


def _batch():
    ns, ks, ps, seeds = I.batch_sizes(40, 3, n_lo=2, n_hi=400, k_lo=0, k_hi=4)
    return I.random_batch(ns, ks, ps, seeds)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # timing aggregation: slowest rank, units of every rank
        ms, units = aggregate(10.0 + 5 * rank, 100.0 * (rank + 1), dist)
        # the sharded batch path: each rank minimizes its share (the oracle runner stands in
        # for the device), results are gathered on every rank
        delta, acc, state_off, ks = _batch()
        seen = []

        def runner(d, a, so, kk):
            seen.append(int(kk.size))
            return oracle_runner(d, a, so, kk)
        labels, per = run_sharded_batch(delta, acc, state_off, ks, dist=dist, runner=runner)
        q.put((rank, ms, units, labels, per, seen))
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
    delta, acc, state_off, ks = _batch()
    want_labels, want_per = oracle_runner(delta, acc, state_off, ks)
    shares = shard_batch(np.diff(state_off), ks, world)
    for rank, ms, units, labels, per, seen in out:
        assert ms == 15.0 and units == 300.0
        assert seen == [shares[rank].size]             # each rank ran its own share once
        assert np.array_equal(labels, want_labels) and np.array_equal(per, want_per)


def test_member_subbatch_and_single_process_sharding():
    delta, acc, state_off, ks = _batch()
    idx = np.array([0, 3, 7, 39])
    sd, sa, so, sk = member_subbatch(delta, acc, state_off, ks, idx)
    for j, i in enumerate(idx):
        a = I.batch_member(delta, acc, state_off, ks, int(i))
        b = I.batch_member(sd, sa, so, sk, j)
        assert (a.n, a.k) == (b.n, b.k)
        assert np.array_equal(a.delta, b.delta) and np.array_equal(a.accept, b.accept)
    labels, per = run_sharded_batch(delta, acc, state_off, ks, runner=oracle_runner)
    want_labels, want_per = oracle_runner(delta, acc, state_off, ks)
    assert np.array_equal(labels, want_labels) and np.array_equal(per, want_per)


def test_aggregate_single_rank():
    assert aggregate(3.0, 7.0, None) == (3.0, 7.0)

"""The continuous-batching server: every result is identical alone and in the mix (bit-exact,
as all outputs are integers) and equal to the oracle; batches in flight overlap their copies
with earlier launches (the launches run one after another); admission
respects the HBM budget; cancellation and a bad request affect nobody else."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2410_22764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin, serve
    return dfamin, serve


def request_mix(seed=0, count=36, max_n=150_000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(10 ** rng.uniform(3, np.log10(max_n)))
        k = int(rng.integers(2, 9))
        u = rng.random()
        if i % 9 == 4:
            out.append(I.path_fib_dfa(4096))                        # deep refinement
        elif u < 0.5:
            out.append(I.random_dfa(n, k, 0.5, int(rng.integers(1 << 30))))
        else:
            out.append(I.inflated_dfa(max(1, n // 4), k, 4, 0.5, int(rng.integers(1 << 30)),
                                      permute=False)[0])
    return out


def solo(serve, d):
    srv = serve.Server(budget_bytes=8 << 30)
    r = srv.submit(d.n, d.k, d.delta, d.accept)
    srv.drain()
    return r


def test_alone_and_in_mix_identical(mods):
    dfamin, serve = mods
    dfas = request_mix(1)
    alone = [solo(serve, d) for d in dfas]
    srv = serve.Server(budget_bytes=8 << 30, streams=4)
    reqs = []
    for i, d in enumerate(dfas):                 # arrivals interleaved with scheduling
        reqs.append(srv.submit(d.n, d.k, d.delta, d.accept))
        if i % 3 == 2:
            srv.step()
    srv.drain()
    assert srv.stats.escalated >= 1
    for d, a, m in zip(dfas, alone, reqs):
        assert a.status == 0 and m.status == 0
        assert a.nblocks == m.nblocks and a.passes == m.passes
        assert np.array_equal(a.out_block, m.out_block)
        want, wn, _ = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert m.nblocks == wn and np.array_equal(m.out_block, want)


def test_alone_and_in_mix_identical_at_served_stream_sizes(mods):
    # the served-stream distribution at its full size range: n log-uniform 10^3 .. 4*10^6,
    # k 2..8, half uniform random, half inflated (c = 4), the largest sizes drawn on purpose,
    # and one path DFA of 65,536 states (escalated to the closure after its pass cap)
    dfamin, serve = mods
    rng = np.random.default_rng(5)
    sizes = [4_000_000, 2_500_000] + [int(10 ** rng.uniform(3, np.log10(4e6))) for _ in range(14)]
    dfas = []
    for i, n in enumerate(sizes):
        k = int(rng.integers(2, 9))
        if i % 2 == 0:
            dfas.append(I.random_dfa(n, k, 0.5, int(rng.integers(1 << 30))))
        else:
            dfas.append(I.inflated_dfa(max(1, n // 4), k, 4, 0.5, int(rng.integers(1 << 30)),
                                       permute=False)[0])
    dfas.insert(5, I.path_fib_dfa(65536))
    alone = [solo(serve, d) for d in dfas]
    srv = serve.Server(budget_bytes=48 << 30, streams=4)
    reqs = []
    for i, d in enumerate(dfas):
        reqs.append(srv.submit(d.n, d.k, d.delta, d.accept))
        if i % 2 == 1:
            srv.step()
    srv.drain()
    assert srv.stats.escalated >= 1
    for d, a, m in zip(dfas, alone, reqs):
        assert a.status == 0 and m.status == 0
        assert a.nblocks == m.nblocks and a.passes == m.passes
        assert np.array_equal(a.out_block, m.out_block)
        want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        assert m.nblocks == wn and np.array_equal(m.out_block, want)


def test_batches_overlap_on_device(mods):
    dfamin, serve = mods
    from oracle.path_depth import path_passes
    # plain deep-refinement requests (36,880 rounds each, long on the device, light on the
    # host) launched one per tick: later batches are in flight, their copies under way, while
    # earlier ones still run (the launches themselves follow one another on one stream)
    d = I.path_fib_dfa(65536)
    srv = serve.Server(budget_bytes=64 << 30, streams=4, pass_cap=100_000)
    for _ in range(3):
        srv.submit(d.n, d.k, d.delta, d.accept)
        srv.step()
    srv.drain()
    assert srv.stats.batches == 3 and srv.stats.max_inflight >= 2
    assert srv.max_device_overlap() >= 2
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    wp, _ = path_passes(I.fibonacci_word(65536))
    for r in srv.completed:
        assert r.status == 0 and r.nblocks == wn and r.passes == wp
        assert np.array_equal(r.out_block, want)


def test_budget_admission_and_rejection(mods):
    dfamin, serve = mods
    a = I.random_dfa(300_000, 4, 0.5, 1)
    b = I.random_dfa(300_000, 4, 0.5, 2)
    probe = serve.Server(budget_bytes=1 << 40)
    need = probe.request_bytes(a.n, a.k, True)
    srv = serve.Server(budget_bytes=int(need * 1.5), streams=4)
    ra = srv.submit(a.n, a.k, a.delta, a.accept)
    rb = srv.submit(b.n, b.k, b.delta, b.accept)
    srv.step()
    assert len(srv.inflight) == 1 and srv.used <= srv.budget and rb.admitted is None
    srv.drain()
    assert ra.status == 0 and rb.status == 0 and rb.admitted >= ra.done - 1e-3
    huge = I.random_dfa(2_000_000, 8, 0.5, 3)
    rh = srv.submit(huge.n, huge.k, huge.delta, huge.accept)
    assert rh.status == dfamin.ENOMEM and srv.stats.rejected == 1


def test_cancel_and_bad_request_are_isolated(mods):
    dfamin, serve = mods
    dfas = request_mix(2, count=10, max_n=50_000)
    bad = I.random_dfa(20_000, 3, 0.5, 9)
    bad_delta = bad.delta.copy()
    bad_delta[5] = -4
    srv = serve.Server(budget_bytes=8 << 30)
    reqs = [srv.submit(d.n, d.k, d.delta, d.accept) for d in dfas[:5]]
    rbad = srv.submit(bad.n, bad.k, bad_delta, bad.accept)
    rc = srv.submit(dfas[5].n, dfas[5].k, dfas[5].delta, dfas[5].accept)
    assert srv.cancel(rc)
    reqs += [srv.submit(d.n, d.k, d.delta, d.accept) for d in dfas[6:]]
    srv.drain()
    assert rbad.status == dfamin.EINVAL and rc.cancelled and rc.out_block is None
    for r, d in zip(reqs, dfas[:5] + dfas[6:]):
        want, wn, _ = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert r.status == 0 and r.nblocks == wn and np.array_equal(r.out_block, want)


@pytest.mark.parametrize("solo_work", [1, 0])
def test_single_dfa_launches_and_batches_agree(mods, solo_work):
    # every request as its own single-DFA launch (solo_work = 1) or none (0): the results,
    # closure reruns of deep refinements included, equal the oracle either way
    dfamin, serve = mods
    dfas = request_mix(seed=3, count=18, max_n=60_000)
    srv = serve.Server(budget_bytes=16 << 30, pass_cap=32, solo_work=solo_work)
    reqs = []
    for i, d in enumerate(dfas):
        reqs.append(srv.submit(d.n, d.k, d.delta, d.accept))
        if i % 3 == 2:
            srv.step()
    srv.drain()
    assert srv.stats.escalated >= 1
    assert (srv.stats.solo == srv.stats.batches) if solo_work else srv.stats.solo == 0
    for d, r in zip(dfas, reqs):
        want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        assert r.status == 0 and r.nblocks == wn and np.array_equal(r.out_block, want)


def test_results_kept_on_the_device(mods):
    # labels stay in device memory (single-DFA launches and batch members alike) and equal
    # the oracle's
    dfamin, serve = mods
    dfas = request_mix(seed=4, count=12, max_n=80_000) + [I.random_dfa(200_000, 4, 0.5, 9)]
    srv = serve.Server(budget_bytes=16 << 30, pass_cap=32, solo_work=1 << 19,
                       results_on_device=True)
    reqs = [srv.submit(d.n, d.k, d.delta, d.accept) for d in dfas]
    srv.drain()
    assert srv.stats.solo >= 1 and srv.stats.batches > srv.stats.solo
    for d, r in zip(dfas, reqs):
        assert isinstance(r.out_block, torch.Tensor) and r.out_block.is_cuda
        want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        assert r.status == 0 and r.nblocks == wn
        assert np.array_equal(r.out_block.cpu().numpy(), want)

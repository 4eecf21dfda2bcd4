"""Parity at the benchmark workloads' full sizes, in the launch configuration bench.py times
(default options), element by element against the oracle.  The batches of 4,096 DFAs are
checked member by member, with the oracle run on every host core (one DFA per process)."""
import numpy as np
import pytest
import torch

import oracle
from oracle.path_depth import path_passes
from paper_2410_22764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin
    return dfamin


def test_inflated_1e7_k4_against_hopcroft(dm):
    # the bench workload: base m = 10^6, k = 4, p = 0.5, c = 10, permuted ids, seed 1
    d, base = I.inflated_dfa(1_000_000, 4, 10, 0.5, 1, permute=True)
    got, nb, ps, st = dm.minimize_host(d.n, d.k, d.delta, d.accept)
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    _, bn = oracle.hopcroft(base.delta, base.accept, base.n, base.k)
    assert st == 0 and nb == wn == bn
    assert np.array_equal(got, want)
    # pass count from Moore on the base DFA: every clone behaves as its base state round by
    # round; a discrete base stops one round earlier than its (non-discrete) inflation
    _, bnb, bp = oracle.moore(base.delta, base.accept, base.n, base.k)
    assert ps == bp + (1 if bnb == base.n else 0)


def test_path_2pow20_closure_full(dm):
    d = I.path_fib_dfa(1 << 20)
    got, nb, ps, st = dm.minimize_host(d.n, d.k, d.delta, d.accept, closure=True)
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert st == 0 and nb == wn == (1 << 20) - 1
    assert np.array_equal(got, want)
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    _, _, wp = oracle.moore(dc, d.accept, d.n, kc)
    assert ps == wp == 8


def test_path_2pow20_plain_full(dm):
    # ~half a million rounds: the pass count is pinned by the distinguishing depth computed
    # from the acceptance string (suffix ranks), the partition by Hopcroft
    d = I.path_fib_dfa(1 << 20)
    got, nb, ps, st = dm.minimize_host(d.n, d.k, d.delta, d.accept)
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    wp, wc = path_passes(I.fibonacci_word(1 << 20))
    assert st == 0 and nb == wn == wc
    assert np.array_equal(got, want)
    assert ps == wp == 534348


@pytest.fixture(scope="module")
def pool():
    from oracle_pool import make_pool
    p = make_pool()
    yield p
    p.close()
    p.join()


def _draws(kind):
    ns, ks, ps, seeds = I.batch_sizes(4096, 1)
    if kind == "capped":
        cap = I.batch_cap_for_transitions(4096, 1, 200_000_000)
        ns, ks, ps, seeds = I.batch_sizes(4096, 1, n_cap=cap)
    return ns, ks, ps, seeds


@pytest.mark.parametrize("kind", ["capped", "drawn"])
def test_batch_4096_every_member(dm, pool, kind):
    # every member of the batch against the oracle, one DFA per host core (Moore up to 300,000
    # states, with its pass count; Hopcroft above, compared through a digest of its labels)
    from oracle_pool import BatchJob, label_digest
    ns, ks, ps, seeds = _draws(kind)
    job = BatchJob(pool, ns, ks, ps, seeds, digest_min_n=300_001)
    delta, acc, state_off, kk = I.random_batch(ns, ks, ps, seeds)
    plan = dm.BatchPlan(state_off, kk, dm.options())
    out, per = plan.run(torch.from_numpy(delta).cuda(), torch.from_numpy(acc.view(np.int32)).cuda())
    torch.cuda.synchronize()
    outs, per = plan.split(out.cpu().numpy()), per.cpu().numpy()
    del delta, acc
    assert (per[2] == 0).all()
    want = job.results()
    for i, (lab, nb, passes) in enumerate(want):
        assert per[0, i] == nb, (i, ns[i], ks[i])
        if isinstance(lab, str):
            assert label_digest(outs[i]) == lab, (i, ns[i], ks[i])
        else:
            assert np.array_equal(outs[i], lab), (i, ns[i], ks[i])
        if passes >= 0:
            assert per[1, i] == passes, (i, ns[i], ks[i])


def test_minimal_dfa_1e7_against_oracle(dm):
    # the bench workload's minimal DFA from q0 = 0 (reachability + refinement + quotient)
    d, _ = I.inflated_dfa(1_000_000, 4, 10, 0.5, 1, permute=True)
    wd, wa, wn, wq0, wr = oracle.minimal_dfa(d.delta, d.accept, d.n, d.k, 0)
    dd, aa = dm.to_device(d.delta, d.accept)
    qd, qa, sc = dm.minimal_dfa(d.n, d.k, dd, aa, 0)
    torch.cuda.synchronize()
    ns, q0m, nr, passes, st = sc.cpu().tolist()
    assert st == 0 and (ns, q0m, nr) == (wn, wq0, wr)
    assert np.array_equal(qd[: wn * d.k].cpu().numpy(), wd)
    assert np.array_equal(qa.cpu().numpy().view(np.uint32)[: wa.size], wa)

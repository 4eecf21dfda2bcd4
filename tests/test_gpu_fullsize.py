"""Parity at the benchmark workloads' full sizes, in the launch configuration bench.py times
(default options).  Where the oracle finishes at full size the comparison is element by element;
otherwise sampled members are compared one by one and every member is checked for properties
that hold at any size (the labelling refines {F, Q\\F} and is stable under delta)."""
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


def _batch(dm, kind):
    ns, ks, ps, seeds = I.batch_sizes(4096, 1)
    if kind == "4b":
        cap = I.batch_cap_for_transitions(4096, 1, 200_000_000)
        ns, ks, ps, seeds = I.batch_sizes(4096, 1, n_cap=cap)
    delta, acc, state_off, kk = I.random_batch(ns, ks, ps, seeds)
    plan = dm.BatchPlan(state_off, kk, dm.options())
    out, per = plan.run(torch.from_numpy(delta).cuda(), torch.from_numpy(acc.view(np.int32)).cuda())
    torch.cuda.synchronize()
    return delta, acc, state_off, kk, plan.split(out.cpu().numpy()), per.cpu().numpy()


@pytest.mark.parametrize("kind,samples,checked", [("4b", 64, 4096), ("4a", 12, 512)])
def test_batch_4096(dm, kind, samples, checked):
    delta, acc, state_off, kk, outs, per = _batch(dm, kind)
    count = kk.size
    assert (per[2] == 0).all()
    rng = np.random.default_rng(3)
    order = np.argsort(np.diff(state_off))
    pick = set(rng.choice(count, size=samples, replace=False).tolist())
    pick |= {int(order[-1]), int(order[0])}           # the largest and the smallest member
    for i in sorted(pick):
        d = I.batch_member(delta, acc, state_off, kk, i)
        if d.n <= 300_000:
            want, wn, wp = oracle.moore(d.delta, d.accept, d.n, d.k)
            assert per[1, i] == wp
        else:
            want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        assert per[0, i] == wn and np.array_equal(outs[i], want), (i, d.n, d.k)
    for i in rng.choice(count, size=min(checked, count), replace=False):
        d = I.batch_member(delta, acc, state_off, kk, int(i))
        assert per[0, i] == outs[i].max() + 1
        assert oracle.check_stable(d.delta, d.accept, d.n, d.k, outs[i])


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

"""Incremental and letter-masked signature rounds and the bounded device waits, on the GPU
through the C ABI.

* A signature round after another one in which few states moved skips the blocks that cannot
  split (their leader's row names no block that split in the round before); a letter-masked
  round gathers, for each member, only the letters whose entry in its leader's row names a block
  that split.  Every case here runs four ways, with the default choice, with
  DFAMIN_FLAG_FULL_ROUNDS, with DFAMIN_FLAG_INCREMENTAL_ROUNDS (incremental whenever possible)
  and with DFAMIN_FLAG_MASKED_ROUNDS (masked whenever the alphabet is compiled in), and each
  must equal the oracle element by element (partition, block count and pass count): neither
  skipping a block nor trusting an unchanged entry changes the result of Alg. sortPR's round.
* Every wait of a CTA for its team is bounded.  A test-only bound of a microsecond makes a
  multi-CTA call end with DFAMIN_ETIMEOUT (no fault, no hang); the next call on the same
  context must be exact again.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_22764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin
    return dfamin


def _oracle(d, closure):
    want, wn, wp = oracle.moore(d.delta, d.accept, d.n, d.k)
    if closure:
        dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
        _, _, wp = oracle.moore(dc, d.accept, d.n, kc)
    return want, wn, wp


def _run(dm, d, **kw):
    dlt, acc = dm.to_device(d.delta, d.accept)
    return dm.minimize_ex(d.n, d.k, dlt, acc, opt=dm.options(**kw)).host()


def WAYS(dm):
    return (0, dm.FLAG_FULL_ROUNDS, dm.FLAG_INCREMENTAL_ROUNDS, dm.FLAG_MASKED_ROUNDS)


def both_ways(dm, d, closure=False, flags=0, **kw):
    want, wn, wp = _oracle(d, closure)
    for extra in WAYS(dm):
        got, gn, gp, st = _run(dm, d, closure=closure, flags=flags | extra, **kw)
        assert st == 0, dm.status_string(st)
        assert (gn, gp) == (wn, wp), (extra, gn, wn, gp, wp)
        assert np.array_equal(got, want), extra


CASES = {
    "inflated_k4": lambda: I.inflated_dfa(20_000, 4, 10, 0.5, 1)[0],
    "inflated_k3": lambda: I.inflated_dfa(30_000, 3, 4, 0.5, 2)[0],
    "inflated_k5_unpermuted": lambda: I.inflated_dfa(20_000, 5, 6, 0.5, 3, permute=False)[0],
    "inflated_k9": lambda: I.inflated_dfa(10_000, 9, 5, 0.5, 4)[0],
    "inflated_k6": lambda: I.inflated_dfa(12_000, 6, 8, 0.5, 14)[0],
    "inflated_k8": lambda: I.inflated_dfa(8_000, 8, 6, 0.3, 15)[0],
    "inflated_k1": lambda: I.inflated_dfa(50_000, 1, 5, 0.5, 16)[0],
    "inflated_k4_1e6": lambda: I.inflated_dfa(100_000, 4, 10, 0.5, 17)[0],
    "random_k2": lambda: I.random_dfa(150_000, 2, 0.5, 5),
    "random_k7_skewed": lambda: I.random_dfa(60_000, 7, 0.1, 6),
    "bitsplitter_b13": lambda: I.bitsplitter_dfa(13),
    "cyclic_fib_n": lambda: I.cyclic_fib_dfa(17),
    "path_fib": lambda: I.path_fib_dfa(9000),
}


@pytest.mark.parametrize("name", list(CASES))
def test_incremental_rounds_match_oracle(dm, name):
    # smem_states=1 keeps every case on the multi-CTA kernel, whose rounds are incremental
    both_ways(dm, CASES[name](), smem_states=1)


@pytest.mark.parametrize("ctas", [1, 3, 64])
def test_incremental_rounds_team_sizes(dm, ctas):
    both_ways(dm, I.inflated_dfa(8_000, 4, 10, 0.5, 7)[0], smem_states=1, ctas=ctas)
    both_ways(dm, I.cyclic_fib_dfa(14), smem_states=1, ctas=ctas)


@pytest.mark.parametrize("flags", [2, 4])
def test_incremental_rounds_with_forced_collisions(dm, flags):
    both_ways(dm, I.inflated_dfa(6_000, 3, 6, 0.5, 8)[0], flags=flags, smem_states=1)


@pytest.mark.parametrize("maker", ["path", "bits", "fib", "inflated"])
def test_incremental_rounds_on_the_closure(dm, maker):
    d = {"path": lambda: I.path_fib_dfa(20_000), "bits": lambda: I.bitsplitter_dfa(11),
         "fib": lambda: I.cyclic_fib_dfa(16),
         "inflated": lambda: I.inflated_dfa(3_000, 2, 4, 0.5, 9)[0]}[maker]()
    both_ways(dm, d, closure=True, smem_states=1)


def test_incremental_rounds_in_a_batch(dm):
    dfas = [I.inflated_dfa(6_000, 4, 10, 0.5, 11)[0], I.cyclic_fib_dfa(15),
            I.random_dfa(40_000, 3, 0.5, 12), I.bitsplitter_dfa(12), I.random_dfa(900, 2, 0.5, 13),
            I.inflated_dfa(4_000, 6, 8, 0.5, 18)[0], I.inflated_dfa(9_000, 2, 7, 0.5, 19)[0]]
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    outs = []
    for flags in WAYS(dm) + (dm.FLAG_MASKED_ROUNDS | dm.FLAG_BATCH_FOUR_CTAS,):
        plan = dm.BatchPlan(state_off, ks, dm.options(flags=flags, team_states=4096))
        out, per = plan.run(dd, aa)
        outs.append((out.cpu().numpy(), per.cpu().numpy()))
        plan.close()
    for (out, per) in outs:
        for i, d in enumerate(dfas):
            want, wn, wp = oracle.moore(d.delta, d.accept, d.n, d.k)
            got = out[state_off[i]: state_off[i + 1]]
            assert per[2, i] == 0 and per[0, i] == wn and per[1, i] == wp
            assert np.array_equal(got, want)


# ------------------------------------------------------------------ bounded waits
def test_barrier_wait_runs_out_and_context_stays_usable(dm):
    d = I.inflated_dfa(100_000, 4, 10, 0.5, 21)[0]            # n = 1e6: hundreds of CTAs
    got, gn, gp, st = _run(dm, d, barrier_timeout_us=1)
    assert st == dm.ETIMEOUT and gn == -dm.ETIMEOUT
    # a closure run waits at every closure level too
    p = I.path_fib_dfa(300_000)
    _, gn2, _, st2 = _run(dm, p, closure=True, barrier_timeout_us=1)
    assert st2 == dm.ETIMEOUT and gn2 == -dm.ETIMEOUT
    # the next calls on the same context are exact
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    got, gn, gp, st = _run(dm, d)
    assert st == 0 and gn == wn and np.array_equal(got, want)


def test_batch_barrier_wait_runs_out_only_for_team_dfas(dm):
    big = I.inflated_dfa(60_000, 4, 10, 0.5, 22)[0]           # a team of many CTAs
    small = [I.random_dfa(500 + 37 * i, 2, 0.5, 30 + i) for i in range(6)]   # one CTA each
    dfas = [big] + small
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    plan = dm.BatchPlan(state_off, ks, dm.options(barrier_timeout_us=1, team_states=8192))
    out, per = plan.run(dd, aa)
    per = per.cpu().numpy()
    out = out.cpu().numpy()
    plan.close()
    assert per[2, 0] == dm.ETIMEOUT and per[0, 0] == -dm.ETIMEOUT
    for i, d in enumerate(small, start=1):
        want, wn, wp = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert per[2, i] == 0 and per[0, i] == wn
        assert np.array_equal(out[state_off[i]: state_off[i + 1]], want)
    # the same batch with the default bound is exact
    plan = dm.BatchPlan(state_off, ks, dm.options(team_states=8192))
    out, per = plan.run(dd, aa)
    per = per.cpu().numpy()
    out = out.cpu().numpy()
    plan.close()
    want, wn = oracle.hopcroft(big.delta, big.accept, big.n, big.k)
    assert per[2, 0] == 0 and per[0, 0] == wn and np.array_equal(out[: big.n], want)

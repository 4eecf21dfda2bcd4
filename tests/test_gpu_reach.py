"""Reachability, quotient and minimal DFA (dfamin_reachable / dfamin_quotient /
dfamin_minimal_dfa) against the oracle, bit-exact."""
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


def union_with_unreachable(d, seed, copies=2):
    """d plus (copies-1) relabelled copies that nothing from the first copy enters."""
    rng = np.random.default_rng(seed)
    parts, accs = [d.delta.astype(np.int64)], [I.unpack_bits(d.accept, d.n)]
    for c in range(1, copies):
        parts.append(d.delta.astype(np.int64) + c * d.n)
        accs.append(rng.random(d.n) < 0.5)
    n = d.n * copies
    return I.Dfa(n, d.k, np.concatenate(parts).astype(np.int32), I.pack_bits(np.concatenate(accs)))


def cases():
    out = [("fig1_q0", I.fig1_dfa(), 0), ("fig1_q5", I.fig1_dfa(), 5),
           ("bits_from0", I.bitsplitter_dfa(9), 0), ("bits_mid", I.bitsplitter_dfa(9), 300),
           ("k0", I.Dfa(7, 0, np.zeros(0, np.int32), I.pack_bits(np.arange(7) % 2 == 0)), 3),
           ("n1", I.random_dfa(1, 2, 1.0, 1), 0),
           ("path_chain", I.path_fib_dfa(5000), 0),
           ("path_long", I.path_fib_dfa(120000), 7)]
    for seed, (n, k) in enumerate([(300, 1), (3000, 2), (20000, 3), (70000, 5)]):
        out.append((f"rand_union{n}", union_with_unreachable(I.random_dfa(n, k, 0.5, seed), seed),
                    seed * 17 % n))
    infl = I.inflated_dfa(4000, 3, 4, 0.5, 9)[0]
    out.append(("inflated_union", union_with_unreachable(infl, 4, copies=3), 11))
    fib = I.cyclic_fib_dfa(16)
    out.append(("fib_union", union_with_unreachable(fib, 5), 100))
    return out


CASES = cases()


@pytest.mark.parametrize("name,d,q0", CASES, ids=[c[0] for c in CASES])
def test_reachable_matches_oracle(dm, name, d, q0):
    want, cnt = oracle.reachable(d.delta, d.n, d.k, q0)
    wd, wa = oracle.induced(d.delta, d.accept, d.n, d.k, want, cnt)
    dd, aa = dm.to_device(d.delta, d.accept)
    newid, rd, ra, sc = dm.reachable(d.n, d.k, dd, aa, q0)
    torch.cuda.synchronize()
    c, st = sc.cpu().tolist()
    assert st == 0 and c == cnt
    assert np.array_equal(newid.cpu().numpy(), want)
    assert np.array_equal(rd.cpu().numpy()[: cnt * d.k], wd)
    got_acc = ra.cpu().numpy().view(np.uint32)
    assert np.array_equal(got_acc[: wa.size], wa)


@pytest.mark.parametrize("name,d,q0", CASES, ids=[c[0] for c in CASES])
def test_minimal_dfa_matches_oracle(dm, name, d, q0):
    wd, wa, wn, wq0, wr = oracle.minimal_dfa(d.delta, d.accept, d.n, d.k, q0)
    dd, aa = dm.to_device(d.delta, d.accept)
    for opt in (dm.options(), dm.options(closure=True), dm.options(leader=True)):
        qd, qa, sc = dm.minimal_dfa(d.n, d.k, dd, aa, q0, opt=opt)
        torch.cuda.synchronize()
        ns, q0m, nr, passes, st = sc.cpu().tolist()
        assert st == 0, dm.status_string(st)
        assert (ns, q0m, nr) == (wn, wq0, wr)
        assert np.array_equal(qd.cpu().numpy()[: wn * d.k], wd)
        got = qa.cpu().numpy().view(np.uint32)
        assert np.array_equal(got[: wa.size], wa)
        assert not (got[wa.size:] != 0).any()


def test_quotient_of_full_partition(dm):
    # fully reachable DFA: the quotient of the canonical partition with newid = None
    d = I.inflated_dfa(3000, 4, 5, 0.5, 2, permute=True)[0]
    dd, aa = dm.to_device(d.delta, d.accept)
    r = dm.minimize_ex(d.n, d.k, dd, aa)
    qd, qa, sc = dm.quotient(d.n, d.k, dd, aa, r.out_block, 17)
    torch.cuda.synchronize()
    block, nb, _, st = r.host()
    wd, wa, wq0 = oracle.quotient(d.delta, d.accept, d.n, d.k, block, nb, 17)
    ns, q0m, st2 = sc.cpu().tolist()
    assert st == 0 and st2 == 0 and ns == nb and q0m == wq0
    assert np.array_equal(qd.cpu().numpy()[: nb * d.k], wd)
    assert np.array_equal(qa.cpu().numpy().view(np.uint32)[: wa.size], wa)


def test_quotient_renumbers_any_labels(dm):
    # labels need not be canonical: classes are numbered by their smallest member
    d = I.random_dfa(5000, 2, 0.5, 8)
    want, nb = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    perm = np.random.default_rng(1).permutation(d.n).astype(np.int32)
    labels = perm[want]
    dd, aa = dm.to_device(d.delta, d.accept)
    qd, qa, sc = dm.quotient(d.n, d.k, dd, aa, torch.from_numpy(labels).cuda(), 0)
    wd, wa, wq0 = oracle.quotient(d.delta, d.accept, d.n, d.k, want, nb, 0)
    torch.cuda.synchronize()
    ns, q0m, st = sc.cpu().tolist()
    assert st == 0 and ns == nb and q0m == wq0
    assert np.array_equal(qd.cpu().numpy()[: nb * d.k], wd)


def test_bad_entries(dm):
    d = union_with_unreachable(I.random_dfa(4000, 2, 0.5, 3), 3)
    dd, aa = dm.to_device(d.delta, d.accept)
    bad_unreached = d.delta.copy()
    bad_unreached[-1] = d.n + 9            # a row of the unreachable copy
    bd = torch.from_numpy(bad_unreached).cuda()
    newid, rd, ra, sc = dm.reachable(d.n, d.k, bd, aa, 0)
    qd, qa, msc = dm.minimal_dfa(d.n, d.k, bd, aa, 0)
    torch.cuda.synchronize()
    assert sc.cpu().tolist()[1] == 0                   # never read by the search
    assert msc.cpu().tolist()[4] == dm.EINVAL          # the refinement reads every row
    assert msc.cpu().tolist()[0] == -dm.EINVAL
    bad_reached = d.delta.copy()
    bad_reached[0] = -4                    # row of q0 = 0
    newid, rd, ra, sc = dm.reachable(d.n, d.k, torch.from_numpy(bad_reached).cuda(), aa, 0)
    torch.cuda.synchronize()
    assert sc.cpu().tolist() == [-dm.EINVAL, dm.EINVAL]
    # the context stays usable
    test_quotient_of_full_partition(dm)


@pytest.mark.parametrize("n,L,seed", [(3000, 4, 1), (50000, 12, 2)])
def test_lts_pipeline(dm, n, L, seed):
    # synthetic LTS -> DFA (host front end) -> minimal DFA on the device, against the oracle's
    # own front end and minimal DFA
    nn, src, lbl, dst = I.lts_synthetic(n, L, 0.7, 0.2, seed)
    ns, delta, acc = dm.lts_determinize(nn, L, src, lbl, dst, 0)
    wns, wdelta, wacc = oracle.lts_to_dfa(nn, L, src, lbl, dst, 0)
    assert ns == wns and np.array_equal(delta, wdelta)
    wd, wa, wn, wq0, wr = oracle.minimal_dfa(wdelta, wacc, wns, L, 0)
    dd, aa = dm.to_device(delta, acc)
    qd, qa, sc = dm.minimal_dfa(ns, L, dd, aa, 0)
    torch.cuda.synchronize()
    got_n, got_q0, got_r, _, st = sc.cpu().tolist()
    assert st == 0 and (got_n, got_q0, got_r) == (wn, wq0, wr)
    assert np.array_equal(qd.cpu().numpy()[: wn * L], wd)

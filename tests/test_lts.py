"""LTS -> DFA front end (Sec. 4.1): the oracle against brute force, and the library's host
routine against the oracle (both run on the CPU; the front end uses no GPU)."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2410_22764_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dm():
    so = os.path.join(ROOT, "paper_2410_22764_gb300", "libdfamin.so")
    if not os.path.exists(so):
        import __graft_entry__
        __graft_entry__.build()
    from paper_2410_22764_gb300 import dfamin
    return dfamin


def random_lts(n, nlabels, m, seed, s0_out=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m).astype(np.int32)
    lbl = rng.integers(0, nlabels, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    return src, lbl, dst


def has_path(src, lbl, dst, s0, word):
    """Is there a path from s0 labelled `word`?  Depth-first over individual paths."""
    edges = {}
    for s, a, t in zip(src.tolist(), lbl.tolist(), dst.tolist()):
        edges.setdefault((s, a), []).append(t)

    def go(s, i):
        if i == len(word):
            return True
        return any(go(t, i + 1) for t in edges.get((s, word[i]), ()))
    return go(s0, 0)


def accepts(delta, k, acc, word):
    q = 0
    for a in word:
        q = int(delta[q * k + a])
    return bool((int(acc[q >> 5]) >> (q & 31)) & 1)


def test_hand_example():
    # 0 -a-> 1, 0 -a-> 2, 1 -b-> 3, 2 -c-> 3: {0} -a-> {1,2} -b,c-> {3}; all else to bottom
    src, lbl, dst = (np.array(x, np.int32) for x in ([0, 0, 1, 2], [0, 0, 1, 2], [1, 2, 3, 3]))
    ns, delta, acc = oracle.lts_to_dfa(4, 3, src, lbl, dst, 0)
    assert ns == 4
    assert delta.tolist() == [1, 3, 3, 3, 2, 2, 3, 3, 3, 3, 3, 3]
    assert int(acc[0]) == 0b0111


@pytest.mark.parametrize("seed", range(10))
def test_oracle_language_is_the_paths_of_the_lts(seed):
    n, L = 6, 2
    src, lbl, dst = random_lts(n, L, 9, seed)
    ns, delta, acc = oracle.lts_to_dfa(n, L, src, lbl, dst, 0)
    for length in range(7):
        for word in itertools.product(range(L), repeat=length):
            assert accepts(delta, L, acc, word) == has_path(src, lbl, dst, 0, word)


def test_deterministic_complete_lts_gives_its_reachable_part():
    # a DFA read as an LTS: the subsets are singletons of the reachable states, bottom is
    # unreachable, and the language is every word
    d = I.random_dfa(200, 2, 0.5, 4)
    src = np.repeat(np.arange(d.n, dtype=np.int32), d.k)
    lbl = np.tile(np.arange(d.k, dtype=np.int32), d.n)
    ns, delta, acc = oracle.lts_to_dfa(d.n, d.k, src, lbl, d.delta, 5)
    _, reach = oracle.reachable(d.delta, d.n, d.k, 5)
    assert ns == reach + 1
    qd, qa, nb, q0, nr = oracle.minimal_dfa(delta, acc, ns, d.k, 0)
    assert (nb, nr) == (1, reach) and int(qa[0]) & 1


@pytest.mark.parametrize("seed,n,L,m", [(1, 5, 2, 8), (2, 40, 3, 90), (3, 12, 4, 40),
                                        (6, 1, 3, 0), (7, 50, 0, 0)])
def test_library_matches_oracle_random(dm, seed, n, L, m):
    # unrestricted nondeterminism, kept tiny (the powerset grows exponentially)
    src, lbl, dst = random_lts(n, max(L, 1), m, seed)
    s0 = seed % n
    want = oracle.lts_to_dfa(n, L, src, lbl, dst, s0)
    got = dm.lts_determinize(n, L, src, lbl, dst, s0)
    assert got[0] == want[0]
    assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])


@pytest.mark.parametrize("seed,n,L", [(1, 100, 3), (2, 2000, 5), (3, 20000, 8), (4, 5000, 26)])
def test_library_matches_oracle_synthetic(dm, seed, n, L):
    nn, src, lbl, dst = I.lts_synthetic(n, L, 0.7, 0.2, seed)
    s0 = seed % n
    want = oracle.lts_to_dfa(nn, L, src, lbl, dst, s0)
    assert want[0] <= 3 * n + 1
    got = dm.lts_determinize(nn, L, src, lbl, dst, s0)
    assert got[0] == want[0]
    assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])


def test_library_errors(dm):
    src, lbl, dst = random_lts(30, 2, 60, 1)
    bad = lbl.copy()
    bad[3] = 2
    with pytest.raises(dm.DfaminError):
        dm.lts_determinize(30, 2, src, bad, dst, 0)
    with pytest.raises(dm.DfaminError):
        dm.lts_determinize(30, 2, src, lbl, dst, 0, max_states=2)

"""Pins for the CPU oracle: each test checks the oracle against something other than itself
(the definition of state equivalence through delta*, worked examples and closed forms printed
in arXiv 2410.22764, brute force on tiny inputs, and algebraic invariants)."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2410_22764_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- definition by words (Sec. 2)
def _delta_star(delta, k, q, word):
    # delta*(q, eps) = q ; delta*(q, a w) = delta*(delta(q, a), w)   (Sec. 2)
    for a in word:
        q = int(delta[q * k + a])
    return q


def _words_classes(n, k, delta, acc):
    """p ~ q iff every word w has delta*(p,w) in F <=> delta*(q,w) in F.  Words up to length n
    suffice: a shortest distinguishing word of an n-state DFA is shorter than n."""
    words = [w for L in range(n + 1) for w in itertools.product(range(k), repeat=L)]
    sig = [tuple(bool(acc[_delta_star(delta, k, s, w)]) for w in words) for s in range(n)]
    first = {}
    out = []
    for s in range(n):
        out.append(first.setdefault(sig[s], len(first)))
    return np.array(out, np.int32), len(first)


def _all_dfas(n, k):
    for succ in itertools.product(range(n), repeat=n * k):
        for accmask in range(1 << n):
            acc = np.array([(accmask >> s) & 1 for s in range(n)], bool)
            yield np.array(succ, np.int32), acc


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 1), (3, 2), (4, 1)])
def test_exhaustive_tiny_against_words_definition(n, k):
    for delta, acc in _all_dfas(n, k):
        bits = I.pack_bits(acc)
        want, wn = _words_classes(n, k, delta, acc)
        m, mn, _ = oracle.moore(delta, bits, n, k)
        h, hn = oracle.hopcroft(delta, bits, n, k)
        t, tn, _ = oracle.tablefill(delta, bits, n, k)
        assert (m == want).all() and mn == wn
        assert (h == want).all() and hn == wn
        assert (t == want).all() and tn == wn


def test_random_small_against_words_definition():
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(1, 7))
        k = int(rng.integers(0, 3))
        delta = rng.integers(0, n, n * k).astype(np.int32)
        acc = rng.random(n) < rng.random()
        want, wn = _words_classes(n, k, delta, acc)
        m, mn, _ = oracle.moore(delta, I.pack_bits(acc), n, k)
        assert (m == want).all() and mn == wn


# ---------------------------------------------------------------- three oracles agree
@pytest.mark.parametrize("p", [0.0, 0.1, 0.5, 0.9, 1.0])
def test_three_oracles_agree_random(p):
    for seed in range(40):
        n = 1 + (seed * 37) % 300
        k = seed % 5
        d = I.random_dfa(n, k, p, seed)
        m, mn, mp = oracle.moore(d.delta, d.accept, n, k)
        h, hn = oracle.hopcroft(d.delta, d.accept, n, k)
        t, tn, rounds = oracle.tablefill(d.delta, d.accept, n, k)
        assert mn == hn == tn
        assert (m == h).all() and (m == t).all()
        # Moore's pass count is the distinguishing depth, plus one confirming pass unless the
        # partition became discrete (the early-exit rule).
        assert mp == rounds + (1 if mn < n else 0)
        assert oracle.check_stable(d.delta, d.accept, n, k, m)


def test_three_oracles_agree_structured():
    # mostly-mergeable DFAs: inflated (many equivalent clones) with small alphabets
    for seed in range(12):
        d, base = I.inflated_dfa(40 + seed, 1 + seed % 3, 3, 0.5, seed, permute=bool(seed % 2))
        m, mn, mp = oracle.moore(d.delta, d.accept, d.n, d.k)
        h, hn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        t, tn, rounds = oracle.tablefill(d.delta, d.accept, d.n, d.k)
        assert mn == hn == tn and (m == h).all() and (m == t).all()
        assert mp == rounds + (1 if mn < d.n else 0)


def test_canonical_labels_are_first_occurrence():
    lab = np.array([5, 5, 2, 7, 2, 0, 7, 1], np.int32)
    out, c = oracle.canonical(lab)
    assert out.tolist() == [0, 0, 1, 2, 1, 3, 2, 4] and c == 5


def test_planted_mistake_is_caught():
    """A labelling that merges two inequivalent states must fail the stability check."""
    d = I.fig1_dfa()
    b, _ = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    bad = b.copy()
    bad[1] = bad[0]  # q0 and q1 are apart by a^8 (Sec. 3.4)
    assert oracle.check_stable(d.delta, d.accept, d.n, d.k, b)
    assert not oracle.check_stable(d.delta, d.accept, d.n, d.k, bad)


# ---------------------------------------------------------------- closed forms and examples
def test_fig1_path_needs_eight_rounds_and_closure_separates_q0_q1_in_one():
    # Fig. 1: accepts a^j with j > 8; every partition refinement needs 8 iterations to split
    # q0 from q1, while with the closure the letter a^8 splits them in the first iteration.
    d = I.fig1_dfa()
    b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    assert nb == 10 and ps == 8
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    assert kc == 4  # a, a^2, a^4, a^8 (floor(log2 10) = 3)
    one, _, _ = oracle.moore(dc, d.accept, d.n, kc, max_passes=1, partial=True)
    assert one[0] != one[1]
    plain_one, _, _ = oracle.moore(d.delta, d.accept, d.n, d.k, max_passes=1, partial=True)
    assert plain_one[0] == plain_one[1]
    bc, nbc, psc = oracle.moore(dc, d.accept, d.n, kc)
    assert nbc == 10 and (bc == b).all() and psc < ps


def _read_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_fig2_bitsplitter_b3_matches_figure():
    d = I.bitsplitter_dfa(3)
    assert d.n == 8 and d.k == 2
    rows = _read_golden("fig2_b3.txt")
    acc = d.accepting()
    for r in rows:
        if r[0] == "edge":
            src, letter, dst = int(r[1], 2), int(r[2][1:]) - 1, int(r[3], 2)
            assert d.delta[src * d.k + letter] == dst, r
        else:
            assert acc[int(r[1], 2)]
    assert acc.sum() == sum(1 for r in rows if r[0] == "accept")
    assert sum(1 for r in rows if r[0] == "edge") == d.n * d.k


def test_fig2_fib5_matches_figure():
    d = I.cyclic_fib_dfa(5)
    rows = _read_golden("fig2_fib5.txt")
    assert d.n == 8
    for r in rows:
        if r[0] == "edge":
            assert d.delta[int(r[1])] == int(r[2])
    assert sorted(np.nonzero(d.accepting())[0].tolist()) == [int(r[1]) for r in rows
                                                             if r[0] == "accept"]


def test_fibonacci_words_match_listing():
    for idx, word in _read_golden("fibonacci_words.txt"):
        assert "".join(map(str, I.fibonacci_word_n(int(idx)))) == word
    inf = I.fibonacci_word(200)
    for i in range(1, 12):
        w = I.fibonacci_word_n(i)
        assert (inf[: w.size] == w).all()


@pytest.mark.parametrize("i", range(2, 16))
def test_cyclic_fibonacci_classes_and_rounds(i):
    # Table 2: size output = N; Sec. 4.2: n-2 parallel iterations on Fib automata
    d = I.cyclic_fib_dfa(i)
    b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    h, hn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert nb == d.n == hn and (b == h).all()
    assert ps == max(d.n - 2, 0)


@pytest.mark.parametrize("nbits", range(1, 13))
def test_bitsplitter_classes_and_rounds(nbits):
    # Table 2: B_n has size output 2^n and takes n-1 iterations
    d = I.bitsplitter_dfa(nbits)
    b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    h, hn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert nb == hn == 1 << nbits and (b == h).all()
    assert ps == nbits - 1


def test_table2_bitsplitter_rows_small():
    for name, N, sig, size_out, iters in _read_golden("table2_rows.txt"):
        if not name.startswith("B") or int(name[1:]) > 16:
            continue
        d = I.bitsplitter_dfa(int(name[1:]))
        assert d.n == int(N) and d.k == int(sig)
        _, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert nb == int(size_out) and ps == int(iters)


def test_table2_fibonacci_sizes():
    # the table's Fib_i has N = |w_{i+1}| states and is minimal (size output = N)
    for name, N, sig, size_out, iters in _read_golden("table2_rows.txt"):
        if not name.startswith("Fib"):
            continue
        i = int(name[3:])
        assert I.fibonacci_word_n(i + 1).size == int(N) == int(size_out)
        # iterations column: one confirming pass after the n-2 splitting rounds
        assert int(iters) == int(N) - 1


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10, 33, 100, 257, 1000, 2048])
def test_path_fibonacci_closed_form(n):
    d = I.path_fib_dfa(n)
    w = I.fibonacci_word(n)
    want = n - (1 if n >= 2 and w[n - 2] == w[n - 1] else 0)
    b, nb, _ = oracle.moore(d.delta, d.accept, d.n, d.k)
    h, hn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert nb == hn == want and (b == h).all()


@pytest.mark.parametrize("seed", range(6))
def test_inflated_classes_equal_base_classes(seed):
    m, k, c = 300 + 50 * seed, 1 + seed % 4, 2 + seed
    d, base = I.inflated_dfa(m, k, c, 0.5, seed, permute=seed % 2 == 0)
    bb, bn = oracle.hopcroft(base.delta, base.accept, m, k)
    b, nb = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert nb == bn
    # every clone sits in the block of its base state
    raw = np.arange(d.n)
    ident = I.seeded_permutation(d.n, seed) if seed % 2 == 0 else raw
    lab = np.empty(d.n, np.int64)
    lab[ident] = bb[raw // c]
    canon, cn = oracle.canonical(lab.astype(np.int32))
    assert cn == bn and (canon == b).all()


def test_uniform_acceptance_gives_one_block():
    for k in range(0, 4):
        for p in (0.0, 1.0):
            d = I.random_dfa(500, k, p, 3)
            b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
            assert nb == 1 and (b == 0).all() and ps == 1


# ---------------------------------------------------------------- closure (Alg. transPR)
def test_closure_columns_are_powers_of_delta():
    for seed in range(5):
        n, k = 50 + 31 * seed, 1 + seed % 3
        d = I.random_dfa(n, k, 0.5, seed)
        cols = oracle.closure(d.delta, n, k)
        levels = oracle.closure_levels(n)
        assert levels == int(np.floor(np.log2(n))) + 1
        for a in range(k):
            for i in range(levels):
                for q in range(0, n, 7):
                    t = q
                    for _ in range(1 << i):
                        t = int(d.delta[t * k + a])
                    assert cols[a * levels + i, q] == t


@pytest.mark.parametrize("maker", ["path", "cyclic", "bits", "random", "inflated"])
def test_closure_preserves_equivalence(maker):
    if maker == "path":
        d = I.path_fib_dfa(777)
    elif maker == "cyclic":
        d = I.cyclic_fib_dfa(12)
    elif maker == "bits":
        d = I.bitsplitter_dfa(9)
    elif maker == "random":
        d = I.random_dfa(900, 3, 0.4, 11)
    else:
        d, _ = I.inflated_dfa(200, 2, 4, 0.5, 5)
    b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    bc, nbc, psc = oracle.moore(dc, d.accept, d.n, kc)
    assert nbc == nb and (bc == b).all()
    assert psc <= ps


def test_moore_cap_reports_nonconvergence():
    d = I.cyclic_fib_dfa(10)
    with pytest.raises(RuntimeError):
        oracle.moore(d.delta, d.accept, d.n, d.k, max_passes=5)


def test_bad_delta_rejected():
    delta = np.array([0, 5], np.int32)
    with pytest.raises(ValueError):
        oracle.moore(delta, I.pack_bits(np.array([1, 0], bool)), 2, 1)
    with pytest.raises(ValueError):
        oracle.hopcroft(delta, I.pack_bits(np.array([1, 0], bool)), 2, 1)


# ---------------------------------------------------------------- path distinguishing depth
def _path_dfa_from_word(w):
    n = w.size
    i = np.arange(n)
    delta = np.stack([np.minimum(i + 1, n - 1), i], 1).astype(np.int32).reshape(-1)
    return delta, I.pack_bits(w.astype(bool))


def test_path_depth_matches_moore_and_tablefill():
    from oracle.path_depth import path_depth, path_passes
    rng = np.random.default_rng(3)
    for _ in range(300):
        n = int(rng.integers(1, 80))
        w = (rng.random(n) < rng.random()).astype(np.uint8)
        delta, acc = _path_dfa_from_word(w)
        _, nb, ps = oracle.moore(delta, acc, n, 2)
        _, tn, rounds = oracle.tablefill(delta, acc, n, 2)
        assert path_passes(w) == (ps, nb)
        assert path_depth(w) == (rounds, tn)


@pytest.mark.parametrize("n", [2, 7, 100, 1000, 4096])
def test_path_depth_fibonacci(n):
    from oracle.path_depth import path_passes
    d = I.path_fib_dfa(n)
    _, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    assert path_passes(I.fibonacci_word(n)) == (ps, nb)


@pytest.mark.parametrize("seed", range(8))
def test_inflated_pass_count_from_base(seed):
    """The relation the full-size test uses: an inflated DFA takes the base DFA's passes, plus
    one confirming round when the base is already discrete."""
    m, k, c = 500 + 37 * seed, 1 + seed % 4, 2 + seed % 5
    d, base = I.inflated_dfa(m, k, c, 0.5, seed, permute=seed % 2 == 0)
    _, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
    _, bnb, bp = oracle.moore(base.delta, base.accept, base.n, base.k)
    assert nb == bnb and ps == bp + (1 if bnb == base.n else 0)


# ---------------------------------------------------------------- Alg. 2 naivePR
@pytest.mark.parametrize("seed", range(30))
def test_naive_partition_equals_hopcroft(seed):
    n, k = 1 + (seed * 53) % 400, seed % 5
    d = I.random_dfa(n, k, [0.0, 0.3, 0.5, 1.0][seed % 4], seed)
    b, nb, it = oracle.naive(d.delta, d.accept, n, k)
    h, hn = oracle.hopcroft(d.delta, d.accept, n, k)
    assert nb == hn and (b == h).all()
    # every iteration but the last splits at least one block
    assert 1 <= it <= max(1, nb - (1 if nb > 1 else 0)) + 1


def test_naive_iterations_table2_fibonacci():
    # Table 2, naivePR column: Fib with N states takes N-1 iterations (the last changes nothing)
    for name, N, sig, size_out, iters in _read_golden("table2_rows.txt"):
        if name.startswith("Fib"):
            assert int(iters) == int(N) - 1
    for i in range(3, 17):
        d = I.cyclic_fib_dfa(i)
        _, nb, it = oracle.naive(d.delta, d.accept, d.n, d.k)
        assert nb == d.n and it == d.n - 1


@pytest.mark.parametrize("nbits", range(1, 13))
def test_naive_iterations_bitsplitter(nbits):
    # Table 2 prints n-1 for B_n; counting, as Alg. 2 does, the final round that changes nothing
    # gives n (the table's B rows omit that round, its Fib rows include it)
    d = I.bitsplitter_dfa(nbits)
    _, nb, it = oracle.naive(d.delta, d.accept, d.n, d.k)
    assert nb == 1 << nbits and it == nbits


def test_naive_fig1_and_closure():
    d = I.fig1_dfa()
    b, nb, it = oracle.naive(d.delta, d.accept, d.n, d.k)
    assert nb == 10 and it == 9
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    bc, nbc, itc = oracle.naive(dc, d.accept, d.n, kc)
    assert nbc == 10 and (bc == b).all() and itc < it


@pytest.mark.parametrize("i", [12, 16, 19])
def test_naive_rounds_at_most_double_the_blocks(i):
    # synchronous rounds split each block at most once, so r splitting rounds reach at most
    # 2 * 2^r blocks; a round that read its own writes could beat this bound
    d = I.cyclic_fib_dfa(i)
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    for delta, k in ((d.delta, d.k), (dc, kc)):
        _, nb, it = oracle.naive(delta, d.accept, d.n, k)
        assert nb == d.n and 2 * 2 ** (it - 1) >= nb


# ---------------------------------------------------------------- reachability and quotient
def _run_word(delta, k, accept, q, word):
    for a in word:
        q = int(delta[q * k + a])
    return bool((int(accept[q >> 5]) >> (q & 31)) & 1)


def _bfs_canonical(delta, accept, n, k, q0):
    """Relabel a fully reachable DFA by first visit in a BFS from q0 taking letters in order:
    two isomorphic DFAs get the same (delta, accept-list)."""
    order, pos = [q0], {q0: 0}
    i = 0
    while i < len(order):
        s = order[i]
        i += 1
        for a in range(k):
            t = int(delta[s * k + a])
            if t not in pos:
                pos[t] = len(order)
                order.append(t)
    assert len(order) == n
    d = [pos[int(delta[s * k + a])] for s in order for a in range(k)]
    acc = [int((int(accept[s >> 5]) >> (s & 31)) & 1) for s in order]
    return d, acc


def test_reachable_hand_example():
    # 0 -> 1 -> 0, 2 loops, 3 -> 0; only 1 accepts; from 0: {0, 1}; 2 and 3 unreachable
    delta = np.array([1, 0, 2, 0], np.int32)
    acc = I.pack_bits(np.array([0, 1, 0, 0], bool))
    newid, cnt = oracle.reachable(delta, 4, 1, 0)
    assert cnt == 2 and newid.tolist() == [0, 1, -1, -1]
    qd, qa, nb, q0, nr = oracle.minimal_dfa(delta, acc, 4, 1, 0)
    assert (nb, q0, nr) == (2, 0, 2) and qd.tolist() == [1, 0] and int(qa[0]) == 0b10
    # from 3: 3 -> 0 -> 1 -> 0 ...; a from 3 rejects but a from 0 accepts, so 3, 0 and 1 are
    # pairwise distinguishable: three states, renumbered 0 (was 0), 1 (was 1), 2 (was 3)
    qd, qa, nb, q0, nr = oracle.minimal_dfa(delta, acc, 4, 1, 3)
    assert (nb, nr, q0) == (3, 3, 2) and qd.tolist() == [1, 0, 0] and int(qa[0]) == 0b010


def test_reachable_union_and_degenerate_cases():
    # a single cycle (Fib) next to a random DFA: from a cycle state exactly the cycle is reached
    a = I.cyclic_fib_dfa(10)
    b = I.random_dfa(500, 1, 0.5, 3)
    n = a.n + b.n
    delta = np.concatenate([a.delta, b.delta + a.n]).astype(np.int32)
    newid, cnt = oracle.reachable(delta, n, 1, 17)
    assert cnt == a.n and (newid[:a.n] == np.arange(a.n)).all() and (newid[a.n:] == -1).all()
    # bit-splitter from state 0: no letter fires, one reachable state, a one-state minimal DFA
    d = I.bitsplitter_dfa(8)
    qd, qa, nb, q0, nr = oracle.minimal_dfa(d.delta, d.accept, d.n, d.k, 0)
    assert (nb, nr, q0) == (1, 1, 0) and (qd == 0).all() and int(qa[0]) == 0
    # k = 0: only q0 is reachable
    newid, cnt = oracle.reachable(np.zeros(0, np.int32), 5, 0, 2)
    assert cnt == 1 and newid.tolist() == [-1, -1, 0, -1, -1]
    # Fig. 1 from q0 = 0: all 10 states, already minimal
    d = I.fig1_dfa()
    qd, qa, nb, q0, nr = oracle.minimal_dfa(d.delta, d.accept, d.n, d.k, 0)
    assert (nb, nr, q0) == (10, 10, 0) and qd.tolist() == d.delta.tolist()


@pytest.mark.parametrize("seed", range(12))
def test_minimal_dfa_language_and_minimality(seed):
    rng = np.random.default_rng(seed)
    n, k = int(rng.integers(2, 300)), int(rng.integers(1, 4))
    if seed % 3 == 0:
        d = I.inflated_dfa(max(1, n // 4), k, 4, 0.5, seed)[0]
    else:
        d = I.random_dfa(n, k, 0.5, seed)
    # make part of the automaton unreachable: a second copy whose states nothing enters
    n2 = 2 * d.n
    delta = np.concatenate([d.delta, d.delta + d.n]).astype(np.int32)
    acc = I.pack_bits(np.concatenate([I.unpack_bits(d.accept, d.n)] * 2))
    q0 = int(rng.integers(0, d.n))
    qd, qa, nb, q0m, nr = oracle.minimal_dfa(delta, acc, n2, d.k, q0)
    assert nr <= d.n
    # same language: random words from q0 and q0'
    for _ in range(300):
        w = rng.integers(0, d.k, size=int(rng.integers(0, 3 * d.n)))
        assert _run_word(delta, d.k, acc, q0, w) == _run_word(qd, d.k, qa, q0m, w)
    # minimal: every state reachable and no two states equivalent
    assert oracle.reachable(qd, nb, d.k, q0m)[1] == nb
    assert oracle.hopcroft(qd, qa, nb, d.k)[1] == nb
    # unique up to isomorphism (Myhill-Nerode): a permuted copy gives the same canonical form
    perm = rng.permutation(n2).astype(np.int32)
    pd = np.empty_like(delta).reshape(n2, d.k)
    pd[perm] = perm[delta.reshape(n2, d.k)]
    pacc = I.pack_bits(np.array([I.unpack_bits(acc, n2)[np.argsort(perm)][i]
                                 for i in range(n2)], bool))
    qd2, qa2, nb2, q0m2, nr2 = oracle.minimal_dfa(pd.reshape(-1), pacc, n2, d.k, int(perm[q0]))
    assert (nb2, nr2) == (nb, nr)
    assert _bfs_canonical(qd, qa, nb, d.k, q0m) == _bfs_canonical(qd2, qa2, nb2, d.k, q0m2)


def test_table1_trans_iterations_are_log_of_distinguishing_depth():
    # Alg. 1 (trans) doubles the length of the words it has examined every iteration, so its
    # iteration count on cyclic Fib is ceil(log2 D) for the deepest distinguishing word D; the
    # table-filling oracle measures D round by round (D = N - 2 on cyclic Fib)
    import math
    for name, N, iters in _read_golden("table1_rows.txt"):
        i = int(name[3:])
        d = I.cyclic_fib_dfa(i + 1)
        assert d.n == int(N)
        _, nb, rounds = oracle.tablefill(d.delta, d.accept, d.n, d.k)
        assert nb == d.n and rounds == d.n - 2
        assert math.ceil(math.log2(rounds)) == int(iters)


def test_bench_table2_context_matches_golden_rows():
    # the benchmark's copy of Table 2 (sizes and alphabets) agrees with the transcribed rows
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench_workloads
    rows = {r[0]: r for r in _read_golden("table2_rows.txt")}
    checked = 0
    for name, (N, k, *_times) in bench_workloads.TABLE2.items():
        if name in rows:
            assert int(rows[name][1]) == N and int(rows[name][2]) == k
            checked += 1
    assert checked >= 10

"""Checks of the seeded input generators against their published definitions."""
import numpy as np
import pytest

from paper_2410_22764_gb300 import inputs as I


def test_splitmix64_matches_published_stream():
    # first outputs of the splitmix64 reference generator seeded with 0 (Vigna's splitmix64.c)
    got = [int(v) for v in I.splitmix64(0, np.arange(3))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_is_counter_based():
    a = I.splitmix64(12345, np.arange(1000))
    b = I.splitmix64(12345, np.arange(500, 1000))
    assert (a[500:] == b).all()


def test_bounded_is_exact_multiply_shift():
    x = I.splitmix64(99, np.arange(2000))
    for m in (1, 2, 3, 10, 1000, 10_000_000, (1 << 32) - 1):
        got = I.bounded(x, m)
        want = np.array([(int(v) * m) >> 64 for v in x], dtype=np.uint64)
        assert (got == want).all()


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(0)
    for n in (1, 31, 32, 33, 1000):
        f = rng.random(n) < 0.5
        assert (I.unpack_bits(I.pack_bits(f), n) == f).all()
        w = I.pack_bits(f)
        for s in range(n):
            assert ((int(w[s >> 5]) >> (s & 31)) & 1) == int(f[s])


def test_random_dfa_shape_and_range():
    d = I.random_dfa(1000, 2, 0.5, 1)
    assert d.delta.dtype == np.int32 and d.delta.size == 2000
    assert d.delta.min() >= 0 and d.delta.max() < 1000
    frac = d.accepting().mean()
    assert 0.4 < frac < 0.6


def test_inflated_dfa_structure():
    d, base = I.inflated_dfa(100, 3, 5, 0.5, 2)
    assert d.n == 500
    perm = I.seeded_permutation(500, 2)
    assert sorted(perm.tolist()) == list(range(500))
    inv = np.empty(500, np.int64)
    inv[perm] = np.arange(500)
    raw_of = inv  # raw index of each id
    for ident in range(0, 500, 13):
        s = raw_of[ident] // 5
        for a in range(3):
            succ = d.delta[ident * 3 + a]
            assert raw_of[succ] // 5 == base.delta[s * 3 + a]
        assert d.accepting()[ident] == base.accepting()[s]


def test_batch_sizes_ranges():
    ns, ks, ps, seeds = I.batch_sizes(4096, 1)
    assert ns.min() >= 100 and ns.max() <= 1_000_000
    assert ks.min() >= 2 and ks.max() <= 26
    assert ps.min() >= 0.1 and ps.max() <= 0.9
    cap = I.batch_cap_for_transitions(4096, 1, 200_000_000)
    ns2, ks2, _, _ = I.batch_sizes(4096, 1, n_cap=cap)
    assert (ns2 * ks2).sum() >= 200_000_000
    ns3, ks3, _, _ = I.batch_sizes(4096, 1, n_cap=cap - 1)
    assert (ns3 * ks3).sum() < 200_000_000


def test_native_batch_generator_matches_numpy():
    ns, ks, ps, seeds = I.batch_sizes(40, 7, n_lo=1, n_hi=3000, k_lo=0, k_hi=6)
    delta, acc, state_off, kk = I.random_batch(ns, ks, ps, seeds, threads=3)
    for i in range(40):
        want = I.random_dfa(int(ns[i]), int(ks[i]), float(ps[i]), int(seeds[i]))
        got = I.batch_member(delta, acc, state_off, kk, i)
        assert got.n == want.n and got.k == want.k
        assert np.array_equal(got.delta, want.delta)
        assert np.array_equal(got.accepting(), want.accepting())


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_native_bitsplitter_matches_numpy(threads):
    for nbits in range(2, 15):
        a = I.bitsplitter_dfa(nbits)
        b = I.bitsplitter_dfa_native(nbits, threads=threads)
        assert (a.n, a.k) == (b.n, b.k)
        assert np.array_equal(a.delta, b.delta) and np.array_equal(a.accept, b.accept)

"""GPU path vs CPU oracle, element by element (bit-exact: all outputs are integers).

Every case runs the CUDA library through the C ABI (``dfamin_minimize_ex`` via the ctypes
binding) and compares out_block, nblocks and the pass count with the oracle on the same
seeded inputs.
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


def run(dm, d, **kw):
    return dm.minimize_host(d.n, d.k, d.delta, d.accept, **kw)


def check(dm, d, closure=False, flags=0, ctas=0, smem_states=0):
    want, wn, wp = oracle.moore(d.delta, d.accept, d.n, d.k)
    if closure:
        dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
        _, _, wp = oracle.moore(dc, d.accept, d.n, kc)
    dlt, acc = dm.to_device(d.delta, d.accept)
    r = dm.minimize_ex(d.n, d.k, dlt, acc,
                       opt=dm.options(closure=closure, flags=flags, ctas=ctas,
                                      smem_states=smem_states))
    got, gn, gp, st = r.host()
    assert st == 0, dm.status_string(st)
    assert gn == wn
    assert np.array_equal(got, want)
    assert gp == wp
    return gp


SIZES = [1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4095, 4096, 4097, 8191, 8193, 20000, 65537]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 7])
def test_random_sizes_ragged(dm, n, k):
    for p in (0.5, 0.0) if n < 300 else (0.5,):
        check(dm, I.random_dfa(n, k, p, 1000 + n + k))


@pytest.mark.parametrize("n", [100, 5000, 30000])
def test_large_alphabet(dm, n):
    check(dm, I.random_dfa(n, 26, 0.3, 5))


def test_random1k_against_three_oracles(dm):
    # random complete DFA, n = 1000, k = 2, p = 0.5, seed 1
    d = I.random_dfa(1000, 2, 0.5, 1)
    got, gn, gp, st = run(dm, d)
    m, mn, mp = oracle.moore(d.delta, d.accept, d.n, d.k)
    h, hn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    t, tn, rounds = oracle.tablefill(d.delta, d.accept, d.n, d.k)
    assert st == 0 and gn == mn == hn == tn
    assert np.array_equal(got, m) and np.array_equal(got, h) and np.array_equal(got, t)
    assert gp == mp == rounds + (1 if mn < d.n else 0)


@pytest.mark.parametrize("permute", [True, False])
@pytest.mark.parametrize("m,k,c", [(300, 2, 4), (2000, 4, 10), (20000, 3, 4)])
def test_inflated(dm, m, k, c, permute):
    d, base = I.inflated_dfa(m, k, c, 0.5, 7, permute=permute)
    check(dm, d)
    _, bn = oracle.hopcroft(base.delta, base.accept, m, k)
    assert run(dm, d)[1] == bn


@pytest.mark.parametrize("i", [5, 10, 14, 17])
def test_cyclic_fibonacci(dm, i):
    d = I.cyclic_fib_dfa(i)
    assert check(dm, d) == d.n - 2
    check(dm, d, closure=True)


@pytest.mark.parametrize("nbits", [3, 8, 12, 15])
def test_bitsplitter(dm, nbits):
    d = I.bitsplitter_dfa(nbits)
    assert check(dm, d) == nbits - 1
    if nbits <= 12:
        check(dm, d, closure=True)


def test_fig1(dm):
    d = I.fig1_dfa()
    assert check(dm, d) == 8
    assert check(dm, d, closure=True) < 8


@pytest.mark.parametrize("n", [2, 3, 10, 257, 1000, 4096, 9000, 50000])
def test_path_plain_and_closure(dm, n):
    d = I.path_fib_dfa(n)
    if n <= 9000:
        check(dm, d)
    check(dm, d, closure=True)
    check(dm, d, closure=True, flags=dm.FLAG_KEEP_IDENTITY)


@pytest.mark.parametrize("flags", [2, 4])
@pytest.mark.parametrize("n", [700, 6000, 30000])
def test_degenerate_hash_needs_full_tuple_check(dm, flags, n):
    # with the hash reduced to the old block id (2) or a constant (4) every regrouping probe
    # collides; results must stay bit-exact because equality is decided on the full signature
    if flags == 4 and n > 6000:
        n = 6000
    d, _ = I.inflated_dfa(n // 4, 3, 4, 0.5, 3)
    check(dm, d, flags=flags)
    check(dm, I.random_dfa(n, 2, 0.5, 9), flags=flags)


@pytest.mark.parametrize("ctas", [1, 2, 7, 64])
def test_team_sizes(dm, ctas):
    # the multi-CTA kernel at several team sizes, including one CTA, forced past the
    # shared-memory kernel
    d, _ = I.inflated_dfa(3000, 3, 4, 0.5, 11)
    check(dm, d, ctas=ctas, smem_states=1)
    check(dm, I.random_dfa(777, 2, 0.5, 3), ctas=ctas, smem_states=1)


def test_smem_threshold_both_paths_agree(dm):
    d = I.random_dfa(4000, 3, 0.5, 21)
    a = check(dm, d, smem_states=8192)
    b = check(dm, d, smem_states=1)
    assert a == b


def test_out_of_range_delta_reports_einval(dm):
    for n in (50, 20000):
        d = I.random_dfa(n, 2, 0.5, 1)
        bad = d.delta.copy()
        bad[n] = n + 5          # out of range: must be reported, never dereferenced
        bad2 = d.delta.copy()
        bad2[-1] = -1
        for b in (bad, bad2):
            got, gn, gp, st = dm.minimize_host(n, 2, b, d.accept)
            assert st == dm.EINVAL and gn == -dm.EINVAL
        # the context stays usable
        check(dm, d)


def test_pass_cap_reports_noconverge(dm):
    d = I.cyclic_fib_dfa(12)
    for smem in (0, 1):
        dlt, acc = dm.to_device(d.delta, d.accept)
        r = dm.minimize_ex(d.n, d.k, dlt, acc,
                           opt=dm.options(max_passes=5, smem_states=smem))
        _, gn, gp, st = r.host()
        assert st == dm.ENOCONVERGE and gp == 5 and gn == -dm.ENOCONVERGE


def test_simple_entry_point(dm):
    d = I.random_dfa(30000, 4, 0.5, 2)
    dlt, acc = dm.to_device(d.delta, d.accept)
    out, nb = dm.minimize(d.n, d.k, dlt, acc)
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    assert int(nb.item()) == wn and np.array_equal(out.cpu().numpy(), want)


def test_workspace_reuse_and_streams(dm):
    ws = dm.Workspace()
    s = torch.cuda.Stream()
    for seed in range(4):
        d = I.random_dfa(12000 + seed, 3, 0.5, seed)
        dlt, acc = dm.to_device(d.delta, d.accept)
        with torch.cuda.stream(s):
            r = dm.minimize_ex(d.n, d.k, dlt, acc, workspace=ws, stream=s)
        s.synchronize()
        got, gn, gp, st = r.host()
        want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
        assert st == 0 and gn == wn and np.array_equal(got, want)


# ---------------------------------------------------------------- leader mode (Alg. 2 naivePR)
def check_leader(dm, d, closure=False, **kw):
    if closure:
        dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
        want, wn, wi = oracle.naive(dc, d.accept, d.n, kc)
    else:
        want, wn, wi = oracle.naive(d.delta, d.accept, d.n, d.k)
    dlt, acc = dm.to_device(d.delta, d.accept)
    r = dm.minimize_ex(d.n, d.k, dlt, acc, opt=dm.options(closure=closure, leader=True, **kw))
    got, gn, gi, st = r.host()
    assert st == 0 and gn == wn and gi == wi and np.array_equal(got, want)
    return gi


@pytest.mark.parametrize("maker", ["rand1", "rand2", "infl", "fib", "bits", "fig1", "path",
                                   "tiny"])
def test_leader_mode_against_naive_oracle(dm, maker):
    d = {"rand1": lambda: I.random_dfa(3000, 3, 0.5, 1),
         "rand2": lambda: I.random_dfa(50000, 12, 0.3, 2),
         "infl": lambda: I.inflated_dfa(5000, 4, 4, 0.5, 3)[0],
         "fib": lambda: I.cyclic_fib_dfa(14),
         "bits": lambda: I.bitsplitter_dfa(12),
         "fig1": I.fig1_dfa,
         "path": lambda: I.path_fib_dfa(3000),
         "tiny": lambda: I.random_dfa(2, 1, 0.5, 5)}[maker]()
    check_leader(dm, d)
    if maker in ("fib", "fig1", "path", "bits", "rand1"):
        check_leader(dm, d, closure=True)             # transPR as Alg. transPR runs it


def test_leader_mode_team_sizes(dm):
    d = I.inflated_dfa(3000, 3, 4, 0.5, 11)[0]
    for ctas in (1, 3, 32):
        check_leader(dm, d, ctas=ctas, smem_states=1)
    check_leader(dm, d, smem_states=65535)            # the one-CTA kernel


@pytest.mark.parametrize("maker", ["fib", "bits", "rand", "path"])
def test_leader_mode_one_cta_and_team_agree(dm, maker):
    d = {"fib": lambda: I.cyclic_fib_dfa(19), "bits": lambda: I.bitsplitter_dfa(13),
         "rand": lambda: I.random_dfa(30000, 2, 0.5, 4), "path": lambda: I.path_fib_dfa(9000)}[maker]()
    a = check_leader(dm, d, smem_states=65535)
    b = check_leader(dm, d, smem_states=1)
    assert a == b


def test_leader_mode_batch(dm):
    from test_gpu_batch import mixed_batch
    dfas = mixed_batch(10, count=30, max_n=20000)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    plan = dm.BatchPlan(state_off, ks, dm.options(leader=True))
    out, per = plan.run(torch.from_numpy(delta).cuda(), torch.from_numpy(acc.view(np.int32)).cuda())
    torch.cuda.synchronize()
    outs, p = plan.split(out.cpu().numpy()), per.cpu().numpy()
    for i, d in enumerate(dfas):
        want, wn, wi = oracle.naive(d.delta, d.accept, d.n, d.k)
        assert p[2, i] == 0 and p[0, i] == wn and p[1, i] == wi and np.array_equal(outs[i], want)


# ---------------------------------------------------------------- closure saturation
def closure_levels_built(dm, d, flags=0, leader=False):
    ws = dm.Workspace()
    opt = dm.options(closure=True, flags=flags | dm.FLAG_TRACE, smem_states=1, leader=leader)
    dlt, acc = dm.to_device(d.delta, d.accept)
    r = dm.minimize_ex(d.n, d.k, dlt, acc, opt=opt, workspace=ws)
    got, gn, gp, st = r.host()
    assert st == 0
    return sum(1 for _, ph, _ in dm.read_trace(ws, d.n, d.k, opt) if ph == "closure"), gp


@pytest.mark.parametrize("nbits", [6, 10, 13])
def test_closure_stops_at_fixed_point_letters(dm, nbits):
    # every bit-splitter letter is idempotent (a^2 = a): one closure level is built, not
    # floor(log2 n); partition and passes still equal Moore on the full A'
    d = I.bitsplitter_dfa(nbits)
    check(dm, d, closure=True)
    lv, gp = closure_levels_built(dm, d)
    assert lv == 1
    lv_all, gp_all = closure_levels_built(dm, d, flags=dm.FLAG_KEEP_IDENTITY)
    assert lv_all == nbits and gp_all == gp


def test_closure_saturation_mixed_letters(dm):
    # letter 0 cycles (never saturates), letter 1 collapses onto a fixed point after a few
    # steps, letter 2 is the identity: results must match the oracle's full closure
    rng = np.random.default_rng(3)
    n = 5000
    delta = np.empty((n, 3), np.int32)
    delta[:, 0] = (np.arange(n) + 1) % n
    delta[:, 1] = np.maximum(np.arange(n) - 7, 0) // 2
    delta[:, 2] = np.arange(n)
    acc = I.pack_bits(rng.random(n) < 0.5)
    d = I.Dfa(n, 3, delta.reshape(-1), acc)
    check(dm, d, closure=True)
    check(dm, d, closure=True, smem_states=1)
    check(dm, d, closure=True, flags=dm.FLAG_KEEP_IDENTITY, smem_states=1)
    check_leader(dm, d, closure=True)
    lv, _ = closure_levels_built(dm, d)
    assert lv == int(np.log2(n))          # letter 0 needs every level


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 9])
@pytest.mark.parametrize("n", [1, 2, 3, 33, 257, 5000])
def test_team_kernel_tiny_and_pattern_round(dm, n, k):
    # the multi-CTA kernel on tiny DFAs (round 1 from acceptance patterns for k <= 8, the
    # general round 1 for k = 9), including all-accepting and all-rejecting DFAs
    for p in (0.5, 0.0, 1.0):
        d = I.random_dfa(n, k, p, 77 * n + k)
        for ctas in (0, 3):
            check(dm, d, ctas=ctas, smem_states=1)


@pytest.mark.parametrize("k", [9, 16, 30, 31, 32, 33])
def test_runtime_width_key_round_boundary(dm, k):
    # round 1 by acceptance keys needs k + 1 <= 32 bits; 31 is the last width it takes
    for n in (3000, 40000):
        d = I.random_dfa(n, k, 0.5, 5 * k + n)
        check(dm, d, smem_states=1)
    d, _ = I.inflated_dfa(2000, k, 4, 0.5, k)
    check(dm, d, smem_states=1)


@pytest.mark.parametrize("nbits", [5, 9, 11])
def test_closure_key_round_on_bitsplitters(dm, nbits):
    # B_n closure rows have k + k columns before the unchanged level is dropped
    d = I.bitsplitter_dfa(nbits)
    check(dm, d, closure=True, smem_states=1)
    check_leader(dm, d, closure=True)


# ---------------------------------------------------------------- one-CTA medium kernel
@pytest.mark.parametrize("n", [4097, 9000, 30001, 65535])
@pytest.mark.parametrize("k", [1, 2, 4, 9])
def test_medium_kernel(dm, n, k):
    # one CTA with 16-bit ids in shared memory, forced by smem_states >= n
    check(dm, I.random_dfa(n, k, 0.5, n + k), smem_states=65535)
    if n <= 30001:
        d, _ = I.inflated_dfa(n // 4, k, 4, 0.5, k, permute=True)
        check(dm, d, smem_states=65535)


@pytest.mark.parametrize("i", [17, 20, 22])
def test_medium_kernel_deep_refinement(dm, i):
    d = I.cyclic_fib_dfa(i)
    assert d.n <= 65535
    assert check(dm, d, smem_states=65535) == d.n - 2
    check(dm, d, closure=True, smem_states=65535)
    check(dm, I.path_fib_dfa(20000), smem_states=65535)


def test_medium_kernel_errors(dm):
    d = I.random_dfa(20000, 2, 0.5, 1)
    bad = d.delta.copy()
    bad[777] = d.n
    dlt, acc = dm.to_device(bad, d.accept)
    r = dm.minimize_ex(d.n, d.k, dlt, acc, opt=dm.options(smem_states=65535))
    _, gn, gp, st = r.host()
    assert st == dm.EINVAL and gn == -dm.EINVAL
    f = I.cyclic_fib_dfa(20)
    dlt, acc = dm.to_device(f.delta, f.accept)
    r = dm.minimize_ex(f.n, f.k, dlt, acc, opt=dm.options(smem_states=65535, max_passes=7))
    _, gn, gp, st = r.host()
    assert st == dm.ENOCONVERGE and gp == 7
    check(dm, d, smem_states=65535)

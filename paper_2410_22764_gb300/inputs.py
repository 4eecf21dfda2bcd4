"""Seeded synthetic DFA generators (inputs only; none of the minimization arithmetic).

Both the GPU path and the CPU oracle consume what these functions return; neither side
generates its own inputs.  Every random value is drawn from a counter-based splitmix64 stream
(Steele, Lea and Flood, OOPSLA 2014): value i of a stream with seed ``x`` is the splitmix64
finalizer applied to ``x + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64), so any element can be
recomputed on its own.  A uniform integer in [0, m) is the high 64 bits of ``value * m``
(Lemire's multiply-shift; bias at most m / 2^64).  A Bernoulli(p) draw is
``(value >> 11) < round(p * 2^53)``.

Families (Sec. 4.1 of arXiv 2410.22764 and the benchmark workloads):

* :func:`random_dfa`     complete DFA with uniform transitions and Bernoulli(p) acceptance.
* :func:`inflated_dfa`   every state of a random base DFA cloned c times; each clone's
                         a-successor is a uniformly chosen clone of the base successor, so every
                         clone is equivalent to its base state.
* :func:`path_fib_dfa`   letter 0 walks i -> i+1 (last state loops), letter 1 loops; state i
                         accepts iff bit i of the infinite Fibonacci word is 1.
* :func:`cyclic_fib_dfa` the automaton Fib_n of Sec. 4.1 (a cycle over the bits of w_n).
* :func:`bitsplitter_dfa` the bit-splitter B_n of Sec. 4.1.
* :func:`fig1_dfa`       the 10-state a-path of Fig. 1.
* :func:`batch_sizes`    the (n, k, p, seed) draws of a batch of random DFAs.

All DFAs are returned as ``Dfa(n, k, delta, accept)`` with ``delta`` int32 state-major
(``delta[s*k + a]``) and ``accept`` a uint32 bitmap, LSB first.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# stream tags: each random quantity of a generator draws from its own stream
TAG_DELTA = 1
TAG_ACCEPT = 2
TAG_CLONE = 3
TAG_PERM = 4
TAG_SIZE = 5
TAG_LETTERS = 6
TAG_PROB = 7
TAG_SEED = 8


@dataclass
class Dfa:
    n: int
    k: int
    delta: np.ndarray   # int32 [n*k], state-major
    accept: np.ndarray  # uint32 [(n+31)//32], LSB-first bitmap

    def accepting(self) -> np.ndarray:
        """Boolean array: state s accepting."""
        return unpack_bits(self.accept, self.n)


def _mix_scalar(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * MIX1) & M64
    z = ((z ^ (z >> 27)) * MIX2) & M64
    return z ^ (z >> 31)


def substream(seed: int, tag: int) -> int:
    """Seed of the stream ``tag`` derived from a user seed."""
    return _mix_scalar((seed & M64) ^ _mix_scalar(tag * GAMMA))


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based splitmix64: element i = finalizer(seed + (i+1)*GAMMA) (uint64)."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & M64)
             + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * np.uint64(GAMMA))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def bounded(x: np.ndarray, m: int) -> np.ndarray:
    """High 64 bits of x*m for uint64 x and 0 < m < 2^32 (uniform in [0, m))."""
    if not 0 < m < (1 << 32):
        raise ValueError("m must be in (0, 2^32)")
    x = np.asarray(x, dtype=np.uint64)
    mm = np.uint64(m)
    with np.errstate(over="ignore"):
        lo = (x & np.uint64(0xFFFFFFFF)) * mm
        hi = (x >> np.uint64(32)) * mm
        return (hi + (lo >> np.uint64(32))) >> np.uint64(32)


def unit_double(x: np.ndarray) -> np.ndarray:
    """(x >> 11) * 2^-53 in [0, 1)."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def bernoulli(x: np.ndarray, p: float) -> np.ndarray:
    thr = np.uint64(min(max(int(round(p * (1 << 53))), 0), 1 << 53))
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)) < thr


def pack_bits(flags: np.ndarray) -> np.ndarray:
    """Boolean array -> uint32 bitmap, bit s of word s>>5 (LSB first)."""
    flags = np.asarray(flags, dtype=bool)
    n = flags.size
    words = (n + 31) // 32
    padded = np.zeros(words * 32, dtype=np.uint32)
    padded[:n] = flags
    shifts = np.arange(32, dtype=np.uint32)
    return (padded.reshape(words, 32) << shifts).sum(axis=1, dtype=np.uint64).astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32)
    shifts = np.arange(32, dtype=np.uint32)
    bits = (words[:, None] >> shifts) & np.uint32(1)
    return bits.reshape(-1)[:n].astype(bool)


def random_dfa(n: int, k: int, p: float, seed: int) -> Dfa:
    """Uniform complete DFA: delta[s*k+a] uniform in [0, n); state s accepts w.p. p."""
    if n < 1 or k < 0:
        raise ValueError("need n >= 1 and k >= 0")
    idx = np.arange(n * k, dtype=np.uint64)
    delta = bounded(splitmix64(substream(seed, TAG_DELTA), idx), n).astype(np.int32)
    acc = bernoulli(splitmix64(substream(seed, TAG_ACCEPT), np.arange(n, dtype=np.uint64)), p)
    return Dfa(n, k, delta, pack_bits(acc))


def seeded_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded permutation of [0, n): the stable argsort of n splitmix64 keys."""
    keys = splitmix64(substream(seed, TAG_PERM), np.arange(n, dtype=np.uint64))
    return np.argsort(keys, kind="stable").astype(np.int64)


def inflated_dfa(m: int, k: int, c: int, p: float, seed: int, permute: bool = True,
                 base: Dfa | None = None) -> tuple[Dfa, Dfa]:
    """Clone every state of a random base DFA c times (n = m*c).

    Clone j of base state s has raw index r = s*c + j and id pi[r] (pi a seeded permutation,
    or the identity when ``permute`` is False).  Its a-successor is clone
    ``uniform[0, c)`` of delta_base(s, a); it accepts iff s does.  Returns (dfa, base).
    """
    if base is None:
        base = random_dfa(m, k, p, seed)
    n = m * c
    raw = np.arange(n, dtype=np.int64)
    ident = seeded_permutation(n, seed) if permute else raw
    s_of = raw // c
    choice = bounded(splitmix64(substream(seed, TAG_CLONE), np.arange(n * k, dtype=np.uint64)),
                     c).astype(np.int64).reshape(n, k)
    base_succ = base.delta.astype(np.int64).reshape(m, k)[s_of]          # [n, k]
    succ = ident[base_succ * c + choice]                                  # ids of successors
    delta = np.empty((n, k), dtype=np.int32)
    delta[ident] = succ
    acc = np.empty(n, dtype=bool)
    acc[ident] = base.accepting()[s_of]
    return Dfa(n, k, delta.reshape(-1), pack_bits(acc)), base


def fibonacci_word(length: int) -> np.ndarray:
    """First ``length`` bits of the infinite Fibonacci word (w_1 = 0, w_{i+1} = w_i w_{i-1},
    so every w_i with i >= 1 is a prefix of the next): 0100101001001...  Built by integer
    concatenation only."""
    prev, cur = [1], [0]          # w_0, w_1
    while len(cur) < length:
        prev, cur = cur, cur + prev
    return np.array(cur[:length], dtype=np.uint8)


def fibonacci_word_n(i: int) -> np.ndarray:
    """The finite word w_i of Sec. 4.1 (w_0 = 1, w_1 = 0, w_{i+1} = w_i w_{i-1})."""
    words = [[1], [0]]
    while len(words) <= i:
        words.append(words[-1] + words[-2])
    return np.array(words[i], dtype=np.uint8)


def path_fib_dfa(n: int) -> Dfa:
    """Deep-refinement path: delta(i,0) = min(i+1, n-1), delta(i,1) = i, F = {i : fib[i] = 1}."""
    i = np.arange(n, dtype=np.int64)
    delta = np.empty((n, 2), dtype=np.int32)
    delta[:, 0] = np.minimum(i + 1, n - 1)
    delta[:, 1] = i
    return Dfa(n, 2, delta.reshape(-1), pack_bits(fibonacci_word(n).astype(bool)))


def cyclic_fib_dfa(i: int) -> Dfa:
    """Fib_i of Sec. 4.1: states q_0..q_{N-1} with N = |w_i|, delta(q_j, a) = q_{(j+1) mod N},
    F = {q_j : w_i[j] = 1}."""
    w = fibonacci_word_n(i)
    n = w.size
    delta = ((np.arange(n, dtype=np.int64) + 1) % n).astype(np.int32)
    return Dfa(n, 1, delta, pack_bits(w.astype(bool)))


def bitsplitter_dfa(nbits: int) -> Dfa:
    """Bit-splitter B_n of Sec. 4.1 with 2^n states and n-1 letters.

    A state is a bit string b_{n-1} ... b_0, stored as the integer with b_{n-1} the most
    significant bit (the string's first bit).  Letter a_m (column m-1, m = 1..n-1) is the
    fresh letter of B_{m+1} and acts on the low m+1 bits: with b = bit m and sigma[0] = bit
    m-1, the low m+1 bits become (not b) followed by m zeros if bit m-1 is 1, and stay
    unchanged otherwise.  Higher bits are kept.  F = {states whose first bit is 1}.
    """
    if nbits < 1:
        raise ValueError("nbits >= 1")
    if nbits >= 16:
        return bitsplitter_dfa_native(nbits)
    n = 1 << nbits
    k = nbits - 1
    x = np.arange(n, dtype=np.int64)
    delta = np.empty((n, max(k, 1)), dtype=np.int64)
    for m in range(1, nbits):
        low_mask = (1 << (m + 1)) - 1
        b = (x >> m) & 1
        trigger = ((x >> (m - 1)) & 1) == 1
        jumped = (x & ~low_mask) | ((1 - b) << m)
        delta[:, m - 1] = np.where(trigger, jumped, x)
    acc = ((x >> (nbits - 1)) & 1) == 1
    return Dfa(n, k, delta[:, :k].astype(np.int32).reshape(-1), pack_bits(acc))


def bitsplitter_dfa_native(nbits: int, threads: int | None = None) -> Dfa:
    """bitsplitter_dfa built by the multithreaded C generator (B_26 has 67M states)."""
    import ctypes
    import os
    n, k = 1 << nbits, nbits - 1
    delta = np.empty(n * k, dtype=np.int32)
    accept = np.empty((n + 31) // 32, dtype=np.uint32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = _native().inputs_bitsplitter(nbits, p(delta), p(accept),
                                      threads or max(1, os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError(f"inputs_bitsplitter failed ({rc})")
    return Dfa(n, k, delta, accept)


def lts_synthetic(n: int, nlabels: int, p_edge: float, p_nd: float, seed: int):
    """A seeded LTS with bounded powerset growth, standing in for the VLTS inputs of Sec. 4.1.

    A partial deterministic system on n states (edge s -a-> t present with probability p_edge,
    t uniform) is doubled into states 0..2n-1 (state s + n mirrors s); each edge s -a-> t of
    the first copy also gets, with probability p_nd, the nondeterministic alternative
    s -a-> t + n.  Reachable subsets are singletons and mirror pairs {t, t + n}, so the DFA has at
    most 3n + 1 states.  Returns (2n, src, lbl, dst) with int32 arrays."""
    rng = np.random.default_rng(seed)
    s = np.repeat(np.arange(n, dtype=np.int64), nlabels)
    a = np.tile(np.arange(nlabels, dtype=np.int64), n)
    keep = rng.random(s.size) < p_edge
    s, a = s[keep], a[keep]
    t = rng.integers(0, n, s.size)
    nd = rng.random(s.size) < p_nd
    src = np.concatenate([s, s + n, s[nd]])
    lbl = np.concatenate([a, a, a[nd]])
    dst = np.concatenate([t, t + n, t[nd] + n])
    order = rng.permutation(src.size)
    return (2 * n, src[order].astype(np.int32), lbl[order].astype(np.int32),
            dst[order].astype(np.int32))


def fig1_dfa() -> Dfa:
    """Fig. 1: q0 -a-> q1 -a-> ... -a-> q9, q9 loops on a and is the only accepting state."""
    delta = np.minimum(np.arange(10) + 1, 9).astype(np.int32)
    acc = np.zeros(10, dtype=bool)
    acc[9] = True
    return Dfa(10, 1, delta, pack_bits(acc))


def batch_sizes(count: int, seed: int, n_lo: int = 100, n_hi: int = 1_000_000,
                k_lo: int = 2, k_hi: int = 26, p_lo: float = 0.1, p_hi: float = 0.9,
                n_cap: int | None = None):
    """Draws for a batch of random DFAs: n log-uniform in [n_lo, n_hi] (rounded), k uniform
    in {k_lo..k_hi}, p uniform in [p_lo, p_hi], and a per-DFA seed.  ``n_cap`` clips n."""
    i = np.arange(count, dtype=np.uint64)
    u = unit_double(splitmix64(substream(seed, TAG_SIZE), i))
    lo, hi = math.log10(n_lo), math.log10(n_hi)
    ns = np.rint(10.0 ** (lo + (hi - lo) * u)).astype(np.int64)
    if n_cap is not None:
        ns = np.minimum(ns, n_cap)
    ks = (k_lo + bounded(splitmix64(substream(seed, TAG_LETTERS), i),
                         k_hi - k_lo + 1)).astype(np.int64)
    ps = p_lo + (p_hi - p_lo) * unit_double(splitmix64(substream(seed, TAG_PROB), i))
    seeds = splitmix64(substream(seed, TAG_SEED), i)
    return ns, ks, ps, seeds


def batch_cap_for_transitions(count: int, seed: int, target: int, **kw) -> int:
    """Smallest n_cap (by bisection) for which sum(n_i * k_i) of the capped draws reaches
    ``target`` transitions."""
    lo, hi = 1, kw.get("n_hi", 1_000_000)
    while lo < hi:
        mid = (lo + hi) // 2
        ns, ks, _, _ = batch_sizes(count, seed, n_cap=mid, **kw)
        if int((ns * ks).sum()) >= target:
            hi = mid
        else:
            lo = mid + 1
    return lo


# ------------------------------------------------------------------------------------------
# Batches of random DFAs, generated by the multithreaded C version of the same streams
# ------------------------------------------------------------------------------------------
_NATIVE = None


def _native():
    """Build (gcc, once) and load inputs_native.c."""
    global _NATIVE
    if _NATIVE is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "inputs_native.c")
        out_dir = os.path.join(here, "_build")
        lib = os.path.join(out_dir, "libinputs.so")
        os.makedirs(out_dir, exist_ok=True)
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp,
                            src], check=True)
            os.replace(tmp, lib)
        h = ctypes.CDLL(lib)
        h.inputs_random_batch.restype = ctypes.c_int
        h.inputs_random_batch.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 8 + [ctypes.c_int32]
        h.inputs_bitsplitter.restype = ctypes.c_int
        h.inputs_bitsplitter.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32]
        _NATIVE = h
    return _NATIVE


def random_batch(ns, ks, ps, seeds, threads: int | None = None):
    """Concatenated batch of random DFAs, DFA i being random_dfa(ns[i], ks[i], ps[i], seeds[i]).

    Returns (delta int32, accept uint32 bitmap over the concatenated states, state_off int64,
    ks int32): the layout of the batch C ABI (successor ids local to each DFA)."""
    import ctypes
    import os
    ns = np.asarray(ns, dtype=np.int64)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    count = ns.size
    state_off = np.zeros(count + 1, dtype=np.int64)
    state_off[1:] = np.cumsum(ns)
    delta_off = np.zeros(count + 1, dtype=np.int64)
    delta_off[1:] = np.cumsum(ns * ks.astype(np.int64))
    sub_d = np.array([substream(int(s), TAG_DELTA) for s in seeds], dtype=np.uint64)
    sub_a = np.array([substream(int(s), TAG_ACCEPT) for s in seeds], dtype=np.uint64)
    thr = np.array([min(max(int(round(float(p) * (1 << 53))), 0), 1 << 53) for p in ps],
                   dtype=np.uint64)
    delta = np.empty(int(delta_off[-1]), dtype=np.int32)
    accept = np.empty((int(state_off[-1]) + 31) // 32, dtype=np.uint32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = _native().inputs_random_batch(count, p(state_off), p(delta_off), p(ks), p(sub_d),
                                       p(sub_a), p(thr), p(delta), p(accept),
                                       threads or max(1, os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError(f"inputs_random_batch failed ({rc})")
    return delta, accept, state_off, ks


def batch_member(delta, accept, state_off, ks, i: int) -> Dfa:
    """DFA i of a concatenated batch, as a standalone Dfa."""
    n, k = int(state_off[i + 1] - state_off[i]), int(ks[i])
    doff = int(np.sum((state_off[1:i + 1] - state_off[:i]) * ks[:i].astype(np.int64)))
    lo, hi = int(state_off[i]), int(state_off[i + 1])
    w0, w1 = lo // 32, (hi + 31) // 32
    bits = unpack_bits(accept[w0:w1], (w1 - w0) * 32)[lo - 32 * w0: hi - 32 * w0]
    return Dfa(n, k, delta[doff: doff + n * k].copy(), pack_bits(bits))

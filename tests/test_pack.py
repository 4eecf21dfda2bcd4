"""Host packing of batches (no GPU): the batch layout of the C ABI is every DFA's rows one after
the other and one acceptance bitmap over all states, DFA i's state q at bit state_off[i] + q.
The word-shifting packer is checked against that definition written bit by bit."""
import numpy as np
import pytest
import torch

from paper_2410_22764_gb300 import dfamin
from paper_2410_22764_gb300 import inputs as I


class _D:
    def __init__(self, n, k, delta, accept):
        self.n, self.k, self.delta, self.accept = n, k, delta, accept


def _bits(d):
    a = np.ascontiguousarray(d.accept, dtype=np.uint32)
    return np.unpackbits(a.view(np.uint8), bitorder="little")[: d.n]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pack_batch_matches_bitwise_definition(seed):
    rng = np.random.default_rng(seed)
    sizes = list(rng.integers(1, 200, 30)) + [32, 64, 31, 33, 1, 96]
    dfas = []
    for i, n in enumerate(sizes):
        n = int(n)
        k = int(rng.integers(1, 6))
        d = I.random_dfa(n, k, float(rng.uniform(0.1, 0.9)), 100 * seed + i)
        acc = np.ascontiguousarray(d.accept, dtype=np.uint32).copy()
        if n % 32:                                   # garbage above n must not leak
            acc[-1] |= np.uint32(~((1 << (n % 32)) - 1) & 0xFFFFFFFF)
        dfas.append(_D(n, k, d.delta, acc))
    delta, accept, state_off, ks = dfamin.pack_batch(dfas)
    assert list(ks) == [d.k for d in dfas]
    assert state_off[0] == 0 and list(np.diff(state_off)) == [d.n for d in dfas]
    assert np.array_equal(delta, np.concatenate([np.asarray(d.delta).reshape(-1) for d in dfas]))
    want = np.concatenate([_bits(d) for d in dfas])
    got = np.unpackbits(accept.view(np.uint8), bitorder="little")
    assert accept.size == (want.size + 31) // 32
    assert np.array_equal(got[: want.size], want) and not got[want.size:].any()


def test_pack_batch_into_preallocated_buffers():
    dfas = [I.random_dfa(n, 3, 0.5, n) for n in (5, 40, 77, 128)]
    ref = dfamin.pack_batch(dfas)
    nd = sum(d.n * d.k for d in dfas)
    words = (sum(d.n for d in dfas) + 31) // 32
    dbuf = np.full(nd + 7, -1, dtype=np.int32)
    abuf = np.full(words + 3, -1, dtype=np.int32)         # stale contents are overwritten
    delta, accept, _, _ = dfamin.pack_batch(dfas, dbuf, abuf)
    assert np.shares_memory(delta, dbuf) and np.shares_memory(accept, abuf)
    assert np.array_equal(delta, ref[0]) and np.array_equal(accept, ref[1])


def test_pack_batch_rows_copied_by_torch():
    dfas = [I.random_dfa(n, k, 0.5, n + k) for n, k in ((3, 2), (500, 4), (64, 1), (1000, 3))]
    ref = dfamin.pack_batch(dfas)
    nd = sum(d.n * d.k for d in dfas)
    buf = torch.full((nd + 5,), -1, dtype=torch.int32)
    delta, accept, state_off, ks = dfamin.pack_batch(dfas, buf)
    assert np.array_equal(delta, ref[0]) and np.array_equal(buf[:nd].numpy(), ref[0])
    assert np.array_equal(accept, ref[1]) and np.array_equal(state_off, ref[2])

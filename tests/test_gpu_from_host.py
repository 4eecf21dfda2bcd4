"""End-to-end calls from host arrays (dfamin_minimize_from_host), on the GPU through the C ABI.

Each case runs with page-locked host arrays (round 1 reads the rows from host memory and the
labels are written straight back, where the kernel allows it) and with pageable ones (copies
around the kernel), and must give exactly the result of the device-array entry point
dfamin_minimize_ex and of the oracle (all outputs are integers: bit-exact).
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


def _host(d, pinned, offset=0):
    """Host tensors for d; `offset` ints of padding before the rows (unaligned rows)."""
    buf = torch.zeros(d.delta.size + offset + 1, dtype=torch.int32)
    delta = buf[offset: offset + d.delta.size]
    delta.copy_(torch.from_numpy(np.ascontiguousarray(d.delta, np.int32)))
    acc = torch.from_numpy(np.ascontiguousarray(d.accept, np.uint32).view(np.int32).copy())
    out = torch.full((d.n,), -7, dtype=torch.int32)
    sc = torch.full((3,), -7, dtype=torch.int32)
    if pinned:
        buf = buf.pin_memory()
        delta = buf[offset: offset + d.delta.size]
        acc, out, sc = acc.pin_memory(), out.pin_memory(), sc.pin_memory()
    return delta, acc, out, sc


def from_host(dm, d, pinned, offset=0, ws=None, **kw):
    delta, acc, out, sc = _host(d, pinned, offset)
    s = torch.cuda.Stream()
    dm.minimize_from_host(d.n, d.k, delta, acc, out, sc, opt=dm.options(**kw), workspace=ws,
                          stream=s)
    s.synchronize()
    return out.numpy().copy(), sc.tolist()


def device_call(dm, d, **kw):
    dd, aa = dm.to_device(d.delta, d.accept)
    got, nb, ps, st = dm.minimize_ex(d.n, d.k, dd, aa, opt=dm.options(**kw)).host()
    return got, [nb, ps, st]


CASES = {
    "multi_cta_k4": (lambda: I.inflated_dfa(100_000, 4, 10, 0.5, 1)[0], {}),
    "multi_cta_k3": (lambda: I.random_dfa(200_000, 3, 0.5, 2), {}),
    "multi_cta_k1": (lambda: I.cyclic_fib_dfa(19), {"smem_states": 1}),
    "multi_cta_k8": (lambda: I.random_dfa(90_000, 8, 0.4, 3), {}),
    "runtime_width_k9": (lambda: I.random_dfa(50_000, 9, 0.5, 4), {}),
    "closure": (lambda: I.path_fib_dfa(20_000), {"closure": True}),
    "one_cta_shared": (lambda: I.random_dfa(1000, 2, 0.5, 5), {}),
    "one_cta_medium": (lambda: I.random_dfa(30_000, 2, 0.5, 6), {}),
    "no_letters": (lambda: I.random_dfa(5000, 0, 0.5, 7), {}),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pinned", [True, False])
def test_from_host_matches_device_call_and_oracle(dm, name, pinned):
    make, kw = CASES[name]
    d = make()
    want, wsc = device_call(dm, d, **kw)
    assert wsc[2] == 0
    got, sc = from_host(dm, d, pinned, **kw)
    assert sc == wsc
    assert np.array_equal(got, want)
    if d.n <= 200_000 and not kw.get("closure"):
        o, on, op = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert np.array_equal(got, o) and sc[:2] == [on, op]


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_pinned_rows(dm, offset):
    # rows that do not start on the vector-load boundary are copied instead of read in place
    d = I.inflated_dfa(20_000, 4, 10, 0.5, 8)[0]
    want, wsc = device_call(dm, d)
    got, sc = from_host(dm, d, True, offset=offset)
    assert sc == wsc and np.array_equal(got, want)


def test_bad_row_from_host_reports_einval(dm):
    d = I.random_dfa(300_000, 4, 0.5, 9)
    bad = d.delta.copy()
    bad[123_457] = d.n + 3
    b = I.Dfa(d.n, d.k, bad, d.accept)
    for pinned in (True, False):
        _, sc = from_host(dm, b, pinned)
        assert sc[2] == dm.EINVAL and sc[0] == -dm.EINVAL
    got, sc = from_host(dm, d, True)                      # the context stays usable
    want, wsc = device_call(dm, d)
    assert sc == wsc and np.array_equal(got, want)


def test_workspace_reuse_across_calls(dm):
    ws = dm.Workspace()
    for seed, (n, k) in enumerate([(400_000, 4), (3000, 2), (250_000, 2), (400_000, 4)]):
        d = I.random_dfa(n, k, 0.5, 20 + seed)
        want, wsc = device_call(dm, d)
        got, sc = from_host(dm, d, True, ws=ws)
        assert sc == wsc and np.array_equal(got, want)

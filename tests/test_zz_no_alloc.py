"""The scratch-free entry point dfamin_minimize_static, called through the C ABI.

Some callers cannot allocate device memory (their host owns the whole device-memory budget, or
cannot afford cudaMalloc's implicit synchronisation); dfamin_minimize_static serves them from a
fixed scratch array inside the library.  This test checks that it gives exactly the result of the
workspace entry point dfamin_minimize_ex (all outputs are integers, so the comparison is
bit-exact), on several calls in a row that reuse the same scratch array, and that a problem too
large for the array is refused before anything runs.  The file sorts last so that a failure here
comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_22764_gb300 import inputs

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _static_call(dm, d, opt):
    dd, aa = dm.to_device(d.delta, d.accept)
    out = torch.full((d.n,), -7, dtype=torch.int32, device="cuda")
    sc = torch.full((3,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = dm.lib().dfamin_minimize_static(
        d.n, d.k, _ptr(dd), _ptr(aa), _ptr(out), _ptr(sc), ctypes.byref(opt),
        ctypes.c_void_p(sc.data_ptr() + 4), ctypes.c_void_p(sc.data_ptr() + 8),
        ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, dm.status_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy(), sc.cpu().tolist()


def _workspace_call(dm, d, opt):
    dd, aa = dm.to_device(d.delta, d.accept)
    r = dm.minimize_ex(d.n, d.k, dd, aa, opt=opt)
    got, nb, ps, st = r.host()
    return got, [nb, ps, st]


def test_static_scratch_matches_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin as dm
    calls = [
        (inputs.inflated_dfa(50_000, 4, 4, 0.5, 3)[0], dm.options()),      # multi-CTA kernel
        (inputs.random_dfa(300_000, 2, 0.5, 8), dm.options()),             # other n, k
        (inputs.random_dfa(1000, 3, 0.5, 5), dm.options()),                # one-CTA kernel
        (inputs.path_fib_dfa(20_000), dm.options(closure=True)),           # closure columns
        (inputs.inflated_dfa(50_000, 4, 4, 0.5, 3)[0], dm.options()),      # first problem again
    ]
    for d, opt in calls:
        got, sc = _static_call(dm, d, opt)
        want, wsc = _workspace_call(dm, d, opt)
        assert sc[2] == 0 and wsc[2] == 0
        assert sc == wsc
        assert np.array_equal(got, want)


def test_static_scratch_rejects_problems_beyond_its_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin as dm
    d = inputs.random_dfa(4_000_000, 4, 0.5, 1)
    assert dm.workspace_size(d.n, d.k) > 64 << 20
    dd, aa = dm.to_device(d.delta, d.accept)
    out = torch.full((d.n,), -7, dtype=torch.int32, device="cuda")
    sc = torch.full((3,), -7, dtype=torch.int32, device="cuda")
    opt = dm.options()
    rc = dm.lib().dfamin_minimize_static(
        d.n, d.k, _ptr(dd), _ptr(aa), _ptr(out), _ptr(sc), ctypes.byref(opt),
        ctypes.c_void_p(sc.data_ptr() + 4), ctypes.c_void_p(sc.data_ptr() + 8),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dm.ENOMEM
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == -7).all() and sc.cpu().tolist() == [-7, -7, -7]

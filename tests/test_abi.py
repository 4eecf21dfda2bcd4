"""The C-ABI library loads and exports every function that include/*.h declares (no GPU)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dfamin_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    so = os.path.join(ROOT, "paper_2410_22764_gb300", "libdfamin.so")
    if not os.path.exists(so):
        import __graft_entry__
        __graft_entry__.build()
    from paper_2410_22764_gb300 import dfamin
    return dfamin


def test_header_declares_functions():
    assert {"dfamin_minimize", "dfamin_minimize_ex", "dfamin_workspace_size",
            "dfamin_status_string"} <= _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib.lib(), name), name
    assert set(lib.ABI_FUNCTIONS) <= _declared()


def test_host_side_queries_without_gpu(lib):
    assert lib.status_string(0) == "DFAMIN_OK"
    assert lib.status_string(4) == "DFAMIN_ETIMEOUT"
    small = lib.workspace_size(1000, 2)
    big = lib.workspace_size(10_000_000, 4)
    clo = lib.workspace_size(10_000_000, 4, lib.options(closure=True))
    assert 0 < small < big < clo
    # closure columns: k * floor(log2 n) extra int32 columns of n states
    assert clo - big >= 4 * 10_000_000 * 4 * 23
    with pytest.raises(lib.DfaminError):
        lib.workspace_size(0, 2)
    with pytest.raises(lib.DfaminError):
        lib.workspace_size(10, -1)


def test_host_argument_checks_need_no_gpu(lib):
    # sizes, options and null pointers are checked on the host before any CUDA call
    import ctypes
    L = lib.lib()
    sz = ctypes.c_size_t(0)
    opt = lib.options()
    assert L.dfamin_workspace_size(0, 2, ctypes.byref(opt), ctypes.byref(sz)) == lib.EINVAL
    assert L.dfamin_workspace_size((1 << 30) + 1, 2, ctypes.byref(opt),
                                   ctypes.byref(sz)) == lib.EINVAL
    assert L.dfamin_workspace_size(100, -1, ctypes.byref(opt), ctypes.byref(sz)) == lib.EINVAL
    bad = lib.options()
    bad.closure = 7
    assert L.dfamin_workspace_size(100, 2, ctypes.byref(bad), ctypes.byref(sz)) == lib.EINVAL
    bad = lib.options()
    bad.algorithm = 9
    assert L.dfamin_workspace_size(100, 2, ctypes.byref(bad), ctypes.byref(sz)) == lib.EINVAL
    bad = lib.options()
    bad.barrier_timeout_us = -1
    assert L.dfamin_workspace_size(100, 2, ctypes.byref(bad), ctypes.byref(sz)) == lib.EINVAL
    # workspace sizes grow with n, and the closure needs more
    sizes = []
    for n in (10, 1000, 100000):
        assert L.dfamin_workspace_size(n, 3, ctypes.byref(opt), ctypes.byref(sz)) == 0
        sizes.append(sz.value)
    assert sizes == sorted(sizes) and sizes[0] > 0
    clo = lib.options(closure=True)
    assert L.dfamin_workspace_size(100000, 3, ctypes.byref(clo), ctypes.byref(sz)) == 0
    assert sz.value > sizes[-1]
    # the entry points refuse bad sizes and null pointers before touching the device
    null = ctypes.c_void_p(0)
    assert L.dfamin_minimize_ex((1 << 30) + 1, 1, null, null, null, null, ctypes.byref(opt),
                                null, 0, null, null, null) == lib.EINVAL
    assert L.dfamin_minimize_ex(10, 1, null, null, null, null, ctypes.byref(opt), null, 0,
                                null, null, null) == lib.EINVAL
    assert L.dfamin_reach_workspace_size(0, ctypes.byref(sz)) == lib.EINVAL
    assert L.dfamin_reach_workspace_size(1000, ctypes.byref(sz)) == 0 and sz.value > 0
    assert L.dfamin_quotient_workspace_size(-5, ctypes.byref(sz)) == lib.EINVAL
    assert L.dfamin_minimize_static(0, 1, null, null, null, null, ctypes.byref(opt), null, null,
                                    null) == lib.EINVAL
    for code in range(7):
        assert L.dfamin_status_string(code).startswith(b"DFAMIN_")

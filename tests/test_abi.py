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

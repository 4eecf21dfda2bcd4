"""The closure under a column budget (dfamin_options.closure_columns), on the GPU through the C ABI.

Alg. transPR (Sec. 3.4) adds the letters a^(2^i); every subset of them leaves the state
equivalence unchanged (each added letter is a word over the original alphabet), so a budget
that keeps only some columns must give exactly the plain partition, with a pass count between
the full closure's and the plain one.  Where the columns the library keeps are known in advance
the pass count is pinned exactly: Moore on the DFA extended by those columns.
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


def _run(dm, d, **kw):
    dlt, acc = dm.to_device(d.delta, d.accept)
    return dm.minimize_ex(d.n, d.k, dlt, acc, opt=dm.options(**kw)).host()


def _extended(d, levels):
    """The DFA with, for every letter, its closure columns of levels 1..levels appended."""
    cols = oracle.closure(d.delta, d.n, d.k)               # row a*L + i = delta^(2^i) of a
    L = oracle.closure_levels(d.n)
    keep = [d.delta.reshape(d.n, d.k)]
    for i in range(1, levels + 1):
        for a in range(d.k):
            keep.append(cols[a * L + i][:, None])
    ext = np.ascontiguousarray(np.concatenate(keep, axis=1))
    return ext.reshape(-1), ext.shape[1]


@pytest.mark.parametrize("n", [3000, 70000])
@pytest.mark.parametrize("budget", [1, 2, 5, 9])
def test_path_budget_pass_count_is_exact(dm, n, budget):
    # path DFA: letter 1 is the identity (no closure columns), letter 0 changes at every level
    # below log2 n, so a budget of b columns keeps exactly levels 1..b of letter 0
    d = I.path_fib_dfa(n)
    want, wn = oracle.hopcroft(d.delta, d.accept, d.n, d.k)
    ext, ke = _extended(d, budget)
    _, _, wp = oracle.moore(ext, d.accept, d.n, ke)
    for smem in (0, 1):
        got, gn, gp, st = _run(dm, d, closure=True, closure_columns=budget, smem_states=smem)
        assert st == 0 and gn == wn and np.array_equal(got, want)
        assert gp == wp, (smem, gp, wp)


@pytest.mark.parametrize("nbits", [10, 13])
def test_bitsplitter_under_a_small_workspace(dm, nbits):
    # B_n with fewer columns than floor(log2 n) * k: the partition is exact, and the pass count
    # lies between the full closure's and the plain one
    d = I.bitsplitter_dfa(nbits)
    want, wn, plain = oracle.moore(d.delta, d.accept, d.n, d.k)
    dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
    _, _, full = oracle.moore(dc, d.accept, d.n, kc)
    full_ws = dm.workspace_size(d.n, d.k, dm.options(closure=True))
    for budget in (1, d.k // 2, d.k):
        opt = dm.options(closure=True, closure_columns=budget, smem_states=1)
        assert dm.workspace_size(d.n, d.k, opt) < full_ws
        got, gn, gp, st = _run(dm, d, closure=True, closure_columns=budget, smem_states=1)
        assert st == 0 and gn == wn and np.array_equal(got, want)
        assert full <= gp <= plain, (budget, full, gp, plain)


def test_budget_in_a_batch(dm):
    dfas = [I.path_fib_dfa(3000), I.path_fib_dfa(40000), I.bitsplitter_dfa(9),
            I.cyclic_fib_dfa(15), I.random_dfa(20000, 3, 0.5, 4)]
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    plan = dm.BatchPlan(state_off, ks, dm.options(closure=True, closure_columns=3))
    out, per = plan.run(dd, aa)
    out, per = out.cpu().numpy(), per.cpu().numpy()
    plan.close()
    for i, d in enumerate(dfas):
        want, wn, plain = oracle.moore(d.delta, d.accept, d.n, d.k)
        assert per[2, i] == 0 and per[0, i] == wn
        assert np.array_equal(out[state_off[i]: state_off[i + 1]], want)
        assert per[1, i] <= plain
    # the path DFAs keep levels 1..3 of letter 0: exact pass counts
    for i in (0, 1):
        d = dfas[i]
        ext, ke = _extended(d, 3)
        _, _, wp = oracle.moore(ext, d.accept, d.n, ke)
        assert per[1, i] == wp

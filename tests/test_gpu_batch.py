"""Batched minimization (dfamin_batch_plan_run, dfamin_minimize_batch) against the oracle,
DFA by DFA, bit-exact.

Every DFA of a batch must get exactly what the oracle (and the single-DFA entry point) gives:
canonical block ids, the block count and the pass count.
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


def mixed_batch(seed=0, count=60, max_n=40000):
    rng = np.random.default_rng(seed)
    dfas = [I.random_dfa(1, 0, 1.0, 1), I.random_dfa(2, 1, 0.5, 2), I.random_dfa(3, 0, 0.5, 3),
            I.fig1_dfa(), I.cyclic_fib_dfa(9), I.bitsplitter_dfa(7), I.path_fib_dfa(300)]
    while len(dfas) < count:
        kind = rng.integers(0, 4)
        n = int(10 ** rng.uniform(0, np.log10(max_n)))
        k = int(rng.integers(0, 11))
        s = int(rng.integers(0, 1 << 30))
        if kind == 0:
            dfas.append(I.random_dfa(n, k, float(rng.uniform(0.1, 0.9)), s))
        elif kind == 1:
            m = max(1, n // 4)
            dfas.append(I.inflated_dfa(m, max(k, 1), 4, 0.5, s)[0])
        elif kind == 2:
            dfas.append(I.path_fib_dfa(max(2, min(n, 3000))))
        else:
            dfas.append(I.random_dfa(n, k, 0.0 if s % 2 else 1.0, s))
    return dfas


def oracle_results(dfas, closure=False):
    out = []
    for d in dfas:
        b, nb, ps = oracle.moore(d.delta, d.accept, d.n, d.k)
        if closure:
            dc, kc = oracle.closure_dfa(d.delta, d.n, d.k)
            _, _, ps = oracle.moore(dc, d.accept, d.n, kc)
        out.append((b, nb, ps))
    return out


def run_batch(dm, dfas, opt):
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    plan = dm.BatchPlan(state_off, ks, opt)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    out, per = plan.run(dd, aa)
    torch.cuda.synchronize()
    return plan, plan.split(out.cpu().numpy()), per.cpu().numpy()


def check_batch(dm, dfas, opt, closure=False):
    want = oracle_results(dfas, closure)
    plan, outs, per = run_batch(dm, dfas, opt)
    for i, (d, (b, nb, ps)) in enumerate(zip(dfas, want)):
        assert per[2, i] == 0, (i, d.n, d.k, dm.status_string(per[2, i]))
        assert per[0, i] == nb, (i, d.n, d.k)
        assert np.array_equal(outs[i], b), (i, d.n, d.k)
        assert per[1, i] == ps, (i, d.n, d.k, per[1, i], ps)
    return plan


def test_mixed_batch_default_schedule(dm):
    check_batch(dm, mixed_batch(1), dm.options())


def test_mixed_batch_closure(dm):
    check_batch(dm, mixed_batch(2, count=40, max_n=8000), dm.options(closure=True), closure=True)


@pytest.mark.parametrize("small,team", [(64, 512), (1, 2000), (4096, 100000)])
def test_mixed_batch_team_shapes(dm, small, team):
    # force many multi-CTA teams (small shared-memory limit, few states per CTA) and the reverse
    plan = check_batch(dm, mixed_batch(3), dm.options(smem_states=small, team_states=team))
    assert plan.tickets >= plan.count


def test_batch_grid_smaller_than_work(dm):
    # a capped grid forces teams to form from CTAs freed by earlier DFAs
    plan = check_batch(dm, mixed_batch(4), dm.options(ctas=16, smem_states=256, team_states=1000))
    assert plan.grid == 16 and plan.tickets > 16


@pytest.mark.parametrize("flags", [2, 4])
def test_batch_degenerate_hash(dm, flags):
    check_batch(dm, mixed_batch(5, count=25, max_n=5000), dm.options(flags=flags,
                                                                     smem_states=512))


def test_batch_error_is_isolated(dm):
    dfas = mixed_batch(6, count=20, max_n=20000)
    bad_i = max(range(len(dfas)), key=lambda i: dfas[i].n * dfas[i].k)
    d = dfas[bad_i]
    bad = I.Dfa(d.n, d.k, d.delta.copy(), d.accept)
    bad.delta[0] = d.n + 3
    dfas[bad_i] = bad
    want = oracle_results([x for i, x in enumerate(dfas) if i != bad_i])
    plan, outs, per = run_batch(dm, dfas, dm.options(smem_states=256))
    assert per[2, bad_i] == dm.EINVAL and per[0, bad_i] == -dm.EINVAL
    j = 0
    for i in range(len(dfas)):
        if i == bad_i:
            continue
        b, nb, ps = want[j]
        j += 1
        assert per[2, i] == 0 and per[0, i] == nb and per[1, i] == ps
        assert np.array_equal(outs[i], b)


def test_batch_matches_single_entry_point(dm):
    dfas = mixed_batch(7, count=30, max_n=60000)
    plan, outs, per = run_batch(dm, dfas, dm.options())
    for i, d in enumerate(dfas):
        got, nb, ps, st = dm.minimize_host(d.n, d.k, d.delta, d.accept)
        assert st == 0 and nb == per[0, i] and ps == per[1, i]
        assert np.array_equal(got, outs[i])


def test_batch_cuda_graph_replay(dm):
    dfas = mixed_batch(8, count=30, max_n=30000)
    want = oracle_results(dfas)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    plan = dm.BatchPlan(state_off, ks, dm.options())
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    ws = dm.Workspace()
    out = torch.empty(plan.states, dtype=torch.int32, device="cuda")
    per = torch.zeros((3, plan.count), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(dd, aa, workspace=ws, out_block=out, per_dfa=per, stream=s)   # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(dd, aa, workspace=ws, out_block=out, per_dfa=per, stream=s)
    for _ in range(2):
        out.fill_(-1)
        per.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        o, p = plan.split(out.cpu().numpy()), per.cpu().numpy()
        for i, (b, nb, ps) in enumerate(want):
            assert p[2, i] == 0 and p[0, i] == nb and p[1, i] == ps
            assert np.array_equal(o[i], b)


def test_plan_destroyed_right_after_launch(dm):
    # a plan released while its launch still runs (a Python temporary) must not free the
    # descriptor table under the running kernel: the free waits for the launch in stream order
    dfas = mixed_batch(9, count=40, max_n=60000)
    want = oracle_results(dfas)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    results = []
    for _ in range(3):
        out, per = dm.BatchPlan(state_off, ks, dm.options()).run(dd, aa)
        results.append((out, per))
    torch.cuda.synchronize()
    for out, per in results:
        o, p = np.split(out.cpu().numpy(), state_off[1:-1]), per.cpu().numpy()
        for i, (b, nb, ps) in enumerate(want):
            assert p[2, i] == 0 and p[0, i] == nb and p[1, i] == ps
            assert np.array_equal(o[i], b)


def test_single_calls_after_graph_captured_plan_is_released(dm):
    # releasing a plan whose launch was captured into a graph must leave no pending CUDA error
    # behind for later, unrelated calls
    dfas = mixed_batch(12, count=10, max_n=5000)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    plan = dm.BatchPlan(state_off, ks, dm.options())
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    ws = dm.Workspace()
    out = torch.empty(plan.states, dtype=torch.int32, device="cuda")
    per = torch.zeros((3, plan.count), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(dd, aa, workspace=ws, out_block=out, per_dfa=per, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(dd, aa, workspace=ws, out_block=out, per_dfa=per, stream=s)
    g.replay()
    torch.cuda.synchronize()
    del g
    plan.close()
    d = I.random_dfa(1, 0, 1.0, 1)
    got, nb, ps, st = dm.minimize_host(d.n, d.k, d.delta, d.accept)
    assert st == 0 and nb == 1


@pytest.mark.parametrize("closure", [False, True])
def test_one_shot_batch_call(dm, closure):
    # dfamin_minimize_batch: no plan object, host offsets, table in the caller's workspace
    dfas = mixed_batch(13, count=40, max_n=20000 if not closure else 5000)
    want = oracle_results(dfas, closure)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    out, nb, st = dm.minimize_batch(state_off, ks, dd, aa, opt=dm.options(closure=closure))
    torch.cuda.synchronize()
    o = np.split(out.cpu().numpy(), state_off[1:-1])
    nb, st = nb.cpu().numpy(), st.cpu().numpy()
    for i, (b, n_b, _) in enumerate(want):
        assert st[i] == 0 and nb[i] == n_b and np.array_equal(o[i], b)


def test_one_shot_batch_call_refuses_stream_capture(dm):
    # the one-shot call copies its table from host memory that dies with the call, so it must
    # not be recorded into a graph: it returns EINVAL on a capturing stream and enqueues nothing
    dfas = mixed_batch(14, count=6, max_n=3000)
    want = oracle_results(dfas)
    delta, acc, state_off, ks = dm.pack_batch(dfas)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    ws = dm.Workspace()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dm.minimize_batch(state_off, ks, dd, aa, workspace=ws, stream=s)   # sizes the workspace
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=s):
        try:
            dm.minimize_batch(state_off, ks, dd, aa, workspace=ws, stream=s)
        except dm.DfaminError as e:
            err = e
    assert err is not None and err.code == dm.EINVAL
    assert "capturing" in dm.lib().dfamin_last_cuda_error().decode()
    out, nb, st = dm.minimize_batch(state_off, ks, dd, aa, workspace=ws)
    torch.cuda.synchronize()
    o = np.split(out.cpu().numpy(), state_off[1:-1])
    nb, st = nb.cpu().numpy(), st.cpu().numpy()
    for i, (b, n_b, _) in enumerate(want):
        assert st[i] == 0 and nb[i] == n_b and np.array_equal(o[i], b)

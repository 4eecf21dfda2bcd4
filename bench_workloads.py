"""Measurement of the other workloads (one JSON line each), selected by
``python bench.py --workload random1k|path|batch200m|batch6g|serve|table2|minimal|trace2``.

* random1k  random DFA n = 1,000, k = 2 (one CTA in shared memory): ms per minimization.
* path      deep-refinement path n = 2^20, k = 2: plain rounds (534,348) against the closure.
* batch200m 4,096 random DFAs (n log-uniform 100..10^6 capped so that sum n*k = 2e8, k in 2..26,
            p in 0.1..0.9): one batched launch against one launch per DFA.
* batch6g   the same 4,096 draws uncapped (~6.5e9 transitions): one batched launch.
* serve     Poisson request stream through the continuous-batching server at
            0.5 / 0.8 / 0.95 of its saturated throughput: p50 / p99 latency and DFAs/s.
* minimal   the minimal DFA of the bench workload (n = 10^7, q0 = 0): reachability, refinement
            of the whole DFA and the quotient on one stream, against the refinement alone; and
            the same with a second, unreachable copy of the DFA appended (n = 2*10^7).
* table2    the paper's own families at the sizes of Table 2 (cyclic Fib with 17,711 ..
            2,178,309 states, bit-splitters B_15 .. B_26 with up to 67M states and 25 letters),
            each minimized by signature refinement (the sortPR rounds), the leader election
            (naivePR), signature refinement on the closure (transPR as built here) and the leader
            election on the closure (transPR as printed); the paper's times are carried as
            context (other hardware).
Timing: CUDA events on the launching stream, warm-up first, L2 flushed between timed steps
(a 512 MB write) unless the inputs are larger than L2.
"""
from __future__ import annotations

import ctypes
import json
import os
import statistics
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2410_22764_gb300 import dfamin, inputs as I  # noqa: E402


def _line(workload, value, unit, ms, steps, warmup, extra, higher=True):
    line = {"metric": bench.METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": higher, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _time_steps(fn, steps, warmup, flush=None, stream=None):
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return ts


def single(args, name, d, closure=False, steps=None, warmup=None):
    dd, aa = dfamin.to_device(d.delta, d.accept)
    ws = dfamin.Workspace()
    opt = dfamin.options(closure=closure)
    out = torch.empty(d.n, dtype=torch.int32, device="cuda")
    sc = torch.zeros(3, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    fn = lambda: dfamin.minimize_ex(d.n, d.k, dd, aa, opt=opt, workspace=ws,  # noqa: E731
                                    out_block=out, scalars=sc)
    ts = _time_steps(fn, steps or args.steps, max(3, warmup or args.warmup), flush)
    nb, ps, st = sc.cpu().tolist()
    assert st == 0
    ms = statistics.median(ts)
    return {"name": name, "ms": ms, "passes": ps, "nblocks": nb, "steps": len(ts),
            "edge_visits_per_s": d.n * d.k * ps / (ms / 1e3), "us_per_pass": 1e3 * ms / max(ps, 1)}


def run_random1k(args):
    d = I.random_dfa(1000, 2, 0.5, 1)
    r = single(args, "random1k", d, steps=max(args.steps, 200))
    _line("random DFA n=1000 k=2 p=0.5 seed 1 (one CTA, shared memory)", r["edge_visits_per_s"],
          "edge-visits/s", r["ms"], r["steps"], max(3, args.warmup), {"result": r})


def run_path(args):
    d = I.path_fib_dfa(1 << 20)
    extra = {}
    clo = plain = None
    if args.path_variant in ("both", "closure"):
        clo = single(args, "closure", d, closure=True, steps=10)
        extra["closure"] = clo
    if args.path_variant in ("both", "plain"):
        plain = single(args, "plain", d, steps=2, warmup=3)
        extra["plain"] = plain
    if clo and plain:
        extra["speedup_closure_vs_plain"] = plain["ms"] / clo["ms"]
    main = clo or plain
    _line("path DFA n=2^20 k=2, Fibonacci acceptance: closure (Alg. transPR) vs plain rounds",
          1e3 / main["ms"], "minimizations/s", main["ms"], main["steps"], 3, extra)


def _per_dfa_launches(delta, acc, state_off, ks, steps):
    """One dfamin_minimize_ex launch per DFA (each DFA's rows and bitmap 16-byte aligned)."""
    count, ns = ks.size, np.diff(state_off)
    doff = np.concatenate([[0], np.cumsum(ns * ks.astype(np.int64))])
    dpad = np.concatenate([[0], np.cumsum((ns * ks + 3) // 4 * 4)])
    aoff = np.concatenate([[0], np.cumsum((ns + 127) // 128 * 4)])
    dbuf = np.zeros(int(dpad[-1]), np.int32)
    abuf = np.zeros(int(aoff[-1]), np.uint32)
    for i in range(count):
        m = I.batch_member(delta, acc, state_off, ks, i)
        dbuf[dpad[i]: dpad[i] + m.delta.size] = m.delta
        abuf[aoff[i]: aoff[i] + m.accept.size] = m.accept
    db, ab = torch.from_numpy(dbuf).cuda(), torch.from_numpy(abuf.view(np.int32)).cuda()
    out = torch.empty(int(state_off[-1]), dtype=torch.int32, device="cuda")
    sc = torch.zeros((count, 3), dtype=torch.int32, device="cuda")
    wsb = max(dfamin.workspace_size(int(ns[i]), int(ks[i])) for i in range(count))
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
    lib, opt = dfamin.lib(), dfamin.options()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p

    def fn():
        for i in range(count):
            base = sc.data_ptr() + 12 * i
            rc = lib.dfamin_minimize_ex(
                int(ns[i]), int(ks[i]), P(db.data_ptr() + 4 * int(dpad[i])),
                P(ab.data_ptr() + 4 * int(aoff[i])), P(out.data_ptr() + 4 * int(state_off[i])),
                P(base), ctypes.byref(opt), P(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                P(base + 4), P(base + 8), st)
            assert rc == 0
    ts = _time_steps(fn, steps, 1)
    return statistics.median(ts), out.cpu().numpy(), sc.cpu().numpy()


def _graph_of(fn, stream):
    """fn captured into a CUDA graph on `stream` (after one uncaptured warm-up call)."""
    with torch.cuda.stream(stream):
        fn(stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn(stream)
    return g


def _oracle_member(task):
    """Pool task (spawn-started worker): regenerate one batch member from its draws with the
    seeded generator and run the CPU oracle (Hopcroft) on it; returns the oracle's seconds and
    block count (the generation is not timed)."""
    n, k, p, seed = task
    import oracle
    delta, acc, _, _ = I.random_batch([n], [k], [p], [seed], threads=1)
    t0 = time.perf_counter()
    _, nb = oracle.hopcroft(delta, acc, n, k)
    return time.perf_counter() - t0, int(nb)


def _cpu_baseline_batch(ns, ks, ps, seeds, stride, nblocks):
    """The CPU oracle as it stands (Hopcroft, one DFA per task) over all host cores on every
    `stride`-th member of the batch; value = DFAs per second on those cores, from the sum of the
    per-DFA oracle times divided by the cores (the pool's own overhead not counted)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    idx = np.arange(0, ns.size, stride)
    tasks = [(int(ns[i]), int(ks[i]), float(ps[i]), int(seeds[i])) for i in idx]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_member, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    cpu_s = sum(t for t, _ in out)
    assert all(nb == int(nblocks[i]) for (_, nb), i in zip(out, idx))
    trans = int(np.sum(ns[idx] * ks[idx].astype(np.int64)))
    return {"value": len(tasks) / (cpu_s / cores), "unit": "DFAs/s", "cores": cores,
            "host_cores": cores, "kind": "oracle", "oracle_cpu_s": cpu_s, "wall_s": wall,
            "transitions_per_s": trans / (cpu_s / cores),
            "sample": f"every {stride}th of the 4,096 DFAs ({len(tasks)} DFAs, {trans} "
                      "transitions), Hopcroft per DFA in a process pool over all host cores; "
                      "value = DFAs / (sum of per-DFA oracle seconds / cores); block counts "
                      "equal the GPU's"}


def run_batch(args, kind):
    """One persistent launch per batch, replayed from a CUDA graph, with the options the
    autotuner picks (timed candidates, cached per GPU and shape bucket), against the default
    options and against one plain launch per DFA (4b).  Under torchrun the batch is sharded:
    every rank generates and minimizes its size-balanced share of the 4,096 DFAs (no collective
    on the data path) and the time is the slowest rank's."""
    from paper_2410_22764_gb300 import autotune, multi
    rank, world, local = bench.dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    ns, ks_all, ps, seeds = I.batch_sizes(4096, 1)
    if kind == "capped":
        cap = I.batch_cap_for_transitions(4096, 1, 200_000_000)
        ns, ks_all, ps, seeds = I.batch_sizes(4096, 1, n_cap=cap)
    mine = multi.shard_batch(ns, ks_all, world)[rank]
    delta, acc, state_off, ks = I.random_batch(ns[mine], ks_all[mine], ps[mine], seeds[mine])
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    tuned_opt, timings = autotune.tune_batch(state_off, ks, dd, aa)
    tune_s = time.perf_counter() - t0
    steps = max(3, min(args.steps, 10 if kind == "capped" else 5))
    warm = max(3, args.warmup)
    side = torch.cuda.Stream()
    res, ref = {}, None
    for name, opt in (("default", dfamin.options()), ("tuned", tuned_opt)):
        plan = dfamin.BatchPlan(state_off, ks, opt)
        ws = dfamin.Workspace()
        out = torch.empty(plan.states, dtype=torch.int32, device="cuda")
        per = torch.zeros((3, plan.count), dtype=torch.int32, device="cuda")

        def launch(stream=None):
            plan.run(dd, aa, workspace=ws, out_block=out, per_dfa=per, stream=stream)
        plain = statistics.median(_time_steps(launch, steps, warm, flush))
        g = _graph_of(launch, side)
        graph = statistics.median(_time_steps(g.replay, steps, warm, flush))
        p = per.cpu().numpy()
        assert (p[2] == 0).all()
        o = out.cpu().numpy()
        if ref is None:
            ref = (o, p)
        else:
            assert np.array_equal(o, ref[0]) and np.array_equal(p, ref[1])
        res[name] = {"plain_launch_ms": plain, "graph_replay_ms": graph, "grid": plan.grid,
                     "tickets": plan.tickets, "workspace_gb": plan.workspace_bytes / 1e9}
        del g
        plan.close()
    ms = res["tuned"]["graph_replay_ms"]
    p = ref[1]
    visits = int((np.diff(state_off) * ks.astype(np.int64) * p[1]).sum())
    # job-wide: the slowest rank's time, every rank's edge visits
    ms, visits = multi.aggregate(ms, float(visits), pg, torch.device("cuda", local))
    best = json.loads(min(timings, key=timings.get))
    extra = {"batched_ms": ms, "dfas": 4096, "states": int(ns.sum()),
             "transitions": int(np.sum(ns * ks_all.astype(np.int64))),
             "dfas_per_s": 4096 / (ms / 1e3), "gpu_launches": steps,
             "tuned_knobs": best, "tuning_s": tune_s, "tuning_candidates": len(timings),
             "default": res["default"], "tuned": res["tuned"],
             "tuned_vs_default": res["default"]["graph_replay_ms"] / res["tuned"]["graph_replay_ms"]}
    if world > 1:
        extra.update({"n_gpus": world, "scaling": "strong",
                      "parallelism": f"batch sharded over {world} ranks (size-balanced)",
                      "rank0_dfas": int(mine.size)})
    if kind == "capped" and world == 1:
        pms, pout, psc = _per_dfa_launches(delta, acc, state_off, ks, 2)
        assert np.array_equal(pout, ref[0]) and np.array_equal(psc[:, 0], p[0])
        extra.update({"per_dfa_launches_ms": pms, "batched_speedup": pms / ms})
    if world == 1 and not getattr(args, "no_cpu_baseline", False):
        nb_by_index = np.zeros(ns.size, dtype=np.int64)
        nb_by_index[mine] = p[0]
        extra["cpu_baseline"] = _cpu_baseline_batch(ns, ks_all, ps, seeds,
                                                    1 if kind == "capped" else 16, nb_by_index)
    desc = ("4,096 random DFAs, n log-uniform 100..1e6, k 2..26, p 0.1..0.9, seed 1" +
            (", n capped so that sum n*k = 2e8" if kind == "capped" else ", as drawn") +
            "; one persistent launch replayed from a CUDA graph with autotuned options")
    if rank == 0:
        _line(desc, visits / (ms / 1e3), "edge-visits/s", ms, steps, warm, extra)
    if pg:
        pg.destroy_process_group()


def _serve_pool(pool, seed=5):
    """Request pool with the served-stream distribution: 5% path DFAs (n = 65,536), the rest
    half uniform random, half inflated (c = 4); n log-uniform 1e3..4e6, k in 2..8."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(pool):
        if rng.random() < 0.05:
            out.append(I.path_fib_dfa(65536))
            continue
        n = int(round(10 ** rng.uniform(3, np.log10(4e6))))
        k = int(rng.integers(2, 9))
        if rng.random() < 0.5:
            out.append(I.random_dfa(n, k, 0.5, int(rng.integers(1 << 30))))
        else:
            m = max(1, n // 4)
            out.append(I.inflated_dfa(m, k, 4, 0.5, int(rng.integers(1 << 30)), permute=False)[0])
    return out


def _latency_stats(lat, t_elapsed, R, rate):
    lat = np.asarray(lat)
    return {"rate_req_per_s": rate, "dfas_per_s": R / t_elapsed,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3)}


def _serve_batched(reqs, rate, max_work, solo_work=None):
    from paper_2410_22764_gb300 import serve
    R = len(reqs)
    kw = {} if solo_work is None else {"solo_work": solo_work}
    srv = serve.Server(budget_bytes=48 << 30, streams=4, max_batch_work=max_work, **kw)
    rng = np.random.default_rng(11)
    gaps = rng.exponential(1.0 / rate, size=R) if rate else np.zeros(R)
    t0 = time.perf_counter()
    arrive = t0 + np.cumsum(gaps)
    i = 0
    while i < R or not srv.idle():
        now = time.perf_counter()
        while i < R and arrive[i] <= now:
            d = reqs[i]
            srv.submit(d.n, d.k, d.delta, d.accept, arrival=float(arrive[i]))
            i += 1
        if not srv.step():
            time.sleep(20e-6)
    t1 = time.perf_counter()
    lat = [r.latency for r in srv.completed if r.status == 0]
    out = _latency_stats(lat, t1 - t0, R, rate)
    out.update({"failed": sum(1 for r in srv.completed if r.status != 0),
                "batches": srv.stats.batches, "max_inflight": srv.stats.max_inflight,
                "max_device_overlap": srv.max_device_overlap(),
                "escalated": srv.stats.escalated, "single_dfa_launches": srv.stats.solo})
    return out


def _serve_plain(reqs, rate, pass_cap=64):
    """The same arrival stream served one request at a time, one dfamin_minimize_ex launch per
    request (plus a closure rerun when the pass cap is hit, as the batching server does):
    pinned host copy, H2D, the launch, D2H, in arrival order on one stream."""
    R = len(reqs)
    s = torch.cuda.Stream()
    ws = dfamin.Workspace()
    sc = torch.zeros(3, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(11)
    gaps = rng.exponential(1.0 / rate, size=R) if rate else np.zeros(R)
    t0 = time.perf_counter()
    arrive = t0 + np.cumsum(gaps)
    lat, failed, escalated = [], 0, 0
    with torch.cuda.stream(s):
        for i, d in enumerate(reqs):
            while time.perf_counter() < arrive[i]:
                time.sleep(20e-6)
            hd = torch.from_numpy(np.ascontiguousarray(d.delta, np.int32)).pin_memory()
            ha = torch.from_numpy(np.ascontiguousarray(d.accept, np.uint32).view(np.int32)).pin_memory()
            dd = hd.to("cuda", non_blocking=True)
            aa = ha.to("cuda", non_blocking=True)
            out = torch.empty(d.n, dtype=torch.int32, device="cuda")
            dfamin.minimize_ex(d.n, d.k, dd, aa, opt=dfamin.options(max_passes=pass_cap),
                               workspace=ws, out_block=out, scalars=sc, stream=s)
            st = int(sc[2].item())
            if st == dfamin.ENOCONVERGE:
                escalated += 1
                dfamin.minimize_ex(d.n, d.k, dd, aa, opt=dfamin.options(closure=True),
                                   workspace=ws, out_block=out, scalars=sc, stream=s)
                st = int(sc[2].item())
            host = out.cpu()
            del host
            if st != 0:
                failed += 1
            lat.append(time.perf_counter() - arrive[i])
    t1 = time.perf_counter()
    out = _latency_stats(lat, t1 - t0, R, rate)
    out.update({"failed": failed, "escalated": escalated})
    return out


def run_serve(args):
    pool = _serve_pool(args.serve_pool)
    R = args.requests
    pick = np.random.default_rng(7).integers(0, len(pool), size=R)
    reqs = [pool[int(i)] for i in pick]
    W = args.max_batch_work
    S = getattr(args, "solo_work", None)
    _serve_batched(reqs[: min(R, 200)], 0, W, S)       # warm-up (allocator, plans, kernels)
    sat = _serve_batched(reqs, 0, W, S)
    batched = {"saturated": sat}
    plain_sat = _serve_plain(reqs, 0)
    plain = {"saturated": plain_sat}
    for rho in (0.5, 0.8, 0.95):
        rate = rho * sat["dfas_per_s"]
        batched[f"rho_{rho}"] = _serve_batched(reqs, rate, W, S)
        plain[f"rho_{rho}"] = _serve_plain(reqs, rate)
    _line(f"served Poisson stream, {R} requests drawn from a pool of {len(pool)} DFAs (n "
          "log-uniform 1e3..4e6, k 2..8, 50% random / 50% inflated c=4, 5% path n=65536), HBM "
          f"budget 48 GB, batches of at most {W} transitions, requests of at least "
          f"{S if S is not None else 'the default'} transitions as single-DFA launches",
          sat["dfas_per_s"], "DFAs/s",
          1e3 / sat["dfas_per_s"], R, 1,
          {"serve": batched, "plain_one_launch_per_request": plain,
           "batched_vs_plain_saturated": sat["dfas_per_s"] / plain_sat["dfas_per_s"],
           "rho_rates_from": "the batching server's saturated DFAs/s (both arms see the same "
                             "arrival times)"})


# Table 2 of the paper: name -> (N, |Sigma|, naivePR ms, sortPR ms, transPR ms); None = t/o or
# OoM there.  Fib_i of the table has N = |w_{i+1}| states.
TABLE2 = {
    "Fib20": (17711, 1, 308.8, 3909.2, 1.7), "Fib21": (28657, 1, 494.2, 6374.2, 2.4),
    "Fib22": (46368, 1, 778.7, 11712.1, 4.1), "Fib23": (75025, 1, 1241.3, 21366.6, 8.0),
    "Fib24": (121393, 1, 2006.7, 34793.1, 12.5), "Fib25": (196418, 1, 3251.3, 64411.7, 18.3),
    "Fib26": (317811, 1, 5277.8, 178367.4, 49.8), "Fib27": (514229, 1, 8607.7, None, 96.1),
    "Fib28": (832040, 1, 22723.0, None, 178.4), "Fib29": (1346269, 1, 59510.8, None, 726.9),
    "Fib30": (2178309, 1, 141601.0, None, 1109.3),
    "B15": (32768, 14, 0.8, 25.8, 1.7), "B16": (65536, 15, 1.4, 29.7, 3.7),
    "B17": (131072, 16, 2.6, 54.3, 9.4), "B18": (262144, 17, 5.0, 107.2, 25.6),
    "B19": (524288, 18, 9.6, 235.7, 60.9), "B20": (1048576, 19, 19.3, 520.2, 139.8),
    "B21": (2097152, 20, 39.8, 1148.6, 312.2), "B22": (4194304, 21, 82.6, 2538.5, 728.7),
    "B23": (8388608, 22, 170.3, 5612.7, 1612.1), "B24": (16777216, 23, 352.6, 12351.8, None),
    "B25": (33554432, 24, 737.4, 27092.2, None), "B26": (67108864, 25, 1541.5, 59203.8, None),
}
VARIANTS = (("sortPR", False, False), ("naivePR", False, True),
            ("transPR", True, False), ("transPR_printed", True, True))


def _table2_dfa(name):
    if name.startswith("Fib"):
        return I.cyclic_fib_dfa(int(name[3:]) + 1)
    return I.bitsplitter_dfa(int(name[1:]))


def _timed_runs(d, dd, aa, opt, reps, warmup):
    """Median of `reps` timed minimizations (after `warmup` untimed ones) and the scalars."""
    ws = dfamin.Workspace()
    out = torch.empty(d.n, dtype=torch.int32, device="cuda")
    sc = torch.zeros(3, dtype=torch.int32, device="cuda")
    fn = lambda: dfamin.minimize_ex(d.n, d.k, dd, aa, opt=opt, workspace=ws,  # noqa: E731
                                    out_block=out, scalars=sc)
    ts = _time_steps(fn, reps, warmup)
    nb, ps, st = sc.cpu().tolist()
    del ws, out
    torch.cuda.empty_cache()
    return statistics.median(ts), nb, ps, st


def run_table2(args):
    rows, total = [], 0.0
    for name, (N, k, p_naive, p_sort, p_trans) in TABLE2.items():
        if args.table2_rows and name not in args.table2_rows.split(","):
            continue
        d = _table2_dfa(name)
        assert d.n == N and d.k == k, (name, d.n, d.k)
        dd, aa = dfamin.to_device(d.delta, d.accept)
        row = {"name": name, "N": N, "k": k,
               "paper_ms": {"naivePR": p_naive, "sortPR": p_sort, "transPR": p_trans}}
        for vname, closure, leader in VARIANTS:
            # deep plain refinement on Fib costs N rounds, and the leader election on the
            # closure about N/2 rounds of N*(1 + log2 N) gathers: bounded by --table2-max-rounds
            rounds = N if name.startswith("Fib") and not closure else 0
            if name.startswith("Fib") and closure and leader:
                rounds = N // 2 * (1 + int(np.log2(N)))
            if rounds > args.table2_max_rounds:
                row[vname] = {"skipped": f"about {rounds} rounds"}
                continue
            budget = 0
            if closure:
                # every column of every level when the workspace fits in device memory (less
                # 2 GB), else a column budget that fits: each column holds one int per state
                # twice (the column and its place in the signature rows)
                need = dfamin.workspace_size(d.n, d.k, dfamin.options(closure=True))
                free = torch.cuda.mem_get_info()[0] - (2 << 30)
                if need > free:
                    base = dfamin.workspace_size(d.n, d.k,
                                                 dfamin.options(closure=True, closure_columns=1))
                    budget = int((free - base) // (8 * d.n)) + 1
                    if budget < 1:
                        row[vname] = {"enomem": f"workspace {base / 1e9:.0f} GB > free "
                                                f"{free / 1e9:.0f} GB"}
                        continue
            opt = dfamin.options(closure=closure, leader=leader, closure_columns=budget)
            # runs of seconds are timed once, without a warm-up run of their own (the kernels
            # were loaded by the rows before)
            long = rounds > 100_000
            reps = 1 if long else 3
            ms, nb, ps, st = _timed_runs(d, dd, aa, opt, reps, 0 if long else 1)
            assert st == 0 and nb == N, (name, vname, st, nb)
            # closed forms of the plain pass counts (pinned by the oracle at small sizes):
            # signature rounds take N - 2 on cyclic Fib and n - 1 on B_n (Table 2, Sec. 4.2),
            # the leader election one more (its final round changes nothing)
            if not closure:
                nbits = int(name[1:]) if name.startswith("B") else 0
                want = (N - 2 if name.startswith("Fib") else nbits - 1) + (1 if leader else 0)
                assert ps == want, (name, vname, ps, want)
            row[vname] = {"ms": ms, "iterations": ps, "steps": reps}
            if budget:
                row[vname]["closure_columns"] = budget
            if vname == "transPR":
                total += ms
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        del dd, aa
        torch.cuda.empty_cache()
    _line("paper families at Table 2 sizes: cyclic Fib (17,711..2,178,309 states, 1 letter) and "
          "bit-splitters B_15..B_26 (2^15..2^26 states, 14..25 letters)", total, "ms",
          total, 1, 1, {"rows": rows,
                        "value_is": "sum over rows of the transPR (closure + signature) times"},
          higher=False)


def _median_ms(fn, steps, warmup, flush):
    return statistics.median(_time_steps(fn, steps, warmup, flush))


def run_minimal(args):
    d = bench.make_workload(bench.BASE_M)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    rows = {}
    for name, dfa in (("reachable", d), ("half_unreachable", None)):
        if dfa is None:
            # a second copy of the DFA that no word from q0 = 0 reaches
            delta = np.concatenate([d.delta, d.delta + np.int32(d.n)])
            acc = I.pack_bits(np.concatenate([I.unpack_bits(d.accept, d.n)] * 2))
            dfa = I.Dfa(2 * d.n, d.k, delta, acc)
        dd, aa = dfamin.to_device(dfa.delta, dfa.accept)
        ws1, ws2 = dfamin.Workspace(), dfamin.Workspace()
        res = {}
        steps, warm = max(3, min(args.steps, 10)), max(3, args.warmup)
        res["refinement_ms"] = _median_ms(
            lambda: dfamin.minimize_ex(dfa.n, dfa.k, dd, aa, workspace=ws1), steps, warm, flush)
        out = {}

        def full():
            out["r"] = dfamin.minimal_dfa(dfa.n, dfa.k, dd, aa, 0, workspace=ws2)
        res["minimal_dfa_ms"] = _median_ms(full, steps, warm, flush)
        res["reachability_ms"] = _median_ms(
            lambda: dfamin.reachable(dfa.n, dfa.k, dd, aa, 0, induced=False, workspace=ws1),
            steps, warm, flush)
        ns, q0m, nr, passes, st = out["r"][2].cpu().tolist()
        assert st == 0
        res.update({"n": dfa.n, "reachable": nr, "minimal_states": ns, "passes": passes})
        rows[name] = res
        del dd, aa, ws1, ws2
        torch.cuda.empty_cache()
    main = rows["reachable"]
    _line("minimal DFA of the inflated random DFA (n = 10^7, k = 4, q0 = 0): reachability + "
          "refinement + quotient on one stream", 1e3 / main["minimal_dfa_ms"], "minimal DFAs/s",
          main["minimal_dfa_ms"], max(3, min(args.steps, 10)), max(3, args.warmup),
          {"minimal": rows})


def run_trace2(args):
    """Per-phase device times of the bench workload (n = 10^7, k = 4) with DFAMIN_FLAG_TRACE,
    for the default choice of rounds, every round full and every round incremental, beside the
    median of untraced launches of each (CUDA events, L2 flushed between launches)."""
    d = bench.make_workload(bench.BASE_M)
    dd, aa = dfamin.to_device(d.delta, d.accept)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")     # > L2
    out = torch.empty(d.n, dtype=torch.int32, device="cuda")
    sc = torch.zeros(3, dtype=torch.int32, device="cuda")
    res, labels = {}, []
    for name, fl in (("default", 0), ("full", dfamin.FLAG_FULL_ROUNDS),
                     ("incremental", dfamin.FLAG_INCREMENTAL_ROUNDS)):
        opt = dfamin.options(flags=fl)
        ws = dfamin.Workspace()
        ms = _time_steps(lambda: dfamin.minimize_ex(d.n, d.k, dd, aa, opt=opt, workspace=ws,
                                                    out_block=out, scalars=sc),
                         30, 3, flush)
        labels.append(out.cpu().numpy())
        topt = dfamin.options(flags=fl | dfamin.FLAG_TRACE)
        tws = dfamin.Workspace()
        for _ in range(2):
            dfamin.minimize_ex(d.n, d.k, dd, aa, opt=topt, workspace=tws)
        torch.cuda.synchronize()
        tr = dfamin.read_trace(tws, d.n, d.k, topt)
        phases, prev = [], tr[0][2]
        for p_, ph, t in tr[1:]:
            phases.append([int(p_), str(ph), round((t - prev) / 1e3, 1)])
            prev = t
        res[name] = {"median_ms": statistics.median(ms), "scalars": sc.cpu().tolist(),
                     "phases_us": phases}
    same = all(np.array_equal(labels[0], x) for x in labels[1:])
    _line("per-phase trace of the inflated random DFA n=10^7 k=4 (default, full and incremental "
          "rounds)", res["default"]["median_ms"], "ms", res["default"]["median_ms"], 30, 3,
          {"trace": res, "labels_equal": same}, higher=False)


def run(args):
    torch.cuda.set_device(bench.dist_env()[2])
    if args.workload == "trace2":
        run_trace2(args)
        return 0
    if args.workload == "random1k":
        run_random1k(args)
    elif args.workload == "path":
        run_path(args)
    elif args.workload in ("batch200m", "batch6g"):
        run_batch(args, "capped" if args.workload == "batch200m" else "drawn")
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "table2":
        run_table2(args)
    elif args.workload == "minimal":
        run_minimal(args)
    return 0

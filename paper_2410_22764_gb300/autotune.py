"""Autotuner for the schedule knobs of the library.

The knobs change no result, only speed:
  * single DFAs: the grid of the multi-CTA kernel (``ctas``) and the size limit of the one-CTA
    kernels (``smem_states``: everything in shared memory up to 8,192 states, 16-bit ids in
    shared memory up to 65,535);
  * batches: the one-CTA limit (``smem_states``), the states per CTA when sizing a team
    (``team_states``), a cap on the grid (``ctas``) and the batch kernel's occupancy (three or
    four resident CTAs per SM, ``flags``).
With ``allow_leader=True`` a single DFA may also be given the leader election (Alg. 2 naivePR,
``algorithm=1``): the partition is the same, the round count is that algorithm's own.

Candidates are timed on the device (CUDA events, median of a few runs after warm-up) and the
fastest is stored in a JSON cache keyed by GPU name and a shape bucket, so later calls with a
similar shape reuse it.  The timing function can be replaced (tests use a fake one).
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

_lock = threading.Lock()
FLAG_BATCH_FOUR_CTAS = 64          # include/dfamin.h: DFAMIN_FLAG_BATCH_FOUR_CTAS


def cache_path() -> str:
    return os.environ.get("DFAMIN_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "dfamin", "tune.json"))


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def single_key(gpu: str, n: int, k: int, closure: bool, leader: bool = False) -> str:
    return (f"{gpu}|single|n2^{round(math.log2(max(n, 1)))}|k{k}|c{int(closure)}"
            + ("|alg" if leader else ""))


def batch_key(gpu: str, ns, ks, closure: bool) -> str:
    count = len(ns)
    trans = sum(int(a) * int(b) for a, b in zip(ns, ks))
    meank = sum(int(b) for b in ks) / max(count, 1)
    return (f"{gpu}|batch|count2^{round(math.log2(max(count, 1)))}"
            f"|t2^{round(math.log2(max(trans, 1)))}|k{round(meank)}|c{int(closure)}")


def single_candidates(n: int, sms: int, leader: bool = False) -> list[dict]:
    cands = [{"ctas": c * sms} for c in (1, 2, 3, 4)]
    if n <= 65535:      # one CTA (shared memory) against the multi-CTA kernel
        cands += [{"smem_states": max(n, 1)}, {"smem_states": 1}]
    if leader:
        cands += [dict(c, algorithm=1) for c in cands if "smem_states" not in c]
    return cands


def batch_candidates(sms: int) -> list[dict]:
    out = []
    for small in (512, 2048, 4096):
        for team in (4096, 16384, 65536):
            out.append({"smem_states": small, "team_states": team})
    out.append({"smem_states": 2048, "team_states": 16384, "ctas": 2 * sms})
    # the batch kernel built for four resident CTAs per SM (fewer registers, more spills)
    for team in (4096, 16384, 65536):
        out.append({"smem_states": 2048, "team_states": team, "flags": FLAG_BATCH_FOUR_CTAS})
    return out


def choose(key: str, candidates: list[dict], measure, path: str | None = None,
           retune: bool = False) -> tuple[dict, dict]:
    """Return (best candidate, {candidate-json: ms}) for `key`, from the cache or by calling
    measure(candidate) -> milliseconds on every candidate (then cached)."""
    path = path or cache_path()
    with _lock:
        data = _load(path)
        if not retune and key in data:
            return data[key]["best"], data[key]["timings"]
    timings = {}
    for c in candidates:
        timings[json.dumps(c, sort_keys=True)] = float(measure(c))
    best = json.loads(min(timings, key=timings.get))
    with _lock:
        data = _load(path)
        data[key] = {"best": best, "timings": timings}
        _store(path, data)
    return best, timings


# ------------------------------------------------------------------------------------------
# device measurement
# ------------------------------------------------------------------------------------------
def _gpu_name_and_sms():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return p.name, p.multi_processor_count


def _time_ms(fn, warmup=2, reps=3) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def tune_single(n: int, k: int, delta, accept, closure: bool = False, retune: bool = False,
                path: str | None = None, allow_leader: bool = False):
    """Tuned options for one DFA (device tensors delta, accept)."""
    from . import dfamin
    gpu, sms = _gpu_name_and_sms()
    ws = dfamin.Workspace()

    def opts(c):
        c = dict(c)
        leader = c.pop("algorithm", 0) == 1
        return dfamin.options(closure=closure, leader=leader, **c)

    def measure(c):
        opt = opts(c)
        return _time_ms(lambda: dfamin.minimize_ex(n, k, delta, accept, opt=opt, workspace=ws))
    best, timings = choose(single_key(gpu, n, k, closure, allow_leader),
                           single_candidates(n, sms, allow_leader), measure, path, retune)
    return opts(best), timings


def cached(key: str, path: str | None = None) -> dict | None:
    """The stored best candidate for `key`, or None (no measurement)."""
    with _lock:
        data = _load(path or cache_path())
    e = data.get(key)
    return e["best"] if e else None


def lookup_batch(state_off, ks, closure: bool = False, path: str | None = None):
    """Options tuned earlier for a batch of this shape bucket on this GPU, or None.  Measures
    nothing, so it is cheap enough for a serving loop."""
    import numpy as np
    from . import dfamin
    gpu, _ = _gpu_name_and_sms()
    ns = np.diff(np.asarray(state_off, dtype=np.int64))
    best = cached(batch_key(gpu, ns.tolist(), list(ks), closure), path)
    return None if best is None else dfamin.options(closure=closure, **best)


def tune_batch(state_off, ks, delta, accept, closure: bool = False, retune: bool = False,
               path: str | None = None):
    """Tuned options for a batch (host state_off / ks, device delta / accept)."""
    import numpy as np
    from . import dfamin
    gpu, sms = _gpu_name_and_sms()
    ns = np.diff(np.asarray(state_off, dtype=np.int64))
    ws = dfamin.Workspace()

    def measure(c):
        plan = dfamin.BatchPlan(state_off, ks, dfamin.options(closure=closure, **c))
        try:
            return _time_ms(lambda: plan.run(delta, accept, workspace=ws))
        finally:
            plan.close()
    best, timings = choose(batch_key(gpu, ns.tolist(), list(ks), closure), batch_candidates(sms),
                           measure, path, retune)
    return dfamin.options(closure=closure, **best), timings

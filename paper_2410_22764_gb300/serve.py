"""Continuous-batching minimization server over the dfamin batch ABI.

Requests (host DFAs) arrive at any time.  The scheduler admits them in arrival order while the
device memory they need fits in an HBM budget, packs everything admitted since the last launch
into one batch (one persistent launch, ``dfamin_batch_plan_run``), and keeps several batches in
flight at once: a batch's host-to-device copies run on a copy stream while earlier batches
compute, and the launches themselves run one after another on one compute stream.  (A batch
launch fills the GPU with CTAs whose teams wait for one another; two such launches side by
side can leave a team's CTAs unscheduled behind the other launch's waiting CTAs until the
team's bounded wait runs out.)  Finished batches are found by polling their events; their
results are copied back asynchronously and their memory returns to the budget.

Deep-refinement requests are run first with a pass cap; those that hit it
(``DFAMIN_ENOCONVERGE``) are rerun on the partial transitive closure (Alg. transPR, Sec. 3.4),
which has the same state equivalence and needs logarithmically many rounds on path-like DFAs.
The returned partition is the same either way; ``passes`` is the count of the run that
finished.

All device work goes through the C ABI; this module only schedules and marshals.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import autotune, dfamin


@dataclass
class Request:
    rid: int
    n: int
    k: int
    delta: np.ndarray
    accept: np.ndarray
    arrival: float
    closure: bool = False
    nbytes: int = 0
    admitted: float | None = None
    done: float | None = None
    out_block: np.ndarray | None = None
    nblocks: int | None = None
    passes: int | None = None
    status: int | None = None
    attempts: int = 0
    cancelled: bool = False

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


@dataclass
class _Batch:
    reqs: list
    closure: bool
    stream_idx: int
    plan: object
    tensors: list
    host_out: torch.Tensor | None      # page-locked labels, or None (labels kept on the device)
    host_per: torch.Tensor
    state_off: np.ndarray
    ev_start: torch.cuda.Event
    ev_end: torch.cuda.Event
    nbytes: int
    dev_out: torch.Tensor | None = None  # the launch's labels on the device


@dataclass
class ServerStats:
    batches: int = 0
    max_inflight: int = 0
    escalated: int = 0
    rejected: int = 0
    solo: int = 0                                   # requests run as single-DFA launches
    intervals: list = field(default_factory=list)   # (start_ms, end_ms) of every batch on device


class Server:
    """Continuous-batching server.

    budget_bytes    device memory the requests in flight may hold together (admission bound)
    streams         batches that may be in flight at once (copies overlap, launches do not)
    max_batch       requests per batch at most
    max_batch_work  transitions (sum of n*k) per batch at most, except that a batch always takes
                    at least one request: a small bound keeps short requests from waiting behind
                    one huge batch, and lets more batches overlap on the device
    pass_cap        plain-refinement passes before a request is rerun on the closure
    solo_work       transitions (n*k) from which a request runs as its own single-DFA launch
                    (`dfamin_minimize_ex`, the whole GPU for one DFA) instead of joining a
                    batch, in which it would get one team and hold the batch up; 0 = never.
    results_on_device  keep every finished request's labels in device memory (a CUDA int32
                    tensor in ``Request.out_block``, owned by the caller and outside the budget)
                    instead of copying them to the host; only the per-request scalars (block
                    count, passes, status) come back
                    On the served size mix (n 1e3..4e6) 2^19 gave the most DFAs per second of
                    2^14..2^22 (3,416/s against 1,499/s batching everything and 1,928/s
                    launching everything alone)
    tuned           use batch options from the autotuner's cache when it has them for the
                    batch's shape (a lookup, no measurement)
    """

    def __init__(self, budget_bytes: int = 32 << 30, streams: int = 4, max_batch: int = 1024,
                 pass_cap: int = 64, device: str | torch.device = "cuda", flags: int = 0,
                 max_batch_work: int = 1 << 62, tuned: bool = True, solo_work: int = 1 << 19,
                 results_on_device: bool = False):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.compute_stream = torch.cuda.Stream(device=self.device)
        self.free = list(range(streams))
        # page-locked staging per stream (rows, acceptance words, labels, per-DFA scalars),
        # grown on demand and reused: a stream's buffers are free again once its batch's end
        # event has been seen, and pinning fresh host memory for every batch costs more than
        # the copy itself
        self._staging = [dict() for _ in range(streams)]
        self.max_batch = max_batch
        self.max_batch_work = int(max_batch_work)
        self.solo_work = int(solo_work)
        self.results_on_device = bool(results_on_device)
        self.pass_cap = pass_cap
        self.flags = flags
        self.tuned = tuned
        self.pending: deque[Request] = deque()
        self.inflight: list[_Batch] = []
        self.used = 0
        self.completed: list[Request] = []
        self.stats = ServerStats()
        self._next_id = 0
        self._base = torch.cuda.Event(enable_timing=True)
        self._base.record(torch.cuda.current_stream(self.device))

    # ---------------------------------------------------------------- requests
    def request_bytes(self, n: int, k: int, closure: bool) -> int:
        """Device bytes one request holds while in flight: inputs, outputs and its share of the
        batch workspace (bounded by the single-DFA workspace)."""
        ws = dfamin.workspace_size(n, k, dfamin.options(closure=closure))
        return ws + 4 * n * k + 4 * ((n + 31) // 32) + 4 * n + 4096

    def submit(self, n: int, k: int, delta: np.ndarray, accept: np.ndarray,
               arrival: float | None = None) -> Request:
        r = Request(self._next_id, n, k, np.ascontiguousarray(delta, dtype=np.int32),
                    np.ascontiguousarray(accept, dtype=np.uint32),
                    time.perf_counter() if arrival is None else arrival)
        self._next_id += 1
        r.nbytes = self.request_bytes(n, k, True)   # admit for the worst case (closure rerun)
        if r.nbytes > self.budget:
            r.status = dfamin.ENOMEM
            r.done = time.perf_counter()
            self.stats.rejected += 1
            self.completed.append(r)
            return r
        self.pending.append(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Withdraw a request that has not been admitted yet."""
        if r in self.pending:
            self.pending.remove(r)
            r.cancelled = True
            r.done = time.perf_counter()
            self.completed.append(r)
            return True
        return False

    # ---------------------------------------------------------------- scheduling
    def idle(self) -> bool:
        return not self.pending and not self.inflight

    def step(self) -> bool:
        """One scheduler iteration: retire finished batches, then launch one new batch if a
        stream is free and something fits.  Returns True if anything happened."""
        progressed = False
        for b in list(self.inflight):
            if b.ev_end.query():
                self._finish(b)
                progressed = True
        if self.free and self.pending:
            reqs = []
            head_closure = self.pending[0].closure
            budget_left = self.budget - self.used
            if self._solo(self.pending[0]):
                if self.pending[0].nbytes <= budget_left:
                    self._launch_solo(self.pending.popleft())
                    progressed = True
                return progressed
            # the batch takes the pending requests of the head's kind in arrival order, passing
            # over the ones that will run as single-DFA launches (they keep their places), until
            # the batch is full by count, budget or work
            work = 0
            passed = []
            while self.pending and len(reqs) < self.max_batch and len(passed) < self.max_batch:
                r = self.pending[0]
                if r.closure != head_closure or self._solo(r):
                    passed.append(self.pending.popleft())
                    continue
                if r.nbytes > budget_left or (reqs and work + r.n * r.k > self.max_batch_work):
                    break
                self.pending.popleft()
                budget_left -= r.nbytes
                work += r.n * r.k
                reqs.append(r)
            self.pending.extendleft(reversed(passed))
            if reqs:
                self._launch(reqs, head_closure)
                progressed = True
        return progressed

    def drain(self, poll_s: float = 20e-6):
        while not self.idle():
            if not self.step():
                time.sleep(poll_s)

    def _launch(self, reqs, closure: bool):
        si = self.free.pop()
        cs, s = self.copy_stream, self.compute_stream
        now = time.perf_counter()
        for r in reqs:
            r.admitted = now
            r.attempts += 1
        nbytes = sum(r.nbytes for r in reqs)
        self.used += nbytes
        # pack straight into page-locked buffers (one host copy of the rows)
        state_off, ks = dfamin.batch_offsets(reqs)
        nd = int(sum(r.n * r.k for r in reqs))
        words = (int(state_off[-1]) + 31) // 32
        h_delta = self._stage(si, "delta", max(nd, 1))
        h_acc = self._stage(si, "acc", max(words, 1))
        delta, acc, state_off, ks = dfamin.pack_batch(reqs, h_delta, h_acc.numpy())
        opt = dfamin.options(closure=closure, max_passes=0 if closure else self.pass_cap,
                             flags=self.flags)
        if self.tuned:
            t = autotune.lookup_batch(state_off, ks, closure)
            if t is not None:
                opt.smem_states, opt.team_states, opt.ctas = t.smem_states, t.team_states, t.ctas
                opt.flags |= t.flags
        plan = dfamin.BatchPlan(state_off, ks, opt)
        host_out = None if self.results_on_device else self._stage(si, "out", plan.states)
        host_per = self._stage(si, "per", 3 * plan.count).view(3, plan.count)
        ev_start = torch.cuda.Event(enable_timing=True)
        ev_copied = torch.cuda.Event()
        ev_end = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            # allocated on the compute stream and filled on the copy stream; a batch's device
            # memory is released only after its end event has been seen (every use finished)
            d_delta = torch.empty(h_delta.numel(), dtype=torch.int32, device=self.device)
            d_acc = torch.empty(h_acc.numel(), dtype=torch.int32, device=self.device)
        with torch.cuda.stream(cs):
            ev_start.record(cs)
            d_delta.copy_(h_delta, non_blocking=True)
            d_acc.copy_(h_acc, non_blocking=True)
            ev_copied.record(cs)
        s.wait_event(ev_copied)
        with torch.cuda.stream(s):
            ws = dfamin.Workspace(self.device)
            out, per = plan.run(d_delta, d_acc, workspace=ws, stream=s)
            if host_out is not None:
                host_out.copy_(out, non_blocking=True)
            host_per.copy_(per, non_blocking=True)
            ev_end.record(s)
        tensors = [h_delta, h_acc, d_delta, d_acc, ws, out, per]
        self.inflight.append(_Batch(reqs, closure, si, plan, tensors, host_out, host_per,
                                    state_off, ev_start, ev_end, nbytes, dev_out=out))
        self.stats.batches += 1
        self.stats.max_inflight = max(self.stats.max_inflight, len(self.inflight))

    def _solo(self, r: Request) -> bool:
        return self.solo_work > 0 and r.n * r.k >= self.solo_work

    def _launch_solo(self, r: Request):
        """One request as its own single-DFA launch, on the same streams as the batches (so that
        launches still run one after another)."""
        si = self.free.pop()
        cs, s = self.copy_stream, self.compute_stream
        r.admitted = time.perf_counter()
        r.attempts += 1
        self.used += r.nbytes
        m, words = r.n * r.k, (r.n + 31) // 32
        h_delta = self._stage(si, "delta", max(m, 1))
        h_acc = self._stage(si, "acc", max(words, 1))
        if m:                                         # torch copies in parallel over host cores
            h_delta[:m].copy_(torch.from_numpy(r.delta.reshape(-1)[:m]))
        h_acc.numpy()[:words] = r.accept.reshape(-1)[:words].view(np.int32)
        host_out = None if self.results_on_device else self._stage(si, "out", r.n)
        host_per = self._stage(si, "per", 3).view(3, 1)
        opt = dfamin.options(closure=r.closure, max_passes=0 if r.closure else self.pass_cap,
                             flags=self.flags)
        ev_start = torch.cuda.Event(enable_timing=True)
        ev_copied = torch.cuda.Event()
        ev_end = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            d_delta = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
            d_acc = torch.empty(max(words, 1), dtype=torch.int32, device=self.device)
        with torch.cuda.stream(cs):
            ev_start.record(cs)
            d_delta.copy_(h_delta, non_blocking=True)
            d_acc.copy_(h_acc, non_blocking=True)
            ev_copied.record(cs)
        s.wait_event(ev_copied)
        with torch.cuda.stream(s):
            ws = dfamin.Workspace(self.device)
            res = dfamin.minimize_ex(r.n, r.k, d_delta[:m] if m else d_delta, d_acc, opt=opt,
                                     workspace=ws, stream=s)
            if host_out is not None:
                host_out.copy_(res.out_block, non_blocking=True)
            host_per.view(-1).copy_(res.scalars, non_blocking=True)
            ev_end.record(s)
        tensors = [h_delta, h_acc, d_delta, d_acc, ws, res.out_block, res.scalars]
        self.inflight.append(_Batch([r], r.closure, si, None, tensors, host_out, host_per,
                                    np.array([0, r.n], dtype=np.int64), ev_start, ev_end,
                                    r.nbytes, dev_out=res.out_block))
        self.stats.batches += 1
        self.stats.solo += 1
        self.stats.max_inflight = max(self.stats.max_inflight, len(self.inflight))

    def _stage(self, si: int, name: str, count: int) -> torch.Tensor:
        """The first `count` int32 of stream si's page-locked buffer `name` (grown by doubling)."""
        buf = self._staging[si].get(name)
        if buf is None or buf.numel() < count:
            size = max(count, 2 * buf.numel() if buf is not None else 0, 1 << 16)
            buf = torch.empty(size, dtype=torch.int32, pin_memory=True)
            self._staging[si][name] = buf
        return buf[:count]

    def _finish(self, b: _Batch):
        now = time.perf_counter()
        per = b.host_per.numpy()
        self.stats.intervals.append((self._base.elapsed_time(b.ev_start),
                                     self._base.elapsed_time(b.ev_end)))
        requeue = []
        for i, r in enumerate(b.reqs):
            st = int(per[2, i])
            if st == dfamin.ENOCONVERGE and not b.closure:
                r.closure = True                      # deep refinement: rerun on the closure
                requeue.append(r)
                self.stats.escalated += 1
                continue
            r.status = st
            r.nblocks = int(per[0, i])
            r.passes = int(per[1, i])
            # the staging buffer is reused by the stream's next batch: keep a copy (torch clones
            # large arrays in parallel over the host's cores)
            lo, hi = int(b.state_off[i]), int(b.state_off[i + 1])
            if b.host_out is None:
                # on the device: a batch's labels share one tensor, so each request gets its
                # own copy (a single-DFA launch's tensor is the request's already)
                r.out_block = b.dev_out if len(b.reqs) == 1 and b.plan is None \
                    else b.dev_out[lo:hi].clone()
            else:
                r.out_block = b.host_out[lo:hi].clone().numpy()
            r.done = now
            self.completed.append(r)
        for r in reversed(requeue):
            self.pending.appendleft(r)
        self.used -= b.nbytes
        self.free.append(b.stream_idx)
        self.inflight.remove(b)
        if b.plan is not None:
            b.plan.close()                            # stream-ordered free: no device sync

    def max_device_overlap(self) -> int:
        """Largest number of batches whose device intervals (start..end events) overlap."""
        ev = []
        for a, z in self.stats.intervals:
            ev.append((a, 1))
            ev.append((z, -1))
        cur = best = 0
        for _, d in sorted(ev, key=lambda x: (x[0], x[1])):
            cur += d
            best = max(best, cur)
        return best

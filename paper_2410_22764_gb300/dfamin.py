"""Thin Python binding of the dfamin C ABI (``include/dfamin.h``).

Argument marshalling only: every step of the minimization runs in the CUDA library
``libdfamin.so`` built from ``csrc/``.  PyTorch supplies device memory and streams.  There is no
CPU fallback: importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DFAMIN_LIBRARY selects another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("DFAMIN_LIBRARY", os.path.join(_HERE, "libdfamin.so"))

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOCONVERGE, EPROBE = range(7)
CLOSURE_OFF, CLOSURE_ON = 0, 1
ALG_SIGNATURE, ALG_LEADER = 0, 1
FLAG_KEEP_IDENTITY = 1
FLAG_HASH_BLOCK_ONLY = 2
FLAG_HASH_CONSTANT = 4
FLAG_TRACE = 8
FLAG_FULL_ROUNDS = 16
FLAG_INCREMENTAL_ROUNDS = 32
FLAG_BATCH_FOUR_CTAS = 64
FLAG_MASKED_ROUNDS = 128
TRACE_BYTES = 262144
TRACE_PHASES = {0: "start", 1: "validate", 2: "init", 3: "closure", 4: "leaders",
                5: "members", 6: "moves", 7: "count", 8: "canonical"}

# names declared in include/dfamin.h (checked against the library's exports by the tests)
ABI_FUNCTIONS = (
    "dfamin_default_options",
    "dfamin_minimize",
    "dfamin_workspace_size",
    "dfamin_minimize_ex",
    "dfamin_status_string",
    "dfamin_last_cuda_error",
    "dfamin_minimize_static",
    "dfamin_minimize_from_host",
    "dfamin_minimize_from_host_workspace_size",
    "dfamin_batch_plan_create",
    "dfamin_batch_plan_destroy",
    "dfamin_batch_workspace_size",
    "dfamin_batch_plan_info",
    "dfamin_batch_plan_run",
    "dfamin_minimize_batch",
    "dfamin_minimize_batch_workspace_size",
    "dfamin_reach_workspace_size",
    "dfamin_reachable",
    "dfamin_quotient_workspace_size",
    "dfamin_quotient",
    "dfamin_minimal_dfa_workspace_size",
    "dfamin_minimal_dfa",
    "dfamin_lts_determinize",
)


class DfaminError(RuntimeError):
    def __init__(self, code: int, what: str):
        detail = ""
        if code in (ECUDA, ENOMEM):
            detail = " [" + _lib.dfamin_last_cuda_error().decode() + "]"
        super().__init__(f"{what}: {status_string(code)} ({code}){detail}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("closure", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("ctas", ctypes.c_int32),
                ("smem_states", ctypes.c_int32), ("team_states", ctypes.c_int32),
                ("algorithm", ctypes.c_int32), ("barrier_timeout_us", ctypes.c_int32),
                ("closure_columns", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    i32, u32, p, sz = ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
    lib.dfamin_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.dfamin_default_options.restype = None
    lib.dfamin_minimize.argtypes = [i32, i32, p, p, p, p, p]
    lib.dfamin_workspace_size.argtypes = [i32, i32, ctypes.POINTER(Options),
                                          ctypes.POINTER(sz)]
    lib.dfamin_minimize_ex.argtypes = [i32, i32, p, p, p, p, ctypes.POINTER(Options), p, sz,
                                       p, p, p]
    lib.dfamin_status_string.argtypes = [ctypes.c_int]
    lib.dfamin_status_string.restype = ctypes.c_char_p
    lib.dfamin_minimize_static.argtypes = [i32, i32, p, p, p, p, ctypes.POINTER(Options), p, p, p]
    lib.dfamin_minimize_static.restype = ctypes.c_int
    lib.dfamin_minimize_from_host.argtypes = [i32, i32, p, p, p, p, ctypes.POINTER(Options), p,
                                              sz, p]
    lib.dfamin_minimize_from_host.restype = ctypes.c_int
    lib.dfamin_minimize_from_host_workspace_size.argtypes = [i32, i32, ctypes.POINTER(Options),
                                                             ctypes.POINTER(sz)]
    lib.dfamin_minimize_from_host_workspace_size.restype = ctypes.c_int
    lib.dfamin_batch_plan_create.argtypes = [i32, p, p, ctypes.POINTER(Options),
                                             ctypes.POINTER(ctypes.c_void_p)]
    lib.dfamin_batch_plan_destroy.argtypes = [p]
    lib.dfamin_batch_workspace_size.argtypes = [p, ctypes.POINTER(sz)]
    lib.dfamin_batch_plan_info.argtypes = [p, p, p, p, p]
    lib.dfamin_batch_plan_run.argtypes = [p, p, p, p, p, p, p, p, sz, p]
    lib.dfamin_minimize_batch.argtypes = [i32, p, p, p, p, p, p, p, ctypes.POINTER(Options), p,
                                          sz, p, p]
    lib.dfamin_minimize_batch_workspace_size.argtypes = [i32, p, p, ctypes.POINTER(Options),
                                                         ctypes.POINTER(sz)]
    for f in (lib.dfamin_batch_plan_create, lib.dfamin_batch_plan_destroy,
              lib.dfamin_batch_workspace_size, lib.dfamin_batch_plan_info,
              lib.dfamin_batch_plan_run, lib.dfamin_minimize_batch,
              lib.dfamin_minimize_batch_workspace_size):
        f.restype = ctypes.c_int
    lib.dfamin_reach_workspace_size.argtypes = [i32, ctypes.POINTER(sz)]
    lib.dfamin_reachable.argtypes = [i32, i32, p, p, i32, p, p, p, p, p, p, sz, p]
    lib.dfamin_quotient_workspace_size.argtypes = [i32, ctypes.POINTER(sz)]
    lib.dfamin_quotient.argtypes = [i32, i32, p, p, p, i32, p, p, p, p, p, p, p, sz, p]
    lib.dfamin_minimal_dfa_workspace_size.argtypes = [i32, i32, ctypes.POINTER(Options),
                                                      ctypes.POINTER(sz)]
    lib.dfamin_minimal_dfa.argtypes = [i32, i32, p, p, i32, ctypes.POINTER(Options), p, p, p, p,
                                       sz, p]
    for f in (lib.dfamin_reach_workspace_size, lib.dfamin_reachable,
              lib.dfamin_quotient_workspace_size, lib.dfamin_quotient,
              lib.dfamin_minimal_dfa_workspace_size, lib.dfamin_minimal_dfa):
        f.restype = ctypes.c_int
    lib.dfamin_lts_determinize.argtypes = [i32, i32, ctypes.c_int64, p, p, p, i32, i32, p, p,
                                           ctypes.POINTER(i32)]
    lib.dfamin_lts_determinize.restype = ctypes.c_int
    lib.dfamin_last_cuda_error.argtypes = []
    lib.dfamin_last_cuda_error.restype = ctypes.c_char_p
    for f in (lib.dfamin_minimize, lib.dfamin_workspace_size, lib.dfamin_minimize_ex):
        f.restype = ctypes.c_int
    del u32
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def status_string(code: int) -> str:
    return _lib.dfamin_status_string(int(code)).decode()


def options(closure: bool = False, max_passes: int = 0, flags: int = 0, ctas: int = 0,
            smem_states: int = 0, team_states: int = 0, leader: bool = False,
            barrier_timeout_us: int = 0, closure_columns: int = 0) -> Options:
    o = Options()
    _lib.dfamin_default_options(ctypes.byref(o))
    o.closure = CLOSURE_ON if closure else CLOSURE_OFF
    o.max_passes, o.flags, o.ctas, o.smem_states = max_passes, flags, ctas, smem_states
    o.team_states = team_states
    o.algorithm = ALG_LEADER if leader else ALG_SIGNATURE
    o.barrier_timeout_us = barrier_timeout_us
    o.closure_columns = closure_columns
    return o


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def workspace_size(n: int, k: int, opt: Options | None = None) -> int:
    out = ctypes.c_size_t(0)
    rc = _lib.dfamin_workspace_size(n, k, ctypes.byref(opt or options()), ctypes.byref(out))
    if rc:
        raise DfaminError(rc, "dfamin_workspace_size")
    return out.value


@dataclass
class Result:
    """Device-side outputs of one call (valid once the stream has passed the call)."""
    out_block: torch.Tensor  # int32 [n]
    scalars: torch.Tensor    # int32 [3] = nblocks, passes, status

    def host(self):
        s = self.scalars.cpu().tolist()
        return self.out_block.cpu().numpy(), s[0], s[1], s[2]


class Workspace:
    """Caller-owned device workspace (torch memory) for dfamin_minimize_ex."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(256, (nbytes + 255) // 256 * 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


def minimize_ex(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor, *,
                opt: Options | None = None, workspace: Workspace | None = None,
                out_block: torch.Tensor | None = None, scalars: torch.Tensor | None = None,
                stream=None) -> Result:
    """Enqueue dfamin_minimize_ex on ``stream``; returns device tensors (no synchronisation).

    ``delta`` int32 [n*k] state-major and ``accept`` a 32-bit bitmap [(n+31)//32] (int32 or
    uint32 storage) must be CUDA tensors.
    """
    opt = opt or options()
    dev = delta.device if k > 0 else accept.device
    if dev.type != "cuda" or accept.device.type != "cuda":
        raise ValueError("delta and accept must be CUDA tensors")
    if k > 0 and (delta.dtype != torch.int32 or delta.numel() != n * k
                  or not delta.is_contiguous()):
        raise ValueError("delta must be a contiguous int32 tensor of n*k entries")
    if accept.element_size() != 4 or accept.numel() < (n + 31) // 32:
        raise ValueError("accept must be a 32-bit bitmap of (n+31)//32 words")
    ws = (workspace or Workspace(dev)).get(workspace_size(n, k, opt))
    if out_block is None:
        out_block = torch.empty(n, dtype=torch.int32, device=dev)
    if scalars is None:
        scalars = torch.zeros(3, dtype=torch.int32, device=dev)
    sp = scalars.data_ptr()
    rc = _lib.dfamin_minimize_ex(
        n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0), _ptr(accept), _ptr(out_block),
        ctypes.c_void_p(sp), ctypes.byref(opt), _ptr(ws), ctypes.c_size_t(ws.numel()),
        ctypes.c_void_p(sp + 4), ctypes.c_void_p(sp + 8), _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_minimize_ex")
    return Result(out_block, scalars)


def minimize_from_host(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor,
                       out_block: torch.Tensor, scalars: torch.Tensor, *,
                       opt: Options | None = None, workspace: Workspace | None = None,
                       stream=None):
    """Enqueue dfamin_minimize_from_host: ``delta`` (int32 [n*k]), ``accept`` (32-bit bitmap),
    ``out_block`` (int32 [n]) and ``scalars`` (int32 [3] = nblocks, passes, status) are CPU
    tensors (page-locked ones, e.g. ``pin_memory()``, for the asynchronous path); the workspace
    is device memory."""
    opt = opt or options()
    for t in (delta, accept, out_block, scalars):
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError("host arrays must be contiguous CPU tensors")
    if k > 0 and (delta.dtype != torch.int32 or delta.numel() != n * k):
        raise ValueError("delta must be an int32 tensor of n*k entries")
    if accept.element_size() != 4 or accept.numel() < (n + 31) // 32:
        raise ValueError("accept must be a 32-bit bitmap of (n+31)//32 words")
    if out_block.dtype != torch.int32 or out_block.numel() < n or scalars.numel() < 3:
        raise ValueError("out_block int32 [n] and scalars int32 [3] expected")
    need = ctypes.c_size_t(0)
    rc = _lib.dfamin_minimize_from_host_workspace_size(n, k, ctypes.byref(opt), ctypes.byref(need))
    if rc:
        raise DfaminError(rc, "dfamin_minimize_from_host_workspace_size")
    ws = (workspace or Workspace()).get(need.value)
    rc = _lib.dfamin_minimize_from_host(
        n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0), _ptr(accept), _ptr(out_block),
        _ptr(scalars), ctypes.byref(opt), _ptr(ws), ctypes.c_size_t(ws.numel()),
        _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_minimize_from_host")


def read_trace(ws: Workspace, n: int, k: int, opt: Options):
    """Decode the phase trace of the last call that used ``ws`` with ``opt`` (FLAG_TRACE set):
    a list of (pass, phase_name, t_ns)."""
    need = workspace_size(n, k, opt)
    raw = ws.buf[need - TRACE_BYTES: need].cpu().numpy().view(np.int64)
    cnt = int(min(raw[0], (TRACE_BYTES // 8 - 1) // 2))
    recs = raw[1: 1 + 2 * cnt].reshape(cnt, 2)
    return [(int(t) >> 8, TRACE_PHASES.get(int(t) & 255, str(int(t) & 255)), int(ns))
            for t, ns in recs]


def minimize(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor, *,
             out_block: torch.Tensor | None = None, nblocks: torch.Tensor | None = None,
             stream=None):
    """Enqueue dfamin_minimize (library-owned workspace); returns (out_block, nblocks)."""
    dev = accept.device
    if out_block is None:
        out_block = torch.empty(n, dtype=torch.int32, device=dev)
    if nblocks is None:
        nblocks = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = _lib.dfamin_minimize(n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0),
                              _ptr(accept), _ptr(out_block), _ptr(nblocks),
                              _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_minimize")
    return out_block, nblocks


def _check_dfa(n, k, delta, accept):
    dev = delta.device if k > 0 else accept.device
    if dev.type != "cuda" or accept.device.type != "cuda":
        raise ValueError("delta and accept must be CUDA tensors")
    if k > 0 and (delta.dtype != torch.int32 or delta.numel() != n * k
                  or not delta.is_contiguous()):
        raise ValueError("delta must be a contiguous int32 tensor of n*k entries")
    if accept.element_size() != 4 or accept.numel() < (n + 31) // 32:
        raise ValueError("accept must be a 32-bit bitmap of (n+31)//32 words")
    return dev


def _size(fn, *args) -> int:
    out = ctypes.c_size_t(0)
    rc = fn(*args, ctypes.byref(out))
    if rc:
        raise DfaminError(rc, fn.__name__)
    return out.value


def reachable(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor, q0: int, *,
              induced: bool = True, workspace: Workspace | None = None, stream=None):
    """Enqueue dfamin_reachable.  Returns device tensors (newid [n], delta' [n*k] or None,
    accept' [(n+31)//32] or None, scalars [2] = count, status)."""
    dev = _check_dfa(n, k, delta, accept)
    ws = (workspace or Workspace(dev)).get(_size(_lib.dfamin_reach_workspace_size, n))
    newid = torch.empty(n, dtype=torch.int32, device=dev)
    rd = torch.empty(max(n * k, 1), dtype=torch.int32, device=dev) if induced else None
    ra = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev) if induced else None
    sc = torch.zeros(2, dtype=torch.int32, device=dev)
    rc = _lib.dfamin_reachable(n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0), _ptr(accept),
                               q0, _ptr(newid), _ptr(rd), _ptr(ra), ctypes.c_void_p(sc.data_ptr()),
                               ctypes.c_void_p(sc.data_ptr() + 4), _ptr(ws),
                               ctypes.c_size_t(ws.numel()), _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_reachable")
    return newid, rd, ra, sc


def quotient(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor, block: torch.Tensor,
             q0: int, newid: torch.Tensor | None = None, *, workspace: Workspace | None = None,
             stream=None):
    """Enqueue dfamin_quotient.  Returns device tensors (delta' [n*k] capacity, accept' bitmap,
    scalars [3] = nstates, q0', status)."""
    dev = _check_dfa(n, k, delta, accept)
    ws = (workspace or Workspace(dev)).get(_size(_lib.dfamin_quotient_workspace_size, n))
    qd = torch.empty(max(n * k, 1), dtype=torch.int32, device=dev)
    qa = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    sc = torch.zeros(3, dtype=torch.int32, device=dev)
    sp = sc.data_ptr()
    rc = _lib.dfamin_quotient(n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0), _ptr(accept),
                              _ptr(block), q0, _ptr(newid), _ptr(qd), _ptr(qa),
                              ctypes.c_void_p(sp), ctypes.c_void_p(sp + 4),
                              ctypes.c_void_p(sp + 8), _ptr(ws), ctypes.c_size_t(ws.numel()),
                              _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_quotient")
    return qd, qa, sc


def minimal_dfa(n: int, k: int, delta: torch.Tensor, accept: torch.Tensor, q0: int, *,
                opt: Options | None = None, workspace: Workspace | None = None, stream=None):
    """Enqueue dfamin_minimal_dfa.  Returns device tensors (delta' [n*k] capacity, accept'
    bitmap, scalars [5] = nstates, q0', reachable states, passes, status)."""
    opt = opt or options()
    dev = _check_dfa(n, k, delta, accept)
    ws = (workspace or Workspace(dev)).get(
        _size(_lib.dfamin_minimal_dfa_workspace_size, n, k, ctypes.byref(opt)))
    qd = torch.empty(max(n * k, 1), dtype=torch.int32, device=dev)
    qa = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    sc = torch.zeros(5, dtype=torch.int32, device=dev)
    rc = _lib.dfamin_minimal_dfa(n, k, _ptr(delta) if k > 0 else ctypes.c_void_p(0),
                                 _ptr(accept), q0, ctypes.byref(opt), _ptr(qd), _ptr(qa),
                                 ctypes.c_void_p(sc.data_ptr()), _ptr(ws),
                                 ctypes.c_size_t(ws.numel()), _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_minimal_dfa")
    return qd, qa, sc


def lts_determinize(n: int, nlabels: int, src, lbl, dst, s0: int, max_states: int = 0):
    """LTS -> DFA (host code, host arrays): powerset construction from s0, every subset
    accepting, plus a non-accepting bottom state.  Returns (nstates, delta int32 [nstates*nlabels],
    accept uint32 bitmap)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    lbl = np.ascontiguousarray(lbl, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if not (src.size == lbl.size == dst.size):
        raise ValueError("src, lbl and dst must have the same length")
    cap = max_states or max(2, 2 * n + 1)
    while True:
        delta = np.empty(max(cap * nlabels, 1), np.int32)
        acc = np.empty((cap + 31) // 32, np.uint32)
        out_n = ctypes.c_int32(0)
        pp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        rc = _lib.dfamin_lts_determinize(n, nlabels, src.size, pp(src), pp(lbl), pp(dst), s0, cap,
                                         pp(delta), pp(acc), ctypes.byref(out_n))
        if rc == ENOMEM and not max_states:
            cap *= 4
            continue
        if rc:
            raise DfaminError(rc, "dfamin_lts_determinize")
        ns = out_n.value
        return ns, delta[: ns * nlabels].copy(), acc[: (ns + 31) // 32].copy()


def to_device(delta: np.ndarray, accept: np.ndarray, device="cuda"):
    """Copy a host DFA (numpy int32 delta, uint32 bitmap) to CUDA tensors."""
    d = torch.from_numpy(np.ascontiguousarray(delta, dtype=np.int32)).to(device)
    a = torch.from_numpy(np.ascontiguousarray(accept, dtype=np.uint32).view(np.int32)).to(device)
    return d, a


def minimize_host(n: int, k: int, delta: np.ndarray, accept: np.ndarray, *,
                  closure: bool = False, flags: int = 0, max_passes: int = 0,
                  leader: bool = False, device="cuda"):
    """Convenience end-to-end call on host arrays; returns (block, nblocks, passes, status)."""
    d, a = to_device(delta, accept, device)
    r = minimize_ex(n, k, d, a, opt=options(closure=closure, flags=flags,
                                            max_passes=max_passes, leader=leader))
    return r.host()


# ------------------------------------------------------------------------------------------
# Batches
# ------------------------------------------------------------------------------------------
def batch_offsets(dfas):
    """(state_off int64[count + 1], k int32[count]) of host DFAs in batch order."""
    ns = np.array([d.n for d in dfas], dtype=np.int64)
    ks = np.array([d.k for d in dfas], dtype=np.int32)
    state_off = np.zeros(len(dfas) + 1, dtype=np.int64)
    state_off[1:] = np.cumsum(ns)
    return state_off, ks


def pack_accept(dfas, state_off, accept_out: np.ndarray | None = None):
    """The batch acceptance bitmap: DFA i's state q at bit state_off[i] + q.  Each DFA's words
    are shifted to its bit offset word by word; bits beyond a DFA's n are cleared.  Written into
    accept_out (at least ceil(sum(n) / 32) 32-bit words) when given."""
    total = int(state_off[-1])
    words = (total + 31) // 32
    acc64 = np.zeros(words + 1, dtype=np.uint64)
    for d, off in zip(dfas, state_off[:-1]):
        n = int(d.n)
        if n == 0:
            continue
        nw = (n + 31) // 32
        a = np.ascontiguousarray(d.accept, dtype=np.uint32).reshape(-1)[:nw].astype(np.uint64)
        if n % 32:
            a[-1] &= np.uint64((1 << (n % 32)) - 1)
        w0, sh = divmod(int(off), 32)
        v = a << np.uint64(sh)
        acc64[w0: w0 + nw] |= v & np.uint64(0xFFFFFFFF)
        acc64[w0 + 1: w0 + nw + 1] |= v >> np.uint64(32)
    if accept_out is None:
        return acc64[:words].astype(np.uint32)
    accept = accept_out.reshape(-1)[:words].view(np.uint32)
    accept[:] = acc64[:words]
    return accept


def pack_batch(dfas, delta_out=None, accept_out: np.ndarray | None = None):
    """Concatenate host DFAs (objects with n, k, delta, accept) into the batch layout of the C
    ABI: (delta int32, accept uint32 bitmap over all states, state_off int64, k int32).

    delta_out / accept_out: optional preallocated outputs (for instance page-locked memory) of
    at least sum(n*k) int32 and ceil(sum(n) / 32) uint32, written in place.  delta_out may be a
    numpy array or a CPU torch tensor (then the rows are copied by torch, in parallel over the
    host's cores, and a numpy view of it is returned)."""
    state_off, ks = batch_offsets(dfas)
    nd = int(sum(int(d.n) * int(d.k) for d in dfas))
    if isinstance(delta_out, torch.Tensor):
        flat = delta_out.reshape(-1)[:nd]
        pos = 0
        for d in dfas:
            m = int(d.n) * int(d.k)
            if m:
                src = np.ascontiguousarray(d.delta, dtype=np.int32).reshape(-1)[:m]
                flat[pos: pos + m].copy_(torch.from_numpy(src))
            pos += m
        delta = flat.numpy()
    else:
        delta = (np.empty(nd, dtype=np.int32) if delta_out is None
                 else delta_out.reshape(-1)[:nd].view(np.int32))
        pos = 0
        for d in dfas:
            m = int(d.n) * int(d.k)
            delta[pos: pos + m] = np.asarray(d.delta, dtype=np.int32).reshape(-1)[:m]
            pos += m
    return delta, pack_accept(dfas, state_off, accept_out), state_off, ks


class BatchPlan:
    """A dfamin batch plan (host schedule + small device table) for one batch shape."""

    def __init__(self, state_off, k, opt: Options | None = None):
        self.state_off = np.ascontiguousarray(state_off, dtype=np.int64)
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        self.count = int(self.k.size)
        self.opt = opt or options()
        self._plan = ctypes.c_void_p(0)
        rc = _lib.dfamin_batch_plan_create(
            self.count, self.state_off.ctypes.data_as(ctypes.c_void_p),
            self.k.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.opt),
            ctypes.byref(self._plan))
        if rc:
            raise DfaminError(rc, "dfamin_batch_plan_create")
        nb = ctypes.c_size_t(0)
        _lib.dfamin_batch_workspace_size(self._plan, ctypes.byref(nb))
        self.workspace_bytes = nb.value
        g, t, st, tr = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _lib.dfamin_batch_plan_info(self._plan, ctypes.byref(g), ctypes.byref(t),
                                    ctypes.byref(st), ctypes.byref(tr))
        self.grid, self.tickets, self.states, self.transitions = g.value, t.value, st.value, tr.value

    def close(self):
        if self._plan and self._plan.value:
            _lib.dfamin_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, delta: torch.Tensor, accept: torch.Tensor, *, workspace: Workspace | None = None,
            out_block: torch.Tensor | None = None, per_dfa: torch.Tensor | None = None,
            stream=None):
        """Enqueue dfamin_batch_plan_run.  Returns (out_block [states], per_dfa [3, count]
        = nblocks, passes, status) as device tensors."""
        dev = accept.device
        ws = (workspace or Workspace(dev)).get(self.workspace_bytes)
        if out_block is None:
            out_block = torch.empty(self.states, dtype=torch.int32, device=dev)
        if per_dfa is None:
            per_dfa = torch.zeros((3, self.count), dtype=torch.int32, device=dev)
        rc = _lib.dfamin_batch_plan_run(
            self._plan, _ptr(delta) if self.transitions > 0 else ctypes.c_void_p(0),
            _ptr(accept), _ptr(out_block), _ptr(per_dfa[0]), _ptr(per_dfa[1]),
            _ptr(per_dfa[2]), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream_handle(stream))
        if rc:
            raise DfaminError(rc, "dfamin_batch_plan_run")
        return out_block, per_dfa

    def split(self, out_block: np.ndarray):
        """Per-DFA views of a concatenated host out_block."""
        return [out_block[self.state_off[i]: self.state_off[i + 1]] for i in range(self.count)]


def minimize_batch(state_off, k, delta: torch.Tensor, accept: torch.Tensor, *,
                   opt: Options | None = None, workspace: Workspace | None = None, stream=None):
    """Enqueue the one-shot dfamin_minimize_batch (host state_off / k, device delta / accept).
    Returns (out_block [states], nblocks [count], status [count]) as device tensors."""
    opt = opt or options()
    state_off = np.ascontiguousarray(state_off, dtype=np.int64)
    k = np.ascontiguousarray(k, dtype=np.int32)
    count = int(k.size)
    pp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    need = ctypes.c_size_t(0)
    rc = _lib.dfamin_minimize_batch_workspace_size(count, pp(state_off), pp(k), ctypes.byref(opt),
                                                   ctypes.byref(need))
    if rc:
        raise DfaminError(rc, "dfamin_minimize_batch_workspace_size")
    dev = accept.device
    ws = (workspace or Workspace(dev)).get(need.value)
    out_block = torch.empty(int(state_off[-1]), dtype=torch.int32, device=dev)
    nblocks = torch.zeros(count, dtype=torch.int32, device=dev)
    status = torch.zeros(count, dtype=torch.int32, device=dev)
    total = int(np.sum(np.diff(state_off) * k.astype(np.int64)))
    rc = _lib.dfamin_minimize_batch(count, pp(state_off), pp(k), ctypes.c_void_p(0),
                                    _ptr(delta) if total > 0 else ctypes.c_void_p(0),
                                    _ptr(accept), _ptr(out_block), _ptr(nblocks),
                                    ctypes.byref(opt), _ptr(ws), ctypes.c_size_t(ws.numel()),
                                    _ptr(status), _stream_handle(stream))
    if rc:
        raise DfaminError(rc, "dfamin_minimize_batch")
    return out_block, nblocks, status

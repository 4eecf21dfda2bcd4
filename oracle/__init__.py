"""CPU oracle for DFA state equivalence (arXiv 2410.22764).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The GPU library never imports it, and the two
share no code: the oracle is the plain sequential C in ``oracle.c`` loaded through ctypes.

Each function follows one passage of the paper:

* :func:`moore`      - Alg. sortPR (Sec. 3.3): signature, sort, adjacent difference, scan.
* :func:`hopcroft`   - Hopcroft's quasi-linear refinement named in Sec. 1.
* :func:`tablefill`  - pairwise marking, the sequential meaning of Alg. 1 ``trans`` (Sec. 3.1).
* :func:`closure`    - the per-letter partial transitive closure of Alg. transPR (Sec. 3.4).
* :func:`naive`      - leader-election refinement, Alg. 2 naivePR (Sec. 3.2).
* :func:`canonical`  - canonical relabelling (block id = rank of the block's smallest state).
* :func:`check_stable` - congruence property check that holds at any size.

All arrays are numpy; ``delta`` is int32 state-major (``delta[s*k+a]``) and ``accept`` is the
uint32 bitmap (LSB first) of the public contract.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ENOCONVERGE = -3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so`` (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, p = ctypes.c_int32, ctypes.c_void_p
            lib.oracle_canonical.argtypes = [i32, p, p, p]
            lib.oracle_moore.argtypes = [i32, i32, p, p, i32, p, p, p]
            lib.oracle_hopcroft.argtypes = [i32, i32, p, p, p, p]
            lib.oracle_tablefill.argtypes = [i32, i32, p, p, p, p, p]
            lib.oracle_closure_levels.argtypes = [i32]
            lib.oracle_closure_levels.restype = i32
            lib.oracle_closure.argtypes = [i32, i32, p, p]
            lib.oracle_check_stable.argtypes = [i32, i32, p, p, p]
            lib.oracle_naive.argtypes = [i32, i32, p, p, i32, p, p, p]
            lib.oracle_naive.restype = ctypes.c_int
            lib.oracle_reachable.argtypes = [i32, i32, p, i32, p, p]
            lib.oracle_reachable.restype = ctypes.c_int
            lib.oracle_quotient.argtypes = [i32, i32, p, p, p, i32, i32, p, p, p]
            lib.oracle_quotient.restype = ctypes.c_int
            for f in (lib.oracle_canonical, lib.oracle_moore, lib.oracle_hopcroft,
                      lib.oracle_tablefill, lib.oracle_closure, lib.oracle_check_stable):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(delta, accept, n, k):
    delta = np.ascontiguousarray(delta, dtype=np.int32).reshape(-1)
    accept = np.ascontiguousarray(accept, dtype=np.uint32).reshape(-1)
    if delta.size != n * k:
        raise ValueError(f"delta has {delta.size} entries, expected n*k = {n * k}")
    if accept.size < (n + 31) // 32:
        raise ValueError("accept bitmap too short")
    if k == 0:
        delta = np.zeros(1, np.int32)
    return delta, accept


def canonical(labels) -> tuple[np.ndarray, int]:
    """Canonical relabelling: id = rank of the block's smallest state. Labels in [0, n)."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = labels.size
    out = np.empty(n, np.int32)
    cnt = ctypes.c_int32(0)
    rc = _load().oracle_canonical(n, _ptr(labels), _ptr(out), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError(f"oracle_canonical failed ({rc})")
    return out, cnt.value


def moore(delta, accept, n: int, k: int, max_passes: int = 0, partial: bool = False):
    """Moore refinement as Alg. sortPR; returns (block, nblocks, passes).  With ``partial``
    the partition reached after ``max_passes`` rounds is returned instead of an error."""
    delta, accept = _prep(delta, accept, n, k)
    out = np.empty(n, np.int32)
    nb, ps = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = _load().oracle_moore(n, k, _ptr(delta), _ptr(accept), max_passes, _ptr(out),
                              ctypes.byref(nb), ctypes.byref(ps))
    if rc == ENOCONVERGE and not partial:
        raise RuntimeError(f"oracle_moore hit max_passes={max_passes}")
    if rc not in (0, ENOCONVERGE):
        raise ValueError(f"oracle_moore failed ({rc})")
    return out, nb.value, ps.value


def naive(delta, accept, n: int, k: int, max_iters: int = 0):
    """Alg. 2 naivePR (smallest writer wins each election); returns (block, nblocks, iters)."""
    delta, accept = _prep(delta, accept, n, k)
    out = np.empty(n, np.int32)
    nb, it = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = _load().oracle_naive(n, k, _ptr(delta), _ptr(accept), max_iters, _ptr(out),
                              ctypes.byref(nb), ctypes.byref(it))
    if rc == ENOCONVERGE:
        raise RuntimeError(f"oracle_naive hit max_iters={max_iters}")
    if rc != 0:
        raise ValueError(f"oracle_naive failed ({rc})")
    return out, nb.value, it.value


def hopcroft(delta, accept, n: int, k: int):
    """Hopcroft's algorithm; returns (block, nblocks)."""
    delta, accept = _prep(delta, accept, n, k)
    out = np.empty(n, np.int32)
    nb = ctypes.c_int32(0)
    rc = _load().oracle_hopcroft(n, k, _ptr(delta), _ptr(accept), _ptr(out), ctypes.byref(nb))
    if rc != 0:
        raise ValueError(f"oracle_hopcroft failed ({rc})")
    return out, nb.value


def tablefill(delta, accept, n: int, k: int):
    """Pairwise marking; returns (block, nblocks, rounds) where rounds is the distinguishing
    depth (length of the longest shortest distinguishing word)."""
    delta, accept = _prep(delta, accept, n, k)
    out = np.empty(n, np.int32)
    nb, rd = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = _load().oracle_tablefill(n, k, _ptr(delta), _ptr(accept), _ptr(out),
                                  ctypes.byref(nb), ctypes.byref(rd))
    if rc != 0:
        raise ValueError(f"oracle_tablefill failed ({rc})")
    return out, nb.value, rd.value


def closure_levels(n: int) -> int:
    """floor(log2 n) + 1: the number of powers a^(2^i), i = 0..floor(log2 n)."""
    return int(_load().oracle_closure_levels(n))


def closure(delta, n: int, k: int) -> np.ndarray:
    """Columns of Alg. transPR: out[a*levels + i, q] = delta^T(q, a^(2^i))."""
    delta = np.ascontiguousarray(delta, dtype=np.int32).reshape(-1)
    levels = closure_levels(n)
    out = np.empty((k * levels, n), np.int32)
    if k == 0:
        return out
    rc = _load().oracle_closure(n, k, _ptr(delta), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_closure failed ({rc})")
    return out


def closure_dfa(delta, n: int, k: int) -> tuple[np.ndarray, int]:
    """The DFA A' of Alg. transPR as a state-major table with k' = k * levels letters."""
    cols = closure(delta, n, k)
    return np.ascontiguousarray(cols.T).reshape(-1), cols.shape[0]


def check_stable(delta, accept, n: int, k: int, labels) -> bool:
    """True iff ``labels`` refines {F, Q\\F} and is stable under delta."""
    delta, accept = _prep(delta, accept, n, k)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    rc = _load().oracle_check_stable(n, k, _ptr(delta), _ptr(accept), _ptr(labels))
    if rc < 0:
        raise ValueError(f"oracle_check_stable failed ({rc})")
    return rc == 1


def reachable(delta, n: int, k: int, q0: int):
    """States reachable from q0 (Sec. 2): (newid, count), newid[s] = rank of s among the
    reachable states in increasing order, -1 if unreachable."""
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    out = np.empty(n, np.int32)
    cnt = ctypes.c_int32(0)
    rc = _load().oracle_reachable(n, k, _ptr(delta), q0, _ptr(out), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError(f"oracle_reachable failed ({rc})")
    return out, cnt.value


def induced(delta, accept, n: int, k: int, newid, count: int):
    """The sub-DFA on the reachable states, renumbered by newid (a plain restriction: every
    successor of a reachable state is reachable)."""
    delta = np.asarray(delta, dtype=np.int32).reshape(n, k) if k else np.zeros((n, 0), np.int32)
    keep = np.flatnonzero(newid >= 0)
    assert keep.size == count
    rdelta = newid[delta[keep]].astype(np.int32).reshape(-1)
    bits = (np.asarray(accept, dtype=np.uint32)[keep >> 5] >> (keep & 31).astype(np.uint32)) & 1
    racc = np.zeros((count + 31) // 32, np.uint32)
    np.bitwise_or.at(racc, np.arange(count) >> 5, (bits << (np.arange(count) & 31)).astype(np.uint32))
    return rdelta, racc


def quotient(delta, accept, n: int, k: int, block, nblocks: int, q0: int):
    """Quotient automaton of a stable partition (Sec. 2): (delta' [nblocks*k], accept' bitmap,
    q0')."""
    delta, accept = _prep(delta, accept, n, k)
    block = np.ascontiguousarray(block, dtype=np.int32)
    qd = np.empty(max(nblocks * k, 1), np.int32)
    qa = np.empty((nblocks + 31) // 32, np.uint32)
    q0o = ctypes.c_int32(0)
    rc = _load().oracle_quotient(n, k, _ptr(delta), _ptr(accept), _ptr(block), nblocks, q0,
                                 _ptr(qd), _ptr(qa), ctypes.byref(q0o))
    if rc != 0:
        raise ValueError(f"oracle_quotient failed ({rc})")
    return qd[: nblocks * k], qa, q0o.value


def minimal_dfa(delta, accept, n: int, k: int, q0: int):
    """The minimal DFA of (delta, accept, q0) (Sec. 2): unreachable states removed, then
    equivalent states merged (Hopcroft, canonical ids).  Returns (delta', accept', nstates,
    q0', nreach)."""
    newid, cnt = reachable(delta, n, k, q0)
    rdelta, racc = induced(delta, accept, n, k, newid, cnt)
    block, nb = hopcroft(rdelta, racc, cnt, k)
    qd, qa, q0m = quotient(rdelta, racc, cnt, k, block, nb, int(newid[q0]))
    return qd, qa, nb, q0m, cnt


def lts_to_dfa(n: int, nlabels: int, src, lbl, dst, s0: int):
    """LTS -> DFA as Sec. 4.1 describes it: the powerset construction from s0 (FIFO order of
    discovery, labels in increasing order), every subset accepting, plus a non-accepting bottom
    state that takes every missing transition.  Returns (nstates, delta, accept bitmap)."""
    succ = {}
    for s, a, t in zip(np.asarray(src).tolist(), np.asarray(lbl).tolist(),
                       np.asarray(dst).tolist()):
        succ.setdefault((s, a), set()).add(t)
    start = frozenset([s0])
    ids, order, rows = {start: 0}, [start], []
    i = 0
    while i < len(order):
        S = order[i]
        i += 1
        row = []
        for a in range(nlabels):
            T = frozenset(t for s in S for t in succ.get((s, a), ()))
            if not T:
                row.append(None)
                continue
            if T not in ids:
                ids[T] = len(order)
                order.append(T)
            row.append(ids[T])
        rows.append(row)
    bottom = len(order)
    total = bottom + 1
    delta = np.array([bottom if t is None else t for row in rows for t in row] +
                     [bottom] * nlabels, dtype=np.int32)
    acc = np.zeros((total + 31) // 32, np.uint32)
    for q in range(bottom):
        acc[q >> 5] |= np.uint32(1 << (q & 31))
    return total, delta, acc

"""The CPU oracle over many DFAs at once: one DFA per task, a process pool over all host cores.

Test infrastructure only.  The oracle's routines stay plain and sequential; the parallelism is
across DFAs.  Workers are started with the ``spawn`` method (a pool forked from a process that
already holds a CUDA context can hang), and every worker regenerates its DFA from the batch
draws (n, k, p, seed) with the same seeded generator that built the batch, so no large array
crosses a process boundary.

A task returns the oracle's canonical labels in full for small DFAs, or their SHA-256 digest
(of the little-endian int32 array) for large ones; the caller compares the GPU's labels the same
way, so the comparison is element by element either way.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np


def label_digest(labels: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(labels, dtype="<i4").tobytes()).hexdigest()


def _member(task):
    """(index, n, k, p, seed, mode) -> (index, labels or digest, nblocks, passes or -1)."""
    i, n, k, p, seed, mode = task
    import oracle
    from paper_2410_22764_gb300 import inputs as I
    delta, acc, _, _ = I.random_batch([n], [k], [p], [seed], threads=1)
    if mode == "moore":
        labels, nb, passes = oracle.moore(delta, acc, n, k)
        return i, labels, nb, passes
    labels, nb = oracle.hopcroft(delta, acc, n, k)
    return i, label_digest(labels), nb, -1


def make_pool(processes: int | None = None):
    """A spawn-started pool over the host's cores (safe to create after CUDA is initialised)."""
    return mp.get_context("spawn").Pool(processes or max(1, os.cpu_count() or 1))


class BatchJob:
    """Oracle results for every member of a batch of random DFAs (member i is
    random_dfa(ns[i], ks[i], ps[i], seeds[i])), computed in the pool while the caller does other
    work.  Members with n <= moore_max_n run Moore (labels and pass count), the others Hopcroft
    (labels only).  Labels of members with n >= digest_min_n come back as digests."""

    def __init__(self, pool, ns, ks, ps, seeds, moore_max_n: int = 300_000,
                 digest_min_n: int = 1 << 62):
        self.ns = np.asarray(ns, dtype=np.int64)
        self.digest_min_n = digest_min_n
        tasks = []
        # largest first, so that the long tasks do not finish last
        for i in np.argsort(-self.ns * np.asarray(ks, dtype=np.int64), kind="stable"):
            i = int(i)
            n, k = int(ns[i]), int(ks[i])
            mode = "moore" if n <= moore_max_n else "hopcroft"
            tasks.append((i, n, k, float(ps[i]), int(seeds[i]), mode))
        self._async = pool.map_async(_member, tasks, chunksize=1)

    def results(self, timeout: float | None = None):
        """A list indexed by member: (labels or digest, nblocks, passes or -1)."""
        out = [None] * int(self.ns.size)
        for i, lab, nb, passes in self._async.get(timeout):
            if not isinstance(lab, str) and int(self.ns[i]) >= self.digest_min_n:
                lab = label_digest(lab)
            out[i] = (lab, nb, passes)
        return out

"""Distinguishing depth of the deep-refinement path DFA (test infrastructure only).

For the path DFA (letter 0: i -> min(i+1, n-1); every other letter the identity; state i
accepting iff w[i] = 1) the only thing a word changes is how far along the path it moves, so
state i sees the acceptance sequence u_i = w[i], w[i+1], ..., w[n-1], w[n-1], w[n-1], ...
Two states are equivalent iff u_i = u_j, and the shortest word that tells them apart has length
LCP(u_i, u_j) (Sec. 2, delta*).  Round r of partition refinement separates exactly the pairs
whose shortest distinguishing word has length r, so the number of rounds that split something
is the distinguishing depth D = max over inequivalent pairs of LCP(u_i, u_j); the number of
executed passes is D + 1 (one confirming pass) unless the final partition is discrete, when it
is D (the same stopping rule as the oracle's Moore loop; Sec. 3.3 ties the iteration count to
the length of the shortest distinguishing word).

Computed without any refinement: ranks of the suffixes of S = w + w[n-1]^n by prefix doubling,
then the LCP of neighbouring suffixes (in sorted order) by binary lifting over the stored rank
levels.  Inequivalent pairs have LCP < n; equivalent pairs run to the end of S.
"""
from __future__ import annotations

import numpy as np


def path_depth(w) -> tuple[int, int]:
    """Returns (D, classes) for the acceptance string w (0/1 array of length n >= 1)."""
    w = np.asarray(w, dtype=np.int64)
    n = int(w.size)
    if n == 1:
        return 0, 1
    S = np.concatenate([w, np.full(n, w[-1], dtype=np.int64)])
    m = S.size
    ranks = [S.copy()]                     # ranks[t][i]: rank of S[i : i + 2^t]
    rank = S.copy()
    t = 0
    while (1 << t) < m:
        h = 1 << t
        second = np.full(m, -1, dtype=np.int64)
        second[: m - h] = rank[h:]
        order = np.lexsort((second, rank))
        a, b = rank[order], second[order]
        new = np.empty(m, dtype=np.int64)
        step = np.ones(m, dtype=np.int64)
        step[0] = 0
        step[1:] = (a[1:] != a[:-1]) | (b[1:] != b[:-1])
        new[order] = np.cumsum(step)
        rank = new
        ranks.append(rank.copy())
        t += 1
    sa = np.argsort(rank, kind="stable")
    sa = sa[sa < n]                        # suffixes that are states
    x, y = sa[:-1].copy(), sa[1:].copy()
    lcp = np.zeros(x.size, dtype=np.int64)
    for lvl in range(len(ranks) - 1, -1, -1):
        h = 1 << lvl
        px, py = x + lcp, y + lcp
        ok = (px + h <= m) & (py + h <= m)
        same = np.zeros(x.size, dtype=bool)
        idx = np.nonzero(ok)[0]
        same[idx] = ranks[lvl][px[idx]] == ranks[lvl][py[idx]]
        lcp[same] += h
    equivalent = lcp >= m - np.maximum(x, y)   # one suffix is a prefix of the other
    classes = n - int(equivalent.sum())
    depth = int(lcp[~equivalent].max()) if (~equivalent).any() else 0
    return depth, classes


def path_passes(w) -> tuple[int, int]:
    """Passes of the refinement loop (stop on an unchanged count or a discrete partition) and
    the class count."""
    depth, classes = path_depth(w)
    n = int(np.asarray(w).size)
    return depth + (1 if classes < n else 0), classes

"""Frontier sizes of the paper's unfused verification loop — TEST INFRASTRUCTURE ONLY.

The same rule as the rest of ``oracle/``: only tests, ``smoke()`` and the benchmark's CPU legs may use it, and it
shares no code with the CUDA library.

Algorithm 1 matches the triangle query by an all-source BFS in rounds (Sec. III-A/III-B): a filter of candidate
sources by NE, then per round an advance over the out-edges of the partial matches, the constraint check per
traversed edge, and a compaction of the survivors.  With the 1- and 2-look-ahead of Sec. III-C and a visiting
order that orients every edge towards the later vertex, the sizes of those frontiers follow from the definitions
alone:

* candidates  |{u : d+(u) >= 2}|                                    (NE filter, 2-look-ahead)
* frontier1   sum of d+(u) over the candidates                       (hop-1 advance: one slot per (u, v))
* partials    |{(u, v) : u a candidate, u -> v, d+(v) > 0}|          (1-look-ahead, compacted)
* frontier2   sum of d+(v) over the partials                         (hop-2 advance: one slot per (u, v, w))
* matches     the triangle count (hop-2 slots closed by u -> w)

The visiting order is the one the library documents for tc_build (a reading of Sec. III-C, which only needs a total
order): vertices ascending by the number of input pairs at the vertex (self-loops excluded, repeated pairs counted
each time), ties by id.  ``unfused_frontiers`` computes the sizes with numpy set operations; ``unfused_frontiers_brute``
enumerates paths with Python loops on tiny graphs.  Both are pinned by closed forms in tests/test_unfused.py.
"""
from __future__ import annotations

import numpy as np


def visiting_rank(src, dst, n: int) -> np.ndarray:
    """rank[x] = position of x in the (input-pair count, id) order."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    cnt = np.bincount(src[keep], minlength=n) + np.bincount(dst[keep], minlength=n)
    order = np.lexsort((np.arange(n), cnt))  # primary key: count, then id
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    return rank


def unfused_frontiers(src, dst, n: int) -> dict:
    """The four frontier sizes above (without matches), vectorised."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    rank = visiting_rank(src, dst, n)
    keep = src != dst
    a, b = rank[src[keep]], rank[dst[keep]]
    key = np.unique(np.minimum(a, b) * max(n, 1) + np.maximum(a, b))
    lo, hi = key // max(n, 1), key % max(n, 1)
    dplus = np.bincount(lo, minlength=n)
    cand = dplus >= 2
    slot1 = cand[lo]
    kept1 = slot1 & (dplus[hi] > 0)
    return {"candidates": int(cand.sum()), "frontier1": int(dplus[cand].sum()), "partials": int(kept1.sum()),
            "frontier2": int(dplus[hi[kept1]].sum())}


def unfused_frontiers_brute(src, dst, n: int) -> dict:
    """The same sizes by enumerating vertex pairs and triples in the visiting order (tiny graphs only)."""
    pairs = [(int(s), int(d)) for s, d in zip(src, dst) if int(s) != int(d)]
    cnt = [0] * n
    for s, d in pairs:
        cnt[s] += 1
        cnt[d] += 1
    order = sorted(range(n), key=lambda x: (cnt[x], x))
    pos = {x: i for i, x in enumerate(order)}
    adj = [set() for _ in range(n)]
    for s, d in pairs:
        adj[s].add(d)
        adj[d].add(s)
    out = {x: [y for y in adj[x] if pos[y] > pos[x]] for x in range(n)}
    res = {"candidates": 0, "frontier1": 0, "partials": 0, "frontier2": 0}
    for u in range(n):
        if len(out[u]) < 2:
            continue
        res["candidates"] += 1
        for v in out[u]:
            res["frontier1"] += 1
            if not out[v]:
                continue
            res["partials"] += 1
            for _w in out[v]:
                res["frontier2"] += 1
    return res

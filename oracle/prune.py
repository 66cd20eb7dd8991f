"""The NE filter applied until it settles (2-core peeling) — TEST INFRASTRUCTURE ONLY.

The same rule as the rest of ``oracle/``: only tests, ``smoke()`` and the benchmark's CPU legs may use it, and it
shares no code with the CUDA library.

Sec. III-A takes NE, the neighbourhood encoding, to be the degree, filters the candidate vertices on it and updates
it after each filtering.  For the triangle query a vertex needs degree >= 2, so one filtering round removes every
edge with an endpoint of degree below 2 in the current simple graph, and the rounds repeat until one removes
nothing: what is left is the 2-core.  ``ne_filter_rounds`` is that procedure, written on numpy arrays of the distinct
undirected edges; it is pinned in tests/test_prune.py by networkx's k_core and by closed forms (paths, stars,
cycles, cliques with tails).
"""
from __future__ import annotations

import numpy as np


def distinct_edges(src, dst, n: int):
    """The simple graph of the pairs: (lo, hi) arrays of the distinct undirected edges, lo < hi."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    a, b = src[keep], dst[keep]
    key = np.unique(np.minimum(a, b) * max(n, 1) + np.maximum(a, b))
    return key // max(n, 1), key % max(n, 1)


def ne_filter_rounds(src, dst, n: int, max_rounds: int = 0):
    """Rounds of the degree >= 2 filter (max_rounds = 0: until a round removes nothing).

    Returns ({"rounds", "edges_removed", "vertices_removed"}, (lo, hi) of the edges kept).  rounds counts the rounds
    that removed at least one edge; vertices_removed counts vertices that had an edge before and have none after.
    """
    lo, hi = distinct_edges(src, dst, n)
    m0 = lo.size

    def with_edge(lo, hi):
        return int(np.count_nonzero(np.bincount(np.concatenate([lo, hi]), minlength=n)))

    nz0 = with_edge(lo, hi)
    rounds = 0
    while not max_rounds or rounds < max_rounds:
        deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
        kill = (deg[lo] < 2) | (deg[hi] < 2)
        if not kill.any():
            break
        lo, hi = lo[~kill], hi[~kill]
        rounds += 1
    return ({"rounds": rounds, "edges_removed": int(m0 - lo.size), "vertices_removed": nz0 - with_edge(lo, hi)},
            (lo, hi))

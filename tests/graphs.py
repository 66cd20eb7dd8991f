"""Small graphs with known triangle counts, for pinning the oracle and for GPU parity cases.

Each constructor returns (src, dst, n, T, t): the edge pairs as int32 arrays, the vertex count, and the closed-form
triangle count and per-vertex counts that graph theory fixes for it (no oracle involved).
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _pack(edges, n, T, t):
    e = np.array(list(edges), dtype=np.int32).reshape(-1, 2)
    return e[:, 0].copy(), e[:, 1].copy(), n, T, np.asarray(t, dtype=np.uint64)


def complete(n):
    """K_n: every 3-set is a triangle, T = C(n,3); each vertex in C(n-1,2)."""
    a, b = np.triu_indices(n, 1)
    return a.astype(np.int32), b.astype(np.int32), n, math.comb(n, 3), np.full(n, math.comb(n - 1, 2), np.uint64)


def wheel(k):
    """Wheel: hub 0 joined to a k-cycle 1..k.  For k >= 4 the triangles are the k hub-spokes-rim ones: T = k,
    t(hub) = k, t(rim) = 2.  k = 3 is K4."""
    if k == 3:
        return complete(4)
    edges = [(0, i) for i in range(1, k + 1)] + [(i, i % k + 1) for i in range(1, k + 1)]
    return _pack(edges, k + 1, k, [k] + [2] * k)


def cycle(n):
    """C_n: one triangle when n = 3, none when n > 3."""
    edges = [(i, (i + 1) % n) for i in range(n)]
    return _pack(edges, n, 1 if n == 3 else 0, [1 if n == 3 else 0] * n)


def complete_bipartite(a, b):
    """K_{a,b}: bipartite, so triangle-free."""
    edges = [(i, a + j) for i in range(a) for j in range(b)]
    return _pack(edges, a + b, 0, [0] * (a + b))


def complete_tripartite(a, b, c):
    """K_{a,b,c}: a triangle takes one vertex per part: T = abc; a vertex of the first part lies in bc, etc."""
    parts = [range(0, a), range(a, a + b), range(a + b, a + b + c)]
    edges = [(x, y) for p, q in itertools.combinations(parts, 2) for x in p for y in q]
    t = [b * c] * a + [a * c] * b + [a * b] * c
    return _pack(edges, a + b + c, a * b * c, t)


def friendship(k):
    """Friendship (windmill) graph F_k: k triangles sharing vertex 0.  T = k; t(0) = k; others 1."""
    edges = []
    for i in range(k):
        x, y = 1 + 2 * i, 2 + 2 * i
        edges += [(0, x), (0, y), (x, y)]
    return _pack(edges, 2 * k + 1, k, [k] + [1] * (2 * k))


def icosahedron():
    """Icosahedron from its vertex coordinates (cyclic permutations of (0, +-1, +-phi)); adjacent = at distance 2.
    Its triangles are exactly its 20 faces, and 5 faces meet at each vertex."""
    phi = (1 + 5 ** 0.5) / 2
    pts = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            pts += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    pts = np.array(pts)
    edges = [(i, j) for i, j in itertools.combinations(range(12), 2)
             if abs(np.linalg.norm(pts[i] - pts[j]) - 2.0) < 1e-9]
    assert len(edges) == 30
    return _pack(edges, 12, 20, [5] * 12)


def disjoint_union(*graphs):
    src, dst, t = [], [], []
    off, T = 0, 0
    for s, d, n, Tg, tg in graphs:
        src.append(s + off)
        dst.append(d + off)
        t.append(tg)
        off += n
        T += Tg
    return (np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32), off, T,
            np.concatenate(t).astype(np.uint64))


def closed_form_cases():
    """(name, graph) pairs covering every closed form above."""
    cases = [(f"K{n}", complete(n)) for n in (1, 2, 3, 4, 5, 8, 13, 40)]
    cases += [(f"W{k}", wheel(k)) for k in (3, 4, 5, 9, 33)]
    cases += [(f"C{n}", cycle(n)) for n in (3, 4, 5, 17)]
    cases += [(f"K{a},{b}", complete_bipartite(a, b)) for a, b in ((1, 1), (3, 4), (10, 17))]
    cases += [(f"K{a},{b},{c}", complete_tripartite(a, b, c)) for a, b, c in ((1, 1, 1), (2, 3, 4), (5, 7, 9))]
    cases += [(f"F{k}", friendship(k)) for k in (1, 2, 7)]
    cases += [("icosahedron", icosahedron())]
    for name in sorted(os.listdir(GOLDEN)):
        if name.endswith(".txt"):
            cases.append((name[:-4], read_golden(name)))
    return cases


def read_golden(name):
    """Golden edge-list file: '# n=.. T=.. [m=..] [t=a,b,..]' header line, then one 'u v' pair per line."""
    n = T = None
    t = None
    pairs = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                for tok in line[1:].split():
                    if tok.startswith("n="):
                        n = int(tok[2:])
                    elif tok.startswith("T="):
                        T = int(tok[2:])
                    elif tok.startswith("t="):
                        t = [int(x) for x in tok[2:].split(",")]
                continue
            u, v = line.split()
            pairs.append((int(u), int(v)))
    if t is None:
        t = [0] * n if T == 0 else None
    return _pack(pairs, n, T, t)


def random_simple_pairs(rng: np.random.Generator, n: int, m: int, noise: bool = True):
    """Random pairs on [0, n), optionally with flips, repeats and self-loops mixed in."""
    src = rng.integers(0, n, size=m, dtype=np.int32)
    dst = rng.integers(0, n, size=m, dtype=np.int32)
    if noise and m > 0:
        k = max(1, m // 10)
        idx = rng.integers(0, m, size=k)
        src = np.concatenate([src, dst[idx], rng.integers(0, n, size=k, dtype=np.int32)])
        loops = src[-k:]
        dst = np.concatenate([dst, src[idx], loops])
    return src.astype(np.int32), dst.astype(np.int32)


def dense_counts(src, dst, n):
    """Brute force from linear algebra: with A the 0/1 adjacency matrix of the simple graph, trace(A^3) counts
    closed 3-walks, 6 per triangle, and (A^3)_xx counts those through x, 2 per triangle containing x."""
    A = np.zeros((n, n), dtype=np.int64)
    A[src, dst] = 1
    A[dst, src] = 1
    np.fill_diagonal(A, 0)
    A3 = A @ A @ A
    return int(np.trace(A3)) // 6, (np.diag(A3) // 2).astype(np.uint64), int(A.sum()) // 2

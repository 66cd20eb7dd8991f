"""Pins for the CPU oracle against facts fixed by graph theory and linear algebra (no GPU).

A plausible slip in the oracle — a dropped per-vertex term, an off-by-one in the suffix start, a missed
symmetrisation, duplicates or self-loops counted — fails at least one of: the closed forms, the dense
trace(A^3)/6 / diag(A^3)/2 brute force, or the invariances below.
"""
import math

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs


@pytest.mark.parametrize("name,g", graphs.closed_form_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_closed_forms(name, g):
    src, dst, n, T, t = g
    got_T, _, got_t = oracle.count(src, dst, n, per_vertex=True)
    assert got_T == T
    if t is not None:
        np.testing.assert_array_equal(got_t, t)
    # the definition-based per-vertex routine agrees on every vertex
    vt, _ = oracle.vertex_triangles(src, dst, n, np.arange(n))
    if t is not None:
        np.testing.assert_array_equal(vt, t)
    assert int(got_t.sum()) == 3 * T


def test_golden_k4_noise_edge_count():
    src, dst, n, T, t = graphs.read_golden("k4_with_noise.txt")
    got_T, m = oracle.count(src, dst, n)
    assert (got_T, m) == (4, 6)


def test_empty_graphs():
    e = np.zeros(0, dtype=np.int32)
    assert oracle.count(e, e, 0) == (0, 0)
    assert oracle.count(e, e, 7) == (0, 0)
    loops = np.arange(5, dtype=np.int32)
    T, m, t = oracle.count(loops, loops, 5, per_vertex=True)
    assert (T, m) == (0, 0) and not t.any()


@pytest.mark.parametrize("seed", range(12))
def test_dense_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 200))
    density = rng.choice([0.02, 0.1, 0.3, 0.7])
    m = int(density * n * (n - 1) / 2)
    src, dst = graphs.random_simple_pairs(rng, n, m)
    T, tv, m_dense = graphs.dense_counts(src, dst, n)
    got_T, got_m, got_t = oracle.count(src, dst, n, per_vertex=True, threads=int(rng.integers(1, 5)))
    assert got_T == T and got_m == m_dense
    np.testing.assert_array_equal(got_t, tv)
    xs = rng.integers(0, n, size=min(n, 20))
    vt, deg = oracle.vertex_triangles(src, dst, n, xs, threads=2)
    np.testing.assert_array_equal(vt, tv[xs])


def _rmat_small(scale=11, ef=12, seed=5):
    spec = graphgen.rmat(scale, ef, seed)
    s, d = spec.edges()
    return s, d, spec.n


def test_invariance_relabel_shuffle_flip_noise():
    src, dst, n = _rmat_small()
    T, m, t = oracle.count(src, dst, n, per_vertex=True)
    assert T > 1000  # the case must be non-trivial
    rng = np.random.default_rng(1)
    perm = rng.permutation(n).astype(np.int32)
    T2, m2, t2 = oracle.count(perm[src], perm[dst], n, per_vertex=True)
    assert (T2, m2) == (T, m)
    np.testing.assert_array_equal(t2[perm], t)
    order = rng.permutation(src.size)
    flip = rng.random(src.size) < 0.5
    s3 = np.where(flip, dst, src)[order]
    d3 = np.where(flip, src, dst)[order]
    assert oracle.count(s3, d3, n)[:2] == (T, m)
    # repeated pairs and self-loops change nothing
    extra = rng.integers(0, src.size, size=src.size // 3)
    loops = rng.integers(0, n, size=1000, dtype=np.int32)
    s4 = np.concatenate([src, dst[extra], loops])
    d4 = np.concatenate([dst, src[extra], loops])
    assert oracle.count(s4, d4, n)[:2] == (T, m)


def test_disjoint_union_additive():
    g1 = graphs.complete(9)
    s, d, n = _rmat_small(9, 8, 3)
    T2, _ = oracle.count(s, d, n)
    g2 = (s, d, n, T2, np.zeros(n, dtype=np.uint64))
    g3 = graphs.wheel(6)
    src, dst, N, T, _ = graphs.disjoint_union(g1, g2, g3)
    assert oracle.count(src, dst, N)[0] == T == math.comb(9, 3) + T2 + 6


def test_edge_deletion_delta():
    """Removing edge {a,b} destroys exactly the triangles a-b-c, one per common neighbour c."""
    src, dst, n = _rmat_small(10, 10, 9)
    T, m = oracle.count(src, dst, n)
    a, b = int(src[0]), int(dst[0])
    assert a != b
    nbr = [set() for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            nbr[u].add(v)
            nbr[v].add(u)
    common = len(nbr[a] & nbr[b])
    keep = ~(((src == a) & (dst == b)) | ((src == b) & (dst == a)))
    T2, m2 = oracle.count(src[keep], dst[keep], n)
    assert m2 == m - 1
    assert T - T2 == common


def test_vertex_triangles_matches_count_per_vertex():
    src, dst, n = _rmat_small(12, 16, 11)
    T, _, t = oracle.count(src, dst, n, per_vertex=True)
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.argsort(-t.astype(np.int64))[:8], rng.integers(0, n, size=40)])
    vt, _ = oracle.vertex_triangles(src, dst, n, xs)
    np.testing.assert_array_equal(vt, t[xs])


def test_thread_count_does_not_change_result():
    src, dst, n = _rmat_small(12, 8, 2)
    ref = oracle.count(src, dst, n, per_vertex=True, threads=1)
    for th in (2, 3, 8):
        got = oracle.count(src, dst, n, per_vertex=True, threads=th)
        assert got[:2] == ref[:2]
        np.testing.assert_array_equal(got[2], ref[2])


def test_out_of_range_ids_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.count(np.array([0, 5], dtype=np.int32), np.array([1, 1], dtype=np.int32), 5)
    with pytest.raises(oracle.OracleError):
        oracle.count(np.array([-1], dtype=np.int32), np.array([1], dtype=np.int32), 5)
    with pytest.raises(oracle.OracleError):
        oracle.vertex_triangles(np.array([0], dtype=np.int32), np.array([1], dtype=np.int32), 2, [2])


def test_er4096_statistical_sanity():
    """Not a parity pin: G(4096, 16/4095) draws no repeats, so the oracle keeps every generated pair (m within 4
    standard deviations of C(n,2) p = 32768), and the expected triangle count is C(n,3) p^3 = 682.7; a 30% band is
    > 7 standard deviations."""
    spec = graphgen.config("er4096")
    s, d = spec.edges()
    T, m = oracle.count(s, d, spec.n)
    p = 16 / 4095
    assert m == s.size and abs(m - 32768) < 4 * math.sqrt(32768 * (1 - p))
    expect = math.comb(4096, 3) * p ** 3
    assert abs(T - expect) < 0.3 * expect

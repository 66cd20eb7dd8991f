"""The NE filter to a fixpoint (2-core peeling, tc_build_pruned).

CPU: the peeling definition in oracle/prune.py against networkx's k_core and closed forms.  GPU: tc_build_pruned
through the C ABI: counts, per-vertex counts and listings unchanged (against the oracle on the unpruned input), the
removal statistics equal to the definition's, and the pruned graph's size reported by tc_graph_get_info.
"""
import math

import numpy as np
import pytest

import graphgen
import oracle
from oracle import prune
from tests import graphs


def _path(k):
    """P_k: k vertices in a line."""
    return np.arange(k - 1, dtype=np.int32), np.arange(1, k, dtype=np.int32), k


def _clique_with_tail(c, tail):
    """K_c on 0..c-1 with a path of `tail` edges hanging from vertex c-1."""
    a, b = np.triu_indices(c, 1)
    pa = np.arange(c - 1, c - 1 + tail)
    src = np.concatenate([a, pa]).astype(np.int32)
    dst = np.concatenate([b, pa + 1]).astype(np.int32)
    return src, dst, c + tail


# ---------------------------------------------------------------------------------------------------------------
# CPU pins
# ---------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [2, 3, 4, 5, 10, 11])
def test_path_peels_two_end_edges_per_round(k):
    st, (lo, hi) = prune.ne_filter_rounds(*_path(k))
    assert st == {"rounds": math.ceil((k - 1) / 2), "edges_removed": k - 1, "vertices_removed": k} and lo.size == 0


@pytest.mark.parametrize("c,tail", [(5, 1), (5, 7), (4, 20)])
def test_clique_tail_peels_one_edge_per_round(c, tail):
    st, (lo, hi) = prune.ne_filter_rounds(*_clique_with_tail(c, tail))
    assert st == {"rounds": tail, "edges_removed": tail, "vertices_removed": tail}
    assert lo.size == c * (c - 1) // 2


def test_star_cycle_clique():
    k = 9
    src = np.zeros(k, np.int32)
    dst = np.arange(1, k + 1, dtype=np.int32)
    assert prune.ne_filter_rounds(src, dst, k + 1)[0] == {"rounds": 1, "edges_removed": k, "vertices_removed": k + 1}
    for g in (graphs.cycle(8), graphs.complete(6)):
        assert prune.ne_filter_rounds(g[0], g[1], g[2])[0] == {"rounds": 0, "edges_removed": 0, "vertices_removed": 0}


def test_max_rounds_stops_early():
    st, _ = prune.ne_filter_rounds(*_clique_with_tail(5, 7), max_rounds=3)
    assert st == {"rounds": 3, "edges_removed": 3, "vertices_removed": 3}


@pytest.mark.parametrize("seed", range(6))
def test_fixpoint_is_the_2core(seed):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(1200 + seed)
    n = int(rng.integers(10, 400))
    src, dst = graphs.random_simple_pairs(rng, n, int(rng.integers(n // 2, 3 * n)))
    st, (lo, hi) = prune.ne_filter_rounds(src, dst, n)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, dst) if a != b)
    core = nx.k_core(G, 2)
    assert set(zip(lo.tolist(), hi.tolist())) == {(min(a, b), max(a, b)) for a, b in core.edges()}
    assert st["edges_removed"] == G.number_of_edges() - core.number_of_edges()
    with_edge = {x for x in G.nodes if G.degree(x) > 0}
    assert st["vertices_removed"] == len(with_edge) - sum(1 for x in core.nodes if core.degree(x) > 0)
    # pruning never changes the triangle count
    assert oracle.count(lo, hi, n)[0] == oracle.count(src, dst, n)[0]


# ---------------------------------------------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


CASES = [("path40", lambda: _path(40)), ("K5tail30", lambda: _clique_with_tail(5, 30)),
         ("wheel30", lambda: graphs.wheel(30)[:3]), ("er4096", lambda: (*graphgen.config("er4096").edges(), 4096)),
         ("rmat14", lambda: (*graphgen.rmat(14, 8, 81).edges(), 1 << 14)),
         ("rmat13p", lambda: (*graphgen.rmat(13, 4, 82, n=7000, permute=True).edges(), 7000)),
         ("er20k_sparse", lambda: (*graphgen.er(20000, 24000, 83).edges(), 20000))]


@pytest.mark.gpu
@pytest.mark.parametrize("rounds", [0, 1, 3])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_gpu_pruned_build(tc, name, make, rounds):
    src, dst, n = make()
    T, m, t = oracle.count(src, dst, n, per_vertex=True)
    want, _ = prune.ne_filter_rounds(src, dst, n, max_rounds=rounds)
    g = tc.tc_load_edges(src, dst, n)
    try:
        got = tc.tc_build_pruned(g, rounds)
        assert got == want
        info = tc.tc_graph_get_info(g)
        assert info["num_edges"] == m - want["edges_removed"]
        assert tc.tc_count(g) == T
        T2, t2 = tc.tc_count_per_vertex(g)
        assert T2 == T
        np.testing.assert_array_equal(t2, t)
        if rounds == 0 and T <= 200000:
            tri, found = tc.tc_list_triangles(g)
            ref, _ = oracle.list_triangles(src, dst, n)
            assert found == T and set(map(tuple, tri.tolist())) == set(map(tuple, ref.tolist()))
    finally:
        tc.tc_free(g)


@pytest.mark.gpu
def test_gpu_pruned_build_errors(tc):
    import ctypes
    lib = tc.load_library()
    assert lib.tc_build_pruned(None, 0, None, None) == tc.TC_ERR_INVALID_ARG
    src, dst, n = _path(5)
    g = tc.tc_load_edges(src, dst, n)
    try:
        assert lib.tc_build_pruned(g, -1, None, None) == tc.TC_ERR_INVALID_ARG
        assert tc.tc_build_pruned(g, 0) == {"rounds": 2, "edges_removed": 4, "vertices_removed": 5}
        assert tc.tc_graph_get_info(g)["num_edges"] == 0 and tc.tc_count(g) == 0
        assert tc.tc_build_pruned(g, 0) == {"rounds": 0, "edges_removed": 0, "vertices_removed": 0}  # already built
    finally:
        tc.tc_free(g)

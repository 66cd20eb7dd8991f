"""The unfused verification loop of Algorithm 1 (tc_count_unfused), the ablation of the fused kernel.

CPU: the frontier-size definitions in oracle/frontiers.py against closed forms (K_n, stars, disjoint unions) and a
loop enumeration on random tiny graphs.  GPU: tc_count_unfused through the C ABI against the oracle's count and the
frontier sizes, whole and cut into many hop-2 passes, and its argument errors.
"""
import math

import numpy as np
import pytest

import graphgen
import oracle
from oracle import frontiers
from tests import graphs


# ---------------------------------------------------------------------------------------------------------------
# CPU: pins of the frontier definitions
# ---------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 4, 5, 9, 30])
def test_frontiers_of_a_clique(n):
    """K_n: every vertex has the same count, so the order is by id and d+(i) = n-1-i.  Candidates are i <= n-3;
    hop 1 has sum_{d=2}^{n-1} d slots; the partials are i < j <= n-2; hop 2 reaches every i < j < k, all
    closed: C(n,3) slots."""
    src, dst, n, T, _ = graphs.complete(n)
    f = frontiers.unfused_frontiers(src, dst, n)
    assert f == {"candidates": n - 2, "frontier1": n * (n - 1) // 2 - 1, "partials": (n - 2) * (n - 1) // 2,
                 "frontier2": math.comb(n, 3)}
    assert f == frontiers.unfused_frontiers_brute(src, dst, n)


def test_frontiers_of_a_star():
    """A star orients every spoke leaf -> hub (the hub has the larger count): no source has two out-edges."""
    k = 12
    src = np.zeros(k, np.int32)
    dst = np.arange(1, k + 1, dtype=np.int32)
    assert frontiers.unfused_frontiers(src, dst, k + 1) == dict(candidates=0, frontier1=0, partials=0, frontier2=0)


def test_frontiers_add_over_disjoint_unions():
    """Frontier sizes are sums over components (the order inside each component is unchanged up to ties)."""
    parts = [graphs.complete(6), graphs.complete(4), graphs.complete(7)]
    src, dst, n, T, _ = graphs.disjoint_union(*parts)
    got = frontiers.unfused_frontiers(src, dst, n)
    want = {k: sum(frontiers.unfused_frontiers(p[0], p[1], p[2])[k] for p in parts) for k in got}
    assert got == want


@pytest.mark.parametrize("seed", range(8))
def test_frontiers_against_enumeration(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 60))
    src, dst = graphs.random_simple_pairs(rng, n, int(rng.integers(0, 5 * n)))
    f = frontiers.unfused_frontiers(src, dst, n)
    assert f == frontiers.unfused_frontiers_brute(src, dst, n)
    T, _ = oracle.count(src, dst, n)
    assert f["frontier2"] >= T  # every triangle is one closed hop-2 slot


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


CASES = [("K40", lambda: graphs.complete(40)[:3]), ("W50", lambda: graphs.wheel(50)[:3]),
         ("icosahedron", lambda: graphs.icosahedron()[:3]),
         ("K333", lambda: graphs.complete_tripartite(3, 3, 3)[:3]),
         ("er4096", lambda: (*graphgen.config("er4096").edges(), 4096)),
         ("rmat14", lambda: (*graphgen.rmat(14, 16, 71).edges(), 1 << 14)),
         ("rmat13p", lambda: (*graphgen.rmat(13, 12, 72, n=6000, permute=True).edges(), 6000)),
         ("er50k", lambda: (*graphgen.er(50000, 400000, 73).edges(), 50000))]


def _check(tc, src, dst, n, budget=0):
    T, _ = oracle.count(src, dst, n)
    want = frontiers.unfused_frontiers(src, dst, n)
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        got, st = tc.tc_count_unfused(g, budget)
        assert got == T == st["matches"] == tc.tc_count(g)
        assert {k: st[k] for k in want} == want
        return st
    finally:
        tc.tc_free(g)


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_gpu_unfused_matches_oracle(tc, name, make):
    src, dst, n = make()
    st = _check(tc, src, dst, n)
    assert st["chunks"] == (1 if st["frontier2"] > 0 else 0)
    assert st["peak_bytes"] >= 4 * st["frontier2"]  # the hop-2 frontier is held whole


@pytest.mark.gpu
def test_gpu_unfused_in_many_passes(tc):
    """A small budget cuts hop 2 into passes of 4096 slots; rows of the frontier straddle the cuts."""
    src, dst = graphgen.rmat(13, 16, 74).edges()
    n = 1 << 13
    st = _check(tc, src, dst, n, budget=16 * 4096)
    assert st["chunks"] == -(-st["frontier2"] // 4096) and st["chunks"] > 10


@pytest.mark.gpu
def test_gpu_unfused_degenerate(tc):
    for src, dst, n in [(np.zeros(0, np.int32), np.zeros(0, np.int32), 5), (*graphs.cycle(7)[:2], 7),
                        (*graphs.complete_bipartite(5, 6)[:2], 11), (*graphs.complete(3)[:2], 3),
                        (np.array([0, 1, 1], np.int32), np.array([1, 0, 1], np.int32), 2)]:
        _check(tc, src, dst, n)


@pytest.mark.gpu
def test_gpu_unfused_errors(tc):
    import ctypes
    lib = tc.load_library()
    T = ctypes.c_uint64()
    assert lib.tc_count_unfused(None, ctypes.byref(T), 0, None, None) == tc.TC_ERR_INVALID_ARG
    src, dst, n, _, _ = graphs.complete(5)
    g = tc.tc_load_edges(src, dst, n)
    try:
        assert lib.tc_count_unfused(g, ctypes.byref(T), 0, None, None) == tc.TC_ERR_STATE
        tc.tc_build(g)
        assert lib.tc_count_unfused(g, ctypes.byref(T), -1, None, None) == tc.TC_ERR_INVALID_ARG
        assert lib.tc_count_unfused(g, None, 0, None, None) == tc.TC_ERR_INVALID_ARG
        assert lib.tc_count_unfused(g, ctypes.byref(T), 0, None, None) == tc.TC_OK and T.value == 10
    finally:
        tc.tc_free(g)

"""Triangle listing (the matched node id lists of Sec. II-A).

CPU: the oracle's listing routine against closed forms and dense brute force (every triple a triangle, none
twice, the right number).  GPU: the listing kernel through the C ABI against the oracle's list, as sets of sorted
triples (the order of the output is unspecified), whole, in rank-range chunks, past its capacity, and into device
memory.
"""
import ctypes
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs


def _as_set(tri):
    return set(map(tuple, np.asarray(tri).tolist()))


def _sorted_rows(tri):
    """The triples as one sorted int64 key each (ids < 2^21), for comparing millions of them."""
    t = np.asarray(tri, dtype=np.int64)
    return np.sort((t[:, 0] << 42) | (t[:, 1] << 21) | t[:, 2])


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_oracle_lists_every_triple_of_a_clique(n):
    src, dst, n, T, _ = graphs.complete(n)
    tri, found = oracle.list_triangles(src, dst, n)
    assert found == T == len(tri)
    assert _as_set(tri) == set(itertools.combinations(range(n), 3))


@pytest.mark.parametrize("seed", range(6))
def test_oracle_listing_against_brute_force(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 120))
    src, dst = graphs.random_simple_pairs(rng, n, int(rng.integers(n, 6 * n)))
    T, _, _ = graphs.dense_counts(src, dst, n)
    tri, found = oracle.list_triangles(src, dst, n)
    assert found == T == len(tri) == len(_as_set(tri))
    A = np.zeros((n, n), dtype=bool)
    A[src, dst] = True
    A[dst, src] = True
    np.fill_diagonal(A, False)
    for a, b, c in tri:
        assert a < b < c and A[a, b] and A[b, c] and A[a, c]


def test_oracle_listing_capacity():
    src, dst, n, T, _ = graphs.complete(9)
    tri, found = oracle.list_triangles(src, dst, n, capacity=10)
    assert found == T == 84 and len(tri) == 10 and _as_set(tri) <= set(itertools.combinations(range(9), 3))


@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


CASES = [("K30", lambda: graphs.complete(30)[:3]), ("W40", lambda: graphs.wheel(40)[:3]),
         ("icosahedron", lambda: graphs.icosahedron()[:3]),
         ("rmat14", lambda: (*graphgen.rmat(14, 16, 61).edges(), 1 << 14)),
         ("rmat13p", lambda: (*graphgen.rmat(13, 12, 62, n=6000, permute=True).edges(), 6000)),
         ("er50k", lambda: (*graphgen.er(50000, 400000, 63).edges(), 50000))]


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_gpu_listing_matches_oracle(tc, name, make):
    src, dst, n = make()
    ref, T = oracle.list_triangles(src, dst, n)
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        if name == "rmat14":  # hub rows stored as bitmaps: listing expands their ANDs bit by bit
            assert tc.tc_graph_get_info(g)["dense_rows"] > 0
        tri, found = tc.tc_list_triangles(g)
        assert found == T == len(tri)
        assert _as_set(tri) == _as_set(ref) and len(_as_set(tri)) == T
        # three rank ranges cover every source once
        parts, total = [], 0
        for lo, hi in ((0, n // 3), (n // 3, 2 * n // 3), (2 * n // 3, n)):
            part, f = tc.tc_list_triangles(g, lo, hi - lo)
            parts.append(part)
            total += f
        assert total == T and _as_set(np.concatenate(parts)) == _as_set(ref)
        if T > 1:  # past its capacity the call writes what fits and still reports the total
            part, f = tc.tc_list_triangles(g, capacity=T // 2)
            assert f == T and len(part) == T // 2 and _as_set(part) <= _as_set(ref)
    finally:
        tc.tc_free(g)


@pytest.mark.gpu
def test_gpu_listing_rmat16_with_dense_rows(tc):
    """Millions of triangles, most of them closed in dense hub rows; compared as sorted keys, each triple
    ascending and listed once."""
    src, dst = graphgen.rmat(16, 16, 65).edges()
    n = 1 << 16
    ref, T = oracle.list_triangles(src, dst, n)
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        assert info["dense_rows"] > 0 and info["dense_wedges"] > 0
        tri, found = tc.tc_list_triangles(g)
        assert found == T == len(tri) and T > 10 ** 6
        assert (tri[:, 0] < tri[:, 1]).all() and (tri[:, 1] < tri[:, 2]).all()
        got = _sorted_rows(tri)
        assert (np.diff(got) > 0).all()
        assert np.array_equal(got, _sorted_rows(ref))
    finally:
        tc.tc_free(g)


@pytest.mark.gpu
def test_gpu_listing_into_device_memory(tc):
    import torch
    src, dst = graphgen.rmat(12, 16, 64).edges()
    n = 1 << 12
    ref, T = oracle.list_triangles(src, dst, n)
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        out = torch.full((T, 3), -1, dtype=torch.int32, device="cuda")
        found = ctypes.c_uint64()
        lib = tc.load_library()
        st = lib.tc_list_triangles(g, 0, n, out.data_ptr(), T, ctypes.byref(found), tc.TC_PTR_DEVICE,
                                   torch.cuda.current_stream().cuda_stream)
        assert st == tc.TC_OK and found.value == T
        assert _as_set(out.cpu().numpy()) == _as_set(ref)
    finally:
        tc.tc_free(g)

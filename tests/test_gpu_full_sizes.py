"""GPU parity at the benchmark's full sizes, in the benchmark's launch configuration (device-resident edges, one
tc_load_edges / tc_build / count per graph).  Where the oracle cannot count the whole graph in seconds it checks
sampled outputs one by one (t(x) for chosen x, from its definition), and properties that hold at any size check
the rest (sum of t(x) = 3T; batched counts = one-by-one counts)."""
import os

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


def test_rmat26_sampled_per_vertex(tc):
    """R-MAT scale 26 (2^30 sampled pairs, permuted ids): T and t(x) for every x on the GPU; t(x) for 40 sampled
    vertices from the oracle; sum of t = 3T; m against the host count of distinct pairs' degrees."""
    import torch
    spec = graphgen.config("rmat26")
    ds, dd = spec.edges(device="cuda")
    g = tc.tc_load_edges(ds, dd, spec.n)
    del ds, dd
    torch.cuda.empty_cache()
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        T = tc.tc_count(g)
        T2, t = tc.tc_count_per_vertex(g)
    finally:
        tc.tc_free(g)
    assert T == T2 and T > 0
    assert int(t.sum()) == 3 * T
    hs, hd = spec.edges()  # host generator (bit-identical to the device one, see test_graphgen)
    # samples: vertices spread over the degree range (by the input's pair counts), plus random ones
    cnt = np.bincount(hs, minlength=spec.n) + np.bincount(hd, minlength=spec.n)
    order = np.argsort(-cnt, kind="stable")
    ranks = [30, 100, 300, 1000, 3000, 10000, 30000, 100000, 300000, 1000000, 3000000, 10000000]
    rng = np.random.default_rng(26)
    xs = np.concatenate([order[ranks], rng.integers(0, spec.n, size=28)]).astype(np.int32)
    ref, deg = oracle.vertex_triangles(hs, hd, spec.n, xs)
    np.testing.assert_array_equal(t[xs], ref)
    assert info["num_edges"] > 0.95 * spec.num_edges


def test_batch_4096_all_graphs(tc):
    """The 4096-graph batch: batched counts equal one-by-one counts for every graph, and the oracle agrees on
    every 16th graph and on the 64 largest."""
    specs = graphgen.batch_mix(4096)
    handles = []
    try:
        for sp in specs:
            s, d = sp.edges(device="cuda")
            handles.append(tc.tc_load_edges(s, d, sp.n))
            tc.tc_build(handles[-1])
        solo = np.array([tc.tc_count(h) for h in handles], dtype=np.uint64)
        batched = tc.tc_count_batch(handles)
        np.testing.assert_array_equal(batched, solo)
        np.testing.assert_array_equal(tc.tc_count_batch(handles), solo)
    finally:
        for h in handles:
            tc.tc_free(h)
    big = np.argsort([-sp.expected_edges for sp in specs])[:64]
    sample = sorted(set(range(0, 4096, 16)) | set(big.tolist()))
    for i in sample:
        sp = specs[i]
        hs, hd = sp.edges()
        assert oracle.count(hs, hd, sp.n)[0] == int(solo[i]), f"graph {i} ({sp})"

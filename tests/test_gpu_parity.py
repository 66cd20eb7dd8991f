"""GPU parity: the CUDA path through the C ABI against the CPU oracle (and closed forms), bit-exact.

Counts are integers with a unique value, so every comparison here is equality (tolerance 0).
"""
import math

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


def gpu_counts(tc, src, dst, n, device=True, per_vertex=True, allocator="torch"):
    import torch
    if device:
        s = torch.as_tensor(np.asarray(src, dtype=np.int32)).cuda()
        d = torch.as_tensor(np.asarray(dst, dtype=np.int32)).cuda()
    else:
        s, d = np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32)
    g = tc.tc_load_edges(s, d, n, allocator=allocator)
    try:
        tc.tc_build(g)
        T = tc.tc_count(g)
        t = None
        if per_vertex:
            T2, t = tc.tc_count_per_vertex(g)
            assert T2 == T
        info = tc.tc_graph_get_info(g)
    finally:
        tc.tc_free(g)
    return T, t, info


@pytest.mark.parametrize("name,g", graphs.closed_form_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_closed_forms(tc, name, g):
    src, dst, n, T, t = g
    got, gt, info = gpu_counts(tc, src, dst, n)
    assert got == T
    if t is not None:
        np.testing.assert_array_equal(gt, t)


@pytest.mark.parametrize("n", [200, 1500, 4300])
def test_complete_graph_block_bin(tc, n):
    """K_n: d+(u) runs from 0 to n-1; with a low threshold the heavy sources go to the block bin (a whole CTA
    each) and the light ones to the warp bin."""
    src, dst, n, T, t = graphs.complete(n)
    saved = tc.tc_get_tuning()
    try:
        tc.tc_set_tuning([(1 << 62, 1 << 12)])
        got, gt, info = gpu_counts(tc, src, dst, n)
    finally:
        tc.tc_set_tuning(saved)
    assert got == math.comb(n, 3)
    np.testing.assert_array_equal(gt, t)
    if n >= 1500:
        assert info["bin_block"] > 0 and info["bin_warp"] > 0


@pytest.mark.parametrize("seed", range(10))
def test_random_small_graphs(tc, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.choice([1, 2, 3, 31, 33, 97, 1000, 5000, 9000, 20000]))
    m = int(rng.integers(0, 8 * n + 1))
    src, dst = graphs.random_simple_pairs(rng, n, m)
    T, mm, t = oracle.count(src, dst, n, per_vertex=True)
    got, gt, info = gpu_counts(tc, src, dst, n, device=bool(seed % 2))
    assert got == T and info["num_edges"] == mm
    np.testing.assert_array_equal(gt, t)


STAGED_CASES = [("rmat16", lambda: (*graphgen.rmat(16, 16, 31).edges(), 1 << 16), None),
                ("rmat17p_block", lambda: (*graphgen.rmat(17, 16, 32, n=120000, permute=True).edges(), 120000),
                 [(1 << 62, 1 << 12)]),
                ("k1500_block", lambda: graphs.complete(1500)[:3], [(1 << 62, 1 << 12)]),
                ("k1500_warp", lambda: graphs.complete(1500)[:3], [(1 << 62, 1 << 40)]),
                ("gnp_dense", lambda: (*graphgen.gnp(3000, 0.2, 33).edges(), 3000), None)]


@pytest.mark.parametrize("name,make,classes", STAGED_CASES, ids=[c[0] for c in STAGED_CASES])
def test_staged_long_rows_give_the_same_counts(tc, name, make, classes):
    """Long hop-2 rows walked through the shared-memory ring filled by asynchronous copies (forced on for every
    graph) give the oracle's count, in warp mode and in block mode, with rows of every length mod 32 quads."""
    hs, hd, n = make()
    T_ref = oracle.count(hs, hd, n)[0]
    saved = tc.tc_get_tuning()
    saved_stage, saved_isect = tc.tc_get_stage_min_csr_bytes(), tc.tc_get_isect_max_wedges_milli()
    try:
        if classes:
            tc.tc_set_tuning(classes)
        for stage in (1, 0, 1):
            tc.tc_set_tuning(tc.tc_get_tuning(), stage_min_csr_bytes=stage, isect_max_wedges_milli=0)
            g = tc.tc_load_edges(hs, hd, n)
            try:
                tc.tc_build(g)
                info = tc.tc_graph_get_info(g)
                assert tc.tc_count(g) == T_ref, f"stage_min_csr_bytes={stage}"
            finally:
                tc.tc_free(g)
    finally:
        tc.tc_set_tuning(saved, stage_min_csr_bytes=saved_stage, isect_max_wedges_milli=saved_isect)
    if classes and classes[0][1] < (1 << 20):
        assert info["bin_block"] > 0


def test_hub_heavy_graph(tc):
    """One hub joined to everything plus a dense core: long N+(v) rows re-read by many sources."""
    rng = np.random.default_rng(7)
    n = 30000
    hub_s = np.zeros(n - 1, dtype=np.int32)
    hub_d = np.arange(1, n, dtype=np.int32)
    core = rng.integers(1, 400, size=(60000, 2)).astype(np.int32)
    rest = rng.integers(0, n, size=(100000, 2)).astype(np.int32)
    src = np.concatenate([hub_s, core[:, 0], rest[:, 0]])
    dst = np.concatenate([hub_d, core[:, 1], rest[:, 1]])
    T, _, t = oracle.count(src, dst, n, per_vertex=True)
    got, gt, _ = gpu_counts(tc, src, dst, n)
    assert got == T
    np.testing.assert_array_equal(gt, t)


def test_sources_with_many_entries_below_the_bitmap_window(tc):
    """A clique K_101 of degree-100 vertices beside 32768 vertices of higher degree: the clique's ranks fall below
    the per-warp bitmap window (the top 32768 ranks), so their sources have up to 100 out-neighbours below it and
    take the binary-search closing test.  The clique adds exactly C(101, 3) triangles to those of the rest."""
    rng = np.random.default_rng(17)
    top = 32768
    m_top = top * 110
    ts = rng.integers(0, top, size=m_top).astype(np.int32)
    td = rng.integers(0, top, size=m_top).astype(np.int32)
    a, b = np.triu_indices(101, 1)
    src = np.concatenate([ts, (a + top).astype(np.int32)])
    dst = np.concatenate([td, (b + top).astype(np.int32)])
    n = top + 101
    T_top, _ = oracle.count(ts, td, top)
    got, gt, info = gpu_counts(tc, src, dst, n, per_vertex=False)
    assert got == T_top + math.comb(101, 3)


def test_ids_at_the_top_of_the_range(tc):
    n = 100003
    rng = np.random.default_rng(3)
    src = (n - 1 - rng.integers(0, 300, size=20000)).astype(np.int32)
    dst = (n - 1 - rng.integers(0, 300, size=20000)).astype(np.int32)
    T, _, t = oracle.count(src, dst, n, per_vertex=True)
    got, gt, _ = gpu_counts(tc, src, dst, n)
    assert got == T
    np.testing.assert_array_equal(gt, t)


def test_duplicate_heavy_input(tc):
    src, dst, n, T, t = graphs.complete(30)
    src, dst = np.tile(np.concatenate([src, dst]), 50), np.tile(np.concatenate([dst, src]), 50)
    T_ref, m_ref, t_ref = oracle.count(src, dst, n, per_vertex=True)
    got, gt, info = gpu_counts(tc, src, dst, n)
    assert got == T_ref and info["num_edges"] == m_ref
    np.testing.assert_array_equal(gt, t_ref)


def test_empty_and_degenerate(tc):
    e = np.zeros(0, dtype=np.int32)
    assert gpu_counts(tc, e, e, 0)[0] == 0
    got, gt, info = gpu_counts(tc, e, e, 9)
    assert got == 0 and not gt.any() and info["num_edges"] == 0
    loops = np.arange(50, dtype=np.int32)
    got, gt, info = gpu_counts(tc, loops, loops, 50)
    assert got == 0 and info["num_edges"] == 0
    one = np.array([0], dtype=np.int32)
    assert gpu_counts(tc, one, one + 1, 2)[0] == 0


@pytest.mark.parametrize("cfg", ["er4096"])
def test_er4096_full(tc, cfg):
    spec = graphgen.config(cfg)
    hs, hd = spec.edges()
    T, m, t = oracle.count(hs, hd, spec.n, per_vertex=True)
    ds, dd = spec.edges(device="cuda")
    g = tc.tc_load_edges(ds, dd, spec.n)
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        assert info["num_edges"] == m
        assert tc.tc_count(g) == T
        T2, gt = tc.tc_count_per_vertex(g)
        assert T2 == T
        np.testing.assert_array_equal(gt, t)
    finally:
        tc.tc_free(g)


@pytest.mark.parametrize("spec", [graphgen.rmat(16, 16, 11), graphgen.rmat(17, 8, 12, n=100000, permute=True),
                                  graphgen.er(200000, 3000000, 13)], ids=["rmat16", "rmat17p", "er200k"])
def test_medium_graphs(tc, spec):
    hs, hd = spec.edges()
    T, m, t = oracle.count(hs, hd, spec.n, per_vertex=True)
    got, gt, info = gpu_counts(tc, hs, hd, spec.n)
    assert got == T and info["num_edges"] == m
    np.testing.assert_array_equal(gt, t)


@pytest.mark.parametrize("spec", [graphgen.rmat(16, 16, 11), graphgen.rmat(17, 8, 12, n=100000, permute=True)],
                         ids=["rmat16", "rmat17p"])
def test_per_vertex_add_modes(tc, spec):
    """Per-vertex counts with the per-block counters of the top ranks added to without read-back (graphs below 2^31
    edges) and with every add checking its counter (forced here by a bound of 0 edges): both equal the oracle."""
    hs, hd = spec.edges()
    T, _, t = oracle.count(hs, hd, spec.n, per_vertex=True)
    saved = tc.tc_get_tuning()
    try:
        for bound in (tc.VERTEX_PLAIN_MAX_EDGES, 0):
            tc.tc_set_tuning(saved, vertex_plain_max_edges=bound)
            got, gt, _ = gpu_counts(tc, hs, hd, spec.n)
            assert got == T, bound
            np.testing.assert_array_equal(gt, t)
    finally:
        tc.tc_set_tuning(saved, vertex_plain_max_edges=tc.VERTEX_PLAIN_MAX_EDGES)


def test_rmat20_full(tc):
    """R-MAT scale 20, edge factor 16: the benchmark workload, counted in the benchmark's launch configuration
    (device-resident edges, one tc_count), every per-vertex count compared."""
    import torch
    spec = graphgen.config("rmat20")
    hs, hd = spec.edges()
    T, m, t = oracle.count(hs, hd, spec.n, per_vertex=True)
    ds, dd = spec.edges(device="cuda")
    g = tc.tc_load_edges(ds, dd, spec.n)
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        assert info["num_edges"] == m
        assert tc.tc_count(g) == T
        d_total = torch.zeros(1, dtype=torch.int64, device="cuda")
        tc.tc_count_device(g, d_total)
        assert int(d_total.item()) == T
        T2, gt = tc.tc_count_per_vertex(g)
        assert T2 == T
        np.testing.assert_array_equal(gt, t)
    finally:
        tc.tc_free(g)
    # the same graph with heavy sources in the block bin: n > 2^19, so the block bitmap starts above 0 and dense
    # rows are addressed through the offset between the two windows
    saved = tc.tc_get_tuning()
    try:
        tc.tc_set_tuning([(1 << 62, 1 << 13)])
        g = tc.tc_load_edges(ds, dd, spec.n)
        try:
            tc.tc_build(g)
            info = tc.tc_graph_get_info(g)
            assert info["bin_block"] > 0 and info["dense_rows"] > 0
            assert tc.tc_count(g) == T
            T2, gt = tc.tc_count_per_vertex(g)
            assert T2 == T
            np.testing.assert_array_equal(gt, t)
            assert int(tc.tc_count_batch([g])[0]) == T
            tc.tc_set_tuning([(1 << 62, 1 << 13)], vertex_plain_max_edges=0)  # every counter add checked
            T2, gt = tc.tc_count_per_vertex(g)
            assert T2 == T
            np.testing.assert_array_equal(gt, t)
        finally:
            tc.tc_free(g)
    finally:
        tc.tc_set_tuning(saved, vertex_plain_max_edges=tc.VERTEX_PLAIN_MAX_EDGES)


def _repeat_heavy_pairs():
    """Hubs whose pairs repeat thousands of times: the build's buckets then span all three sizes (up to 32 pairs,
    up to a few thousand, and longer), with most of each long bucket being repeats."""
    rng = np.random.default_rng(2100)
    n = 6000
    hubs = np.arange(12, dtype=np.int32)
    parts_s, parts_d = [], []
    for i in range(12):
        for j in range(i + 1, 12):
            k = int(rng.integers(50, 4000))
            parts_s.append(np.full(k, hubs[i]))
            parts_d.append(np.full(k, hubs[j]))
    parts_s.append(np.repeat(hubs, 700))
    parts_d.append(rng.integers(12, n, 12 * 700))
    parts_s.append(rng.integers(12, n, 40000))
    parts_d.append(rng.integers(12, n, 40000))
    parts_s.append(rng.integers(12, 400, 30000))  # mid-size buckets among the next tier
    parts_d.append(rng.integers(12, 400, 30000))
    src = np.concatenate(parts_s).astype(np.int32)
    dst = np.concatenate(parts_d).astype(np.int32)
    perm = rng.permutation(src.size)
    return src[perm], dst[perm], n


def _counts_past_the_clamp():
    """Six vertices whose input-pair counts pass 65535, each a different amount (the rank sort clamps counts there
    and orders those vertices afterwards), among random pairs."""
    rng = np.random.default_rng(2200)
    n = 20000
    s, d = [], []
    for k in range(6):
        reps = 66000 + 997 * (5 - k)
        s.append(np.full(reps, 100 + 7 * k))
        d.append(rng.integers(0, n, reps))
    s.append(rng.integers(0, n, 50000))
    d.append(rng.integers(0, n, 50000))
    return np.concatenate(s).astype(np.int32), np.concatenate(d).astype(np.int32), n


CSR_CASES = [("rmat13", lambda: (*graphgen.rmat(13, 12, 21).edges(), 1 << 13)),
             ("counts_past_clamp", _counts_past_the_clamp),
             ("rmat16p", lambda: (*graphgen.rmat(16, 8, 23, n=60000, permute=True).edges(), 60000)),
             ("repeat_heavy", _repeat_heavy_pairs),
             ("er_sparse", lambda: (*graphgen.er(30000, 20000, 22).edges(), 30000))]


BUILD_PATHS = {"compact": dict(bucket_max_pairs=0, compact_max_pairs=1 << 40, tiny_max_pairs=0),  # one host sync
               "buckets": dict(bucket_max_pairs=0, compact_max_pairs=0, tiny_max_pairs=0),        # sizes as known
               "sort": dict(bucket_max_pairs=1, compact_max_pairs=0, tiny_max_pairs=0),           # radix sort
               "tiny": dict(bucket_max_pairs=0, compact_max_pairs=0, tiny_max_pairs=(1 << 18) - 1)}  # one launch


def _tiny_eligible(tc, n, pairs):
    return 0 < n <= tc.TINY_MAX_VERTICES and 0 < pairs <= tc.TINY_MAX_PAIRS


def _build_with(tc, path, hs, hd, n, launches=None):
    """(off, col, perm, info, T) of the graph built on the given path; launches (a list) receives the number of
    kernels tc_build launched."""
    saved = dict(bucket_max_pairs=tc.tc_get_bucket_max_pairs(), compact_max_pairs=tc.tc_get_compact_max_pairs(),
                 tiny_max_pairs=tc.tc_get_tiny_max_pairs())
    tc.tc_set_tuning(tc.tc_get_tuning(), **BUILD_PATHS[path])
    try:
        g = tc.tc_load_edges(hs, hd, n)
        try:
            k0 = tc.tc_kernel_launches()
            tc.tc_build(g)
            if launches is not None:
                launches.append(tc.tc_kernel_launches() - k0)
            off, col, perm = tc.tc_copy_csr(g)
            info = tc.tc_graph_get_info(g)
            T = tc.tc_count(g)
        finally:
            tc.tc_free(g)
    finally:
        tc.tc_set_tuning(tc.tc_get_tuning(), **saved)
    return off, col, perm, info, T


@pytest.mark.parametrize("path", list(BUILD_PATHS))
@pytest.mark.parametrize("name,make", CSR_CASES, ids=[c[0] for c in CSR_CASES])
def test_csr_structure(tc, name, make, path):
    """The oriented CSR: vertices relabelled by rank in the (count, id) order, each undirected edge stored once
    from its lower to its higher rank, rows ascending, 16-byte aligned and padded with the id n.  The three ways of
    building it (per-source buckets with one host synchronisation or with sizes read as they become known, a
    radix sort of all pairs, and for small graphs one cooperative launch) give this same CSR."""
    hs, hd, n = make()
    if path == "tiny" and not _tiny_eligible(tc, n, hs.size):
        pytest.skip("beyond the one-launch build's bounds")
    off, col, perm, info, T = _build_with(tc, path, hs, hd, n)
    assert T == oracle.count(hs, hd, n)[0]
    lo = np.minimum(hs, hd)
    hi = np.maximum(hs, hd)
    keep = lo != hi
    und = np.unique(lo[keep].astype(np.int64) * n + hi[keep])
    deg = np.bincount(np.concatenate([und // n, und % n]), minlength=n)
    # perm is the (count, id) order, count = input pairs at the vertex (self-loops excluded, repeats included)
    cnt = np.bincount(np.concatenate([hs[keep], hd[keep]]), minlength=n)
    np.testing.assert_array_equal(np.sort(perm), np.arange(n))
    key = cnt[perm].astype(np.int64) * n + perm
    assert np.all(np.diff(key) > 0)
    assert off[0] == 0 and np.all(off % 4 == 0) and off[-1] == col.size == info["csr_entries"]
    real = col < n
    assert int(real.sum()) == und.size == info["num_edges"]
    rows = np.repeat(np.arange(n), np.diff(off))
    pads_per_row = np.bincount(rows[~real], minlength=n)
    dplus = np.bincount(rows[real], minlength=n)
    assert np.all(pads_per_row < 4) and np.all(np.diff(off) == dplus + pads_per_row)
    assert np.all(col[real] > rows[real])
    for r in np.flatnonzero(dplus > 1)[-3000:]:
        seg = col[off[r]:off[r] + dplus[r]]
        assert np.all(np.diff(seg) > 0) and np.all(col[off[r] + dplus[r]:off[r + 1]] == n)
    a, b = perm[rows[real]].astype(np.int64), perm[col[real]].astype(np.int64)
    np.testing.assert_array_equal(np.sort(np.minimum(a, b) * n + np.maximum(a, b)), und)
    assert info["max_out_degree"] == dplus.max()
    assert info["num_wedges"] == int(dplus[col[real]].sum())
    # dense rows: v in the warp window (its base a multiple of 128 at or above n - 2^15) whose bitmap quads over
    # (v, n) hold no more words than v has out-neighbours (and at least 16 of them)
    base = ((n - (1 << 15) + 127) & ~127) if n > (1 << 15) else 0
    wtopq = ((n - 1 - base) >> 7) + 1
    v = np.arange(n)
    quads = np.where(v >= base, wtopq - ((v + 1 - base) >> 7), 0)
    dense = (v >= base) & (dplus >= 16) & (4 * quads <= dplus)
    targets = col[real]
    assert info["dense_rows"] == int(dense.sum())
    assert info["dense_wedges"] == int(dplus[targets][dense[targets]].sum())
    assert info["dense_quads"] == int(quads[targets][dense[targets]].sum())
    if name.startswith("rmat"):
        assert info["dense_rows"] > 0


COMPACT_CASES = CSR_CASES + [("er4096", lambda: (*graphgen.config("er4096").edges(), 4096)),
                             ("k40", lambda: graphs.complete(40)[:3]),
                             ("wheel9", lambda: graphs.wheel(9)[:3]),
                             ("one_edge", lambda: (np.array([3], np.int32), np.array([5], np.int32), 9)),
                             ("self_loops_only", lambda: (np.arange(7, dtype=np.int32), np.arange(7, dtype=np.int32),
                                                          7))]


@pytest.mark.parametrize("name,make", COMPACT_CASES, ids=[c[0] for c in COMPACT_CASES])
def test_compact_build_equals_synchronising_build(tc, name, make):
    """The build with one host synchronisation (buffers at size bounds, sizes read back at the end) gives exactly
    the graph of the build that reads each size as it becomes known: offsets, columns, visiting order, every
    reported size and bin, and the count (also against the oracle)."""
    hs, hd, n = make()
    a = _build_with(tc, "compact", hs, hd, n)
    b = _build_with(tc, "buckets", hs, hd, n)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3]
    assert a[4] == b[4] == oracle.count(hs, hd, n)[0]


def _hub_and_clique(n, seed):
    """A hub joined to every vertex, a 90-clique among the top ids, random pairs with repeats and self-loops."""
    rng = np.random.default_rng(seed)
    a, b = np.triu_indices(90, 1)
    s = np.concatenate([np.zeros(n - 1, np.int64), n - 90 + a, rng.integers(0, n, 6000)])
    d = np.concatenate([np.arange(1, n), n - 90 + b, rng.integers(0, n, 6000)])
    return s.astype(np.int32), d.astype(np.int32), n


TINY_CASES = [("er4096", lambda: (*graphgen.config("er4096").edges(), 4096)),
              ("k200_dense_rows", lambda: graphs.complete(200)[:3]),
              ("n8192_m65536", lambda: (*graphgen.er(8192, 65536, 91).edges(), 8192)),
              ("rmat13_ef7", lambda: (*graphgen.rmat(13, 7, 92).edges(), 1 << 13)),
              ("gnp_small_dense", lambda: (*graphgen.gnp(300, 0.6, 93).edges(), 300)),
              ("hub_and_clique", lambda: _hub_and_clique(5000, 94)),
              ("n1_self_loop", lambda: (np.array([0], np.int32), np.array([0], np.int32), 1)),
              ("two_vertices", lambda: (np.array([0, 1, 1], np.int32), np.array([1, 0, 1], np.int32), 2)),
              ("wheel50", lambda: graphs.wheel(50)[:3])]


@pytest.mark.parametrize("name,make", TINY_CASES, ids=[c[0] for c in TINY_CASES])
def test_small_graphs_every_build_path(tc, name, make):
    """Small graphs at the edges of the compact build's bounds (n up to 8192, up to 65536 pairs, dense rows, a hub,
    a clique, repeats, self-loops, one and two vertices): the compact build, the build that reads sizes as known,
    the radix-sort build and the one-launch build give the same graph, and its counts and per-vertex counts are the
    oracle's."""
    hs, hd, n = make()
    a = _build_with(tc, "compact", hs, hd, n)
    for other in ("buckets", "sort", "tiny"):
        b = _build_with(tc, other, hs, hd, n)
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)
        assert a[3] == b[3] and a[4] == b[4]
    T, _, t = oracle.count(hs, hd, n, per_vertex=True)
    assert a[4] == T
    g = tc.tc_load_edges(hs, hd, n)
    try:
        tc.tc_build(g)
        T2, t2 = tc.tc_count_per_vertex(g)
    finally:
        tc.tc_free(g)
    assert T2 == T
    np.testing.assert_array_equal(t2, t)


def _star_and_repeats(n, seed):
    """A star over all n vertices, one pair repeated 70000 times (an input-pair count above 2^16: three passes of the
    rank sort), and random pairs."""
    rng = np.random.default_rng(seed)
    s = np.concatenate([np.zeros(n - 1, np.int64), np.full(70000, 5), rng.integers(0, n, 20000)])
    d = np.concatenate([np.arange(1, n), np.full(70000, 9), rng.integers(0, n, 20000)])
    return s.astype(np.int32), d.astype(np.int32), n


def _at_the_bounds(seed):
    """n = 2^14 and 2^18 - 1 pairs (the one-launch build's largest input): an R-MAT-like skew with long buckets."""
    spec = graphgen.rmat(14, 16, seed)
    hs, hd = spec.edges()
    k = (1 << 18) - 1
    assert hs.size >= k
    return hs[:k].copy(), hd[:k].copy(), 1 << 14


ONE_LAUNCH_CASES = [("n16384_max_pairs", lambda: _at_the_bounds(95)),
                    ("star_and_repeats", lambda: _star_and_repeats(16384, 96)),
                    ("rmat14_ef8", lambda: (*graphgen.rmat(14, 8, 97).edges(), 1 << 14)),
                    ("gnp_2000_dense", lambda: (*graphgen.gnp(2000, 0.05, 98).edges(), 2000)),
                    ("isolated_vertices", lambda: (np.array([100, 200, 300], np.int32),
                                                   np.array([200, 300, 100], np.int32), 16384))]


@pytest.mark.parametrize("name,make", ONE_LAUNCH_CASES, ids=[c[0] for c in ONE_LAUNCH_CASES])
def test_one_launch_build(tc, name, make):
    """The one-launch build at its bounds (16384 vertices, 2^18 - 1 pairs, an input-pair count above 2^16, a star,
    isolated vertices): one kernel launch, the compact build's graph, and the oracle's count."""
    hs, hd, n = make()
    assert _tiny_eligible(tc, n, hs.size)
    launches = []
    a = _build_with(tc, "tiny", hs, hd, n, launches)
    assert launches == [1]
    b = _build_with(tc, "compact", hs, hd, n)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3]
    assert a[4] == b[4] == oracle.count(hs, hd, n)[0]


@pytest.mark.parametrize("scale,ef", [(14, 10), (11, 8)], ids=["compact", "one_launch"])
def test_host_and_device_inputs_and_allocators_agree(tc, scale, ef):
    """Host and device inputs with the library's pool and with torch's allocator, on a graph built compactly and on
    one small enough for the one-launch build."""
    spec = graphgen.rmat(scale, ef, 31)
    hs, hd = spec.edges()
    ref = oracle.count(hs, hd, spec.n)[0]
    for device in (False, True):
        for allocator in ("torch", None):
            assert gpu_counts(tc, hs, hd, spec.n, device=device, per_vertex=False, allocator=allocator)[0] == ref


def test_pinned_host_inputs(tc):
    """Page-locked host arrays are read by the device in place; a slice inside a larger pinned buffer, and a pinned
    array paired with a pageable one (staged), give the same count; ids out of range are still reported."""
    import torch
    spec = graphgen.rmat(15, 12, 32)
    hs, hd = spec.edges()
    ref = oracle.count(hs, hd, spec.n)[0]
    ps = torch.from_numpy(hs).pin_memory()
    pd = torch.from_numpy(hd).pin_memory()
    big = torch.zeros(2 * hs.size + 64, dtype=torch.int32).pin_memory()
    big[32:32 + hs.size] = ps
    big[hs.size + 48:hs.size + 48 + hd.size] = pd
    cases = [(ps, pd), (big[32:32 + hs.size], big[hs.size + 48:hs.size + 48 + hd.size]), (ps, torch.from_numpy(hd))]
    for s_, d_ in cases:
        g = tc.tc_load_edges(s_, d_, spec.n)
        try:
            tc.tc_build(g)
            assert tc.tc_count(g) == ref
        finally:
            tc.tc_free(g)
    bad = ps.clone().pin_memory()
    bad[7] = spec.n + 3
    with pytest.raises(tc.TCError):
        tc.tc_load_edges(bad, pd, spec.n)


def test_ingest_alignment_and_ragged_tiles(tc):
    """Ingest takes four pairs per thread as 16-byte loads when both arrays are 16-byte aligned and a tile of 1024
    pairs is whole, scalar loads otherwise: unaligned device views and ragged lengths give the oracle's count, and an
    invalid id (negative or >= n) inside a whole aligned tile is reported like one in a ragged tail."""
    import torch
    src, dst = graphgen.rmat(14, 16, 81).edges()
    n = 1 << 14
    for cut in (len(src), len(src) - 1, 5 * 1024 + 3):
        ref, _ = oracle.count(src[:cut], dst[:cut], n)
        for shift in (0, 1, 2, 3):
            pad = np.zeros(shift, np.int32)
            s = torch.from_numpy(np.concatenate([pad, src[:cut]])).cuda()[shift:]
            d = torch.from_numpy(np.concatenate([pad, dst[:cut]])).cuda()[shift:]
            assert (s.data_ptr() % 16 == 0) == (shift == 0)
            g = tc.tc_load_edges(s, d, n)
            try:
                tc.tc_build(g)
                assert tc.tc_count(g) == ref, (cut, shift)
            finally:
                tc.tc_free(g)
    for pos, bad_id in ((2048 + 517, n), (3 * 1024, -1), (len(src) - 1, n + 7)):
        for arr in ("src", "dst"):
            a, b = src.copy(), dst.copy()
            (a if arr == "src" else b)[pos] = bad_id
            with pytest.raises(tc.TCError) as e:
                tc.tc_load_edges(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), n)
            assert e.value.status == tc.TC_ERR_OUT_OF_RANGE


def test_errors(tc):
    import torch
    s = torch.tensor([0, 1, 5], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError) as e:
        tc.tc_load_edges(s, d, 5)
    assert e.value.status == tc.TC_ERR_OUT_OF_RANGE
    with pytest.raises(tc.TCError) as e:
        tc.tc_load_edges(s - 1, d, 6)
    assert e.value.status == tc.TC_ERR_OUT_OF_RANGE
    g = tc.tc_load_edges(s, d, 6)
    try:
        with pytest.raises(tc.TCError) as e:
            tc.tc_count(g)
        assert e.value.status == tc.TC_ERR_STATE
        tc.tc_build(g)
        tc.tc_build(g)  # idempotent
        assert tc.tc_count(g) == 0
    finally:
        tc.tc_free(g)


def test_batch_equals_solo(tc):
    specs = graphgen.batch_mix(48)
    extra = [graphs.complete(150), graphs.wheel(40), graphs.complete(5000)]
    handles, expect = [], []
    try:
        for sp in specs:
            hs, hd = sp.edges()
            handles.append(tc.tc_load_edges(hs, hd, sp.n))
            tc.tc_build(handles[-1])
            expect.append(oracle.count(hs, hd, sp.n)[0])
        for src, dst, n, T, _ in extra:
            handles.append(tc.tc_load_edges(src, dst, n))
            tc.tc_build(handles[-1])
            expect.append(T)
        solo = [tc.tc_count(h) for h in handles]
        assert solo == expect
        got = tc.tc_count_batch(handles)
        assert got.tolist() == expect
        plan = tc.tc_batch_plan_create(handles)
        try:
            for _ in range(3):  # the captured sequence zeroes its counters on every replay
                assert tc.tc_batch_plan_run(plan, len(handles)).tolist() == expect
        finally:
            tc.tc_batch_plan_free(plan)
        # repeated handles and reversed order
        rev = handles[::-1] + handles[:5]
        got = tc.tc_count_batch(rev)
        assert got.tolist() == expect[::-1] + expect[:5]
    finally:
        for h in handles:
            tc.tc_free(h)


def test_counts_do_not_depend_on_tuning(tc):
    spec = graphgen.rmat(15, 16, 51)
    hs, hd = spec.edges()
    T, _, t = oracle.count(hs, hd, spec.n, per_vertex=True)
    saved = tc.tc_get_tuning()
    try:
        for table in ([(1 << 62, 0)], [(1 << 62, 1 << 40)], [(1 << 62, 1 << 12)], [(100, 0), (1 << 62, 1 << 40)]):
            tc.tc_set_tuning(table)
            got, gt, info = gpu_counts(tc, hs, hd, spec.n)
            assert got == T
            np.testing.assert_array_equal(gt, t)
            if table == [(1 << 62, 0)]:
                assert info["bin_warp"] == 0 and info["bin_block"] > 0
            if table == [(1 << 62, 1 << 40)]:
                assert info["bin_block"] == 0
    finally:
        tc.tc_set_tuning(saved)


@pytest.mark.parametrize("scale", [16, 18])
def test_build_then_count_on_another_stream(tc, scale):
    """tc_build synchronises its stream before returning, so a graph built on one stream can be counted on another
    at once (the serving loop does exactly that) — including the dense row bitmaps written last."""
    import torch
    src, dst = graphgen.rmat(scale, 16, 2200 + scale).edges()
    n = 1 << scale
    T = oracle.count(src, dst, n)[0]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        g = tc.tc_load_edges(src, dst, n, stream=s1)
        try:
            tc.tc_build(g, s1)
            assert tc.tc_graph_get_info(g)["dense_rows"] > 0
            tc.tc_count_device(g, out, s2)
            s2.synchronize()
            assert int(out.item()) == T
        finally:
            tc.tc_free(g)


@pytest.mark.parametrize("scale,ef", [(14, 4), (16, 8), (18, 16)])
def test_thread_bin_sources(tc, scale, ef):
    """Sparse R-MAT graphs put many sources in the thread bin (a handful of out-neighbours next to heavy rows): one
    lane tests each pair of their out-neighbours by a lookup.  Totals, per-vertex counts and batches stay exact."""
    src, dst = graphgen.rmat(scale, ef, 2300 + scale).edges()
    n = 1 << scale
    T, m, t = oracle.count(src, dst, n, per_vertex=True)
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        assert info["bin_thread"] > 0
        assert info["bin_thread"] + info["bin_warp"] + info["bin_block"] == info["active_sources"]
        assert tc.tc_count(g) == T
        T2, t2 = tc.tc_count_per_vertex(g)
        assert T2 == T
        np.testing.assert_array_equal(t2, t)
        assert tc.tc_count_intersect(g) == T
        assert int(tc.tc_count_batch([g, g])[1]) == T
    finally:
        tc.tc_free(g)

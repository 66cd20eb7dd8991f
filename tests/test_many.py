"""tc_count_many: several graphs ingested, built and counted as one pipeline (their disjoint union).  Each graph's
count must equal the oracle's T for that graph alone (Def. 2, Sec. II-A) and tc_count's on the graph alone, for
mixes of sizes and kinds, empty and degenerate graphs, every kind of input memory, both build paths of the union,
and out-of-range ids."""
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


def _mix(seed, k):
    """k graphs of mixed kinds and sizes, with empty, edgeless and self-loop-only graphs among them."""
    rng = np.random.default_rng(seed)
    out = [(np.zeros(0, np.int32), np.zeros(0, np.int32), 0),          # no vertices
           (np.zeros(0, np.int32), np.zeros(0, np.int32), 17),         # no edges
           (np.arange(5, dtype=np.int32), np.arange(5, dtype=np.int32), 5),  # self-loops only
           graphs.complete(30)[:3], graphs.wheel(12)[:3], graphs.friendship(9)[:3]]
    for i in range(k - len(out)):
        kind = i % 3
        if kind == 0:
            n = int(rng.integers(2, 3000))
            sp = graphgen.gnp(n, min(0.5, float(rng.uniform(2, 40)) / n), seed * 1000 + i)
        elif kind == 1:
            scale = int(rng.integers(4, 13))
            sp = graphgen.rmat(scale, int(rng.integers(4, 24)), seed * 1000 + i, n=int(rng.integers(1 << (scale - 1),
                                                                                                  (1 << scale) + 1)))
        else:
            n = int(rng.integers(1, 2000))
            sp = graphgen.er(n, int(rng.integers(0, 6 * n + 1)), seed * 1000 + i)
        s, d = sp.edges()
        out.append((s, d, sp.n))
    return out


@pytest.mark.parametrize("seed,k", [(1, 40), (2, 300)])
def test_many_equals_oracle_and_solo(tc, seed, k):
    mix = _mix(seed, k)
    got = tc.tc_count_many(mix)
    ref = np.array([oracle.count(s, d, n)[0] for s, d, n in mix], dtype=np.uint64)
    np.testing.assert_array_equal(got, ref)
    for (s, d, n), c in list(zip(mix, ref))[5:25]:  # the solo path agrees
        if n > 0:
            g = tc.tc_load_edges(s, d, n)
            try:
                tc.tc_build(g)
                assert tc.tc_count(g) == int(c)
            finally:
                tc.tc_free(g)


def test_many_input_memory_kinds(tc):
    """Pageable host arrays (copied), page-locked mapped host arrays (read in place) and device tensors agree."""
    import torch
    mix = _mix(3, 24)
    ref = np.array([oracle.count(s, d, n)[0] for s, d, n in mix], dtype=np.uint64)
    np.testing.assert_array_equal(tc.tc_count_many(mix), ref)
    pinned = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory(), n) for s, d, n in mix]
    np.testing.assert_array_equal(tc.tc_count_many(pinned), ref)
    dev = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n) for s, d, n in mix]
    np.testing.assert_array_equal(tc.tc_count_many(dev), ref)
    side = torch.cuda.Stream()
    np.testing.assert_array_equal(tc.tc_count_many(dev, stream=side), ref)


@pytest.mark.parametrize("path", ["compact", "sorted"])
def test_many_union_build_paths(tc, path):
    """A union above the compact build's limit (built with sizes read as known) and one sorted by radix sort give
    the same per-graph counts: the same R-MAT 14 graph thirty times, with a G(n, p) graph between copies."""
    s, d = graphgen.rmat(14, 16, 77).edges()
    T = oracle.count(s, d, 1 << 14)[0]
    gs, gd = graphgen.gnp(500, 0.05, 78).edges()
    Tg = oracle.count(gs, gd, 500)[0]
    mix = []
    for _ in range(30):
        mix += [(s, d, 1 << 14), (gs, gd, 500)]
    saved = (tc.tc_get_bucket_max_pairs(), tc.tc_get_compact_max_pairs())
    try:
        if path == "compact":
            tc.tc_set_tuning(tc.tc_get_tuning(), compact_max_pairs=1 << 40)
        else:
            tc.tc_set_tuning(tc.tc_get_tuning(), bucket_max_pairs=1, compact_max_pairs=0)
        got = tc.tc_count_many(mix)
    finally:
        tc.tc_set_tuning(tc.tc_get_tuning(), bucket_max_pairs=saved[0], compact_max_pairs=saved[1])
    np.testing.assert_array_equal(got, np.array([T, Tg] * 30, dtype=np.uint64))


def test_many_out_of_range_and_repeat_calls(tc):
    mix = _mix(4, 12)
    ref = np.array([oracle.count(s, d, n)[0] for s, d, n in mix], dtype=np.uint64)
    bad = list(mix)
    s, d, n = bad[7]
    d = d.copy()
    d[len(d) // 2] = n  # one id just past its graph's range
    bad[7] = (s, d, n)
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_many(bad)
    assert e.value.status == tc.TC_ERR_OUT_OF_RANGE
    for _ in range(2):  # the library is unaffected
        np.testing.assert_array_equal(tc.tc_count_many(mix), ref)
    np.testing.assert_array_equal(tc.tc_count_many(mix[3:4]), ref[3:4])

"""tc_count_per_vertex_noalloc: per-vertex counts for callers that may not allocate device memory while they run
(a serving loop that reserves all of its memory at start-up, or a host whose device memory belongs to another
framework's allocator).  Its scratch is a static device array shared by every call, so this file checks, on two
calls in a row, that it gives exactly the oracle's T and t(x) (Def. 2, Sec. II-A) and the output of
tc_count_per_vertex; that it asks the allocator for nothing; that it works on a side stream and on an empty graph;
and that it rejects graphs larger than the array.  The file name makes pytest collect it last."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


def _outputs(n):
    import torch
    out = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    return out, total


@pytest.mark.parametrize("spec", [graphgen.rmat(16, 16, 41), graphgen.er(200000, 2000000, 42)],
                         ids=["rmat16", "er200k"])
def test_noalloc_matches_oracle_twice(tc, spec):
    import torch
    hs, hd = spec.edges()
    T_or, _, t_or = oracle.count(hs, hd, spec.n, per_vertex=True)
    g = tc.tc_load_edges(hs, hd, spec.n, allocator="torch")  # allocations visible to the counter below
    try:
        tc.tc_build(g)
        T_pv, t_pv = tc.tc_count_per_vertex(g)
        assert T_pv == T_or
        np.testing.assert_array_equal(t_pv, t_or)
        alloc = tc.torch_allocator()
        for _ in range(2):  # the second call finds the first call's counts in the shared scratch
            out, total = _outputs(spec.n)
            torch.cuda.synchronize()
            before = alloc.allocations
            tc.tc_count_per_vertex_noalloc(g, out, total)
            torch.cuda.synchronize()
            assert alloc.allocations == before
            assert int(total.item()) == T_or
            np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), t_or)
    finally:
        tc.tc_free(g)


def test_noalloc_on_a_side_stream(tc):
    """Outputs are valid in the order of the stream given: read only after that stream has finished."""
    import torch
    spec = graphgen.rmat(14, 16, 43)
    hs, hd = spec.edges()
    T_or, _, t_or = oracle.count(hs, hd, spec.n, per_vertex=True)
    g = tc.tc_load_edges(hs, hd, spec.n)
    try:
        tc.tc_build(g)
        side = torch.cuda.Stream()
        for _ in range(2):
            with torch.cuda.stream(side):
                out, total = _outputs(spec.n)
            torch.cuda.synchronize()
            tc.tc_count_per_vertex_noalloc(g, out, total, stream=side)
            side.synchronize()
            assert int(total.item()) == T_or
            np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), t_or)
    finally:
        tc.tc_free(g)


def test_noalloc_empty_graph(tc):
    """n = 0: nothing to count, T = 0, and no per-vertex pointer is needed (passed as 0)."""
    import torch
    empty = np.zeros(0, dtype=np.int32)
    g = tc.tc_load_edges(empty, empty, 0)
    try:
        tc.tc_build(g)
        total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            tc.tc_count_per_vertex_noalloc(g, 0, total.data_ptr())
            torch.cuda.synchronize()
            assert int(total.item()) == 0
    finally:
        tc.tc_free(g)


def test_noalloc_rejects_graphs_above_its_scratch(tc):
    import torch
    n = (1 << 20) + 1
    s = np.array([0, 1, 2], dtype=np.int32)
    d = np.array([1, 2, 0], dtype=np.int32)
    g = tc.tc_load_edges(s, d, n)
    try:
        tc.tc_build(g)
        out = torch.zeros(n, dtype=torch.int64, device="cuda")
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(tc.TCError) as e:
            tc.tc_count_per_vertex_noalloc(g, out, total)
        assert e.value.status == tc.TC_ERR_INVALID_ARG and "1048576" in str(e.value)
        assert tc.tc_count(g) == 1  # the graph is still usable through the allocating path
    finally:
        tc.tc_free(g)

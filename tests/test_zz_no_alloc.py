"""tc_count_per_vertex_noalloc: the per-vertex count for callers that may not allocate device memory while they
run.  Its scratch is a static device array, so this file checks, on two calls in a row, that it gives exactly the
output of tc_count_per_vertex, that it asks the allocator for nothing, and that it rejects graphs larger than the
array.  The file name makes pytest collect it last."""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    import paper_1909_02127_gb300 as tc
    from paper_1909_02127_gb300 import build
    build.build()
    torch.cuda.init()
    return tc


@pytest.mark.parametrize("spec", [graphgen.rmat(16, 16, 41), graphgen.er(200000, 2000000, 42)],
                         ids=["rmat16", "er200k"])
def test_noalloc_matches_per_vertex_twice(tc, spec):
    import torch
    hs, hd = spec.edges()
    g = tc.tc_load_edges(hs, hd, spec.n, allocator="torch")  # allocations visible to the counter below
    try:
        tc.tc_build(g)
        T_ref, t_ref = tc.tc_count_per_vertex(g)
        alloc = tc.torch_allocator()
        for _ in range(2):
            out = torch.full((spec.n,), -1, dtype=torch.int64, device="cuda")
            total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            before = alloc.allocations
            tc.tc_count_per_vertex_noalloc(g, out, total)
            torch.cuda.synchronize()
            assert alloc.allocations == before
            assert int(total.item()) == T_ref
            np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), t_ref)
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

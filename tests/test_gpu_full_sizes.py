"""GPU parity at the benchmark's full sizes, in the benchmark's launch configuration (device-resident edges, one
tc_load_edges / tc_build / count per graph).  R-MAT 26 is compared with the oracle's full result, computed once on
the host by a committed script and stored under tests/golden/; the 4096-graph batch with one-by-one counts on every
graph and with the oracle on a sample of them."""
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


GOLDEN_RMAT26 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rmat26_oracle.json")


def test_rmat26_bit_exact_against_the_oracle(tc):
    """R-MAT scale 26 (2^30 sampled pairs, permuted ids), in the benchmark's launch configuration: T, m and every
    t(x) on the GPU equal the oracle's (Def. 2, Sec. II-A; the |M|/|Q| result of Algorithm 1), as stored by
    tests/golden/make_rmat26.py, which calls only the oracle: T and m exactly, t(x) by the sha256 of all n counts and
    value by value at 256 stored vertices.  The input is first checked against the stored fingerprint, so a changed
    generator and a wrong count cannot be confused."""
    import hashlib
    import json

    import torch
    with open(GOLDEN_RMAT26) as f:
        gold = json.load(f)
    spec = graphgen.config("rmat26")
    assert (spec.n, spec.num_edges, spec.seed, spec.scale, spec.permute) == (
        gold["spec"]["n"], gold["spec"]["num_edges"], gold["spec"]["seed"], gold["spec"]["scale"],
        gold["spec"]["permute"])
    ds, dd = spec.edges(device="cuda")
    idx = torch.from_numpy(np.unique(np.linspace(0, spec.num_edges - 1, 65536).astype(np.int64))).cuda()
    fp = hashlib.sha256()
    fp.update(ds[idx].cpu().numpy().astype("<i4").tobytes())
    fp.update(dd[idx].cpu().numpy().astype("<i4").tobytes())
    assert fp.hexdigest() == gold["input_fingerprint"]["sha256"], "the generated input differs from the stored one"
    g = tc.tc_load_edges(ds, dd, spec.n)
    del ds, dd, idx
    torch.cuda.empty_cache()
    try:
        tc.tc_build(g)
        info = tc.tc_graph_get_info(g)
        T = tc.tc_count(g)
        T2, t = tc.tc_count_per_vertex(g)
    finally:
        tc.tc_free(g)
    assert info["num_edges"] == gold["m"]
    assert T == gold["T"] and T2 == gold["T"]
    np.testing.assert_array_equal(t[np.array(gold["sample_x"])], np.array(gold["sample_t"], dtype=np.uint64))
    assert hashlib.sha256(np.ascontiguousarray(t).astype("<u8").tobytes()).hexdigest() == gold["t_sha256"]


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

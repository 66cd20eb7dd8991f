"""Serving loop: every request's count is the same alone and in the mix (tolerance 0), with continuous batching
and with one graph per launch, and under a tight device-memory budget."""
import time

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


@pytest.fixture(scope="module")
def requests_and_solo(tc):
    pool = [sp for sp in graphgen.serve_pool(96) if sp.num_edges <= 400_000]
    edges = [sp.edges() for sp in pool]
    solo = []
    for sp, (s, d) in zip(pool, edges):
        g = tc.tc_load_edges(s, d, sp.n)
        tc.tc_build(g)
        solo.append(tc.tc_count(g))
        tc.tc_free(g)
    # the solo path itself against the oracle, on every request graph of the pool
    for sp, (s, d), T in zip(pool, edges, solo):
        assert oracle.count(s, d, sp.n)[0] == T, sp
    return pool, edges, solo


def _run(tc, pool, edges, order, **cfg):
    got = {}
    with tc.Server(**cfg) as srv:
        ids = {}
        for k in order:
            s, d = edges[k]
            ids[srv.submit(s, d, pool[k].n)] = k
        deadline = time.time() + 120
        received = 0
        while received < len(ids) and time.time() < deadline:
            for r in srv.poll(timeout_ms=100):
                received += 1
                assert r["status"] == 0, r
                assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_built_ns"] <= r["t_done_ns"]
                got.setdefault(ids[r["id"]], []).append(r["triangles"])
        stats = srv.stats()
    assert sum(len(v) for v in got.values()) == len(order)
    return got, stats


def test_alone_equals_in_the_mix(tc, requests_and_solo):
    pool, edges, solo = requests_and_solo
    rng = np.random.default_rng(5)
    order = list(rng.permutation(len(pool))) + list(rng.integers(0, len(pool), size=64))  # with repeats
    for batching in ("pipeline", True, False):
        got, stats = _run(tc, pool, edges, order, batching=batching, build_workers=4)
        for k, counts in got.items():
            assert all(c == solo[k] for c in counts), (k, counts, solo[k])
        if batching:
            assert stats["max_batch_seen"] > 1  # requests did share launches
        else:
            assert stats["max_batch_seen"] == 1


def test_pipeline_batch_with_a_bad_request(tc, requests_and_solo):
    """With the whole path batched, a request with an out-of-range id fails alone; its batch-mates still get their
    counts."""
    pool, edges, solo = requests_and_solo
    order = list(range(min(40, len(pool))))
    bad_k = order[len(order) // 2]
    s, d = edges[bad_k]
    d_bad = d.copy()
    d_bad[0] = pool[bad_k].n  # one id past the range
    statuses = {}
    with tc.Server(batching="pipeline", build_workers=1) as srv:
        ids = {}
        for k in order:
            ss, dd = (s, d_bad) if k == bad_k else edges[k]
            ids[srv.submit(ss, dd, pool[k].n)] = k
        deadline = time.time() + 120
        while len(statuses) < len(ids) and time.time() < deadline:
            for r in srv.poll(timeout_ms=100):
                statuses[ids[r["id"]]] = (r["status"], r["triangles"])
    assert statuses[bad_k][0] == tc.TC_ERR_OUT_OF_RANGE
    for k in order:
        if k != bad_k:
            assert statuses[k] == (0, solo[k])


@pytest.mark.parametrize("batching", [True, "pipeline"])
def test_tight_memory_budget(tc, requests_and_solo, batching):
    pool, edges, solo = requests_and_solo
    budget = 48 << 20
    order = [k for k in range(len(pool)) if 32 * pool[k].num_edges + 48 * pool[k].n + (1 << 20) <= budget]
    assert len(order) > 10
    got, stats = _run(tc, pool, edges, order, hbm_budget_bytes=budget, build_workers=8, batching=batching)
    for k, counts in got.items():
        assert counts == [solo[k]]
    assert stats["peak_held_bytes"] <= budget
    # a request larger than the whole budget is refused at submission
    big = max(range(len(pool)), key=lambda k: pool[k].num_edges)
    with tc.Server(hbm_budget_bytes=1 << 20) as srv:
        s, d = edges[big]
        with pytest.raises(tc.TCError) as e:
            srv.submit(s, d, pool[big].n)
        assert e.value.status == tc.TC_ERR_NO_MEMORY

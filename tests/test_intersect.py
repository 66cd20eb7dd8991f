"""The segmented-intersection counter (tc_count_intersect) against the oracle, bit-exact.

It walks the same oriented CSR as tc_count with a different kernel (one lane per oriented edge, galloping search),
so the cases cover its own edges: rows staged in shared memory and rows too long for it (K_n with d+ > 1024),
empty intersections, hubs, and the workloads' graph families.
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


def _count(tc, src, dst, n):
    g = tc.tc_load_edges(src, dst, n)
    try:
        tc.tc_build(g)
        return tc.tc_count_intersect(g), tc.tc_count(g)
    finally:
        tc.tc_free(g)


@pytest.mark.parametrize("name,g", graphs.closed_form_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_closed_forms(tc, name, g):
    src, dst, n, T, _ = g
    assert _count(tc, src, dst, n) == (T, T)


@pytest.mark.parametrize("n", [33, 1030, 2100])
def test_cliques_staged_and_unstaged(tc, n):
    src, dst, n, T, _ = graphs.complete(n)
    assert _count(tc, src, dst, n) == (math.comb(n, 3), math.comb(n, 3))


CASES = [("er4096", lambda: (*graphgen.config("er4096").edges(), 4096)),
         ("rmat16", lambda: (*graphgen.rmat(16, 16, 91).edges(), 1 << 16)),
         ("rmat15p", lambda: (*graphgen.rmat(15, 24, 92, n=30000, permute=True).edges(), 30000)),
         ("er100k", lambda: (*graphgen.er(100000, 1600000, 93).edges(), 100000))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_against_oracle(tc, name, make):
    src, dst, n = make()
    T, _ = oracle.count(src, dst, n)
    assert _count(tc, src, dst, n) == (T, T)


@pytest.mark.parametrize("seed", range(6))
def test_random(tc, seed):
    rng = np.random.default_rng(1300 + seed)
    n = int(rng.choice([3, 50, 700, 6000]))
    src, dst = graphs.random_simple_pairs(rng, n, int(rng.integers(0, 10 * n)))
    T, _ = oracle.count(src, dst, n)
    assert _count(tc, src, dst, n) == (T, T)


def test_hub_heavy(tc):
    rng = np.random.default_rng(1400)
    n = 20000
    hubs = rng.integers(0, n, 8)
    src = np.concatenate([np.repeat(hubs, 3000), rng.integers(0, n, 60000)]).astype(np.int32)
    dst = np.concatenate([rng.integers(0, n, 24000), rng.integers(0, n, 60000)]).astype(np.int32)
    T, _ = oracle.count(src, dst, n)
    assert _count(tc, src, dst, n) == (T, T)


def test_state_and_null(tc):
    import ctypes
    lib = tc.load_library()
    T = ctypes.c_uint64()
    assert lib.tc_count_intersect(None, ctypes.byref(T), None) == tc.TC_ERR_INVALID_ARG
    src, dst, n, _, _ = graphs.complete(4)
    g = tc.tc_load_edges(src, dst, n)
    try:
        assert lib.tc_count_intersect(g, ctypes.byref(T), None) == tc.TC_ERR_STATE
        tc.tc_build(g)
        assert lib.tc_count_intersect(g, None, None) == tc.TC_ERR_INVALID_ARG
        assert lib.tc_count_intersect(g, ctypes.byref(T), None) == tc.TC_OK and T.value == 4
    finally:
        tc.tc_free(g)


def test_tc_count_dispatches_by_the_tuning(tc):
    """With the ratio threshold above every graph's, tc_count and tc_count_device run the intersection kernel; the
    counts stay exact either way."""
    import torch
    src, dst = graphgen.rmat(14, 16, 94).edges()
    n = 1 << 14
    T, _ = oracle.count(src, dst, n)
    saved = tc.tc_get_isect_max_wedges_milli()
    d = torch.zeros(1, dtype=torch.int64, device="cuda")
    try:
        for ratio in (0, 1 << 40):
            tc.tc_set_tuning(tc.tc_get_tuning(), isect_max_wedges_milli=ratio)
            g = tc.tc_load_edges(src, dst, n)
            try:
                tc.tc_build(g)
                assert tc.tc_count(g) == T
                tc.tc_count_device(g, d)
                assert int(d.item()) == T
            finally:
                tc.tc_free(g)
    finally:
        tc.tc_set_tuning(tc.tc_get_tuning(), isect_max_wedges_milli=saved)

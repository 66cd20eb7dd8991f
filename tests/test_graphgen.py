"""Input generators: determinism, ranges, bijectivity, chunking, host == device."""
import numpy as np
import pytest

import graphgen


def test_mix64_python_matches_published_values():
    # SplitMix64 with seed 0: the first outputs of the reference sequence x_i = mix64(i * GAMMA), i = 1, 2, 3
    # (Steele, Lea & Flood 2014; widely reproduced test vector).
    assert graphgen.mix64(graphgen.GAMMA) == 0xE220A8397B1DCDAF
    assert graphgen.mix64((2 * graphgen.GAMMA) & graphgen.M64) == 0x6E789E6AA1B965F4
    assert graphgen.mix64((3 * graphgen.GAMMA) & graphgen.M64) == 0x06C45D188009454F


def test_er_deterministic_and_in_range():
    spec = graphgen.er(1000, 5000, 42)
    a1, b1 = spec.edges()
    a2, b2 = spec.edges()
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(b1, b2)
    assert a1.min() >= 0 and a1.max() < 1000 and b1.min() >= 0 and b1.max() < 1000
    a3, _ = graphgen.er(1000, 5000, 43).edges()
    assert (a3 != a1).mean() > 0.9


def test_chunked_equals_whole():
    for spec in (graphgen.er(777, 3001, 1), graphgen.rmat(12, 4, 2), graphgen.rmat(10, 8, 3, n=700)):
        s, d = spec.edges()
        s1, d1 = spec.edges(e0=0, length=1000)
        s2, d2 = spec.edges(e0=1000)
        np.testing.assert_array_equal(np.concatenate([s1, s2]), s)
        np.testing.assert_array_equal(np.concatenate([d1, d2]), d)


def test_rmat_thresholds_and_skew():
    thr = graphgen.rmat_thresholds(7, 16)
    t = thr.reshape(16, 3).astype(np.int64)
    assert (t[:, 0] < t[:, 1]).all() and (t[:, 1] < t[:, 2]).all()
    # noise stays within +-5% of each probability before renormalisation
    a = t[:, 0] / 2 ** 32
    assert ((a > 0.57 * 0.95 / 1.05 - 1e-9) & (a < 0.57 * 1.05 / 0.95 + 1e-9)).all()
    s, d = graphgen.rmat(14, 8, 7).edges()
    deg = np.bincount(np.concatenate([s, d]), minlength=1 << 14)
    assert deg.max() > 50 * deg.mean()  # power-law-like skew


def test_rmat_non_power_of_two_in_range():
    s, d = graphgen.rmat(11, 16, 9, n=1500).edges()
    assert s.max() < 1500 and d.max() < 1500 and s.min() >= 0


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 1024, 4097])
def test_permutation_is_bijection(n):
    ids = np.arange(n, dtype=np.int32)
    spec = graphgen.GraphSpec("er", n, 0, 99, permute=True)
    lib = graphgen._host()
    out = ids.copy()
    assert lib.gg_permute_host(spec.seed, n, graphgen._i32p(out), n, 2) == 0
    assert sorted(out.tolist()) == list(range(n))


def test_batch_and_serve_mixes():
    b = graphgen.batch_mix(4096)
    ns = np.array([s.n for s in b])
    assert ns.min() >= 64 and ns.max() <= 65536
    assert 1200 < np.median(ns) < 3500  # log-uniform on [64, 65536] has median 2048
    assert sum(s.kind == "er" for s in b) == 2048
    pool = graphgen.serve_pool(256)
    ms = np.array([s.num_edges for s in pool])
    assert ms.min() >= 1000 and ms.max() <= 4_000_000
    arr = graphgen.poisson_arrivals(2000.0, 1.0)
    assert 1800 < arr.size < 2200 and np.all(np.diff(arr) > 0)


@pytest.mark.gpu
def test_device_generator_matches_host():
    import torch
    for spec in (graphgen.er(4096, 32768, 5), graphgen.rmat(16, 16, 6), graphgen.rmat(13, 9, 7, n=5000),
                 graphgen.rmat(12, 16, 8, permute=True)):
        hs, hd = spec.edges()
        ds, dd = spec.edges(device="cuda")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ds.cpu().numpy(), hs)
        np.testing.assert_array_equal(dd.cpu().numpy(), hd)

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
    assert sum(s.kind == "gnp" for s in b) == 2048
    degs = np.array([s.p * (s.n - 1) for s in b if s.kind == "gnp"])
    assert degs.min() >= 4.0 - 1e-9 and degs.max() <= 64.0 + 1e-9  # mean degree d ~ U[4, 64] (below n - 1)
    pool = graphgen.serve_pool(256)
    ms = np.array([s.expected_edges for s in pool])
    assert ms.min() >= 900 and ms.max() <= 4_000_000
    arr = graphgen.poisson_arrivals(2000.0, 1.0)
    assert 1800 < arr.size < 2200 and np.all(np.diff(arr) > 0)


@pytest.mark.gpu
def test_device_generator_matches_host():
    import torch
    for spec in (graphgen.er(4096, 32768, 5), graphgen.rmat(16, 16, 6), graphgen.rmat(13, 9, 7, n=5000),
                 graphgen.rmat(12, 16, 8, permute=True), graphgen.config("er4096"), graphgen.gnp(65536, 1e-3, 9),
                 graphgen.gnp(300, 0.9, 10), graphgen.gnp(5000, 0.0, 11)):
        hs, hd = spec.edges()
        ds, dd = spec.edges(device="cuda")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ds.cpu().numpy(), hs)
        np.testing.assert_array_equal(dd.cpu().numpy(), hd)


# ---- G(n, p) by geometric skipping -----------------------------------------------------------------------------
def test_log2_q40_pins():
    """Powers of two are exact; other values agree with the real logarithm to the 2^-40 truncation; the C and
    Python versions take the same integer steps (bit-identical)."""
    import math
    lib = graphgen._host()
    one = 1 << graphgen.LOG_FRAC_BITS
    for k in range(64):
        assert graphgen.log2_q40(1 << k) == k * one
        assert lib.gg_log2_q40_host(1 << k) == k * one
    rng = np.random.default_rng(1)
    xs = [3, 5, 10, 1000, (1 << 63) - 1, (1 << 64) - 1] + [int(v) for v in rng.integers(1, 1 << 63, 300, dtype=np.int64)]
    for x in xs:
        r = graphgen.log2_q40(x)
        assert lib.gg_log2_q40_host(x) == r
        # truncated: below the true value by less than 2^-38 (each of 40 squarings truncates at 2^-63)
        err = math.log2(x) - r / one
        assert -1e-12 <= err < 2.0 ** -38 + 1e-12 * math.log2(x), x


def test_geometric_gap_law():
    """P(gap >= k) = (1-p)^k: the mean gap is (1-p)/p and a gap of 0 has probability p."""
    lib = graphgen._host()
    for p in (0.5, 0.1, 0.004):
        lq = graphgen.gnp_lq(p)
        key = graphgen.stream_key(77, 9)
        gaps = np.array([lib.gg_geometric_host(graphgen.draw(key, i), lq) for i in range(40000)], dtype=np.float64)
        mean, sd = (1 - p) / p, np.sqrt(1 - p) / p
        assert abs(gaps.mean() - mean) < 5 * sd / np.sqrt(gaps.size)
        assert abs((gaps == 0).mean() - p) < 5 * np.sqrt(p * (1 - p) / gaps.size)


def test_gnp_simple_and_in_range():
    spec = graphgen.gnp(3000, 0.01, 5)
    s, d = spec.edges()
    assert s.size == spec.num_edges and s.size > 0
    assert (s < d).all() and s.min() >= 0 and d.max() < 3000  # pairs i < j: no self-loops
    assert np.unique(s.astype(np.int64) * 3000 + d).size == s.size  # no repeats
    s2, d2 = spec.edges()
    np.testing.assert_array_equal(s, s2)
    np.testing.assert_array_equal(d, d2)
    s3, _ = graphgen.gnp(3000, 0.01, 6).edges()
    assert s3.size != s.size or (s3 != s).any()


@pytest.mark.parametrize("n,p", [(4096, 16.0 / 4095.0), (20000, 1e-4), (500, 0.5), (65536, 4.0 / 65535.0)])
def test_gnp_edge_count_binomial(n, p):
    """m ~ Binomial(n(n-1)/2, p): within 4 sigma of its mean."""
    spec = graphgen.gnp(n, p, 1000 + n)
    pairs = n * (n - 1) / 2
    assert abs(spec.num_edges - pairs * p) < 4 * np.sqrt(pairs * p * (1 - p))


def test_er4096_config_is_gnp():
    spec = graphgen.config("er4096")
    assert spec.kind == "gnp" and spec.n == 4096 and abs(spec.p - 16 / 4095) < 1e-15
    m = spec.num_edges
    assert abs(m - 32768) < 4 * np.sqrt(32768 * (1 - 16 / 4095))
    s, d = spec.edges()
    assert np.unique(s.astype(np.int64) * 4096 + d).size == m  # no duplicates arise


def test_gnp_pairs_independent_and_uniform():
    """Each pair's frequency over many seeds is p, with no dependence between neighbouring pairs of a row (their
    joint frequency is p^2) and none between rows."""
    n, p, reps = 24, 0.3, 3000
    cnt = np.zeros((n, n))
    both = 0
    both_rows = 0
    for r in range(reps):
        s, d = graphgen.gnp(n, p, 50000 + r).edges()
        a = np.zeros((n, n), dtype=bool)
        a[s, d] = True
        cnt += a
        both += a[0, 1] and a[0, 2]
        both_rows += a[0, 5] and a[1, 5]
    iu = np.triu_indices(n, 1)
    freq = cnt[iu] / reps
    sd = np.sqrt(p * (1 - p) / reps)
    assert np.abs(freq - p).max() < 5 * sd
    assert abs(cnt[np.tril_indices(n)].sum()) == 0
    sd2 = np.sqrt(p * p * (1 - p * p) / reps)
    assert abs(both / reps - p * p) < 5 * sd2 and abs(both_rows / reps - p * p) < 5 * sd2


def test_gnp_degenerate_cases():
    assert graphgen.gnp(5000, 0.0, 1).num_edges == 0
    assert graphgen.gnp(1, 0.5, 1).num_edges == 0
    s, d = graphgen.gnp(2, 0.999999, 1).edges()
    assert s.size <= 1
    spec = graphgen.gnp(200, 0.999, 2)  # nearly complete
    assert spec.num_edges > 0.99 * 200 * 199 / 2
    with pytest.raises(ValueError):
        graphgen.gnp(10, 1.0, 1)


def test_gnp_slices():
    spec = graphgen.gnp(2000, 0.02, 3)
    s, d = spec.edges()
    s1, d1 = spec.edges(e0=0, length=1000)
    s2, d2 = spec.edges(e0=1000)
    np.testing.assert_array_equal(np.concatenate([s1, s2]), s)
    np.testing.assert_array_equal(np.concatenate([d1, d2]), d)

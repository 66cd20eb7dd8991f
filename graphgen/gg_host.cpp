// gg_host.cpp — multi-threaded host evaluation of the generators in gg.h (C ABI, loaded by graphgen/__init__.py).
// Each edge is a pure function of its index, so threads split the index range with no shared state.
#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "gg.h"

namespace {

template <class F>
void parallel_range(int64_t len, int threads, F f) {
  if (threads < 1) threads = 1;
  const int64_t min_chunk = 1 << 16;
  int64_t t = std::min<int64_t>(threads, std::max<int64_t>(1, (len + min_chunk - 1) / min_chunk));
  if (t <= 1) {
    f(0, len);
    return;
  }
  std::vector<std::thread> pool;
  const int64_t chunk = (len + t - 1) / t;
  for (int64_t i = 0; i < t; ++i) {
    const int64_t lo = i * chunk, hi = std::min(len, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([=] { f(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

// G(n, p) with lq = -log2(1-p) in Q.40.  Row i has n-1-i candidates, so rows are dealt to threads round-robin.
template <class F>
void gnp_rows(uint32_t n, int threads, F f) {
  int64_t t = threads < 1 ? 1 : threads;
  if (t > (int64_t)n / 256 + 1) t = (int64_t)n / 256 + 1;
  std::vector<std::thread> pool;
  for (int64_t k = 1; k < t; ++k)
    pool.emplace_back([=] {
      for (int64_t i = k; i < (int64_t)n; i += t) f((uint32_t)i);
    });
  for (int64_t i = 0; i < (int64_t)n; i += t) f((uint32_t)i);
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// Edges [e0, e0+len) of the uniform edge sampler on n vertices.
int gg_er_host(uint64_t seed, uint32_t n, int64_t e0, int64_t len, int32_t* src, int32_t* dst, int threads) {
  if (n == 0 || len < 0 || (len > 0 && (!src || !dst))) return 1;
  parallel_range(len, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) gg_er_edge(seed, n, (uint64_t)(e0 + i), &src[i], &dst[i]);
  });
  return 0;
}

// Edges [e0, e0+len) of an R-MAT graph (thresholds: 3*scale uint32 values).
int gg_rmat_host(uint64_t seed, int scale, uint32_t n, const uint32_t* thr, int64_t e0, int64_t len, int32_t* src,
                 int32_t* dst, int threads) {
  if (n == 0 || scale < 1 || scale > 31 || (1ULL << scale) < n || len < 0 || !thr ||
      (len > 0 && (!src || !dst)))
    return 1;
  parallel_range(len, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) gg_rmat_edge(seed, scale, n, thr, (uint64_t)(e0 + i), &src[i], &dst[i]);
  });
  return 0;
}

// The fixed-point helpers of gg.h, exported for the tests.
uint64_t gg_log2_q40_host(uint64_t x) { return x ? gg_log2_q40(x) : 0; }
uint64_t gg_geometric_host(uint64_t r, uint64_t lq) { return lq ? gg_geometric(r, lq) : 0; }

// Row offsets of G(n, p): row_off[0..n] (row_off[n] = the number of pairs, also returned); -1 on a bad argument.
int64_t gg_gnp_count_host(uint64_t seed, uint32_t n, uint64_t lq, int64_t* row_off, int threads) {
  if (!row_off) return -1;
  row_off[0] = 0;
  gnp_rows(n, threads, [&](uint32_t i) { row_off[i + 1] = gg_gnp_row(seed, n, lq, i, nullptr, nullptr); });
  for (int64_t i = 0; i < (int64_t)n; ++i) row_off[i + 1] += row_off[i];
  return row_off[n];
}

// The pairs of G(n, p), row i at row_off[i] (the offsets from gg_gnp_count_host).  Returns 0, or 1 on a bad
// argument.
int gg_gnp_write_host(uint64_t seed, uint32_t n, uint64_t lq, const int64_t* row_off, int32_t* src, int32_t* dst,
                      int threads) {
  if (!row_off || ((!src || !dst) && row_off[n] > 0)) return 1;
  gnp_rows(n, threads, [&](uint32_t i) { gg_gnp_row(seed, n, lq, i, src + row_off[i], dst + row_off[i]); });
  return 0;
}

// ids[i] <- perm(ids[i]) in place, for ids in [0, n).
int gg_permute_host(uint64_t seed, uint32_t n, int32_t* ids, int64_t len, int threads) {
  if (n == 0 || len < 0 || (len > 0 && !ids)) return 1;
  parallel_range(len, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) ids[i] = (int32_t)gg_permute(seed, n, (uint32_t)ids[i]);
  });
  return 0;
}

}  // extern "C"

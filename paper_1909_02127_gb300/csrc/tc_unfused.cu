// tc_unfused.cu — the paper's unfused verification loop, kept beside the fused kernel as its ablation.
//
// Algorithm 1 answers the triangle query with rounds of Gunrock operators over an all-source BFS, and every round
// writes its frontier to memory: a filter of candidate sources by NE, then per round an advance from the partial
// matches over their out-edges with the stored constraints checked per traversed edge, a compaction of the
// survivors (Compute), their write to the partial results and a mask of the incomplete ones (Sec. III-A/III-B).
// On the oriented CSR of tc_build (the visiting order stands in for the UMO id constraint) the rounds are:
//   filter    c_set = {u : d+(u) >= 2}                          NE filter with the 2-look-ahead (Sec. III-C)
//   hop 1   advance c_set over N+(u): one slot per (u, v), kept if d+(v) > 0 (the 1-look-ahead);
//             compact the kept slots to the partial matches M2 = [(u, v)]
//   hop 2   advance M2 over N+(v): one slot per (u, v, w), kept if u -> w is an edge (the stored non-tree
//             connection); compact the kept slots to the complete matches M3 = [(u, v, w)]
//   result    |M3| triangles (|M|/|Q| with M counted in nodes)
// Each frontier holds one 32-bit slot per traversed edge: the memory the fused kernel never writes.  Hop 2 has
// W = sum over M2 of d+(v) slots; it runs in chunks whose slots and survivors fit the caller's budget (the paper
// keeps the frontier whole), at most 2^31 - 1 slots per chunk because positions come from a 32-bit scan.
#include <cstring>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kUfThreads = 256;
constexpr int64_t kUfTile = 2048;                      // frontier slots per block step (8 per thread)
constexpr int64_t kUfMaxChunk = (int64_t(1) << 31) - 1;
constexpr int64_t kUfMinChunk = 4096;

// True out-degree of u: the padded row less its trailing pad ids (at most three).
__device__ __forceinline__ int64_t out_degree(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                              int32_t pad, int64_t u) {
  const int64_t a = off[u];
  int64_t e = off[u + 1];
  while (e > a && col[e - 1] == pad) --e;
  return e - a;
}

// Largest j in [lo, hi] with o[j] <= e, for non-decreasing o with o[lo] <= e: the frontier row holding slot e.
__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ o, int64_t lo, int64_t hi, int64_t e) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (o[mid] <= e)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Filter: the sizes of the hop-1 frontier rows (0 for u outside c_set) and |c_set|.
__global__ void k_uf_filter(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                            int32_t* __restrict__ sz, unsigned long long* __restrict__ candidates) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = out_degree(off, col, (int32_t)n, u);
    const bool in = d >= 2;
    sz[u] = in ? (int32_t)d : 0;
    const unsigned b = __ballot_sync(__activemask(), in);
    if (in && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(candidates, (unsigned long long)__popc(b));
  }
}

// Slots [t0, t1) of a frontier with row prefix o (rows 0..rows-1) are handled by one block; the rows they span are
// found once per block and each slot searches only between them.
struct TileRange {
  int64_t lo, hi;
};
__device__ __forceinline__ TileRange tile_rows(const int64_t* o, int64_t rows, int64_t t0, int64_t t1,
                                               int64_t* shared2) {
  if (threadIdx.x == 0) {
    shared2[0] = row_of(o, 0, rows - 1, t0);
    shared2[1] = row_of(o, 0, rows - 1, t1 - 1);
  }
  __syncthreads();
  TileRange r{shared2[0], shared2[1]};
  return r;
}

// Hop 1 advance: slot e is (u, v) with v the (e - o1[u])-th out-neighbour of u; kept if v has out-neighbours.
__global__ void __launch_bounds__(kUfThreads) k_uf_advance1(const int64_t* __restrict__ o1, int64_t n,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ col, int64_t E1,
                                                            uint32_t* __restrict__ keep) {
  __shared__ int64_t rows[2];
  for (int64_t t0 = (int64_t)blockIdx.x * kUfTile; t0 < E1; t0 += (int64_t)gridDim.x * kUfTile) {
    const int64_t t1 = t0 + kUfTile < E1 ? t0 + kUfTile : E1;
    const TileRange r = tile_rows(o1, n, t0, t1, rows);
    for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
      const int64_t u = row_of(o1, r.lo, r.hi, e);
      const int32_t v = col[off[u] + (e - o1[u])];
      keep[e] = off[v + 1] > off[v] ? 1u : 0u;
    }
    __syncthreads();
  }
}

// Hop 1 compaction: kept slots to M2 at their scanned positions.
__global__ void __launch_bounds__(kUfThreads) k_uf_compact1(const int64_t* __restrict__ o1, int64_t n,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ col, int64_t E1,
                                                            const uint32_t* __restrict__ pos,
                                                            int32_t* __restrict__ m2u, int32_t* __restrict__ m2v) {
  __shared__ int64_t rows[2];
  for (int64_t t0 = (int64_t)blockIdx.x * kUfTile; t0 < E1; t0 += (int64_t)gridDim.x * kUfTile) {
    const int64_t t1 = t0 + kUfTile < E1 ? t0 + kUfTile : E1;
    const TileRange r = tile_rows(o1, n, t0, t1, rows);
    for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
      const uint32_t p = pos[e];
      if (pos[e + 1] == p) continue;
      const int64_t u = row_of(o1, r.lo, r.hi, e);
      m2u[p] = (int32_t)u;
      m2v[p] = col[off[u] + (e - o1[u])];
    }
    __syncthreads();
  }
}

// Sizes of the hop-2 frontier rows: d+(v) for each partial match (u, v).
__global__ void k_uf_sizes2(const int32_t* __restrict__ m2v, int64_t P2, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ col, int32_t pad, int32_t* __restrict__ sz) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P2; j += (int64_t)gridDim.x * blockDim.x)
    sz[j] = (int32_t)out_degree(off, col, pad, m2v[j]);
}

// Is w in the sorted row of u?  (Pad ids equal n and sort after every real id.)
__device__ __forceinline__ bool has_edge(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                         int32_t u, int32_t w) {
  int64_t lo = off[u], hi = off[u + 1];
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < w)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < end && col[lo] == w;
}

// Hop 2 advance over slots [c0, c0 + cnt): slot e is (u, v, w) with w the (e - o2[j])-th out-neighbour of v for
// the partial match j = (u, v); kept if the closing edge u -> w exists.
__global__ void __launch_bounds__(kUfThreads) k_uf_advance2(const int64_t* __restrict__ o2, int64_t P2,
                                                            const int32_t* __restrict__ m2u,
                                                            const int32_t* __restrict__ m2v,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ col, int64_t c0,
                                                            int64_t cnt, uint32_t* __restrict__ keep) {
  __shared__ int64_t rows[2];
  for (int64_t t0 = (int64_t)blockIdx.x * kUfTile; t0 < cnt; t0 += (int64_t)gridDim.x * kUfTile) {
    const int64_t t1 = t0 + kUfTile < cnt ? t0 + kUfTile : cnt;
    const TileRange r = tile_rows(o2, P2, c0 + t0, c0 + t1, rows);
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
      const int64_t e = c0 + i;
      const int64_t j = row_of(o2, r.lo, r.hi, e);
      const int32_t v = m2v[j];
      const int32_t w = col[off[v] + (e - o2[j])];
      keep[i] = has_edge(off, col, m2u[j], w) ? 1u : 0u;
    }
    __syncthreads();
  }
}

// Hop 2 compaction: kept slots to M3 as (u, v, w) rank triples.
__global__ void __launch_bounds__(kUfThreads) k_uf_compact2(const int64_t* __restrict__ o2, int64_t P2,
                                                            const int32_t* __restrict__ m2u,
                                                            const int32_t* __restrict__ m2v,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ col, int64_t c0,
                                                            int64_t cnt, const uint32_t* __restrict__ pos,
                                                            int32_t* __restrict__ m3) {
  __shared__ int64_t rows[2];
  for (int64_t t0 = (int64_t)blockIdx.x * kUfTile; t0 < cnt; t0 += (int64_t)gridDim.x * kUfTile) {
    const int64_t t1 = t0 + kUfTile < cnt ? t0 + kUfTile : cnt;
    const TileRange r = tile_rows(o2, P2, c0 + t0, c0 + t1, rows);
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
      const uint32_t p = pos[i];
      if (pos[i + 1] == p) continue;
      const int64_t e = c0 + i;
      const int64_t j = row_of(o2, r.lo, r.hi, e);
      const int32_t v = m2v[j];
      m3[3 * (int64_t)p + 0] = m2u[j];
      m3[3 * (int64_t)p + 1] = v;
      m3[3 * (int64_t)p + 2] = col[off[v] + (e - o2[j])];
    }
    __syncthreads();
  }
}

int tiles_grid(int64_t slots) {
  const int64_t t = (slots + kUfTile - 1) / kUfTile;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(t < 1 ? 1 : (t > cap ? cap : t));
}

// Intermediate buffers with a running total of the bytes held, for the peak the stats report.
struct Held {
  const Allocator& a;
  cudaStream_t s;
  int64_t now = 0, peak = 0;
  tc_status take(Buf& b, size_t bytes) {
    TC_TRY(buf_alloc(a, b, bytes, s));
    now += (int64_t)b.bytes;
    if (now > peak) peak = now;
    return TC_OK;
  }
  void drop(Buf& b) {
    now -= (int64_t)b.bytes;
    buf_release(a, b, s);
  }
};

// Copies one device int64/uint32 value to the host and waits for it.
template <class T>
tc_status read_back(const T* d, uint64_t* pinned, cudaStream_t s, int64_t* out) {
  TC_CUDA(cudaMemcpyAsync(pinned, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  T v;
  memcpy(&v, pinned, sizeof(T));
  *out = (int64_t)v;
  return TC_OK;
}

tc_status run_unfused(tc_graph* g, int64_t max_chunk_bytes, tc_unfused_stats* st, uint64_t* out_total,
                      cudaStream_t s) {
  const int64_t n = g->n;
  const int32_t pad = (int32_t)n;
  const int64_t* off = g->off.as<int64_t>();
  const int32_t* col = g->col.as<int32_t>();
  uint64_t* pinned = g->host_total;
  Held h{g->alloc, s};
  Buf sz1, o1, cand, keep1, m2u, m2v, sz2, o2, keep2, m3;
  tc_status rc = TC_OK;
  uint64_t total = 0;
  auto fail = [&](tc_status e) {
    rc = e;
    return e;
  };
  do {
    // filter
    if (fail(h.take(cand, 8)) != TC_OK) break;
    if (fail(cuda_status(cudaMemsetAsync(cand.p, 0, 8, s), "memset")) != TC_OK) break;
    if (fail(h.take(sz1, (size_t)n * 4)) != TC_OK || fail(h.take(o1, (size_t)(n + 1) * 8)) != TC_OK) break;
    k_uf_filter<<<grid_for(n, 256), 256, 0, s>>>(off, col, n, sz1.as<int32_t>(), cand.as<unsigned long long>());
    note_launch();
    if (fail(cuda_status(cudaGetLastError(), "k_uf_filter")) != TC_OK) break;
    if (fail(exclusive_scan_i32_to_i64(g->alloc, sz1.as<int32_t>(), o1.as<int64_t>(), n, s)) != TC_OK) break;
    h.drop(sz1);
    if (fail(read_back(cand.as<unsigned long long>(), pinned, s, &st->candidates)) != TC_OK) break;
    if (fail(read_back(o1.as<int64_t>() + n, pinned, s, &st->frontier1)) != TC_OK) break;
    const int64_t E1 = st->frontier1;
    if (E1 == 0) break;
    if (E1 >= kUfMaxChunk) {
      set_error("tc_count_unfused: the hop-1 frontier exceeds 2^31 - 1 slots");
      rc = TC_ERR_INVALID_ARG;
      break;
    }
    // hop 1: advance, compact
    if (fail(h.take(keep1, (size_t)(E1 + 1) * 4)) != TC_OK) break;
    if (fail(cuda_status(cudaMemsetAsync(keep1.as<uint32_t>() + E1, 0, 4, s), "memset")) != TC_OK) break;
    k_uf_advance1<<<tiles_grid(E1), kUfThreads, 0, s>>>(o1.as<int64_t>(), n, off, col, E1, keep1.as<uint32_t>());
    note_launch();
    if (fail(cuda_status(cudaGetLastError(), "k_uf_advance1")) != TC_OK) break;
    if (fail(exclusive_scan_u32(g->alloc, keep1.as<uint32_t>(), E1 + 1, s)) != TC_OK) break;
    if (fail(read_back(keep1.as<uint32_t>() + E1, pinned, s, &st->partials)) != TC_OK) break;
    const int64_t P2 = st->partials;
    if (P2 == 0) break;
    if (fail(h.take(m2u, (size_t)P2 * 4)) != TC_OK || fail(h.take(m2v, (size_t)P2 * 4)) != TC_OK) break;
    k_uf_compact1<<<tiles_grid(E1), kUfThreads, 0, s>>>(o1.as<int64_t>(), n, off, col, E1, keep1.as<uint32_t>(),
                                                        m2u.as<int32_t>(), m2v.as<int32_t>());
    note_launch();
    if (fail(cuda_status(cudaGetLastError(), "k_uf_compact1")) != TC_OK) break;
    h.drop(keep1);
    h.drop(o1);
    // hop 2: row sizes, then advance + compaction per chunk
    if (fail(h.take(sz2, (size_t)P2 * 4)) != TC_OK || fail(h.take(o2, (size_t)(P2 + 1) * 8)) != TC_OK) break;
    k_uf_sizes2<<<grid_for(P2, 256), 256, 0, s>>>(m2v.as<int32_t>(), P2, off, col, pad, sz2.as<int32_t>());
    note_launch();
    if (fail(cuda_status(cudaGetLastError(), "k_uf_sizes2")) != TC_OK) break;
    if (fail(exclusive_scan_i32_to_i64(g->alloc, sz2.as<int32_t>(), o2.as<int64_t>(), P2, s)) != TC_OK) break;
    h.drop(sz2);
    if (fail(read_back(o2.as<int64_t>() + P2, pinned, s, &st->frontier2)) != TC_OK) break;
    const int64_t E2 = st->frontier2;
    // 4 bytes per slot plus up to 12 bytes per survivor
    int64_t chunk = max_chunk_bytes > 0 ? max_chunk_bytes / 16 : kUfMaxChunk;
    if (chunk > kUfMaxChunk) chunk = kUfMaxChunk;
    if (chunk < kUfMinChunk) chunk = kUfMinChunk;
    if (chunk > E2) chunk = E2;
    if (E2 > 0 && fail(h.take(keep2, (size_t)(chunk + 1) * 4)) != TC_OK) break;
    for (int64_t c0 = 0; c0 < E2 && rc == TC_OK; c0 += chunk) {
      const int64_t cnt = E2 - c0 < chunk ? E2 - c0 : chunk;
      ++st->chunks;
      uint32_t* keep = keep2.as<uint32_t>();
      if (fail(cuda_status(cudaMemsetAsync(keep + cnt, 0, 4, s), "memset")) != TC_OK) break;
      k_uf_advance2<<<tiles_grid(cnt), kUfThreads, 0, s>>>(o2.as<int64_t>(), P2, m2u.as<int32_t>(),
                                                           m2v.as<int32_t>(), off, col, c0, cnt, keep);
      note_launch();
      if (fail(cuda_status(cudaGetLastError(), "k_uf_advance2")) != TC_OK) break;
      if (fail(exclusive_scan_u32(g->alloc, keep, cnt + 1, s)) != TC_OK) break;
      int64_t found = 0;
      if (fail(read_back(keep + cnt, pinned, s, &found)) != TC_OK) break;
      if (found > 0) {
        if (fail(h.take(m3, (size_t)found * 12)) != TC_OK) break;
        k_uf_compact2<<<tiles_grid(cnt), kUfThreads, 0, s>>>(o2.as<int64_t>(), P2, m2u.as<int32_t>(),
                                                             m2v.as<int32_t>(), off, col, c0, cnt, keep,
                                                             m3.as<int32_t>());
        note_launch();
        if (fail(cuda_status(cudaGetLastError(), "k_uf_compact2")) != TC_OK) break;
        h.drop(m3);
      }
      total += (uint64_t)found;
    }
  } while (false);
  Buf* all[] = {&sz1, &o1, &cand, &keep1, &m2u, &m2v, &sz2, &o2, &keep2, &m3};
  for (Buf* b : all)
    if (b->p) h.drop(*b);
  st->matches = (int64_t)total;
  st->peak_bytes = h.peak;
  if (rc == TC_OK) rc = cuda_status(cudaStreamSynchronize(s), "tc_count_unfused sync");
  if (rc == TC_OK) *out_total = total;
  return rc;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_count_unfused(tc_graph* g, uint64_t* out_total, int64_t max_chunk_bytes,
                                             tc_unfused_stats* stats, void* stream) {
  if (!g) {
    set_error("tc_count_unfused: graph handle is NULL");
    return TC_ERR_INVALID_ARG;
  }
  if (!g->built) {
    set_error("tc_count_unfused: graph is not built: call tc_build first");
    return TC_ERR_STATE;
  }
  if (!out_total || max_chunk_bytes < 0) {
    set_error("tc_count_unfused: out_total is NULL or max_chunk_bytes is negative");
    return TC_ERR_INVALID_ARG;
  }
  tc_unfused_stats local;
  memset(&local, 0, sizeof(local));
  cudaStream_t s = (cudaStream_t)stream;
  g->last_stream = s;
  const tc_status rc = run_unfused(g, max_chunk_bytes, &local, out_total, s);
  if (stats) *stats = local;
  return rc;
}

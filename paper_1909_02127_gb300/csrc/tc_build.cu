// tc_build.cu — from an edge list to the oriented CSR and the source bins.
//
// Steps (all on the caller's stream):
//   pack      validate ids, drop self-loops, key = (min << B) | max                       (Def. 1: undirected)
//   sort      LSD radix sort on bits [0, 2B)
//   unique    keep the first of each run of equal keys                                     (simple graph)
//   degree    deg(x) = number of distinct edges at x                                       (NE, Sec. III-A)
//   orient    edge {a,b} goes from the lower to the higher (deg, id): key (s << B) | d     (UMO, Sec. III-A/C)
//   sort      stable radix sort on the s bits only; each row is then already ascending in d (see below)
//   csr       int64 offsets by an exclusive scan of d+(s); int32 columns (padded to whole 16-byte quads)
//   bins      w(u) = sum of d+(v) over v in N+(u); sources with d+(u) >= 2 and w(u) > 0 are kept (the
//             2-look-ahead of Sec. III-C: a source needs two out-neighbours to close a triangle) and binned by
//             d+(u) and w(u) into warp-per-source and block-per-source lists.
//
// Why one stable pass on s suffices: the unique keys are sorted by (lo, hi).  Row s receives d < s from edges
// (d, s), which appear in increasing d, all before the block lo = s; and d > s from edges (s, d), which appear
// in increasing d inside that block.  The input order of row s's entries is therefore ascending in d, and a
// stable sort on s keeps it.
#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace {

__global__ void k_pack(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t len, int64_t n,
                       int B, uint64_t* __restrict__ keys, uint32_t* __restrict__ err) {
  const uint64_t sentinel = (2 * B >= 64) ? ~0ull : ((1ull << (2 * B)) - 1ull);
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = src[i], b = dst[i];
    uint64_t key = sentinel;
    if (a < 0 || b < 0 || a >= n || b >= n) {
      bad = true;
    } else if (a != b) {
      const uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
      key = (lo << B) | hi;
    }
    keys[i] = key;
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1u);
}

// ---- unique: count then scatter the first key of each run (sentinel keys dropped) ----------------------------
constexpr int kUThreads = 256;
constexpr int kUItems = 8;
constexpr int kUTile = kUThreads * kUItems;

__device__ __forceinline__ bool is_first(const uint64_t* keys, int64_t i, uint64_t sentinel) {
  const uint64_t k = keys[i];
  return k != sentinel && (i == 0 || keys[i - 1] != k);
}

__global__ void __launch_bounds__(kUThreads) k_unique_count(const uint64_t* __restrict__ keys, int64_t n,
                                                            uint64_t sentinel, uint32_t* __restrict__ part) {
  __shared__ uint32_t ws[kUThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kUTile;
  uint32_t c = 0;
  for (int i = 0; i < kUItems; ++i) {
    const int64_t idx = base + i * kUThreads + threadIdx.x;
    if (idx < n && is_first(keys, idx, sentinel)) ++c;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kUThreads / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kUThreads) k_unique_scatter(const uint64_t* __restrict__ keys, int64_t n,
                                                              uint64_t sentinel, const uint32_t* __restrict__ part,
                                                              uint64_t* __restrict__ out, int64_t* __restrict__ m) {
  __shared__ uint32_t ws[kUThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kUTile + (int64_t)threadIdx.x * kUItems;  // blocked
  uint32_t f = 0;
  for (int i = 0; i < kUItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n && is_first(keys, idx, sentinel)) f |= 1u << i;
  }
  uint32_t tot;
  uint32_t pos = part[blockIdx.x] + block_exclusive_scan((uint32_t)__popc(f), ws, &tot);
  for (int i = 0; i < kUItems; ++i)
    if (f & (1u << i)) out[pos++] = keys[base + i];
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *m = (int64_t)part[blockIdx.x] + tot;
}

// ---- degree / orientation -------------------------------------------------------------------------------------
// Warp-aggregated increment: lanes with the same target add once.
__device__ __forceinline__ void agg_inc(int32_t* cnt, uint32_t idx, bool active) {
  const uint32_t key = active ? idx : 0xffffffffu;
  const unsigned peers = __match_any_sync(kFull, key);
  if (active && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[idx], __popc(peers));
}

__global__ void k_degree(const uint64_t* __restrict__ ukeys, int64_t m, int B, int32_t* __restrict__ deg) {
  const uint64_t mask = (1ull << B) - 1ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < m;
    const uint64_t k = ok ? ukeys[i] : 0;
    agg_inc(deg, (uint32_t)(k >> B), ok);
    agg_inc(deg, (uint32_t)(k & mask), ok);
  }
}

__global__ void k_orient(const uint64_t* __restrict__ ukeys, int64_t m, int B, const int32_t* __restrict__ deg,
                         uint64_t* __restrict__ okeys, int32_t* __restrict__ odeg) {
  const uint64_t mask = (1ull << B) - 1ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < m;
    uint32_t s = 0;
    if (ok) {
      const uint64_t k = ukeys[i];
      const uint32_t lo = (uint32_t)(k >> B), hi = (uint32_t)(k & mask);
      const int32_t dl = deg[lo], dh = deg[hi];
      // (deg, id) order; lo < hi breaks ties
      const bool lo_first = dl < dh || (dl == dh);
      s = lo_first ? lo : hi;
      const uint32_t d = lo_first ? hi : lo;
      okeys[i] = ((uint64_t)s << B) | d;
    }
    agg_inc(odeg, s, ok);
  }
}

__global__ void k_columns(const uint64_t* __restrict__ okeys, int64_t m, int64_t padded, int B,
                          int32_t* __restrict__ col) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < padded; i += (int64_t)gridDim.x * blockDim.x)
    col[i] = i < m ? (int32_t)(okeys[i] & mask) : 0;
}

// ---- work estimate and binning ----------------------------------------------------------------------------------
struct BinCounters {
  unsigned long long wedges;
  unsigned long long active;
  unsigned int nb;
  unsigned int nw;
  unsigned int nwide;
  int max_out;
};

__global__ void k_bins(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                       int32_t* __restrict__ list, BinCounters* __restrict__ bc) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long wsum = 0, act = 0;
  int dmax = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t u = base + threadIdx.x;
    int64_t d = 0, w = 0;
    if (u < n) {
      const int64_t b = off[u], e = off[u + 1];
      d = e - b;
      for (int64_t j = b; j < e; ++j) {
        const int32_t v = col[j];
        w += off[v + 1] - off[v];
      }
    }
    wsum += (unsigned long long)w;
    if (d > dmax) dmax = (int)d;
    const bool keep = d >= 2 && w > 0;
    const bool blk = keep && (d > kWarpMaxDeg || w > kBlockMinWork);
    const bool wrp = keep && !blk;
    act += keep ? 1 : 0;
    const unsigned mb = __ballot_sync(kFull, blk);
    const unsigned mw = __ballot_sync(kFull, wrp);
    const unsigned mx = __ballot_sync(kFull, keep && d > kBlockMaxDeg);
    unsigned pb = 0, pw = 0;
    if (lane == 0) {
      if (mb) pb = atomicAdd(&bc->nb, (unsigned)__popc(mb));
      if (mw) pw = atomicAdd(&bc->nw, (unsigned)__popc(mw));
      if (mx) atomicAdd(&bc->nwide, (unsigned)__popc(mx));
    }
    pb = __shfl_sync(kFull, pb, 0);
    pw = __shfl_sync(kFull, pw, 0);
    // block bin from the front of `list`, warp bin from the back
    if (blk) list[pb + __popc(mb & lt)] = (int32_t)u;
    if (wrp) list[n - 1 - (pw + __popc(mw & lt))] = (int32_t)u;
  }
  wsum = warp_sum(wsum);
  act = warp_sum(act);
  for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(kFull, dmax, o));
  if (lane == 0) {
    atomicAdd(&bc->wedges, wsum);
    atomicAdd(&bc->active, act);
    atomicMax(&bc->max_out, dmax);
  }
}

}  // namespace

tc_status pack_edges(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t len, int64_t offset,
                     uint32_t* d_err, cudaStream_t s) {
  if (len <= 0) return TC_OK;
  k_pack<<<grid_for(len, 256), 256, 0, s>>>(src, dst, len, g->n, g->key_bits, g->keys.as<uint64_t>() + offset,
                                            d_err); note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status build_graph(tc_graph* g, cudaStream_t s) {
  const Allocator& a = g->alloc;
  const int B = g->key_bits;
  const int64_t M = g->num_pairs;
  const int64_t n = g->n;
  const uint64_t sentinel = (2 * B >= 64) ? ~0ull : ((1ull << (2 * B)) - 1ull);
  tc_status st = TC_OK;
  Buf alt, part, counters, deg, odeg, ukeys;
  uint64_t* sorted = nullptr;
  int64_t m = 0;
  BinCounters hb{};

  // The pipeline below frees what it allocated on every path.
  do {
    if (M > 0) {
      if ((st = buf_alloc(a, alt, (size_t)M * 8, s))) break;
      if ((st = radix_sort_u64(a, g->keys.as<uint64_t>(), alt.as<uint64_t>(), M, 0, 2 * B, &sorted, s))) break;
      // unique -> the other buffer
      uint64_t* uout = sorted == g->keys.as<uint64_t>() ? alt.as<uint64_t>() : g->keys.as<uint64_t>();
      const int64_t tiles = (M + kUTile - 1) / kUTile;
      if ((st = buf_alloc(a, part, (size_t)tiles * 4, s))) break;
      if ((st = buf_alloc(a, counters, 64, s))) break;
      k_unique_count<<<(unsigned)tiles, kUThreads, 0, s>>>(sorted, M, sentinel, part.as<uint32_t>()); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_unique_count"))) break;
      if ((st = exclusive_scan_u32(a, part.as<uint32_t>(), tiles, s))) break;
      k_unique_scatter<<<(unsigned)tiles, kUThreads, 0, s>>>(sorted, M, sentinel, part.as<uint32_t>(), uout,
                                                              counters.as<int64_t>()); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_unique_scatter"))) break;
      if ((st = cuda_status(cudaMemcpyAsync(&m, counters.p, 8, cudaMemcpyDeviceToHost, s), "copy m"))) break;
      if ((st = cuda_status(cudaStreamSynchronize(s), "sync m"))) break;
      // keep the unique keys in `ukeys`, drop the other buffer
      if (uout == alt.as<uint64_t>()) {
        ukeys = alt;
        alt = Buf{};
      } else {
        ukeys = g->keys;
        g->keys = Buf{};
      }
      buf_release(a, part, s);
    }
    g->m = m;
    // degrees and orientation
    if ((st = buf_alloc(a, deg, (size_t)(n > 0 ? n : 1) * 4, s))) break;
    if ((st = buf_alloc(a, odeg, (size_t)(n > 0 ? n : 1) * 4, s))) break;
    if (n > 0) {
      if ((st = cuda_status(cudaMemsetAsync(deg.p, 0, (size_t)n * 4, s), "memset deg"))) break;
      if ((st = cuda_status(cudaMemsetAsync(odeg.p, 0, (size_t)n * 4, s), "memset odeg"))) break;
    }
    Buf okeys_buf;
    if (m > 0) {
      k_degree<<<grid_for(m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), m, B, deg.as<int32_t>()); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_degree"))) break;
      // orient into whichever of the two key buffers is free
      Buf& free_buf = g->keys.p ? g->keys : alt;
      okeys_buf = free_buf;
      free_buf = Buf{};
      k_orient<<<grid_for(m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), m, B, deg.as<int32_t>(),
                                                okeys_buf.as<uint64_t>(), odeg.as<int32_t>()); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_orient"))) {
        buf_release(a, okeys_buf, s);
        break;
      }
      uint64_t* osorted = nullptr;
      st = radix_sort_u64(a, okeys_buf.as<uint64_t>(), ukeys.as<uint64_t>(), m, B, 2 * B, &osorted, s);
      if (st) {
        buf_release(a, okeys_buf, s);
        break;
      }
      const int64_t padded = ((m + 3) / 4) * 4 + 4;
      if ((st = buf_alloc(a, g->col, (size_t)padded * 4, s))) {
        buf_release(a, okeys_buf, s);
        break;
      }
      k_columns<<<grid_for(padded, 256), 256, 0, s>>>(osorted, m, padded, B, g->col.as<int32_t>()); note_launch();
      st = cuda_status(cudaGetLastError(), "k_columns");
      buf_release(a, okeys_buf, s);
      if (st) break;
    } else {
      if ((st = buf_alloc(a, g->col, 16, s))) break;
      if ((st = cuda_status(cudaMemsetAsync(g->col.p, 0, 16, s), "memset col"))) break;
    }
    buf_release(a, ukeys, s);
    buf_release(a, alt, s);
    buf_release(a, g->keys, s);
    buf_release(a, deg, s);
    // offsets
    if ((st = buf_alloc(a, g->off, (size_t)(n + 1) * 8, s))) break;
    if (n > 0) {
      if ((st = exclusive_scan_i32_to_i64(a, odeg.as<int32_t>(), g->off.as<int64_t>(), n, s))) break;
    } else if ((st = cuda_status(cudaMemsetAsync(g->off.p, 0, 8, s), "memset off"))) {
      break;
    }
    buf_release(a, odeg, s);
    // bins
    if ((st = buf_alloc(a, g->list, (size_t)(n > 0 ? n : 1) * 4, s))) break;
    if (!counters.p && (st = buf_alloc(a, counters, 64, s))) break;
    if ((st = cuda_status(cudaMemsetAsync(counters.p, 0, sizeof(BinCounters), s), "memset bins"))) break;
    if (n > 0) {
      k_bins<<<grid_for(n, 256), 256, 0, s>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), n,
                                              g->list.as<int32_t>(), counters.as<BinCounters>()); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_bins"))) break;
    }
    if ((st = cuda_status(cudaMemcpyAsync(&hb, counters.p, sizeof(BinCounters), cudaMemcpyDeviceToHost, s),
                          "copy bins")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "sync bins"))) break;
  } while (0);

  buf_release(a, alt, s);
  buf_release(a, part, s);
  buf_release(a, counters, s);
  buf_release(a, deg, s);
  buf_release(a, odeg, s);
  buf_release(a, ukeys, s);
  buf_release(a, g->keys, s);
  if (st != TC_OK) return st;
  g->wedges = (int64_t)hb.wedges;
  g->active = (int64_t)hb.active;
  g->nb = hb.nb;
  g->nw = hb.nw;
  g->nwide = hb.nwide;
  g->max_out_degree = hb.max_out;
  return TC_OK;
}

}  // namespace tc

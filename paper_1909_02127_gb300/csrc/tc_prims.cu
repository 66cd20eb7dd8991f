// tc_prims.cu — device exclusive scans and a stable LSD radix sort for uint64 keys.
//
// Radix sort: one pass per 8-bit digit over only the requested bit range.  Each pass is reduce-then-scan:
//   k_rs_hist     per-tile digit histogram (4096 keys per tile), stored digit-major: hist[d * ntiles + tile]
//   scan          one flat exclusive scan of that array gives, for every (digit, tile), the global output offset
//   k_rs_scatter  the tile ranks its keys stably (warp match on the digit, per-warp running counts), sorts them
//                 in shared memory, and writes each digit's run to its global offset with coalesced stores.
#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {

int grid_for(int64_t items, int threads, int max_blocks) {
  if (max_blocks < 0) max_blocks = num_sms() * 16;
  int64_t b = (items + threads - 1) / threads;
  if (b > max_blocks) b = max_blocks;
  return b < 1 ? 1 : (int)b;
}

namespace {

// ------------------------------------------------------------------------------------------------------------
// Exclusive scan (three phases; tiles of 2048 elements)
// ------------------------------------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Tin* __restrict__ in, int64_t n,
                                                              Tout* __restrict__ partial) {
  __shared__ Tout ws[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i * kScanThreads + threadIdx.x;
    if (idx < n) s += (Tout)in[idx];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    Tout t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// out may alias in.  partial: exclusive prefix per tile (null for a single tile).  total: out[n] if non-null.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin* in, Tout* out, int64_t n,
                                                            const Tout* __restrict__ partial, Tout* total) {
  __shared__ Tout tile[kScanTile];
  __shared__ Tout ws[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i * kScanThreads + threadIdx.x;
    tile[i * kScanThreads + threadIdx.x] = idx < n ? (Tout)in[idx] : Tout(0);
  }
  __syncthreads();
  Tout v[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = tile[threadIdx.x * kScanItems + i];
    s += v[i];
  }
  Tout tot;
  Tout run = block_exclusive_scan(s, ws, &tot);
  if (partial) run += partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    tile[threadIdx.x * kScanItems + i] = run;
    run += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i * kScanThreads + threadIdx.x;
    if (idx < n) out[idx] = tile[i * kScanThreads + threadIdx.x];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) *total = run;
}

// tmp: scratch for the partial sums of this level and the levels below (scan_temp_bytes), or null to allocate it.
template <class Tin, class Tout>
tc_status scan_rec(const Allocator& a, const Tin* in, Tout* out, int64_t n, Tout* total, cudaStream_t s,
                   void* tmp) {
  if (n <= 0) {
    if (total) TC_CUDA(cudaMemsetAsync(total, 0, sizeof(Tout), s));
    return TC_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_scan_down<Tin, Tout><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total); note_launch();
    TC_CUDA(cudaGetLastError());
    return TC_OK;
  }
  Buf part;
  if (tmp) {
    part.p = tmp;
    part.owned = false;
  } else {
    TC_TRY(buf_alloc(a, part, (size_t)tiles * sizeof(Tout), s));
  }
  void* below = tmp ? static_cast<char*>(tmp) + (((size_t)tiles * 8 + 255) & ~size_t(255)) : nullptr;
  k_scan_reduce<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, part.as<Tout>()); note_launch();
  tc_status st = cuda_status(cudaGetLastError(), "k_scan_reduce");
  if (st == TC_OK) st = scan_rec<Tout, Tout>(a, part.as<Tout>(), part.as<Tout>(), tiles, nullptr, s, below);
  if (st == TC_OK) {
    k_scan_down<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, part.as<Tout>(), total); note_launch();
    st = cuda_status(cudaGetLastError(), "k_scan_down");
  }
  buf_release(a, part, s);
  return st;
}

// ------------------------------------------------------------------------------------------------------------
// Radix sort
// ------------------------------------------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096 keys
constexpr int kRsBins = 256;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                        uint32_t mask, uint32_t* __restrict__ hist,
                                                        int64_t ntiles) {
  __shared__ uint32_t h[kRsBins];
  for (int i = threadIdx.x; i < kRsBins; i += kRsThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  const int lane = threadIdx.x & 31;
#pragma unroll 4
  for (int i = 0; i < kRsItems; ++i) {
    const int64_t idx = base + i * kRsThreads + threadIdx.x;
    const uint32_t d = idx < n ? (uint32_t)((keys[idx] >> shift) & mask) : kRsBins;
    const unsigned peers = __match_any_sync(kFull, d);
    if (d < kRsBins && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRsBins; d += kRsThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ in,
                                                           uint64_t* __restrict__ out, int64_t n, int shift,
                                                           uint32_t mask, const uint32_t* __restrict__ offs,
                                                           int64_t ntiles) {
  __shared__ uint64_t sk[kRsTile];
  __shared__ uint32_t wc[kRsWarps][kRsBins + 1];
  __shared__ uint32_t tbase[kRsBins];
  __shared__ uint32_t gbase[kRsBins];
  __shared__ uint32_t ws[kRsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * (kRsBins + 1); i += kRsThreads) (&wc[0][0])[i] = 0;
  for (int d = threadIdx.x; d < kRsBins; d += kRsThreads) gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  __syncthreads();

  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  const int64_t base = tile0 + warp * (kRsItems * 32);
  uint64_t k[kRsItems];
  uint32_t dg[kRsItems];
  uint32_t r[kRsItems];
#pragma unroll
  for (int i = 0; i < kRsItems; ++i) {
    const int64_t idx = base + i * 32 + lane;
    const bool valid = idx < n;
    k[i] = valid ? in[idx] : 0ull;
    dg[i] = valid ? (uint32_t)((k[i] >> shift) & mask) : (uint32_t)kRsBins;
  }
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kRsItems; ++i) {
    const unsigned peers = __match_any_sync(kFull, dg[i]);
    const uint32_t before = wc[warp][dg[i]];
    r[i] = before + (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (lane == __ffs(peers) - 1) wc[warp][dg[i]] = before + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: prefix over warps, then over digits (tile-local start of each digit's run)
  {
    const int d = threadIdx.x;  // kRsThreads == kRsBins
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t t = wc[w][d];
      wc[w][d] = run;
      run += t;
    }
    uint32_t tot;
    tbase[d] = block_exclusive_scan(run, ws, &tot);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRsItems; ++i)
    if (dg[i] < kRsBins) sk[tbase[dg[i]] + wc[warp][dg[i]] + r[i]] = k[i];
  __syncthreads();
  const int64_t rem = n - tile0;
  const int tile_n = rem < kRsTile ? (int)rem : kRsTile;
  for (int j = threadIdx.x; j < tile_n; j += kRsThreads) {
    const uint64_t key = sk[j];
    const uint32_t d = (uint32_t)((key >> shift) & mask);
    out[(int64_t)gbase[d] + (j - (int64_t)tbase[d])] = key;
  }
}

}  // namespace

tc_status exclusive_scan_i32_to_i64(const Allocator& a, const int32_t* in, int64_t* out, int64_t n,
                                    cudaStream_t s, void* tmp) {
  return scan_rec<int32_t, int64_t>(a, in, out, n, out + n, s, tmp);
}

tc_status exclusive_scan_u64(const Allocator& a, const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                             void* tmp) {
  return scan_rec<uint64_t, uint64_t>(a, in, out, n, out + n, s, tmp);
}

tc_status exclusive_scan_u32(const Allocator& a, uint32_t* data, int64_t n, cudaStream_t s, void* tmp) {
  return scan_rec<uint32_t, uint32_t>(a, data, data, n, nullptr, s, tmp);
}

size_t scan_temp_bytes(int64_t n) {
  size_t bytes = 0;
  for (int64_t tiles = (n + kScanTile - 1) / kScanTile; tiles > 1; tiles = (tiles + kScanTile - 1) / kScanTile)
    bytes += ((size_t)tiles * 8 + 255) & ~size_t(255);
  return bytes;
}

size_t radix_temp_bytes(int64_t n) {
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  return (((size_t)ntiles * kRsBins * sizeof(uint32_t) + 255) & ~size_t(255)) + scan_temp_bytes(ntiles * kRsBins);
}

tc_status radix_sort_u64(const Allocator& a, uint64_t* keys, uint64_t* alt, int64_t n, int bit_lo, int bit_hi,
                         uint64_t** result, cudaStream_t s, void* tmp) {
  *result = keys;
  if (n <= 1 || bit_hi <= bit_lo) return TC_OK;
  if (n >= (int64_t)0xffffffffLL) {
    set_error("radix sort: more than 2^32-2 keys");
    return TC_ERR_INVALID_ARG;
  }
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  Buf hist;
  void* scan_tmp = nullptr;
  if (tmp) {
    hist.p = tmp;
    hist.owned = false;
    scan_tmp = static_cast<char*>(tmp) + (((size_t)ntiles * kRsBins * sizeof(uint32_t) + 255) & ~size_t(255));
  } else {
    TC_TRY(buf_alloc(a, hist, (size_t)ntiles * kRsBins * sizeof(uint32_t), s));
  }
  uint64_t* src = keys;
  uint64_t* dst = alt;
  tc_status st = TC_OK;
  for (int shift = bit_lo; shift < bit_hi && st == TC_OK; shift += 8) {
    const int nbits = bit_hi - shift < 8 ? bit_hi - shift : 8;
    const uint32_t mask = (1u << nbits) - 1u;
    k_rs_hist<<<(unsigned)ntiles, kRsThreads, 0, s>>>(src, n, shift, mask, hist.as<uint32_t>(), ntiles); note_launch();
    st = cuda_status(cudaGetLastError(), "k_rs_hist");
    if (st != TC_OK) break;
    st = exclusive_scan_u32(a, hist.as<uint32_t>(), ntiles * kRsBins, s, scan_tmp);
    if (st != TC_OK) break;
    k_rs_scatter<<<(unsigned)ntiles, kRsThreads, 0, s>>>(src, dst, n, shift, mask, hist.as<uint32_t>(), ntiles); note_launch();
    st = cuda_status(cudaGetLastError(), "k_rs_scatter");
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  buf_release(a, hist, s);
  *result = src;
  return st;
}

}  // namespace tc

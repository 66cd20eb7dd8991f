// tc_count.cu — the single-graph counting launch.
//
// One persistent kernel, 2 CTAs of 512 threads per SM.  CTAs first take block-bin sources one at a time from an
// atomic cursor (heavy sources: many candidate 2-paths), then every warp takes warp-bin sources in chunks of
// four.  Each thread accumulates its closed 2-paths in a register; at the end the block reduces them (warp
// shuffles, then shared memory) and adds its total with one 64-bit atomic.
#include "tc_count.cuh"

namespace tc {
namespace {

template <int MODE>
__global__ void __launch_bounds__(kCountThreads, 2)
    k_count(CsrView g, unsigned long long* __restrict__ total, dev::Sink sk, uint32_t* __restrict__ cursors) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t ws[32];
  __shared__ unsigned long long red[kWarpsPerCTA];
  __shared__ int s_idx;
  int nhub = 0;
  if (MODE == dev::kModeVertex) {  // zeroed hub counters after the counting layout
    sk.hub = smem + dev::kCountSmem / 4;
    sk.hub0 = g.n > dev::kHubRanks ? (int32_t)(g.n - dev::kHubRanks) : 0;
    nhub = (int)(g.n - sk.hub0);
    for (int i = threadIdx.x; i < nhub; i += kCountThreads) sk.hub[i] = 0u;
    __syncthreads();
  }
  unsigned long long acc = dev::count_graph<MODE>(g, sk, cursors, smem, ws, &s_idx);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kWarpsPerCTA; ++w) s += red[w];
    if (s) atomicAdd(total, s);
  }
  if (MODE == dev::kModeVertex) {  // every add of this CTA is in (the barrier above)
    for (int i = threadIdx.x; i < nhub; i += kCountThreads) {
      const uint32_t c = sk.hub[i];
      if (c) atomicAdd(&sk.pv[sk.hub0 + i], (unsigned long long)c);
    }
  }
}

}  // namespace

int count_grid(const tc_graph* g) {
  const int64_t want = g->nb + (g->nw + kWarpsPerCTA - 1) / kWarpsPerCTA + (g->nt + kCountThreads - 1) / kCountThreads;
  return (int)(want < 2 * kNumSMs ? (want < 1 ? 1 : want) : 2 * kNumSMs);
}

tc_status launch_count(const tc_graph* g, uint64_t* d_total, uint64_t* d_per_vertex, uint32_t* d_cursors,
                       cudaStream_t s) {
  TC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s));
  if (d_per_vertex && g->n > 0) TC_CUDA(cudaMemsetAsync(d_per_vertex, 0, (size_t)g->n * sizeof(uint64_t), s));
  if (g->nb + g->nw + g->nt == 0) return TC_OK;
  TC_CUDA(cudaMemsetAsync(d_cursors, 0, 3 * sizeof(uint32_t), s));
  const int grid = count_grid(g);
  dev::Sink sk;
  if (d_per_vertex) {
    sk.pv = (unsigned long long*)d_per_vertex;
    TC_CUDA(cudaFuncSetAttribute(k_count<dev::kModeVertex>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dev::kVertexSmem));
    k_count<dev::kModeVertex><<<grid, kCountThreads, dev::kVertexSmem, s>>>(g->view(), (unsigned long long*)d_total,
                                                                            sk, d_cursors);
  } else {
    TC_CUDA(cudaFuncSetAttribute(k_count<dev::kModeCount>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dev::kCountSmem));
    k_count<dev::kModeCount><<<grid, kCountThreads, dev::kCountSmem, s>>>(g->view(), (unsigned long long*)d_total,
                                                                          sk, d_cursors);
  }
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

// ---- listing -------------------------------------------------------------------------------------------------------
namespace tc {
namespace {

// Triangles whose first vertex in the visiting order lies in ranks [first, first + count), one source per warp,
// four at a time from a cursor.  MODE kModeCount writes each source's number of triangles to cnt[k]; kModeList
// writes them as triples starting at offs[k] (the exclusive scan of those counts), so each source fills its own
// range of the output and no global cursor is contended.  A source with fewer than two out-neighbours closes no
// 2-path.
template <int MODE>
__global__ void __launch_bounds__(kCountThreads, 2)
    k_list(CsrView g, int64_t first, int64_t count, dev::Sink sk, unsigned long long* __restrict__ cursor,
           uint32_t* __restrict__ cnt, const int64_t* __restrict__ offs) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long wpos[kWarpsPerCTA];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* region = smem + warp * dev::kWarpRegionWords;
  const dev::Rows r = dev::warp_rows(region);
  int32_t* ltab = dev::warp_low(region);
  dev::zero_words(region, dev::kWarpBitmapWords, lane, 32);
  for (int i = lane; i < kWarpLowSlots; i += 32) ltab[i] = -1;
  sk.slot = &wpos[warp];
  __syncwarp();
  constexpr int kChunk = 4;
  while (true) {
    long long idx = 0;
    if (lane == 0) idx = (long long)atomicAdd(cursor, (unsigned long long)kChunk);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= count) break;
    const int64_t e = idx + kChunk < count ? idx + kChunk : count;
    for (int64_t k = idx; k < e; ++k) {
      const int32_t u = (int32_t)(first + k);
      const int64_t beg = __ldg(&g.off[u]);
      if (__ldg(&g.off[u + 1]) - beg < 4 || __ldg(&g.col[beg + 1]) >= g.n) {  // d+(u) < 2
        if (MODE == dev::kModeCount && lane == 0) cnt[k] = 0u;
        continue;
      }
      if (MODE == dev::kModeList) {
        if (lane == 0) wpos[warp] = (unsigned long long)offs[k];
        __syncwarp();
      }
      const uint32_t h = dev::warp_source<MODE>(u, g, region, ltab, r, sk);
      if (MODE == dev::kModeCount) {
        const uint32_t t = warp_sum(h);
        if (lane == 0) cnt[k] = t;
      }
    }
  }
}

}  // namespace

tc_status launch_list(const tc_graph* g, int64_t first, int64_t count, int32_t* d_triples, int64_t capacity,
                      uint64_t* d_found, uint64_t* d_cursor, cudaStream_t s) {
  TC_CUDA(cudaMemsetAsync(d_found, 0, sizeof(uint64_t), s));
  if (count <= 0) return TC_OK;
  const int64_t want = (count + kWarpsPerCTA - 1) / kWarpsPerCTA;
  const int grid = (int)(want < 2 * kNumSMs ? want : 2 * kNumSMs);
  Buf cnt, offs;
  tc_status st = TC_OK;
  do {
    // pass 1: triangles per source (the counting kernel's tests, dense rows included)
    if ((st = buf_alloc(g->alloc, cnt, (size_t)count * 4, s))) break;
    if ((st = buf_alloc(g->alloc, offs, (size_t)(count + 1) * 8, s))) break;
    if ((st = cuda_status(cudaMemsetAsync(d_cursor, 0, sizeof(uint64_t), s), "memset cursor"))) break;
    dev::Sink none;
    if ((st = cuda_status(cudaFuncSetAttribute(k_list<dev::kModeCount>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kWarpSmem),
                          "k_list attribute")))
      break;
    k_list<dev::kModeCount><<<grid, kCountThreads, dev::kWarpSmem, s>>>(
        g->view(), first, count, none, (unsigned long long*)d_cursor, cnt.as<uint32_t>(), nullptr);
    note_launch();
    if ((st = cuda_status(cudaGetLastError(), "k_list count"))) break;
    // per-source output offsets; their total is the number found (per-source counts are below 2^31: C(d+, 2)
    // with d+(u) at most sqrt(2m))
    if ((st = exclusive_scan_i32_to_i64(g->alloc, cnt.as<int32_t>(), offs.as<int64_t>(), count, s))) break;
    if ((st = cuda_status(cudaMemcpyAsync(d_found, offs.as<int64_t>() + count, 8, cudaMemcpyDeviceToDevice, s),
                          "copy found")))
      break;
    // pass 2: the triples, each source into its own range
    dev::Sink sk;
    sk.tri = d_triples;
    sk.capacity = (unsigned long long)(capacity > 0 ? capacity : 0);
    sk.perm = g->perm.as<int32_t>();
    if ((st = cuda_status(cudaMemsetAsync(d_cursor, 0, sizeof(uint64_t), s), "memset cursor"))) break;
    if ((st = cuda_status(cudaFuncSetAttribute(k_list<dev::kModeList>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kWarpSmem),
                          "k_list attribute")))
      break;
    k_list<dev::kModeList><<<grid, kCountThreads, dev::kWarpSmem, s>>>(
        g->view(), first, count, sk, (unsigned long long*)d_cursor, nullptr, offs.as<int64_t>());
    note_launch();
    st = cuda_status(cudaGetLastError(), "k_list");
  } while (0);
  buf_release(g->alloc, cnt, s);
  buf_release(g->alloc, offs, s);
  return st;
}

}  // namespace tc

// tc_count.cu — the single-graph counting launch.
//
// One persistent kernel, 2 CTAs of 512 threads per SM.  CTAs first take block-bin sources one at a time from an
// atomic cursor (heavy sources: many candidate 2-paths), then every warp takes warp-bin sources in chunks of
// four.  Each thread accumulates its closed 2-paths in a register; at the end the block reduces them (warp
// shuffles, then shared memory) and adds its total with one 64-bit atomic.
#include "tc_count.cuh"

namespace tc {
namespace {

template <int MODE, bool STAGED>
__global__ void __launch_bounds__(kCountThreads, 2)
    k_count(CsrView g, unsigned long long* __restrict__ total, dev::Sink sk, uint32_t* __restrict__ cursors) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t ws[32];
  __shared__ unsigned long long red[kWarpsPerCTA];
  __shared__ int s_idx;
  int nhub = 0;
  if (dev::is_vertex(MODE)) {  // zeroed hub counters after the counting layout
    sk.hub = smem + dev::kCountSmem / 4;
    sk.hub0 = g.n > dev::kHubRanks ? (int32_t)(g.n - dev::kHubRanks) : 0;
    nhub = (int)(g.n - sk.hub0);
    for (int i = threadIdx.x; i < nhub; i += kCountThreads) sk.hub[i] = 0u;
    __syncthreads();
  }
  unsigned long long acc = dev::count_graph<MODE, STAGED>(g, sk, cursors, smem, ws, &s_idx);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kWarpsPerCTA; ++w) s += red[w];
    if (s) atomicAdd(total, s);
  }
  if (dev::is_vertex(MODE)) {  // every add of this CTA is in (the barrier above)
    for (int i = threadIdx.x; i < nhub; i += kCountThreads) {
      const uint32_t c = sk.hub[i];
      if (c) atomicAdd(&sk.pv[sk.hub0 + i], (unsigned long long)c);
    }
  }
}

}  // namespace

bool use_staged_rows(const tc_graph* g) {
  const int64_t t = stage_min_csr_bytes();
  return t > 0 && 8 * (g->n + 1) + 4 * g->csr_entries >= t;
}

int count_grid(const tc_graph* g) {
  const int64_t want = g->nb + (g->nw + kWarpsPerCTA - 1) / kWarpsPerCTA + (g->nt + kCountThreads - 1) / kCountThreads;
  return (int)(want < 2 * num_sms() ? (want < 1 ? 1 : want) : 2 * num_sms());
}

tc_status launch_count(const tc_graph* g, uint64_t* d_total, uint64_t* d_per_vertex, uint32_t* d_cursors,
                       cudaStream_t s) {
  const bool adjacent = reinterpret_cast<uint64_t*>(d_cursors) == d_total + 1;  // the graph's own count words
  TC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t) + (adjacent ? 3 * sizeof(uint32_t) : 0), s));
  if (d_per_vertex && g->n > 0) TC_CUDA(cudaMemsetAsync(d_per_vertex, 0, (size_t)g->n * sizeof(uint64_t), s));
  if (g->nb + g->nw + g->nt == 0) return TC_OK;
  if (!adjacent) TC_CUDA(cudaMemsetAsync(d_cursors, 0, 3 * sizeof(uint32_t), s));
  const int grid = count_grid(g);
  dev::Sink sk;
  if (d_per_vertex && g->m <= vertex_plain_max_edges()) {  // no counter can reach 2^32: plain adds
    sk.pv = (unsigned long long*)d_per_vertex;
    TC_TRY((smem_attribute_once<k_count<dev::kModeVertex, false>>(dev::kVertexSmem)));
    k_count<dev::kModeVertex, false><<<grid, kCountThreads, dev::kVertexSmem, s>>>(
        g->view(), (unsigned long long*)d_total, sk, d_cursors);
  } else if (d_per_vertex) {
    sk.pv = (unsigned long long*)d_per_vertex;
    TC_TRY((smem_attribute_once<k_count<dev::kModeVertexChecked, false>>(dev::kVertexSmem)));
    k_count<dev::kModeVertexChecked, false><<<grid, kCountThreads, dev::kVertexSmem, s>>>(
        g->view(), (unsigned long long*)d_total, sk, d_cursors);
  } else if (use_staged_rows(g)) {  // CSR beyond L2: long hop-2 rows staged through shared memory
    TC_TRY((smem_attribute_once<k_count<dev::kModeCount, true>>(dev::kCountStagedSmem)));
    k_count<dev::kModeCount, true><<<grid, kCountThreads, dev::kCountStagedSmem, s>>>(
        g->view(), (unsigned long long*)d_total, sk, d_cursors);
  } else {
    TC_TRY((smem_attribute_once<k_count<dev::kModeCount, false>>(dev::kCountSmem)));
    k_count<dev::kModeCount, false><<<grid, kCountThreads, dev::kCountSmem, s>>>(
        g->view(), (unsigned long long*)d_total, sk, d_cursors);
  }
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

// ---- listing -------------------------------------------------------------------------------------------------------
namespace tc {
namespace {

// A warp-bin source closing many triangles is listed by a whole CTA: listing costs per triangle, and the bins were
// cut by 2-paths, which dense rows make cheap to test but not to write out.  "Many" is 1/kListShare of a CTA's
// average share of the range's triangles, within [kListBlockMinLo, kListBlockMinHi]: a warp-bin source at the end of
// the queue then finishes in a small fraction of the pass, while the CTAs' per-chunk barriers are paid only where a
// source has that much to write (measured on R-MAT 16, 18 and 20: the best fixed thresholds were 1024, 4096 and
// 16384).
constexpr uint32_t kListBlockMinLo = 1024;
constexpr uint32_t kListBlockMinHi = 16384;
constexpr uint64_t kListShare = 64;

// Triangles whose first vertex in the visiting order lies in ranks [first, first + count), taken by the counting
// kernel's bins: CTAs take the sources of blist one at a time, then warps take warp-bin sources four at a time,
// then lanes take thread-bin sources; a source outside the range is skipped.  MODE kModeCount (blist: the block
// bin) writes each source's number of triangles to cnt[u - first] (zeroed beforehand: a source in no bin closes no
// 2-path).  kModeList (blist: k_list_heavy's list) writes them as triples from offs[u - first] on (the exclusive
// scan of those counts), so each source fills its own range of the output and no global cursor is contended; it
// skips sources with no triangle and leaves warp-bin sources with *list_min or more to the CTAs.  The output
// position of a source lives in shared memory (one per warp; one per CTA for a source of blist, whose warps
// reserve runs of it with shared atomics).
template <int MODE>
__global__ void __launch_bounds__(kCountThreads, 2)
    k_list(CsrView g, int64_t first, int64_t count, dev::Sink sk, uint32_t* __restrict__ cursors,
           uint32_t* __restrict__ cnt, const int64_t* __restrict__ offs, const int32_t* __restrict__ blist,
           const uint32_t* __restrict__ nblist, const uint32_t* __restrict__ list_min) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t ws[32];
  __shared__ unsigned long long pos[kWarpsPerCTA + 1];  // [warp]: warp-bin sources; [kWarpsPerCTA]: block bin
  __shared__ int s_idx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t last = first + count;
  const uint32_t block_min = list_min ? *list_min : kListBlockMinHi;
  const int nb = nblist ? (int)*nblist : g.nb;
  if (nb > 0) {
    const dev::BlockRows br = dev::block_rows(smem);
    dev::zero_words(smem, dev::kBlockBitmapWords, tid, kCountThreads);
    for (int i = tid; i < kBlockLowSlots; i += kCountThreads) br.ltab[i] = -1;
    __syncthreads();
    dev::Sink bsk = sk;
    bsk.slot = &pos[kWarpsPerCTA];
    while (true) {
      if (tid == 0) s_idx = (int)atomicAdd(&cursors[0], 1u);
      __syncthreads();
      const int idx = s_idx;
      __syncthreads();
      if (idx >= nb) break;
      const int32_t u = __ldg(&blist[idx]);
      if (u < first || u >= last) continue;  // uniform over the CTA
      if (MODE == dev::kModeList) {
        if (tid == 0) pos[kWarpsPerCTA] = (unsigned long long)offs[u - first];
        __syncthreads();
      }
      const uint32_t h = dev::block_source<MODE>(u, g, smem, br, ws, bsk);
      if (MODE == dev::kModeCount) {
        uint32_t total;
        block_exclusive_scan<uint32_t>(h, ws, &total);
        if (tid == 0) cnt[u - first] = total;
      }
    }
  }
  if (g.nw > 0) {
    uint32_t* region = smem + warp * dev::kWarpRegionWords;
    const dev::Rows r = dev::warp_rows(region);
    int32_t* ltab = dev::warp_low(region);
    dev::zero_words(region, dev::kWarpBitmapWords, lane, 32);
    for (int i = lane; i < kWarpLowSlots; i += 32) ltab[i] = -1;
    __syncwarp();
    dev::Sink wsk = sk;
    wsk.slot = &pos[warp];
    const int32_t* wlist = g.list + (g.n - g.nw);
    constexpr int kChunk = 4;
    while (true) {
      int idx = 0;
      if (lane == 0) idx = (int)atomicAdd(&cursors[1], (unsigned)kChunk);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= g.nw) break;
      const int e = min(idx + kChunk, g.nw);
      for (int k = idx; k < e; ++k) {
        const int32_t u = __ldg(&wlist[k]);
        if (u < first || u >= last) continue;
        if (MODE == dev::kModeList) {
          const uint32_t c = __ldg(&cnt[u - first]);
          if (c == 0 || c >= block_min) continue;
          if (lane == 0) pos[warp] = (unsigned long long)offs[u - first];
          __syncwarp();
        }
        const uint32_t h = dev::warp_source<MODE>(u, g, region, ltab, r, wsk);
        if (MODE == dev::kModeCount) {
          const uint32_t t = warp_sum(h);
          if (lane == 0) cnt[u - first] = t;
        }
      }
    }
  }
  if (g.nt > 0) {  // thread bin: one source per lane, its triangles written in order from its own offset
    while (true) {
      int idx = 0;
      if (lane == 0) idx = (int)atomicAdd(&cursors[2], 32u);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= g.nt) break;
      if (idx + lane < g.nt) {
        const int32_t u = __ldg(&g.tlist[idx + lane]);
        if (u >= first && u < last) {
          if (MODE == dev::kModeCount)
            cnt[u - first] = dev::tiny_source<MODE>(u, g, sk);
          else if (__ldg(&cnt[u - first]) > 0)
            dev::tiny_source<MODE>(u, g, sk, (unsigned long long)offs[u - first]);
        }
      }
    }
  }
}

// The CTA work of the listing pass: the block-bin sources of the range that close a triangle and the warp-bin
// sources that close at least the threshold, appended to heavy in no particular order (*nheavy: zeroed count).  The
// threshold follows the range's triangles (*found) over the listing kernel's CTAs (grid); *list_min receives it.
__global__ void k_list_heavy(CsrView g, int64_t first, int64_t count, const uint32_t* __restrict__ cnt,
                             const unsigned long long* __restrict__ found, int grid, int32_t* __restrict__ heavy,
                             uint32_t* __restrict__ nheavy, uint32_t* __restrict__ list_min) {
  const unsigned long long share = *found / ((unsigned long long)(grid > 0 ? grid : 1) * kListShare);
  const uint32_t thr = share < kListBlockMinLo ? kListBlockMinLo
                                               : (share > kListBlockMinHi ? kListBlockMinHi : (uint32_t)share);
  if (blockIdx.x == 0 && threadIdx.x == 0) *list_min = thr;
  const int64_t total = (int64_t)g.nb + g.nw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const bool blk = i < g.nb;
    const int32_t u = __ldg(&g.list[blk ? i : g.n - g.nw + (i - g.nb)]);
    if (u < first || u >= first + count) continue;
    const uint32_t c = __ldg(&cnt[u - first]);
    if (blk ? c > 0 : c >= thr) heavy[atomicAdd(nheavy, 1u)] = u;
  }
}

// Per-graph sums of per-source triangle counts: the source of rank r is the original (union) vertex perm[r], which
// belongs to the graph j with voff[j] <= perm[r] < voff[j + 1].  Lanes of a warp that land on the same graph add
// once.
__global__ void k_graph_sums(const uint32_t* __restrict__ cnt, const int32_t* __restrict__ perm, int64_t n,
                             const int64_t* __restrict__ voff, int32_t k, unsigned long long* __restrict__ counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {  // warp-uniform trip count
    const int64_t r = base + threadIdx.x;
    const uint32_t c = r < n ? __ldg(&cnt[r]) : 0u;
    int j = -1;
    if (c) {
      const int64_t x = __ldg(&perm[r]);
      int a = 0, b = k;  // the last j with voff[j] <= x
      while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (__ldg(&voff[mid]) <= x)
          a = mid;
        else
          b = mid;
      }
      j = a;
    }
    // the lanes of one graph sum their counts (each below 2^31) in 16-bit halves, so no 32-bit sum can wrap;
    // lanes without a count form the group j = -1 and add nothing
    const unsigned peers = __match_any_sync(kFull, j);
    const unsigned lo = __reduce_add_sync(peers, c & 0xffffu);
    const unsigned hi = __reduce_add_sync(peers, c >> 16);
    const unsigned long long sum = ((unsigned long long)hi << 16) + lo;
    if (j >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1 && sum) atomicAdd(&counts[j], sum);
  }
}

}  // namespace

tc_status launch_graph_counts(const tc_graph* g, const int64_t* d_voff, int32_t k, uint64_t* d_counts,
                              uint32_t* d_cnt, uint32_t* d_cursors, cudaStream_t s) {
  if (g->n == 0 || g->nb + g->nw + g->nt == 0) return TC_OK;
  TC_CUDA(cudaMemsetAsync(d_cnt, 0, (size_t)g->n * 4, s));
  TC_CUDA(cudaMemsetAsync(d_cursors, 0, 3 * sizeof(uint32_t), s));
  TC_TRY((smem_attribute_once<k_list<dev::kModeCount>>(dev::kCountSmem)));
  dev::Sink none;
  k_list<dev::kModeCount><<<count_grid(g), kCountThreads, dev::kCountSmem, s>>>(
      g->view(), 0, g->n, none, d_cursors, d_cnt, nullptr, g->list.as<int32_t>(), nullptr, nullptr);
  note_launch();
  TC_CUDA(cudaGetLastError());
  k_graph_sums<<<grid_for(g->n, 256), 256, 0, s>>>(d_cnt, g->perm.as<int32_t>(), g->n, d_voff, k,
                                                   (unsigned long long*)d_counts);
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status launch_list(const tc_graph* g, int64_t first, int64_t count, int32_t* d_triples, int64_t capacity,
                      uint64_t* d_found, uint32_t* d_cursors, cudaStream_t s) {
  TC_CUDA(cudaMemsetAsync(d_found, 0, sizeof(uint64_t), s));
  if (count <= 0 || g->nb + g->nw + g->nt == 0) return TC_OK;
  const int grid = count_grid(g);
  Buf cnt, offs, heavy;
  tc_status st = TC_OK;
  do {
    // pass 1: triangles per source (the counting kernel's tests, dense rows included)
    if ((st = buf_alloc(g->alloc, cnt, (size_t)count * 4, s))) break;
    if ((st = buf_alloc(g->alloc, offs, (size_t)(count + 1) * 8, s))) break;
    if ((st = buf_alloc(g->alloc, heavy, (size_t)(g->nb + g->nw + 1) * 4, s))) break;
    if ((st = cuda_status(cudaMemsetAsync(cnt.p, 0, (size_t)count * 4, s), "memset counts"))) break;
    if ((st = cuda_status(cudaMemsetAsync(d_cursors, 0, 3 * sizeof(uint32_t), s), "memset cursors"))) break;
    dev::Sink none;
    if ((st = cuda_status(cudaFuncSetAttribute(k_list<dev::kModeCount>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kCountSmem),
                          "k_list attribute")))
      break;
    k_list<dev::kModeCount><<<grid, kCountThreads, dev::kCountSmem, s>>>(
        g->view(), first, count, none, d_cursors, cnt.as<uint32_t>(), nullptr, g->list.as<int32_t>(), nullptr,
        nullptr);
    note_launch();
    if ((st = cuda_status(cudaGetLastError(), "k_list count"))) break;
    // per-source output offsets; their total is the number found (per-source counts are below 2^31: C(d+, 2)
    // with d+(u) at most sqrt(2m))
    if ((st = exclusive_scan_i32_to_i64(g->alloc, cnt.as<int32_t>(), offs.as<int64_t>(), count, s))) break;
    if ((st = cuda_status(cudaMemcpyAsync(d_found, offs.as<int64_t>() + count, 8, cudaMemcpyDeviceToDevice, s),
                          "copy found")))
      break;
    // the CTAs' sources for pass 2 (their number in d_cursors[3])
    if ((st = cuda_status(cudaMemsetAsync(d_cursors + 3, 0, sizeof(uint32_t), s), "memset heavy"))) break;
    k_list_heavy<<<2 * num_sms(), 256, 0, s>>>(g->view(), first, count, cnt.as<uint32_t>(),
                                               reinterpret_cast<const unsigned long long*>(d_found), grid,
                                               heavy.as<int32_t>(), d_cursors + 3, d_cursors + 4);
    note_launch();
    if ((st = cuda_status(cudaGetLastError(), "k_list_heavy"))) break;
    // pass 2: the triples, each source into its own range
    dev::Sink sk;
    sk.tri = d_triples;
    sk.capacity = (unsigned long long)(capacity > 0 ? capacity : 0);
    sk.perm = g->perm.as<int32_t>();
    if ((st = cuda_status(cudaMemsetAsync(d_cursors, 0, 3 * sizeof(uint32_t), s), "memset cursors"))) break;
    if ((st = cuda_status(cudaFuncSetAttribute(k_list<dev::kModeList>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kCountSmem),
                          "k_list attribute")))
      break;
    k_list<dev::kModeList><<<grid, kCountThreads, dev::kCountSmem, s>>>(
        g->view(), first, count, sk, d_cursors, cnt.as<uint32_t>(), offs.as<int64_t>(), heavy.as<int32_t>(),
        d_cursors + 3, d_cursors + 4);
    note_launch();
    st = cuda_status(cudaGetLastError(), "k_list");
  } while (0);
  buf_release(g->alloc, cnt, s);
  buf_release(g->alloc, offs, s);
  buf_release(g->alloc, heavy, s);
  return st;
}

}  // namespace tc

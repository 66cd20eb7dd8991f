// tc_batch.cu — count many graphs in one persistent launch.
//
// The work queue is the concatenation, over the graphs of the batch, of their block-bin sources and (separately)
// of their warp-bin sources.  pb[g] / pw[g] are exclusive prefixes of the per-graph bin sizes, so a global source
// index maps to its graph by binary search.  CTAs first drain the block-bin space one source at a time; then each
// warp drains the warp-bin space four sources at a time.  Per-source counts are added to counts[g] (one atomic per
// warp per run of consecutive sources of the same graph).  The loops end when the cursors pass the totals: there
// is no waiting on other CTAs.
#include <vector>

#include "tc_count.cuh"

namespace tc {
namespace {

struct BatchTable {
  const CsrView* views;
  const int64_t* pb;  // num_graphs + 1
  const int64_t* pw;  // num_graphs + 1
  int32_t num_graphs;
};

__device__ __forceinline__ int find_graph(const int64_t* p, int G, int64_t i) {
  int a = 0, b = G;  // last g with p[g] <= i
  while (a + 1 < b) {
    const int mid = (a + b) >> 1;
    if (__ldg(&p[mid]) <= i)
      a = mid;
    else
      b = mid;
  }
  return a;
}

__global__ void __launch_bounds__(kCountThreads, 2)
    k_count_batch(BatchTable t, unsigned long long* __restrict__ counts, unsigned long long* __restrict__ cursors) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t ws[32];
  __shared__ unsigned long long red[kWarpsPerCTA];
  __shared__ long long s_idx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = t.num_graphs;
  const int64_t NB = __ldg(&t.pb[G]), NW = __ldg(&t.pw[G]);

  if (NB > 0) {
    const dev::BlockRows br = dev::block_rows(smem);
    dev::zero_words(smem, dev::kBlockBitmapWords, tid, kCountThreads);
    for (int k = tid; k < kBlockLowSlots; k += kCountThreads) br.ltab[k] = -1;
    __syncthreads();
    while (true) {
      if (tid == 0) s_idx = (long long)atomicAdd(&cursors[0], 1ull);
      __syncthreads();
      const int64_t i = s_idx;
      __syncthreads();
      if (i >= NB) break;
      const int g = find_graph(t.pb, G, i);
      const CsrView v = t.views[g];
      unsigned long long h = dev::block_source<false>(v.list[i - __ldg(&t.pb[g])], v, smem, br, ws, nullptr);
      h = warp_sum(h);
      if (lane == 0) red[warp] = h;
      __syncthreads();
      if (tid == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kWarpsPerCTA; ++w) s += red[w];
        if (s) atomicAdd(&counts[g], s);
      }
      // the next iteration's barriers order this read of red[] before it is rewritten
    }
  }
  if (NW > 0) {
    uint32_t* region = smem + warp * dev::kWarpRegionWords;
    const dev::Rows r = dev::warp_rows(region);
    int32_t* ltab = dev::warp_low(region);
    dev::zero_words(region, dev::kWarpBitmapWords, lane, 32);
    for (int k = lane; k < kWarpLowSlots; k += 32) ltab[k] = -1;
    __syncwarp();
    int cur_g = -1;
    unsigned long long acc = 0;
    constexpr int kChunk = 4;
    while (true) {
      long long idx = 0;
      if (lane == 0) idx = (long long)atomicAdd(&cursors[1], (unsigned long long)kChunk);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= NW) break;
      const int64_t e = idx + kChunk < NW ? idx + kChunk : NW;
      for (int64_t i = idx; i < e; ++i) {
        const int g = find_graph(t.pw, G, i);
        if (g != cur_g) {
          acc = warp_sum(acc);
          if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
          acc = 0;
          cur_g = g;
        }
        const CsrView v = t.views[g];
        const int32_t u = v.list[v.n - v.nw + (i - __ldg(&t.pw[g]))];
        acc += dev::warp_source<false>(u, v, region, ltab, r, nullptr);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
  }
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_count_batch(tc_graph* const* gs, int32_t num_graphs, uint64_t* out_counts,
                                           void* stream) {
  if (num_graphs < 0 || (num_graphs > 0 && (!gs || !out_counts))) {
    set_error("tc_count_batch: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  if (num_graphs == 0) return TC_OK;
  for (int32_t i = 0; i < num_graphs; ++i) {
    if (!gs[i]) {
      set_error("tc_count_batch: NULL graph handle");
      return TC_ERR_INVALID_ARG;
    }
    if (!gs[i]->built) {
      set_error("tc_count_batch: a graph is not built");
      return TC_ERR_STATE;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const Allocator& a = gs[0]->alloc;
  const size_t G = (size_t)num_graphs;
  // host table: views | pb | pw, then device: counts | cursors
  const size_t views_bytes = ((G * sizeof(CsrView)) + 255) / 256 * 256;
  const size_t pre_bytes = ((G + 1) * 8 + 255) / 256 * 256;
  const size_t table_bytes = views_bytes + 2 * pre_bytes;
  const size_t counts_bytes = (G * 8 + 255) / 256 * 256;
  std::vector<unsigned char> host(table_bytes, 0);
  CsrView* hv = reinterpret_cast<CsrView*>(host.data());
  int64_t* hpb = reinterpret_cast<int64_t*>(host.data() + views_bytes);
  int64_t* hpw = reinterpret_cast<int64_t*>(host.data() + views_bytes + pre_bytes);
  hpb[0] = hpw[0] = 0;
  for (size_t i = 0; i < G; ++i) {
    hv[i] = gs[i]->view();
    hpb[i + 1] = hpb[i] + gs[i]->nb;
    hpw[i + 1] = hpw[i] + gs[i]->nw;
  }
  Buf dev;
  TC_TRY(buf_alloc(a, dev, table_bytes + counts_bytes + 64, s));
  tc_status st = TC_OK;
  do {
    unsigned char* base = dev.as<unsigned char>();
    if ((st = cuda_status(cudaMemcpyAsync(base, host.data(), table_bytes, cudaMemcpyHostToDevice, s), "H2D table")))
      break;
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(base + table_bytes);
    unsigned long long* cursors = reinterpret_cast<unsigned long long*>(base + table_bytes + counts_bytes);
    if ((st = cuda_status(cudaMemsetAsync(counts, 0, counts_bytes + 64, s), "memset counts"))) break;
    BatchTable t;
    t.views = reinterpret_cast<const CsrView*>(base);
    t.pb = reinterpret_cast<const int64_t*>(base + views_bytes);
    t.pw = reinterpret_cast<const int64_t*>(base + views_bytes + pre_bytes);
    t.num_graphs = num_graphs;
    if (hpb[G] + hpw[G] > 0) {
      if ((st = cuda_status(cudaFuncSetAttribute(k_count_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 dev::kCountSmem),
                            "smem attr")))
        break;
      const int64_t want = hpb[G] + (hpw[G] + kWarpsPerCTA - 1) / kWarpsPerCTA;
      const int grid = (int)(want < 2 * kNumSMs ? want : 2 * kNumSMs);
      k_count_batch<<<grid, kCountThreads, dev::kCountSmem, s>>>(t, counts, cursors); note_launch();
      if ((st = cuda_status(cudaGetLastError(), "k_count_batch"))) break;
    }
    if ((st = cuda_status(cudaMemcpyAsync(out_counts, counts, G * 8, cudaMemcpyDeviceToHost, s), "D2H counts")))
      break;
    st = cuda_status(cudaStreamSynchronize(s), "tc_count_batch sync");
  } while (0);
  buf_release(a, dev, s);
  return st;
}

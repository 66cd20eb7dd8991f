// tc_count.cu — the single-graph counting launch.
//
// One persistent kernel, 2 CTAs of 512 threads per SM.  CTAs first take block-bin sources one at a time from an
// atomic cursor (heavy sources: many candidate 2-paths), then every warp takes warp-bin sources in chunks of
// four.  Each thread accumulates its closed 2-paths in a register; at the end the block reduces them (warp
// shuffles, then shared memory) and adds its total with one 64-bit atomic.
#include "tc_count.cuh"

namespace tc {
namespace {

template <bool PV>
__global__ void __launch_bounds__(kCountThreads, 2)
    k_count(CsrView g, unsigned long long* __restrict__ total, unsigned long long* __restrict__ pv,
            uint32_t* __restrict__ cursors) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t ws[32];
  __shared__ unsigned long long red[kWarpsPerCTA];
  __shared__ int s_idx;
  unsigned long long acc = dev::count_graph<PV>(g, pv, cursors, smem, ws, &s_idx);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kWarpsPerCTA; ++w) s += red[w];
    if (s) atomicAdd(total, s);
  }
}

}  // namespace

int count_grid(const tc_graph* g) {
  const int64_t want = g->nb + (g->nw + kWarpsPerCTA - 1) / kWarpsPerCTA;
  return (int)(want < 2 * kNumSMs ? (want < 1 ? 1 : want) : 2 * kNumSMs);
}

tc_status launch_count(const tc_graph* g, uint64_t* d_total, uint64_t* d_per_vertex, uint32_t* d_cursors,
                       cudaStream_t s) {
  TC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s));
  if (d_per_vertex && g->n > 0) TC_CUDA(cudaMemsetAsync(d_per_vertex, 0, (size_t)g->n * sizeof(uint64_t), s));
  if (g->nb + g->nw == 0) return TC_OK;
  TC_CUDA(cudaMemsetAsync(d_cursors, 0, 2 * sizeof(uint32_t), s));
  const int grid = count_grid(g);
  if (d_per_vertex) {
    TC_CUDA(cudaFuncSetAttribute(k_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kCountSmem));
    k_count<true><<<grid, kCountThreads, dev::kCountSmem, s>>>(g->view(), (unsigned long long*)d_total,
                                                                (unsigned long long*)d_per_vertex, d_cursors);
  } else {
    TC_CUDA(cudaFuncSetAttribute(k_count<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kCountSmem));
    k_count<false><<<grid, kCountThreads, dev::kCountSmem, s>>>(g->view(), (unsigned long long*)d_total, nullptr,
                                                                 d_cursors);
  }
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

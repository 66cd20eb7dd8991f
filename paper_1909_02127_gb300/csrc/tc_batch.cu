// tc_batch.cu — count many graphs in one persistent launch.
//
// The work queue is the concatenation, over the graphs of the batch, of their block-bin sources and (separately)
// of their warp-bin sources and of their thread-bin sources in tasks of 32.  pb[g] / pw[g] / pt[g] are exclusive
// prefixes of the per-graph sizes, so a global index maps to its graph by binary search.  CTAs first drain the
// block-bin space one source at a time; then each warp drains the warp-bin space sixteen sources at a time, and the
// thread-bin space one task (one source per lane) at a time.  Per-source counts are added to counts[g] (one atomic per
// warp per run of consecutive sources of the same graph).  The loops end when the cursors pass the totals: there
// is no waiting on other CTAs.
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "tc_count.cuh"

namespace tc {
namespace {

struct BatchTable {
  const CsrView* views;
  const int64_t* pb;  // num_graphs + 1
  const int64_t* pw;  // num_graphs + 1
  const int64_t* pt;  // num_graphs + 1: thread-bin tasks of 32 sources
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
      unsigned long long h =
          dev::block_source<dev::kModeCount>(v.list[i - __ldg(&t.pb[g])], v, smem, br, ws, dev::Sink{});
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
    // Chunks of consecutive sources: the graph is found by one search per chunk and then followed forward, and its
    // view stays in registers while the chunk stays inside it.
    constexpr int kChunk = 16;
    CsrView v{};
    int64_t gbeg = 0, gend = 0;  // [pw[cur_g], pw[cur_g + 1])
    while (true) {
      long long idx = 0;
      if (lane == 0) idx = (long long)atomicAdd(&cursors[1], (unsigned long long)kChunk);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= NW) break;
      const int64_t e = idx + kChunk < NW ? idx + kChunk : NW;
      for (int64_t i = idx; i < e; ++i) {
        if (i < gbeg || i >= gend) {
          const int g = (cur_g >= 0 && i >= gend && i < __ldg(&t.pw[cur_g + 2])) ? cur_g + 1
                                                                                 : find_graph(t.pw, G, i);
          acc = warp_sum(acc);
          if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
          acc = 0;
          cur_g = g;
          v = t.views[g];
          gbeg = __ldg(&t.pw[g]);
          gend = __ldg(&t.pw[g + 1]);
        }
        const int64_t k = i - gbeg;  // the graph's warp work: nbw block-bin sources, then its warp bin
        const int32_t u = k < v.nbw ? v.list[k] : v.list[v.n - v.nw + (k - v.nbw)];
        acc += dev::warp_source<dev::kModeCount>(u, v, region, ltab, r, dev::Sink{});
      }
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
  }
  const int64_t NT = __ldg(&t.pt[G]);
  if (NT > 0) {  // thread-bin sources: one task of 32 per warp, one source per lane
    int cur_g = -1;
    unsigned long long acc = 0;
    CsrView v{};
    int64_t gbeg = 0, gend = 0;  // [pt[cur_g], pt[cur_g + 1])
    while (true) {
      long long idx = 0;
      if (lane == 0) idx = (long long)atomicAdd(&cursors[2], 1ull);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= NT) break;
      if (idx < gbeg || idx >= gend) {
        acc = warp_sum(acc);
        if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
        acc = 0;
        cur_g = find_graph(t.pt, G, idx);
        v = t.views[cur_g];
        gbeg = __ldg(&t.pt[cur_g]);
        gend = __ldg(&t.pt[cur_g + 1]);
      }
      const int64_t k = (idx - gbeg) * 32 + lane;
      if (k < v.nt) acc += dev::tiny_source<dev::kModeCount>(v.tlist[k], v, dev::Sink{});
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc && cur_g >= 0) atomicAdd(&counts[cur_g], acc);
  }
}

// Device layout of a batch: views | pb | pw | counts | cursors, built from host handles.
struct BatchLayout {
  size_t views_bytes, pre_bytes, table_bytes, counts_bytes, total_bytes;
  int64_t nb_total, nw_total, nt_total;
};

tc_status check_batch(tc_graph* const* gs, int32_t num_graphs, const char* who) {
  for (int32_t i = 0; i < num_graphs; ++i) {
    if (!gs[i]) {
      set_error(std::string(who) + ": NULL graph handle");
      return TC_ERR_INVALID_ARG;
    }
    if (!gs[i]->built) {
      set_error(std::string(who) + ": a graph is not built");
      return TC_ERR_STATE;
    }
  }
  return TC_OK;
}

BatchLayout batch_table(tc_graph* const* gs, int32_t num_graphs, std::vector<unsigned char>& host) {
  const size_t G = (size_t)num_graphs;
  BatchLayout L{};
  L.views_bytes = ((G * sizeof(CsrView)) + 255) / 256 * 256;
  L.pre_bytes = ((G + 1) * 8 + 255) / 256 * 256;
  L.table_bytes = L.views_bytes + 3 * L.pre_bytes;
  L.counts_bytes = (G * 8 + 255) / 256 * 256;
  L.total_bytes = L.table_bytes + L.counts_bytes + 64;
  host.assign(L.table_bytes, 0);
  CsrView* hv = reinterpret_cast<CsrView*>(host.data());
  int64_t* hpb = reinterpret_cast<int64_t*>(host.data() + L.views_bytes);
  int64_t* hpw = reinterpret_cast<int64_t*>(host.data() + L.views_bytes + L.pre_bytes);
  int64_t* hpt = reinterpret_cast<int64_t*>(host.data() + L.views_bytes + 2 * L.pre_bytes);
  hpb[0] = hpw[0] = hpt[0] = 0;
  const int64_t warp_max = batch_warp_max_edges();
  for (size_t i = 0; i < G; ++i) {
    hv[i] = gs[i]->view();
    if (gs[i]->m <= warp_max) hv[i].nbw = hv[i].nb;  // this graph's block-bin sources run one warp each
    hpb[i + 1] = hpb[i] + (hv[i].nb - hv[i].nbw);
    hpw[i + 1] = hpw[i] + hv[i].nw + hv[i].nbw;
    hpt[i + 1] = hpt[i] + (hv[i].nt + 31) / 32;
  }
  L.nb_total = hpb[G];
  L.nw_total = hpw[G];
  L.nt_total = hpt[G];
  return L;
}

// Zero the counts and cursors, launch the persistent kernel, copy the counts to `host_counts` (stream-ordered).
tc_status batch_launch(unsigned char* base, const BatchLayout& L, int32_t num_graphs, uint64_t* host_counts,
                       cudaStream_t s) {
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(base + L.table_bytes);
  unsigned long long* cursors = reinterpret_cast<unsigned long long*>(base + L.table_bytes + L.counts_bytes);
  TC_CUDA(cudaMemsetAsync(counts, 0, L.counts_bytes + 64, s));
  if (L.nb_total + L.nw_total + L.nt_total > 0) {
    BatchTable t;
    t.views = reinterpret_cast<const CsrView*>(base);
    t.pb = reinterpret_cast<const int64_t*>(base + L.views_bytes);
    t.pw = reinterpret_cast<const int64_t*>(base + L.views_bytes + L.pre_bytes);
    t.pt = reinterpret_cast<const int64_t*>(base + L.views_bytes + 2 * L.pre_bytes);
    t.num_graphs = num_graphs;
    const int64_t want = L.nb_total + (L.nw_total + L.nt_total + kWarpsPerCTA - 1) / kWarpsPerCTA;
    const int grid = (int)(want < 2 * num_sms() ? want : 2 * num_sms());
    k_count_batch<<<grid, kCountThreads, dev::kCountSmem, s>>>(t, counts, cursors);
    TC_CUDA(cudaGetLastError());
  }
  TC_CUDA(cudaMemcpyAsync(host_counts, counts, (size_t)num_graphs * 8, cudaMemcpyDeviceToHost, s));
  return TC_OK;
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
  TC_TRY(check_batch(gs, num_graphs, "tc_count_batch"));
  cudaStream_t s = (cudaStream_t)stream;
  const Allocator& a = gs[0]->alloc;
  std::vector<unsigned char> host;
  const BatchLayout L = batch_table(gs, num_graphs, host);
  TC_TRY(smem_attribute_once<k_count_batch>(dev::kCountSmem));
  Buf dev;
  TC_TRY(buf_alloc(a, dev, L.total_bytes, s));
  tc_status st = cuda_status(cudaMemcpyAsync(dev.p, host.data(), L.table_bytes, cudaMemcpyHostToDevice, s), "H2D");
  if (st == TC_OK) st = batch_launch(dev.as<unsigned char>(), L, num_graphs, out_counts, s);
  if (st == TC_OK) {
    if (L.nb_total + L.nw_total + L.nt_total > 0) note_launch();
    st = cuda_status(cudaStreamSynchronize(s), "tc_count_batch sync");
  }
  buf_release(a, dev, s);
  return st;
}

// ---- batch plans: the launch sequence of a fixed set of graphs, captured once as a CUDA graph ---------------------
struct tc_batch_plan {
  std::vector<tc_graph*> graphs;
  tc::Allocator alloc;
  tc::Buf dev;
  uint64_t* host_counts = nullptr;  // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool launches_kernel = false;
};

extern "C" TC_API void tc_batch_plan_free(tc_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->host_counts) cudaFreeHost(p->host_counts);
  cudaStream_t s = p->graphs.empty() ? nullptr : p->graphs[0]->last_stream;
  tc::buf_release(p->alloc, p->dev, s);
  delete p;
}

extern "C" TC_API tc_status tc_batch_plan_create(tc_graph* const* gs, int32_t num_graphs, void* stream,
                                                 tc_batch_plan** out) {
  if (!out || num_graphs <= 0 || !gs) {
    set_error("tc_batch_plan_create: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  TC_TRY(check_batch(gs, num_graphs, "tc_batch_plan_create"));
  cudaStream_t s = (cudaStream_t)stream;
  tc_batch_plan* p = new (std::nothrow) tc_batch_plan();
  if (!p) {
    set_error("tc_batch_plan_create: host allocation failed");
    return TC_ERR_NO_MEMORY;
  }
  p->graphs.assign(gs, gs + num_graphs);
  p->alloc = gs[0]->alloc;
  std::vector<unsigned char> host;
  const BatchLayout L = batch_table(gs, num_graphs, host);
  p->launches_kernel = L.nb_total + L.nw_total + L.nt_total > 0;
  tc_status st = TC_OK;
  do {
    if ((st = cuda_status(cudaFuncSetAttribute(k_count_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               dev::kCountSmem),
                          "smem attr")))
      break;
    if ((st = buf_alloc(p->alloc, p->dev, L.total_bytes, s))) break;
    if ((st = cuda_status(cudaMallocHost((void**)&p->host_counts, (size_t)num_graphs * 8), "pinned counts"))) break;
    if ((st = cuda_status(cudaMemcpyAsync(p->dev.p, host.data(), L.table_bytes, cudaMemcpyHostToDevice, s), "H2D")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "sync table"))) break;
    // capture: memset counts and cursors -> persistent kernel -> D2H of the counts.  Capture happens on a private
    // stream (the legacy default stream cannot be captured); the plan is replayed on the caller's stream.
    cudaStream_t cap = nullptr;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream"))) break;
    cudaError_t begin = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    tc_status launch = TC_OK;
    cudaError_t end = cudaSuccess;
    if (begin == cudaSuccess) {
      launch = batch_launch(p->dev.as<unsigned char>(), L, num_graphs, p->host_counts, cap);
      end = cudaStreamEndCapture(cap, &p->graph);
    }
    cudaStreamDestroy(cap);
    if ((st = cuda_status(begin, "begin capture"))) break;
    if ((st = launch)) break;
    if ((st = cuda_status(end, "end capture"))) break;
    if ((st = cuda_status(cudaGraphInstantiate(&p->exec, p->graph, 0), "instantiate"))) break;
  } while (0);
  if (st != TC_OK) {
    tc_batch_plan_free(p);
    return st;
  }
  *out = p;
  return TC_OK;
}

extern "C" TC_API tc_status tc_batch_plan_run(tc_batch_plan* p, uint64_t* out_counts, void* stream) {
  if (!p || !out_counts) {
    set_error("tc_batch_plan_run: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  TC_CUDA(cudaGraphLaunch(p->exec, s));
  if (p->launches_kernel) note_launch();
  TC_CUDA(cudaStreamSynchronize(s));
  memcpy(out_counts, p->host_counts, p->graphs.size() * 8);
  return TC_OK;
}

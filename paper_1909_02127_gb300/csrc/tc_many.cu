// tc_many.cu — many graphs counted as one pipeline.
//
// The graphs are ingested, built and counted together as their disjoint union: graph j's vertices become
// voff[j] .. voff[j+1] - 1 of one graph, whose CSR is built and counted once.  No triangle spans two graphs, and
// each triangle is found once, from its first vertex in the visiting order (Sec. III-A, III-C), so crediting every
// source's triangles to the graph holding that source gives each graph its own count.  For many small graphs this
// replaces a launch sequence per graph (ingest, about twenty build kernels, count) with one for the whole batch.
#include <string.h>

#include <new>
#include <vector>

#include "tc_build.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

// Page-locked host staging for a call's small host<->device copies (pointer table and offsets up, counts down), one
// per host thread, grown when a call needs more and kept for the thread's later calls: copies from pageable memory
// would be synchronous and go through the driver's shared staging, which serialises concurrent callers.
struct PinnedStage {
  void* p = nullptr;
  size_t cap = 0;
  ~PinnedStage() {
    if (p) (void)cudaFreeHost(p);
  }
  void* get(size_t bytes) {
    if (bytes > cap) {
      size_t want = cap ? cap : 4096;
      while (want < bytes) want *= 2;
      void* q = nullptr;
      if (cudaMallocHost(&q, want) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
      }
      if (p) (void)cudaFreeHost(p);
      p = q;
      cap = want;
    }
    return p;
  }
};
thread_local PinnedStage t_stage;

}  // namespace

// The union pipeline for k graphs whose arrays are device-readable (srcs[j], dsts[j]; stage[j] != 0: host arrays
// that must first be copied to the device).  counts: k host uint64.  Blocks until the counts are valid.
tc_status count_many(const int32_t* const* srcs, const int32_t* const* dsts, const int64_t* num_edges,
                     const int64_t* num_vertices, const uint8_t* stage, int32_t k, uint64_t* counts,
                     const tc_allocator* user_alloc, cudaStream_t s) {
  memset(counts, 0, (size_t)k * sizeof(uint64_t));
  // pinned staging: [pointer table 2k | offsets 2(k+1) | counts k]
  const size_t ptr_bytes = 2 * (size_t)k * sizeof(void*), off_bytes = 2 * ((size_t)k + 1) * 8;
  char* pin = static_cast<char*>(t_stage.get(ptr_bytes + off_bytes + (size_t)k * 8));
  if (!pin) {
    set_error("tc_count_many: pinned host allocation failed");
    return TC_ERR_NO_MEMORY;
  }
  const int32_t** h_ptrs = reinterpret_cast<const int32_t**>(pin);
  int64_t* eoff = reinterpret_cast<int64_t*>(pin + ptr_bytes);  // eoff then voff
  int64_t* voff = eoff + k + 1;
  uint64_t* h_counts = reinterpret_cast<uint64_t*>(pin + ptr_bytes + off_bytes);
  eoff[0] = voff[0] = 0;
  int64_t staged_pairs = 0;
  for (int32_t j = 0; j < k; ++j) {
    eoff[j + 1] = eoff[j] + num_edges[j];
    voff[j + 1] = voff[j] + num_vertices[j];
    if (stage && stage[j]) staged_pairs += num_edges[j];
  }
  const int64_t n = voff[k], M = eoff[k];
  if (n > 0x7fffffffLL) {
    set_error("tc_count_many: the graphs' vertices together exceed the int32 id range");
    return TC_ERR_INVALID_ARG;
  }
  if (M >= 0xffffffffLL) {
    set_error("tc_count_many: the graphs' pairs together must be below 2^32-1");
    return TC_ERR_INVALID_ARG;
  }
  if (M == 0) return TC_OK;
  tc_graph* g = new (std::nothrow) tc_graph();
  if (!g) {
    set_error("tc_count_many: host allocation failed");
    return TC_ERR_NO_MEMORY;
  }
  if (user_alloc) {
    g->alloc.user = *user_alloc;
    g->alloc.has_user = true;
  }
  if (cudaGetDevice(&g->device) != cudaSuccess) (void)cudaGetLastError();
  g->n = n;
  g->num_pairs = M;
  g->key_bits = bits_for(n);
  g->last_stream = s;
  const Allocator& a = g->alloc;
  Buf table;
  tc_status st = TC_OK;
  do {
    if (!(g->host_total = slot_acquire())) {
      set_error("tc_count_many: pinned host allocation failed");
      st = TC_ERR_NO_MEMORY;
      break;
    }
    // one block: pointer tables, offsets, counts, the error word and cursors, per-source counts, staged pairs
    Arena lay;
    lay.take<const int32_t*>(2 * (size_t)k);
    lay.take<int64_t>(2 * ((size_t)k + 1));
    lay.take<uint64_t>((size_t)k + 2);
    lay.take<uint32_t>((size_t)n);
    lay.take<int32_t>(2 * (size_t)staged_pairs);
    if ((st = buf_alloc(a, table, lay.used, s))) break;
    Arena ar{table.as<char>()};
    const int32_t** d_ptrs = ar.take<const int32_t*>(2 * (size_t)k);
    int64_t* d_off = ar.take<int64_t>(2 * ((size_t)k + 1));
    uint64_t* d_counts = ar.take<uint64_t>((size_t)k + 2);
    uint32_t* d_words = reinterpret_cast<uint32_t*>(d_counts + k);  // [0] error, [1..3] cursors, after the counts
    uint32_t* d_cnt = ar.take<uint32_t>((size_t)n);
    int32_t* d_stage = ar.take<int32_t>(2 * (size_t)staged_pairs);
    const int32_t** ptrs = h_ptrs;
    int64_t so = 0;
    for (int32_t j = 0; j < k; ++j) {
      if (stage && stage[j] && num_edges[j] > 0) {
        int32_t* ds = d_stage + 2 * so;
        int32_t* dd = ds + num_edges[j];
        if ((st = cuda_status(cudaMemcpyAsync(ds, srcs[j], (size_t)num_edges[j] * 4, cudaMemcpyHostToDevice, s),
                              "tc_count_many copy")))
          break;
        if ((st = cuda_status(cudaMemcpyAsync(dd, dsts[j], (size_t)num_edges[j] * 4, cudaMemcpyHostToDevice, s),
                              "tc_count_many copy")))
          break;
        ptrs[j] = ds;
        ptrs[k + j] = dd;
        so += num_edges[j];
      } else {
        ptrs[j] = srcs[j];
        ptrs[k + j] = dsts[j];
      }
    }
    if (st) break;
    // the pointer table and the offsets are adjacent in the pinned staging and in the device block: one copy
    static_assert(sizeof(void*) == 8, "pointer table entries are 8 bytes");
    if ((st = cuda_status(cudaMemcpyAsync(d_ptrs, h_ptrs, ptr_bytes, cudaMemcpyHostToDevice, s), "tc_count_many table")))
      break;
    if ((st = cuda_status(cudaMemcpyAsync(d_off, eoff, off_bytes, cudaMemcpyHostToDevice, s), "tc_count_many offsets")))
      break;
    if ((st = cuda_status(cudaMemsetAsync(d_counts, 0, ((size_t)k + 2) * 8, s), "tc_count_many zero"))) break;
    // ingest: the counts and keys of the union
    Arena isz;
    isz.view((size_t)n * 4);
    const size_t clear = isz.used;
    isz.view((size_t)M * 8);
    if ((st = buf_alloc(a, g->ingest, isz.used, s))) break;
    Arena ia{g->ingest.as<char>()};
    g->indeg = ia.view((size_t)n * 4);
    g->keys = ia.view((size_t)M * 8);
    if ((st = cuda_status(cudaMemsetAsync(g->ingest.p, 0, clear, s), "tc_count_many counts"))) break;
    if ((st = pack_edges_many(g, d_ptrs, d_ptrs + k, d_off, d_off + k + 1, k, d_words, s))) break;
    // the error word lands with the build's synchronisation
    uint32_t* h_err = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(g->host_total) + kHostErrOffset);
    *h_err = 0;
    if ((st = cuda_status(cudaMemcpyAsync(h_err, d_words, 4, cudaMemcpyDeviceToHost, s), "tc_count_many error")))
      break;
    if ((st = build_graph(g, s))) break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "tc_count_many sync"))) break;
    if (*h_err) {
      set_error("tc_count_many: an edge endpoint lies outside its graph's [0, num_vertices)");
      st = TC_ERR_OUT_OF_RANGE;
      break;
    }
    g->built = true;
    if (k == 1)  // one graph: its total, from the counting kernel itself
      st = launch_count(g, d_counts, nullptr, d_words + 1, s);
    else
      st = launch_graph_counts(g, d_off + k + 1, k, d_counts, d_cnt, d_words + 1, s);
    if (st) break;
    if ((st = cuda_status(cudaMemcpyAsync(h_counts, d_counts, (size_t)k * 8, cudaMemcpyDeviceToHost, s),
                          "tc_count_many counts")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "tc_count_many sync"))) break;
    memcpy(counts, h_counts, (size_t)k * 8);
  } while (0);
  buf_release(a, table, s);
  release_graph(g, s);
  delete g;
  return st;
}

}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_count_many(const int32_t* const* srcs, const int32_t* const* dsts,
                                          const int64_t* num_edges, const int64_t* num_vertices, int32_t k,
                                          uint32_t flags, uint64_t* counts, void* stream) {
  if (k < 0 || (k > 0 && (!srcs || !dsts || !num_edges || !num_vertices || !counts))) {
    set_error("tc_count_many: bad arguments");
    return TC_ERR_INVALID_ARG;
  }
  if (flags != TC_PTR_HOST && flags != TC_PTR_DEVICE) {
    set_error("tc_count_many: flags must be exactly one of TC_PTR_HOST, TC_PTR_DEVICE");
    return TC_ERR_INVALID_ARG;
  }
  std::vector<const int32_t*> s(k), d(k);
  std::vector<uint8_t> stage(k, 0);
  for (int32_t j = 0; j < k; ++j) {
    if (num_edges[j] < 0 || num_vertices[j] < 0 || (num_edges[j] > 0 && (!srcs[j] || !dsts[j]))) {
      set_error("tc_count_many: bad sizes or arrays for graph " + std::to_string(j));
      return TC_ERR_INVALID_ARG;
    }
    if (num_edges[j] > 0 && num_vertices[j] == 0) {
      set_error("tc_count_many: edges given for an empty vertex set (graph " + std::to_string(j) + ")");
      return TC_ERR_OUT_OF_RANGE;
    }
    s[j] = srcs[j];
    d[j] = dsts[j];
    if (flags == TC_PTR_HOST && num_edges[j] > 0) {
      const int32_t* ms = mapped_for_device(srcs[j], num_edges[j]);
      const int32_t* md = ms ? mapped_for_device(dsts[j], num_edges[j]) : nullptr;
      if (ms && md) {
        s[j] = ms;
        d[j] = md;
      } else {
        stage[j] = 1;
      }
    }
  }
  if (k == 0) return TC_OK;
  return count_many(s.data(), d.data(), num_edges, num_vertices, stage.data(), k, counts, nullptr,
                    (cudaStream_t)stream);
}

// tc_internal.cuh — internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "tc.h"

namespace tc {

// Bytes of a graph's page-locked landing slot (see tc_graph::host_total).
constexpr size_t kHostSlotBytes = 256;
constexpr size_t kHostErrOffset = kHostSlotBytes - 8;  // an error word's place in the slot (after the build sizes)

// Streaming multiprocessors of the current device (queried once per device, cached).  Persistent grids are sized
// in multiples of it.
int num_sms();

// ------------------------------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
// Counts kernel launches made by this library (reported by tc_kernel_launches).
void note_launch();
tc_status cuda_status(cudaError_t e, const char* what);

#define TC_CUDA(call)                                              \
  do {                                                             \
    cudaError_t tc_e_ = (call);                                    \
    if (tc_e_ != cudaSuccess) return ::tc::cuda_status(tc_e_, #call); \
  } while (0)

#define TC_TRY(call)                         \
  do {                                       \
    tc_status tc_s_ = (call);                \
    if (tc_s_ != TC_OK) return tc_s_;        \
  } while (0)

// ------------------------------------------------------------------------------------------------------------
// Device memory through the graph's allocator
// ------------------------------------------------------------------------------------------------------------
struct Allocator {
  tc_allocator user{};
  bool has_user = false;
  void* alloc(size_t bytes, cudaStream_t s) const;
  void free(void* p, cudaStream_t s) const;
};

// A buffer owned by the code that allocated it (freed in stream order by buf_release()), or a view into another
// buffer (owned = false: buf_release forgets it, and its owner frees the memory).
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  bool owned = true;
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Pieces of one region of device memory, handed out in order at 256-byte boundaries with no allocation call.  With
// base null it only adds up the sizes asked for, so one layout function can first size the region and then carve
// it.
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
  Buf view(size_t bytes) {
    Buf b;
    b.p = take<char>(bytes);
    b.bytes = bytes;
    b.owned = false;
    return b;
  }
};

tc_status buf_alloc(const Allocator& a, Buf& b, size_t bytes, cudaStream_t s);
void buf_release(const Allocator& a, Buf& b, cudaStream_t s);

// ------------------------------------------------------------------------------------------------------------
// Count-kernel parameters (shared by tc_count and tc_count_batch)
// ------------------------------------------------------------------------------------------------------------
constexpr int kCountThreads = 512;                 // threads per CTA of the counting kernel
constexpr int kWarpsPerCTA = kCountThreads / 32;
constexpr int kWarpBitmapBits = 1 << 15;           // per-warp bitmap of N+(u) over the top 32768 ranks (4 KB)
constexpr int kBlockBitmapBits = 1 << 19;          // per-CTA bitmap of N+(u) over the top 524288 ranks (64 KB)
constexpr int kBitmapSlackWords = 32;              // room for the padding id n (its bit is never set)
constexpr int kWarpLowSlots = 128;                 // per-warp hash of N+(u) entries below the bitmap window
constexpr int kBlockLowSlots = 2048;               // per-CTA hash of the same
constexpr int kBlockRows = kCountThreads;          // rows (v in N+(u)) staged per CTA pass
constexpr int kLongQuads = 16;                     // rows of >= 16 quads (64 ids) are walked by a whole warp
// The warp/block split of sources (w(u) above the threshold -> a whole CTA) comes from the tuning table.
int64_t block_min_work_for(int64_t m);
int64_t batch_warp_max_edges();
int64_t stage_min_csr_bytes();
// Per-vertex counting adds to its per-CTA counters without read-back for graphs of at most this many edges (the
// tuning table; at most kVertexPlainMaxEdges, below which no counter can reach 2^32).
constexpr int64_t kVertexPlainMaxEdges = (int64_t(1) << 31) - 1;
int64_t vertex_plain_max_edges();

// Per-graph view used by the counting kernels.  Vertices are relabelled by rank in the (input-pair count, id)
// order, so every oriented edge goes from a lower to a higher id and rows hold ascending ids.  Rows start on
// 16-byte boundaries and are padded to a multiple of 4 entries with the id n, which no bitmap ever marks.
// Dense rows: a row N+(v) with v in the warp window [base_w, n) whose bitmap over its range (v, n) takes no more
// words than it has entries is also stored as that bitmap, aligned to the windows (both bases are multiples of
// 128, so bitmap quad q of the row lines up with quad (v + 1 - base_w) / 128 + q of a source's warp bitmap and
// dq_delta quads further on in its block bitmap).  Counting (not per-vertex counts or listing) tests such a row by
// ANDing words instead of looking up ids.
struct CsrView {
  const int64_t* off;   // n+1 padded row offsets (multiples of 4)
  const int32_t* col;   // off[n] column ids (+ one spare quad)
  const int32_t* list;  // sources: [0, nb) block bin, [n - nw, n) warp bin
  int64_t n;
  int32_t nb;           // block-bin sources
  int32_t nw;           // warp-bin sources
  int32_t base_w;       // per-warp bitmap covers ids [base_w, n]
  int32_t base_b;       // per-CTA bitmap covers ids [base_b, n]
  int32_t nbw;          // batches only: block-bin sources that are run one warp each (0 or nb)
  int32_t wtopq;        // dense rows end at window quad wtopq (the quad holding id n - 1)
  const int32_t* dq0;   // n - base_w entries: first quad of v's dense row in `dense`, or -1; null if none
  const int4* dense;    // dense row bitmaps, 128 ids per quad
  int32_t dq_delta;     // (base_w - base_b) / 128
  int32_t nt;           // thread-bin sources
  const int32_t* tlist; // thread-bin sources: few out-neighbours, each pair tested by one lookup
};
constexpr int kDenseMinDegree = 16;  // rows with fewer entries stay id lists
constexpr int kTinyMaxDegree = 8;    // thread-bin sources have at most this many out-neighbours

// ------------------------------------------------------------------------------------------------------------
// Primitives (tc_prims.cu)
// ------------------------------------------------------------------------------------------------------------
// LSD radix sort of uint64 keys on bits [bit_lo, bit_hi), stable.  keys/alt: n elements each; the sorted result
// is in *result (either keys or alt).
tc_status radix_sort_u64(const Allocator& a, uint64_t* keys, uint64_t* alt, int64_t n, int bit_lo, int bit_hi,
                         uint64_t** result, cudaStream_t s, void* tmp = nullptr);
// Exclusive scan of n int32 values into n+1 int64 values (out[n] = total).  tmp: device scratch of
// scan_temp_bytes(n) bytes, or null to allocate it through `a`.
tc_status exclusive_scan_i32_to_i64(const Allocator& a, const int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                                    void* tmp = nullptr);
// Exclusive scan of n uint32 values in place; *total (device, may be null) receives the sum.
tc_status exclusive_scan_u32(const Allocator& a, uint32_t* data, int64_t n, cudaStream_t s, void* tmp = nullptr);
// out[0..n] = exclusive scan of in[0..n), out[n] = the total.
tc_status exclusive_scan_u64(const Allocator& a, const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                             void* tmp = nullptr);
// Scratch bytes of a scan of n elements (partial sums of every level; 8-byte elements, enough for both scans).
size_t scan_temp_bytes(int64_t n);
// Scratch bytes of radix_sort_u64 over n keys (tile histograms and their scan).
size_t radix_temp_bytes(int64_t n);

// max_blocks < 0: 16 CTAs per SM of the current device.
int grid_for(int64_t items, int threads, int max_blocks = -1);

// cudaFuncSetAttribute(kernel, MaxDynamicSharedMemorySize, bytes) once per device: the attribute stays set, and a
// build of a small graph should not pay a host call for it every time.
template <auto Kernel>
tc_status smem_attribute_once(int bytes) {
  static std::atomic<int> done[64] = {};
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire) >= bytes) return TC_OK;
  TC_CUDA(cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  if (dev >= 0 && dev < 64) done[dev].store(bytes, std::memory_order_release);
  return TC_OK;
}


}  // namespace tc

// ------------------------------------------------------------------------------------------------------------
// The graph handle
// ------------------------------------------------------------------------------------------------------------
struct tc_graph {
  tc::Allocator alloc;
  int device = -1;           // the device current at tc_load_edges: every buffer of the graph lives there
  cudaStream_t last_stream = nullptr;
  int64_t n = 0;
  int64_t num_pairs = 0;
  int key_bits = 1;          // B: bits per vertex id in packed keys
  tc::Buf keys;              // packed (lo << B) | hi keys, until tc_build
  tc::Buf indeg;             // int32[n]: input pairs at each vertex (self-loops excluded), until tc_build
  tc::Buf ingest;            // small graphs: one block holding keys and indeg (then views), until tc_build
  tc::Buf block;             // compact builds: one block holding off, col, perm, list, tlist, dq0, dense (views)
  bool tiny = false;         // a small graph laid out in `block` from ingest on (keys, counts, scratch, CSR)
  bool built = false;
  // built state
  int64_t m = 0;
  int64_t max_out_degree = 0;
  int64_t wedges = 0;
  int64_t active = 0;
  int64_t nb = 0, nw = 0;
  int64_t csr_entries = 0;   // off[n]: column entries including padding
  tc::Buf off;               // int64[n+1], padded row offsets
  tc::Buf col;               // int32[csr_entries + 4]
  tc::Buf list;              // int32[n]: block bin at the front, warp bin at the back
  tc::Buf tlist;             // int32[n]: thread bin
  int64_t nt = 0;
  tc::Buf perm;              // int32[n]: perm[r] = original id of the vertex of rank r
  tc::Buf acc;               // uint64 scratch word(s) for counting: [0] total, [1..2] work cursors
  tc::Buf dq0;               // int32[n - base_w]: dense row start (quads) or -1
  tc::Buf dense;             // int4[dense_quads]: dense row bitmaps
  int64_t dense_rows = 0, dense_quads = 0;       // rows stored dense; quads of storage
  int64_t dense_wedges = 0, dense_visits = 0;    // 2-paths through dense rows; quads read for them per count
  uint64_t* host_total = nullptr;  // pinned landing slot of kHostSlotBytes: [0, 8) results, [8, ...) build sizes
  // The bitmap windows start at a multiple of 128 ids at or above n - (bitmap bits), so they end at id n.
  static int64_t window_base(int64_t n, int64_t bits) { return n > bits ? ((n - bits + 127) & ~int64_t(127)) : 0; }
  tc::CsrView view() const {
    tc::CsrView v;
    v.off = off.as<int64_t>();
    v.col = col.as<int32_t>();
    v.list = list.as<int32_t>();
    v.n = n;
    v.nb = (int32_t)nb;
    v.nw = (int32_t)nw;
    v.base_w = (int32_t)window_base(n, tc::kWarpBitmapBits);
    v.base_b = (int32_t)window_base(n, tc::kBlockBitmapBits);
    v.nbw = 0;
    v.wtopq = n > v.base_w ? (int32_t)(((n - 1 - v.base_w) >> 7) + 1) : 0;
    v.dq0 = dense_rows > 0 ? dq0.as<int32_t>() : nullptr;
    v.dense = dense.as<int4>();
    v.dq_delta = (v.base_w - v.base_b) >> 7;
    v.nt = (int32_t)nt;
    v.tlist = tlist.as<int32_t>();
    return v;
  }
};

namespace tc {
// tc_capi.cu
int bits_for(int64_t n);                                  // bits per vertex id in packed keys
const int32_t* mapped_for_device(const int32_t* p, int64_t len);  // device address of mapped host memory, or null
uint64_t* slot_acquire();                                 // a page-locked landing slot (kHostSlotBytes)
void slot_release(uint64_t* p);
void release_graph(tc_graph* g, cudaStream_t s);           // every buffer of g, in stream order
// tc_many.cu: k graphs counted as their disjoint union (arrays device-readable, or host arrays to copy where
// stage[j] != 0); counts: k host uint64.  Blocks until the counts are valid.
tc_status count_many(const int32_t* const* srcs, const int32_t* const* dsts, const int64_t* num_edges,
                     const int64_t* num_vertices, const uint8_t* stage, int32_t k, uint64_t* counts,
                     const tc_allocator* user_alloc, cudaStream_t s);
// tc_build.cu
tc_status pack_edges(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t len, int64_t offset,
                     uint32_t* d_err, cudaStream_t s);
tc_status build_graph(tc_graph* g, cudaStream_t s);
// The disjoint union of k graphs into g's keys and counts (g->n and g->num_pairs are the union's sizes): pairs
// [eoff[j], eoff[j+1]) come from d_srcs[j], d_dsts[j] (device-readable) with ids in [0, voff[j+1] - voff[j]),
// offset by voff[j].  Out-of-range ids set *d_err.  All arrays device-resident.
tc_status pack_edges_many(tc_graph* g, const int32_t* const* d_srcs, const int32_t* const* d_dsts,
                          const int64_t* d_eoff, const int64_t* d_voff, int32_t k, uint32_t* d_err, cudaStream_t s);
// by_id[perm[r]] = by_rank[r] for the n vertices (device arrays)
tc_status unpermute_counts(const tc_graph* g, const uint64_t* by_rank, uint64_t* by_id, cudaStream_t s);
// tc_count.cu
// d_per_vertex (if not null) receives counts in rank space.
tc_status launch_count(const tc_graph* g, uint64_t* d_total, uint64_t* d_per_vertex, uint32_t* d_cursors,
                       cudaStream_t s);
int count_grid(const tc_graph* g);
// Whether tc_count stages long hop-2 rows through shared memory for this graph: its CSR (offsets and columns) is
// at least the tuning table's stage_min_csr_bytes (0: never).
bool use_staged_rows(const tc_graph* g);
// Per-graph counts of a disjoint union: each source's triangles (the counting kernel's closing tests) are added to
// d_counts[j] of the graph j holding it, j found from the union's vertex offsets d_voff (k + 1 entries).
// d_counts: k zeroed uint64; d_cursors: three scratch words; d_cnt: n uint32 of scratch.
tc_status launch_graph_counts(const tc_graph* g, const int64_t* d_voff, int32_t k, uint64_t* d_counts,
                              uint32_t* d_cnt, uint32_t* d_cursors, cudaStream_t s);
// Lists into d_triples (capacity triples) the triangles whose first vertex has rank in [first, first + count);
// *d_found receives how many there are (also past capacity).  d_cursors: four scratch words.
tc_status launch_list(const tc_graph* g, int64_t first, int64_t count, int32_t* d_triples, int64_t capacity,
                      uint64_t* d_found, uint32_t* d_cursors, cudaStream_t s);
}  // namespace tc

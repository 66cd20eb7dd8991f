// tc_build.cuh — build variants beyond tc_build (declared apart from the counting kernels' shared header), and the
// pieces the bucketed builds share: the counters their kernels fill and the sizes they read back.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc.h"
#include "tc_internal.cuh"

namespace tc {

// tc_build on the graph's 2-core: after the repeats are removed, the NE filter (degree >= 2) is applied in rounds,
// each dropping the edges of vertices left with degree below 2, for at most peel_rounds rounds (0: until a round
// removes nothing, capped at 2^16 rounds); peel_rounds < 0 builds without pruning.  ps (may be null) receives what
// was removed.
tc_status build_graph_pruned(tc_graph* g, int32_t peel_rounds, tc_prune_stats* ps, cudaStream_t s);

// Whether tc_build groups `pairs` input pairs by per-source buckets (true) or by a radix sort (the tuning table).
bool use_buckets(int64_t pairs);

// tc_build with one host synchronisation (sizes bounded from n and the pair count, read back once at the end), for
// graphs of at most compact_max_pairs() input pairs (the tuning table) on the bucketed path.
tc_status build_graph_compact(tc_graph* g, cudaStream_t s);
int64_t compact_max_pairs();

// tc_build of a small graph as one cooperative kernel (grid-wide barriers between the steps), for graphs with at
// most kTinyMaxVertices vertices and at most tiny_max_pairs() input pairs (the tuning table, capped at
// kTinyMaxPairs); the same CSR as build_graph_compact.
constexpr int kTinyIdBits = 14;
constexpr int64_t kTinyMaxVertices = int64_t(1) << kTinyIdBits;
constexpr int64_t kTinyMaxPairs = (int64_t(1) << (32 - kTinyIdBits)) - 1;  // (count << 14 | id) fits 32 bits
bool tiny_eligible(int64_t n, int64_t pairs);
tc_status build_graph_tiny(tc_graph* g, cudaStream_t s);
// Ingest side of it: the graph's one block (head, error word, counts, keys, count words, build scratch, CSR views)
// allocated and its head cleared; *d_err receives the ingest error word.
tc_status tiny_ingest(tc_graph* g, uint32_t** d_err, cudaStream_t s);
int64_t tiny_max_pairs();

// Per-bucket de-duplication: distinct edges, the buckets handed to the warp and block kernels, and an error flag.
struct RowCounters {
  unsigned long long m;  // distinct edges
  unsigned int nwarp;    // buckets for k_rows_warp
  unsigned int nblock;   // buckets for k_rows_block
  unsigned int err;      // a bucket broke the size bound (cannot happen for consistent counts)
  unsigned int pad;
};

// Work estimate and bins: 2-paths, active sources, bin sizes, the largest out-degree, and what dense rows take.
struct BinCounters {
  unsigned long long wedges;
  unsigned long long active;
  unsigned int nb;
  unsigned int nw;
  int max_out;
  unsigned int nt;
  unsigned long long dense_wedges;  // 2-paths through dense rows
  unsigned long long dense_visits;  // quads of dense rows read per count
};

// w(u) summed over the out-neighbours v of u from rowinfo[v] = {d+(v), padded length or minus dense quads}: the
// padded entries to walk (four per dense quad), the true 2-paths, and those through dense rows.
struct RowWork {
  int64_t pad = 0, wtrue = 0, wdense = 0, qdense = 0;
  __device__ __forceinline__ void add(int2 ri) {
    wtrue += ri.x;
    if (ri.y >= 0) {
      pad += ri.y;
    } else {
      pad += -4 * (int64_t)ri.y;
      wdense += ri.x;
      qdense += -ri.y;
    }
  }
};

// What a one-synchronisation build reads back once, at its end (it lands in the graph's pinned slot after the count
// word).
struct CompactSizes {
  RowCounters rc;
  BinCounters bc;
  int64_t entries;              // padded column entries: off[n]
  int64_t dquads;               // quads of the dense rows
  unsigned long long dense_rows;
  unsigned long long bucket_alloc;  // bucket room claimed so far (compact builds place buckets by claim)
  uint32_t rank_tail;           // vertices whose input-pair count reaches the rank sort's clamp
  uint32_t rank_err;            // the clamped vertices outnumbered the fix-up sort (cannot happen within its bound)
};
static_assert(sizeof(CompactSizes) + 8 <= kHostErrOffset, "the compact build's sizes must fit the landing slot");

// Bits needed for x (0 for x = 0).
int bits_of(int64_t x);
// The read-back sizes into the graph.
void apply_sizes(tc_graph* g, const CompactSizes& hs);
// The graph's arrays as views into one block: off, col (at the column bound), perm, the source lists, the
// dense-row index and store (at the dense bound).
void csr_views(Arena& ar, tc_graph* g, int64_t n, int64_t bound_entries, int64_t wn, int64_t dense_quads);

}  // namespace tc

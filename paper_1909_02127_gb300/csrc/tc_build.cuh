// tc_build.cuh — build variants beyond tc_build (declared apart from the counting kernels' shared header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc.h"

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

}  // namespace tc

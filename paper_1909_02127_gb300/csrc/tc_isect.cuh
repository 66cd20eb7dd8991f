// tc_isect.cuh — the segmented-intersection counter (tc_isect.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc.h"

namespace tc {

// T = sum over oriented edges u -> v of |N+(u) ∩ N+(v)| into d_total (device); d_cursor: one scratch word.
tc_status launch_count_isect(const tc_graph* g, uint64_t* d_total, uint32_t* d_cursor, cudaStream_t s);

}  // namespace tc

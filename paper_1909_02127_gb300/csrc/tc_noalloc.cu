// tc_noalloc.cu — per-vertex counting that allocates no memory.
//
// tc_count_per_vertex produces its counts in rank space in a scratch buffer it allocates for the call, then
// scatters them to original ids.  Some callers cannot allocate device memory while they run: a serving loop that
// reserves all of its memory at start-up and must not allocate afterwards, or a host program whose device memory
// is owned by another framework's allocator.  For them, tc_count_per_vertex_noalloc keeps that scratch in the
// file-scope device array below, of a fixed maximum size, which every GPU that loads this library holds until the
// process exits.
#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxVertices = int64_t(1) << 20;  // 8 MiB of uint64 counts
constexpr int kMaxDevices = 64;

// Rank-space per-vertex counts of the current call.  Shared by every call on a device.
static __device__ __align__(256) unsigned long long g_rank_counts[kNoAllocMaxVertices];

std::mutex g_mutex;
void* g_scratch[kMaxDevices] = {};

// Device address of g_rank_counts on the current device.  In host code the array's name only stands in for the
// symbol, so the address is looked up once per device with that device current.
tc_status scratch_for_current_device(void** out) {
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    tc::set_error("tc_count_per_vertex_noalloc: device ordinal out of range");
    return TC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    TC_CUDA(cudaGetSymbolAddress(&p, g_rank_counts));
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return TC_OK;
}

}  // namespace

using namespace tc;

extern "C" TC_API tc_status tc_count_per_vertex_noalloc(tc_graph* g, uint64_t* d_per_vertex, uint64_t* d_total,
                                                        void* stream) {
  if (!g) {
    set_error("tc_count_per_vertex_noalloc: graph handle is NULL");
    return TC_ERR_INVALID_ARG;
  }
  if (!g->built) {
    set_error("tc_count_per_vertex_noalloc: graph is not built: call tc_build first");
    return TC_ERR_STATE;
  }
  if (!d_total || (g->n > 0 && !d_per_vertex)) {
    set_error("tc_count_per_vertex_noalloc: output pointer is NULL");
    return TC_ERR_INVALID_ARG;
  }
  if (g->n > kNoAllocMaxVertices) {
    set_error("tc_count_per_vertex_noalloc: the graph has more than 1048576 vertices, the size of the static "
              "scratch; use tc_count_per_vertex");
    return TC_ERR_INVALID_ARG;
  }
  int dev = -1;
  TC_CUDA(cudaGetDevice(&dev));
  if (dev != g->device) {
    set_error("tc_count_per_vertex_noalloc: the graph was loaded on device " + std::to_string(g->device) +
              " but device " + std::to_string(dev) + " is current; make the graph's device current first");
    return TC_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  TC_TRY(scratch_for_current_device(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  g->last_stream = s;
  uint32_t* cursors = reinterpret_cast<uint32_t*>(g->acc.as<uint64_t>() + 1);
  if (g->n == 0) return launch_count(g, d_total, nullptr, cursors, s);
  // launch_count zeroes the first n scratch entries before counting into them
  TC_TRY(launch_count(g, d_total, static_cast<uint64_t*>(scratch), cursors, s));
  return unpermute_counts(g, static_cast<const uint64_t*>(scratch), d_per_vertex, s);
}

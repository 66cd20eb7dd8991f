// tc_isect.cu — triangle counting by segmented intersection: the edge-centric family beside the fused traversal.
//
// Gunrock's segmented-intersection operator computes, for each pair of frontier elements, the intersection of
// their neighbour lists (Sec. II-B).  Applied to triangles on the oriented CSR, every oriented edge u -> v
// contributes |N+(u) ∩ N+(v)|: each common w is the triangle u < v < w in the visiting order, counted once.  Only
// the part of N+(u) above v can meet N+(v) (rows hold ascending ranks and every w in N+(v) is above v), so the
// lane that owns the edge at position i of N+(u) intersects N+(v) with N+(u)[i+1 ..].
//
// Layout of the work: a warp takes sources four at a time from an atomic cursor over the active sources (all bins
// of tc_build), stages N+(u) in shared memory when it fits (1024 ranks per warp), and its lanes take the edges
// u -> v of that source one each.  A lane walks the shorter of its two lists and finds each entry in the longer by
// galloping from the previous hit (both lists ascend), so an edge costs about min(a, b) * log(max(a, b) / min(a, b))
// probes.  Each lane reads its own N+(v) row: that scattered access is what this family trades against the fused
// kernel's warp-wide row walk and shared-memory bitmap.
#include "tc_internal.cuh"
#include "tc_isect.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace {

constexpr int kIsThreads = 512;
constexpr int kIsWarps = kIsThreads / 32;
constexpr int kIsStage = 1024;  // ranks of N+(u) staged per warp (4 KB)
constexpr int kIsChunk = 4;     // sources per cursor grab
constexpr size_t kIsSmem = sizeof(int32_t) * kIsWarps * kIsStage + sizeof(unsigned long long) * kIsWarps;

__device__ __forceinline__ int32_t true_len(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                            int32_t pad, int64_t u) {
  const int64_t a = off[u];
  int64_t e = off[u + 1];
  while (e > a && col[e - 1] == pad) --e;
  return (int32_t)(e - a);
}

// First index j in [lo, n) with x[j] >= key, by galloping from lo then binary search; n if none.
template <class P>
__device__ __forceinline__ int32_t gallop(P x, int32_t lo, int32_t n, int32_t key) {
  int32_t step = 1, hi = lo;
  while (hi < n && x[hi] < key) {
    lo = hi + 1;
    hi += step;
    step <<= 1;
  }
  if (hi > n) hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (x[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// |a ∩ b| for ascending lists a (length na) and b (length nb).
template <class PA, class PB>
__device__ __forceinline__ uint32_t intersect(PA a, int32_t na, PB b, int32_t nb) {
  uint32_t c = 0;
  if (na <= nb) {
    int32_t j = 0;
    for (int32_t i = 0; i < na && j < nb; ++i) {
      j = gallop(b, j, nb, a[i]);
      if (j < nb && b[j] == a[i]) {
        ++c;
        ++j;
      }
    }
  } else {
    int32_t j = 0;
    for (int32_t i = 0; i < nb && j < na; ++i) {
      j = gallop(a, j, na, b[i]);
      if (j < na && a[j] == b[i]) {
        ++c;
        ++j;
      }
    }
  }
  return c;
}

// Offset pointer into a list (shared or global memory).
struct SPtr {
  const int32_t* p;
  __device__ __forceinline__ int32_t operator[](int32_t i) const { return p[i]; }
};

__global__ void __launch_bounds__(kIsThreads, 2)
    k_count_isect(CsrView g, unsigned long long* __restrict__ total, uint32_t* __restrict__ cursor) {
  extern __shared__ __align__(16) int32_t is_smem[];  // kIsWarps x kIsStage staged rows, then kIsWarps partials
  int32_t(*stage)[kIsStage] = reinterpret_cast<int32_t(*)[kIsStage]>(is_smem);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(is_smem + kIsWarps * kIsStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t pad = (int32_t)g.n;
  const int64_t sources = (int64_t)g.nb + g.nw + g.nt;
  uint64_t mine = 0;
  for (;;) {
    uint32_t first = 0;
    if (lane == 0) first = atomicAdd(cursor, (uint32_t)kIsChunk);
    first = __shfl_sync(kFull, first, 0);
    if ((int64_t)first >= sources) break;
    const int64_t last = (int64_t)first + kIsChunk < sources ? (int64_t)first + kIsChunk : sources;
    for (int64_t k = first; k < last; ++k) {
      const int32_t u = k < g.nb ? g.list[k]
                        : k < (int64_t)g.nb + g.nw ? g.list[g.n - g.nw + (k - g.nb)]
                                                   : g.tlist[k - g.nb - g.nw];
      const int64_t base = g.off[u];
      const int32_t du = true_len(g.off, g.col, pad, u);
      const bool staged = du <= kIsStage;
      if (staged) {
        for (int32_t i = lane; i < du; i += 32) stage[warp][i] = g.col[base + i];
      }
      __syncwarp();
      const int32_t* nu = staged ? &stage[warp][0] : g.col + base;
      for (int32_t i = lane; i < du - 1; i += 32) {
        const int32_t v = nu[i];
        const int64_t vb = g.off[v];
        const int32_t dv = true_len(g.off, g.col, pad, v);
        if (dv == 0) continue;
        mine += intersect(SPtr{nu + i + 1}, du - i - 1, SPtr{g.col + vb}, dv);
      }
      __syncwarp();
    }
  }
  mine = warp_sum(mine);
  if (lane == 0) part[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kIsWarps; ++w) s += part[w];
    if (s) atomicAdd(total, s);
  }
}

}  // namespace

tc_status launch_count_isect(const tc_graph* g, uint64_t* d_total, uint32_t* d_cursor, cudaStream_t s) {
  TC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s));
  if (g->nb + g->nw + g->nt == 0) return TC_OK;
  TC_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(uint32_t), s));
  const int64_t want = (g->nb + g->nw + g->nt + kIsChunk * kIsWarps - 1) / (kIsChunk * kIsWarps);
  const int grid = (int)(want < 2 * num_sms() ? (want < 1 ? 1 : want) : 2 * num_sms());
  TC_TRY(smem_attribute_once<k_count_isect>((int)kIsSmem));
  k_count_isect<<<grid, kIsThreads, kIsSmem, s>>>(g->view(), (unsigned long long*)d_total, d_cursor);
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

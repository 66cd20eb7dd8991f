// tc_tiny.cu — tc_build of a small graph as one cooperative kernel.
//
// For a graph of a few thousand vertices the bucketed build's kernels do little work each, and their launches and
// the gaps between them set the time (ER-4096: about 25 launches).  Here the same steps run in one launch whose
// CTAs are all resident (a cooperative launch), separated by grid-wide barriers, and no step is left to one CTA:
//   0  rank      with every key (count << 14) | id in shared memory, each CTA counts for 32 vertices at a time the
//                keys below theirs, the key range split over its warps: rank(x) and perm, the (count, id) order
//                (Sec. III-A).  Bucket starts are claimed in any order, a warp's 32 vertices with one atomic add.
//   1  bucket    every pair into the bucket of its lower-ranked endpoint as the higher rank        (Sec. III-A/C)
//   2  rows      one warp per bucket: sorted and de-duplicated in place (a bitonic sort in registers up to 32
//                pairs, else a bitmap over the target range in the warp's shared memory); d+(u), and the row's
//                hop-2 cost code and dense quads as k_dense_select decides them                 (Def. 1, Sec. III-B)
//   3  CSR, bins each CTA takes a contiguous range of ranks: the padded lengths and dense quads of all ranks below
//                it summed (each CTA for itself), then scanned over its own rows to give off and dq0; one warp per
//                row writes the row with its padding, w(u) from its out-neighbours' codes and the bin it goes to
//                (as k_bins decides), and its dense bitmap when it has one                       (Sec. III-C)
// The result is the CSR of build_graph_compact, the bin lists up to their order.  Ids fit 14 bits and input-pair
// counts 18, so a rank key is one 32-bit word and every target range fits a warp's 2 KB bitmap.
//
// Each barrier waits a bounded number of polls; a CTA that gives up sets an error word and leaves, and the CTAs
// still waiting leave at their next poll of that word, so the launch always ends and the host reports the error.
#include <atomic>
#include <climits>

#include "tc_build.cuh"
#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace {

constexpr int kTinyThreads = 1024;
constexpr int kTinyWarps = kTinyThreads / 32;
constexpr int kTinyRowWords = (int)(kTinyMaxVertices / 32);      // a warp's bitmap: 512 words
constexpr unsigned kTinySpinLimit = 1u << 20;                    // barrier polls before giving up (~1 s)

struct TinyCtl {
  unsigned arrive;  // CTA arrivals at the barriers so far: barrier k is passed at (k + 1) * gridDim.x
  unsigned err;     // 1: a barrier gave up waiting
  unsigned alloc;   // bucket entries claimed so far
  unsigned pad;
};

// What the host clears before the launch and reads back after it: the sizes and the barrier word.
struct TinyHead {
  CompactSizes sz;
  TinyCtl ctl;
};
static_assert(sizeof(TinyHead) + 8 <= kHostErrOffset, "the one-launch build's read-back must fit the landing slot");

struct TinyArgs {
  const uint64_t* keys;   // M pair keys (lo << B) | hi, or the sentinel
  const int32_t* indeg;   // input-pair count of each vertex
  int64_t M;
  int32_t n;
  int32_t B;
  int32_t wtopq;          // quads of the top bitmap window row (the window is every vertex: n <= 32768)
  int32_t pad_;
  int64_t block_min_work;
  int32_t* rank;          // [n] by id
  uint32_t* bstart;       // [n] bucket start, by id (buckets in any order)
  uint32_t* cur;          // [n] bucket cursor, by id
  uint32_t* rstart;       // [n] the de-duplicated row's start in tgt, by rank
  int32_t* tgt;           // [sum of counts] bucket targets, rows de-duplicated in place
  int2* rowinfo;          // [n] {d+(u), padded length or minus dense quads}, by rank
  // the graph
  int64_t* off;           // [n + 1]
  int32_t* col;
  int32_t* perm;          // [n]
  int32_t* list;          // [n] block bin from the front, warp bin from the back
  int32_t* tlist;         // [n] thread bin
  int32_t* dq0;           // [n] first quad of the dense row, or -1
  uint32_t* dense;        // dense rows
  CompactSizes* sizes;
  TinyCtl* ctl;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier number k (0, 1, ...) of the cooperative launch: every CTA's writes before it are visible to
// every CTA after it.  One thread per CTA arrives with a release-acquire add on a counter that is never reset and
// waits, polling with acquire loads, until all CTAs have arrived at barrier k.  Returns false in every thread of
// the CTA when the wait gave up or another CTA reported that it had.
__device__ bool grid_barrier(TinyCtl* ctl, unsigned k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (k + 1) * gridDim.x;
    if (atom_add_acq_rel(&ctl->arrive, 1u) + 1 < target) {
      unsigned spins = 0;
      while (ld_acquire(&ctl->arrive) < target) {
        if (++spins > kTinySpinLimit || ld_acquire(&ctl->err) != 0u) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (!ok) atomicOr(&ctl->err, 1u);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// (padded length << 32) | dense quads of a row from its code: summed over rows, the low half never carries into the
// high one (the quads total below 2^32).
__device__ __forceinline__ unsigned long long row_sizes(int2 ri) {
  return ((unsigned long long)(uint32_t)((ri.x + 3) & ~3) << 32) | (uint32_t)(ri.y < 0 ? -ri.y : 0);
}

__global__ void __launch_bounds__(kTinyThreads, 1) k_tiny_build(TinyArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long ws64[kTinyWarps];
  __shared__ unsigned long long s_acc[6];  // m, wedges, active, dense wedges, dense visits, max d+
  __shared__ uint32_t s_cnt[3];            // block, warp, thread bin entries of this CTA
  __shared__ uint32_t s_base[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int64_t M = a.M;
  const int gwarp = blockIdx.x * kTinyWarps + warp, nwarps = gridDim.x * kTinyWarps;
  if (tid < 6) s_acc[tid] = 0ull;
  if (tid < 3) s_cnt[tid] = 0u;

  // ---- 0: ranks (every CTA for its own vertices) and bucket starts ----
  {
    const int npad = (n + 4 * kTinyWarps - 1) & ~(4 * kTinyWarps - 1);  // whole uint4 steps for every warp
    uint32_t* key = smem;                                              // [npad]; the padding is above every key
    uint32_t* part = smem + npad;                                      // [kTinyWarps][32] partial counts
    constexpr int kLoads = 8;  // counts loaded side by side before they are stored
    for (int i0 = tid; i0 < npad; i0 += kLoads * kTinyThreads) {
      int c[kLoads];
#pragma unroll
      for (int k = 0; k < kLoads; ++k) {
        const int i = i0 + k * kTinyThreads;
        c[k] = i < n ? __ldg(&a.indeg[i]) : 0;
      }
#pragma unroll
      for (int k = 0; k < kLoads; ++k) {
        const int i = i0 + k * kTinyThreads;
        if (i < npad) key[i] = i < n ? ((uint32_t)c[k] << kTinyIdBits) | (uint32_t)i : 0xffffffffu;
      }
    }
    __syncthreads();
    // rank(x) = #{y : key(y) < key(x)}: lane l takes vertex xb + l, warp w the keys [w * per, (w + 1) * per)
    const int per4 = npad / (4 * kTinyWarps);
    const uint4* mine = reinterpret_cast<const uint4*>(key) + warp * per4;
    for (int xb = blockIdx.x * 32; xb < n; xb += gridDim.x * 32) {
      const int x = xb + lane;
      const uint32_t kx = x < n ? key[x] : 0u;
      uint32_t c0 = 0, c1 = 0;
      for (int j = 0; j < per4; ++j) {
        const uint4 v = mine[j];
        c0 += (v.x < kx ? 1u : 0u) + (v.y < kx ? 1u : 0u);
        c1 += (v.z < kx ? 1u : 0u) + (v.w < kx ? 1u : 0u);
      }
      part[warp * 32 + lane] = c0 + c1;
      __syncthreads();
      if (warp == 0 && x < n) {
        uint32_t r = 0;
        for (int w = 0; w < kTinyWarps; ++w) r += part[w * 32 + lane];
        a.rank[x] = (int32_t)r;
        a.perm[r] = x;
      }
      __syncthreads();
    }
    // bucket starts: room for each vertex's input-pair count, one atomic claim per warp of 32 vertices
    for (int xb = gwarp * 32; xb < n; xb += nwarps * 32) {
      const int x = xb + lane;
      const uint32_t c = x < n ? key[x] >> kTinyIdBits : 0u;
      const uint32_t incl = warp_inclusive_scan(c);
      uint32_t base = 0;
      if (lane == 31 && incl) base = atomicAdd(&a.ctl->alloc, incl);
      base = __shfl_sync(kFull, base, 31) + incl - c;
      if (x < n) {
        a.bstart[x] = base;
        a.cur[x] = base;
      }
    }
  }
  if (!grid_barrier(a.ctl, 0)) return;

  // ---- 1: buckets (four pairs per thread, their chains of accesses side by side) ----
  {
    const uint64_t mask = (1ull << a.B) - 1ull;
    const uint64_t sentinel = (1ull << (2 * a.B)) - 1ull;
    constexpr int kItems = 4;
    const int64_t stride = (int64_t)gridDim.x * kTinyThreads;
    for (int64_t i0 = (int64_t)blockIdx.x * kTinyThreads + tid; i0 < M; i0 += kItems * stride) {
      uint64_t k[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) k[j] = i0 + j * stride < M ? __ldg(&a.keys[i0 + j * stride]) : sentinel;
      int32_t ra[kItems], rb[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        ra[j] = k[j] != sentinel ? a.rank[k[j] >> a.B] : 0;
        rb[j] = k[j] != sentinel ? a.rank[k[j] & mask] : 0;
      }
      uint32_t slot[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (k[j] != sentinel) slot[j] = atomicAdd(&a.cur[ra[j] < rb[j] ? k[j] >> a.B : k[j] & mask], 1u);
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (k[j] != sentinel) a.tgt[slot[j]] = ra[j] < rb[j] ? rb[j] : ra[j];
    }
  }
  if (!grid_barrier(a.ctl, 1)) return;

  // ---- 2: rows sorted and de-duplicated, d+(u) and the row codes ----
  {
    const unsigned lt = lanemask_lt();
    uint32_t* bm = smem + warp * kTinyRowWords;
    unsigned long long msum = 0;
    for (int x = gwarp; x < n; x += nwarps) {
      const uint32_t ps = a.bstart[x];
      const int L = (int)(a.cur[x] - ps);
      const int u = a.rank[x];
      int32_t* row = a.tgt + ps;
      int dd;
      if (L <= 1) {
        dd = L;
      } else if (L <= 32) {
        int32_t v = lane < L ? row[lane] : INT_MAX;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
          for (int j = kk >> 1; j > 0; j >>= 1) {
            const int32_t y = __shfl_xor_sync(kFull, v, j);
            v = (((lane & j) == 0) == ((lane & kk) == 0)) ? min(v, y) : max(v, y);
          }
        }
        const int32_t prev = __shfl_up_sync(kFull, v, 1);
        const bool keep = v != INT_MAX && (lane == 0 || v != prev);
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) row[__popc(km & lt)] = v;
        dd = __popc(km);
      } else {  // targets lie in (u, n): a bitmap over that range
        const int range = n - 1 - u;
        const int words = (range + 31) >> 5;
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        __syncwarp();
        for (int i = lane; i < L; i += 32) {
          const int b = row[i] - u - 1;
          atomicOr(&bm[b >> 5], 1u << (b & 31));
        }
        __syncwarp();
        const int per = (words + 31) >> 5;
        const int w0 = min(words, lane * per), w1 = min(words, w0 + per);
        uint32_t c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
        const uint32_t incl = warp_inclusive_scan(c);
        uint32_t pos = incl - c;
        dd = (int)__shfl_sync(kFull, incl, 31);
        for (int w = w0; w < w1; ++w) {
          uint32_t bits = bm[w];
          while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            row[pos++] = u + 1 + w * 32 + b;
          }
        }
        __syncwarp();
      }
      if (lane == 0) {
        // the window is every vertex (base 0): dense when it has enough entries for its bitmap quads
        int32_t code = (dd + 3) & ~3;
        const int32_t q = a.wtopq - (int32_t)((u + 1) >> 7);
        if (dd >= kDenseMinDegree && 4 * (int64_t)q <= dd) code = -q;
        a.rowinfo[u] = make_int2(dd, code);
        a.rstart[u] = ps;
        msum += (unsigned long long)dd;
      }
    }
    if (lane == 0 && msum) atomicAdd(&s_acc[0], msum);
  }
  if (!grid_barrier(a.ctl, 2)) return;

  // ---- 3: the CSR rows, bins and dense bitmaps of this CTA's ranks [r0, r1) ----
  {
    const int R = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = min(n, (int)blockIdx.x * R), r1 = min(n, r0 + R);
    uint32_t* s_off = smem;                                       // [R] row offsets
    int32_t* s_dq = reinterpret_cast<int32_t*>(smem + R);         // [R] dense row starts, or -1
    int32_t* lb = reinterpret_cast<int32_t*>(smem + 2 * R);       // [3][R] bin entries: block, warp, thread
    // the sizes of every row below r0, then a scan over this CTA's rows (R <= kTinyThreads)
    unsigned long long below = 0;
    for (int r = tid; r < r0; r += kTinyThreads) below += row_sizes(a.rowinfo[r]);
    below = warp_sum(below);
    if (lane == 0) ws64[warp] = below;
    __syncthreads();
    unsigned long long prefix = 0;
    for (int w = 0; w < kTinyWarps; ++w) prefix += ws64[w];
    __syncthreads();
    const int r = r0 + tid;
    const unsigned long long mine = r < r1 ? row_sizes(a.rowinfo[r]) : 0ull;
    unsigned long long total;
    const unsigned long long pos = prefix + block_exclusive_scan<unsigned long long>(mine, ws64, &total);
    uint32_t dense_here = 0;
    if (r < r1) {
      s_off[tid] = (uint32_t)(pos >> 32);
      const bool dense = (uint32_t)mine != 0u;
      s_dq[tid] = dense ? (int32_t)(uint32_t)pos : -1;
      a.off[r] = (int64_t)(pos >> 32);
      a.dq0[r] = dense ? (int32_t)(uint32_t)pos : -1;
      dense_here = dense ? 1u : 0u;
    }
    dense_here = warp_sum(dense_here);
    if (lane == 0 && dense_here) atomicAdd(&a.sizes->dense_rows, (unsigned long long)dense_here);
    if (r0 < r1 && r1 == n) {  // the CTA holding the last rank: the totals and the spare quad after the last row
      const unsigned long long all = prefix + total;
      const uint32_t tp = (uint32_t)(all >> 32);
      if (tid < 4) a.col[tp + tid] = n;
      if (tid == 0) {
        a.off[n] = tp;
        a.sizes->entries = tp;
        a.sizes->dquads = (uint32_t)all;
      }
    }
    __syncthreads();
    unsigned long long wsum = 0, act = 0, dw = 0, dv = 0;
    int dmax = 0;
    for (int u = r0 + warp; u < r1; u += kTinyWarps) {
      const uint32_t ps = a.rstart[u];
      const int2 ri = a.rowinfo[u];
      const int d = ri.x;
      const int pl = (d + 3) & ~3;
      const int64_t o = s_off[u - r0];
      RowWork w;
      for (int j = lane; j < pl; j += 32) {
        int32_t v = n;
        if (j < d) {
          v = a.tgt[ps + j];
          w.add(a.rowinfo[v]);
        }
        a.col[o + j] = v;
      }
      const int64_t wpad = warp_sum(w.pad), wtrue = warp_sum(w.wtrue);
      const int64_t wdense = warp_sum(w.wdense), qdense = warp_sum(w.qdense);
      if (ri.y < 0) {  // its dense row: zeroed, then its bits
        const int32_t q0 = s_dq[u - r0], nq = -ri.y;
        uint4* qz = reinterpret_cast<uint4*>(a.dense) + q0;
        for (int j = lane; j < nq; j += 32) qz[j] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        const int64_t w0 = 4 * (int64_t)q0 - 4 * (int64_t)((u + 1) >> 7);
        for (int j = lane; j < d; j += 32) {
          const int32_t b = a.tgt[ps + j];
          atomicOr(&a.dense[w0 + (b >> 5)], 1u << (b & 31));
        }
      }
      if (lane == 0) {
        wsum += (unsigned long long)wtrue;
        dw += (unsigned long long)wdense;
        dv += (unsigned long long)qdense;
        dmax = max(dmax, d);
        const bool keep = d >= 2 && wtrue > 0;
        const bool tny = keep && d <= kTinyMaxDegree && 8 * (int64_t)d * (d - 1) <= wpad;
        const bool blk = keep && !tny && wpad > a.block_min_work;
        act += keep ? 1 : 0;
        if (keep) {
          const int which = blk ? 0 : (tny ? 2 : 1);
          lb[which * R + atomicAdd(&s_cnt[which], 1u)] = u;
        }
      }
    }
    if (lane == 0) {
      if (wsum) atomicAdd(&s_acc[1], wsum);
      if (act) atomicAdd(&s_acc[2], act);
      if (dw) atomicAdd(&s_acc[3], dw);
      if (dv) atomicAdd(&s_acc[4], dv);
      if (dmax) atomicMax(&s_acc[5], (unsigned long long)dmax);
    }
    __syncthreads();
    BinCounters* bc = &a.sizes->bc;
    if (tid == 0) {
      s_base[0] = s_cnt[0] ? atomicAdd(&bc->nb, s_cnt[0]) : 0u;
      s_base[1] = s_cnt[1] ? atomicAdd(&bc->nw, s_cnt[1]) : 0u;
      s_base[2] = s_cnt[2] ? atomicAdd(&bc->nt, s_cnt[2]) : 0u;
      if (s_acc[0]) atomicAdd(&a.sizes->rc.m, s_acc[0]);
      if (s_acc[1]) atomicAdd(&bc->wedges, s_acc[1]);
      if (s_acc[2]) atomicAdd(&bc->active, s_acc[2]);
      if (s_acc[3]) atomicAdd(&bc->dense_wedges, s_acc[3]);
      if (s_acc[4]) atomicAdd(&bc->dense_visits, s_acc[4]);
      if (s_acc[5]) atomicMax(&bc->max_out, (int)s_acc[5]);
    }
    __syncthreads();
    for (uint32_t i = tid; i < s_cnt[0]; i += kTinyThreads) a.list[s_base[0] + i] = lb[i];
    for (uint32_t i = tid; i < s_cnt[1]; i += kTinyThreads) a.list[n - 1 - (s_base[1] + i)] = lb[R + i];
    for (uint32_t i = tid; i < s_cnt[2]; i += kTinyThreads) a.tlist[s_base[2] + i] = lb[2 * R + i];
  }
}

// Dynamic shared memory of a launch: every key and the warps' partial counts (step 0), the warps' bitmaps (step 2),
// a CTA's offsets, dense starts and bin entries (step 3), whichever is largest.
size_t tiny_smem_bytes(int64_t n, int grid) {
  const size_t npad = (size_t)((n + 4 * kTinyWarps - 1) & ~int64_t(4 * kTinyWarps - 1));
  const size_t ranks = (npad + (size_t)kTinyWarps * 32) * 4;
  const size_t bitmaps = (size_t)kTinyWarps * kTinyRowWords * 4;
  const size_t rows = 5 * (size_t)((n + grid - 1) / grid) * 4;
  size_t b = ranks > bitmaps ? ranks : bitmaps;
  return b > rows ? b : rows;
}

constexpr size_t kTinySmemMax = (kTinyMaxVertices + kTinyWarps * 32) * 4;  // 68 KB

// CTAs of a launch: a warp per row and a thread per pair at most, no more than can be resident at once.
int tiny_grid(int64_t n, int64_t M) {
  static std::atomic<int> per_sm_cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int per_sm = (dev >= 0 && dev < 64) ? per_sm_cache[dev].load(std::memory_order_relaxed) : 0;
  if (per_sm == 0) {
    if (smem_attribute_once<k_tiny_build>((int)kTinySmemMax) != TC_OK) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiny_build, kTinyThreads, kTinySmemMax) !=
        cudaSuccess)
      return 0;
    if (dev >= 0 && dev < 64) per_sm_cache[dev].store(per_sm, std::memory_order_relaxed);
  }
  const int64_t want_rows = (n + kTinyWarps - 1) / kTinyWarps;
  const int64_t want_pairs = (M + kTinyThreads - 1) / kTinyThreads;
  int64_t g = want_rows > want_pairs ? want_rows : want_pairs;
  const int64_t cap = (int64_t)per_sm * num_sms();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  // step 3 scans a CTA's ranks with one per thread
  return (n + g - 1) / g <= kTinyThreads ? (int)g : 0;
}

}  // namespace

bool tiny_eligible(int64_t n, int64_t pairs) {
  const int64_t cap = tiny_max_pairs();
  if (!(n > 0 && n <= kTinyMaxVertices && pairs > 0 && pairs <= cap && pairs <= kTinyMaxPairs)) return false;
  // the device must hold the launch's CTAs at once with their shared memory
  const int grid = tiny_grid(n, pairs);
  if (grid <= 0) (void)cudaGetLastError();
  return grid > 0 && tiny_smem_bytes(n, grid) <= kTinySmemMax;
}

namespace {

// A small graph's one block: the head (sizes and barrier word), the ingest error word and the input-pair counts
// (cleared together), the keys, the count words, the build's scratch, and the CSR views.  The same n and M give
// the same layout, so ingest and build each lay it out again over the block.
struct TinyLayout {
  TinyHead* head;
  uint32_t* err;
  size_t clear_bytes;  // head, error word and counts
  TinyArgs a;          // scratch and CSR pointers filled in
};

// The build's scratch: ranks, bucket starts and cursors by id, row starts and codes by rank, bucket targets.
void tiny_scratch(Arena& ar, TinyArgs& a, int64_t n, int64_t M) {
  a.rank = ar.take<int32_t>(n);
  a.bstart = ar.take<uint32_t>(n);
  a.cur = ar.take<uint32_t>(n);
  a.rstart = ar.take<uint32_t>(n);
  a.rowinfo = ar.take<int2>(n);
  a.tgt = ar.take<int32_t>(2 * M);
}

TinyLayout tiny_layout(Arena& ar, tc_graph* g, int64_t n, int64_t M) {
  TinyLayout L{};
  L.head = ar.take<TinyHead>(1);
  L.err = ar.take<uint32_t>(4);
  g->indeg = ar.view((size_t)n * 4);
  L.clear_bytes = ar.used;
  g->keys = ar.view((size_t)M * 8);
  g->acc = ar.view(64);
  tiny_scratch(ar, L.a, n, M);
  csr_views(ar, g, n, M + 3 * (n < M ? n : M), n, M / 4 + 1);
  L.a.sizes = L.head ? &L.head->sz : nullptr;
  L.a.ctl = L.head ? &L.head->ctl : nullptr;
  return L;
}

}  // namespace

tc_status tiny_ingest(tc_graph* g, uint32_t** d_err, cudaStream_t s) {
  Arena sizing;
  tiny_layout(sizing, g, g->n, g->num_pairs);
  TC_TRY(buf_alloc(g->alloc, g->block, sizing.used, s));
  Arena ar{g->block.as<char>()};
  const TinyLayout L = tiny_layout(ar, g, g->n, g->num_pairs);
  TC_CUDA(cudaMemsetAsync(g->block.p, 0, L.clear_bytes, s));
  *d_err = L.err;
  g->tiny = true;
  return TC_OK;
}

tc_status build_graph_tiny(tc_graph* g, cudaStream_t s) {
  const Allocator& al = g->alloc;
  const int64_t M = g->num_pairs;
  const int64_t n = g->n;
  tc_status st = TC_OK;
  const int64_t bound_entries = M + 3 * (n < M ? n : M);
  const int64_t bound_quads = M / 4 + 1;
  const int grid = tiny_grid(n, M);
  if (grid <= 0 || tiny_smem_bytes(n, grid) > kTinySmemMax) {
    set_error("tc_build: the device cannot hold the one-launch build");
    return TC_ERR_CUDA;
  }
  Buf scratch;
  do {
    TinyHead* head;
    TinyArgs a{};
    if (g->tiny) {  // laid out at ingest, head cleared there
      Arena ar{g->block.as<char>()};
      const Buf keys = g->keys, indeg = g->indeg;
      const TinyLayout L = tiny_layout(ar, g, n, M);
      g->keys = keys;
      g->indeg = indeg;
      head = L.head;
      a = L.a;
    } else {  // keys and counts from elsewhere (tc_count_many): the scratch and the CSR block allocated here
      Arena sizing;
      sizing.take<TinyHead>(1);
      tiny_scratch(sizing, a, n, M);
      if ((st = buf_alloc(al, scratch, sizing.used, s))) break;
      Arena sa{scratch.as<char>()};
      head = sa.take<TinyHead>(1);
      a.sizes = &head->sz;
      a.ctl = &head->ctl;
      tiny_scratch(sa, a, n, M);
      Arena bsizing;
      csr_views(bsizing, g, n, bound_entries, n, bound_quads);
      if ((st = buf_alloc(al, g->block, bsizing.used, s))) break;
      Arena ba{g->block.as<char>()};
      csr_views(ba, g, n, bound_entries, n, bound_quads);
      if ((st = cuda_status(cudaMemsetAsync(head, 0, sizeof(TinyHead), s), "memset sizes"))) break;
    }
    a.keys = g->keys.as<uint64_t>();
    a.indeg = g->indeg.as<int32_t>();
    a.M = M;
    a.n = (int32_t)n;
    a.B = g->key_bits;
    a.wtopq = (int32_t)(((n - 1) >> 7) + 1);
    a.block_min_work = block_min_work_for(M);
    a.off = g->off.as<int64_t>();
    a.col = g->col.as<int32_t>();
    a.perm = g->perm.as<int32_t>();
    a.list = g->list.as<int32_t>();
    a.tlist = g->tlist.as<int32_t>();
    a.dq0 = g->dq0.as<int32_t>();
    a.dense = g->dense.as<uint32_t>();
    void* params[] = {&a};
    if ((st = cuda_status(cudaLaunchCooperativeKernel((const void*)k_tiny_build, dim3(grid), dim3(kTinyThreads),
                                                      params, tiny_smem_bytes(n, grid), s),
                          "k_tiny_build")))
      break;
    note_launch();
    // ---- the sizes and the barrier word at once, then the one synchronisation ----
    TinyHead* hb = reinterpret_cast<TinyHead*>(g->host_total + 1);
    if ((st = cuda_status(cudaMemcpyAsync(hb, head, sizeof(TinyHead), cudaMemcpyDeviceToHost, s), "copy sizes")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "tc_build sync"))) break;
    if (hb->ctl.err) {
      set_error("tc_build: a grid barrier of the one-launch build gave up waiting");
      st = TC_ERR_INTERNAL;
      break;
    }
    if (hb->sz.entries > bound_entries || hb->sz.dquads > bound_quads) {
      set_error("tc_build: the one-launch build's size bounds were exceeded");
      st = TC_ERR_INTERNAL;
      break;
    }
    apply_sizes(g, hb->sz);
  } while (0);
  buf_release(al, scratch, s);
  buf_release(al, g->keys, s);
  buf_release(al, g->indeg, s);
  buf_release(al, g->ingest, s);
  return st;
}

}  // namespace tc

// tc_count.cuh — device side of the fused two-hop traversal with the closing-edge test.
//
// For a source u (Algorithm 1's verification loop, specialised to Q = K3 and fused into one pass):
//   hop 1   v ranges over N+(u)                      (Advance from the candidate set, Sec. III-A/III-B)
//   hop 2   w ranges over N+(v)                      (the second Advance of the spanning path u-v-w)
//   verify  keep u->v->w iff w is in N+(u)           (the stored non-tree edge u-w, Sec. III-A)
// Nothing is materialised: the 2-paths live in registers only, so Algorithm 1's Compute / Write_to_Partial /
// Mask steps, which exist to store and compact intermediate matches, have no counterpart here.
//
// N+(u) is put in shared memory as a set (a hash table with linear probing, or a bitmap over [0, n) when n is
// small; for very large N+(u), binary search in the sorted global row) and every w is tested against it.
//
// Load balance inside a source: the rows N+(v), v in N+(u), are concatenated and cut into 16-byte quads of the
// column array (a row [rs, re) covers quads rs/4 .. (re-1)/4; elements outside the row are masked).  A warp walks
// this quad stream 32 quads at a time, one int4 load per lane, so short rows do not leave lanes idle.  The row
// that owns a lane's quad is found without a search: with the rows' quad prefix P (strictly increasing, empty
// rows removed), the lanes that hold the next 32 rows OR together one bit per row start inside the window, and a
// lane's owner is the current row plus the number of starts below it (a popcount).
#pragma once

#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace dev {

// Row descriptors in shared memory (structure of arrays).  Row k covers quads [q0, q0 + P[k+1] - P[k]) of the
// column array and, inside that span, elements [lo, hi) (relative to 4*q0).
struct Rows {
  uint32_t* q0;
  uint32_t* P;
  uint32_t* lo;
  uint32_t* hi;
  int32_t* v;
};

// Fibonacci hashing of a vertex id into 2^bits slots.
struct HashSet {
  int32_t* tab;
  uint32_t mask;
  int shift;
  __device__ __forceinline__ uint32_t slot(int32_t k) const { return ((uint32_t)k * 2654435761u) >> shift; }
  // The table always has more than twice as many slots as keys, so the probe sequences below end.
  __device__ __forceinline__ void insert(int32_t k) const {
    uint32_t s = slot(k);
    while (true) {
      const int32_t old = atomicCAS(&tab[s], -1, k);
      if (old == -1) return;
      s = (s + 1) & mask;
    }
  }
  __device__ __forceinline__ bool contains(int32_t k) const {
    uint32_t s = slot(k);
    while (true) {
      const int32_t x = tab[s];
      if (x == k) return true;
      if (x < 0) return false;
      s = (s + 1) & mask;
    }
  }
};

struct BitSet {
  uint32_t* bm;
  __device__ __forceinline__ void insert(int32_t k) const { atomicOr(&bm[k >> 5], 1u << (k & 31)); }
  __device__ __forceinline__ bool contains(int32_t k) const { return (bm[k >> 5] >> (k & 31)) & 1u; }
};

// Closing test by binary search in the sorted global row N+(u) (rows too long for shared memory).
struct SortedGlobal {
  const int32_t* a;
  int32_t len;
  __device__ __forceinline__ bool contains(int32_t k) const {
    int lo = 0, hi = len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(&a[mid]) < k)
        lo = mid + 1;
      else
        hi = mid;
    }
    return lo < len && __ldg(&a[lo]) == k;
  }
};

template <bool PV, class Set>
__device__ __forceinline__ void test_one(int32_t w, int e, uint32_t lo, uint32_t hi, const Set& set,
                                         uint32_t& hits, unsigned long long* pv, int32_t v) {
  if ((uint32_t)e >= lo && (uint32_t)e < hi && set.contains(w)) {
    ++hits;
    if (PV) {
      atomicAdd(&pv[w], 1ull);
      atomicAdd(&pv[v], 1ull);
    }
  }
}

// Walk quads [x0, x1) of the concatenated rows 0..R-1 with one warp.  Returns this lane's number of closed
// 2-paths.
template <bool PV, class Set>
__device__ __forceinline__ uint32_t walk(const Rows& r, int R, uint32_t x0, uint32_t x1,
                                         const int4* __restrict__ col4, const Set& set, unsigned long long* pv) {
  uint32_t hits = 0;
  if (x0 >= x1) return 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  // cur = last row with P <= x0
  int a = 0, b = R;
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (r.P[mid] <= x0)
      a = mid + 1;
    else
      b = mid;
  }
  int cur = a - 1;
  for (uint32_t base = x0; base < x1; base += 32) {
    // lane l (l >= 1) looks at row cur + l, lane 0 at row cur + 32: the rows that may start in (base, base+32]
    const int j = cur + (lane == 0 ? 32 : lane);
    uint32_t bit = 0;
    if (j < R) {
      const uint32_t pj = r.P[j];
      if (pj <= base + 32) bit = 1u << (pj - base - 1);
    }
    const uint32_t starts = __reduce_or_sync(kFull, bit);
    const uint32_t x = base + lane;
    if (x < x1) {
      const int own = cur + __popc(starts & lt);
      const uint32_t rel = x - r.P[own];
      const int4 q = __ldg(&col4[r.q0[own] + rel]);
      const uint32_t lo = r.lo[own], hi = r.hi[own];
      const int32_t v = PV ? r.v[own] : 0;
      const int e = 4 * (int)rel;
      test_one<PV>(q.x, e + 0, lo, hi, set, hits, pv, v);
      test_one<PV>(q.y, e + 1, lo, hi, set, hits, pv, v);
      test_one<PV>(q.z, e + 2, lo, hi, set, hits, pv, v);
      test_one<PV>(q.w, e + 3, lo, hi, set, hits, pv, v);
    }
    cur += __popc(starts);
  }
  return hits;
}

// Row descriptor of v (or an empty row for v < 0).
struct RowOf {
  uint32_t q0, nq, lo, hi;
  bool nonempty;
};
__device__ __forceinline__ RowOf row_of(const int64_t* __restrict__ off, int32_t v) {
  RowOf r{0, 0, 0, 0, false};
  if (v >= 0) {
    const int64_t rs = __ldg(&off[v]), re = __ldg(&off[v + 1]);
    if (re > rs) {
      r.nonempty = true;
      r.q0 = (uint32_t)(rs >> 2);
      r.nq = (uint32_t)(((re + 3) >> 2) - (rs >> 2));
      r.lo = (uint32_t)(rs - 4 * (rs >> 2));
      r.hi = (uint32_t)(re - 4 * (rs >> 2));
    }
  }
  return r;
}

// One source u, one warp.  `set` is the warp's private, empty set; it is emptied again before returning.
template <bool PV, class Set>
__device__ __forceinline__ uint32_t warp_source(int32_t u, const CsrView& g, const Set& set, uint32_t* words,
                                                int nwords, uint32_t empty_word, const Rows& r,
                                                unsigned long long* pv) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t beg = __ldg(&g.off[u]), end = __ldg(&g.off[u + 1]);
  const int d = (int)(end - beg);
  for (int i = lane; i < d; i += 32) set.insert(__ldg(&g.col[beg + i]));
  __syncwarp();
  uint32_t hits = 0;
  const int4* col4 = reinterpret_cast<const int4*>(g.col);
  for (int vb = 0; vb < d; vb += 32) {
    const int j = vb + lane;
    const int32_t v = j < d ? __ldg(&g.col[beg + j]) : -1;
    const RowOf ro = row_of(g.off, v);
    const unsigned ne = __ballot_sync(kFull, ro.nonempty);
    const uint32_t incl = warp_inclusive_scan(ro.nq);
    const uint32_t Q = __shfl_sync(kFull, incl, 31);
    if (ro.nonempty) {
      const int k = __popc(ne & lt);
      r.q0[k] = ro.q0;
      r.P[k] = incl - ro.nq;
      r.lo[k] = ro.lo;
      r.hi[k] = ro.hi;
      if (PV) r.v[k] = v;
    }
    __syncwarp();
    hits += walk<PV>(r, __popc(ne), 0, Q, col4, set, pv);
    __syncwarp();
  }
  for (int i = lane; i < nwords; i += 32) words[i] = empty_word;
  __syncwarp();
  if (PV) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) atomicAdd(&pv[u], (unsigned long long)s);
  }
  return hits;
}

// One source u, the whole block.  `tab` is the block's hash region (kBlockHashSlotsMax slots, all -1 on entry and
// on return); `ws` is shared scratch for block scans (32 entries).
template <bool PV>
__device__ __forceinline__ uint32_t block_source(int32_t u, const CsrView& g, int32_t* tab, const Rows& r,
                                                 uint32_t* ws, unsigned long long* pv) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t beg = __ldg(&g.off[u]), end = __ldg(&g.off[u + 1]);
  const int d = (int)(end - beg);
  const bool wide = d > kBlockMaxDeg;
  int slots = 256, bits = 8;
  while (slots < 2 * d && slots < kBlockHashSlotsMax) {
    slots <<= 1;
    ++bits;
  }
  const HashSet hs{tab, (uint32_t)(slots - 1), 32 - bits};
  const SortedGlobal gs{g.col + beg, d};
  if (!wide)
    for (int i = tid; i < d; i += kCountThreads) hs.insert(__ldg(&g.col[beg + i]));
  __syncthreads();
  uint32_t hits = 0;
  const int4* col4 = reinterpret_cast<const int4*>(g.col);
  for (int cb = 0; cb < d; cb += kBlockRows) {
    const int j = cb + tid;
    const int32_t v = j < d ? __ldg(&g.col[beg + j]) : -1;
    const RowOf ro = row_of(g.off, v);
    uint32_t R, Q;
    const uint32_t rank = block_exclusive_scan<uint32_t>(ro.nonempty ? 1u : 0u, ws, &R);
    const uint32_t pre = block_exclusive_scan<uint32_t>(ro.nq, ws, &Q);
    if (ro.nonempty) {
      r.q0[rank] = ro.q0;
      r.P[rank] = pre;
      r.lo[rank] = ro.lo;
      r.hi[rank] = ro.hi;
      if (PV) r.v[rank] = v;
    }
    __syncthreads();
    const uint32_t per = (Q + kWarpsPerCTA - 1) / kWarpsPerCTA;
    const uint32_t x0 = min(Q, (uint32_t)warp * per), x1 = min(Q, x0 + per);
    if (wide)
      hits += walk<PV>(r, (int)R, x0, x1, col4, gs, pv);
    else
      hits += walk<PV>(r, (int)R, x0, x1, col4, hs, pv);
    __syncthreads();
  }
  if (!wide)
    for (int i = tid; i < slots; i += kCountThreads) tab[i] = -1;
  if (PV) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) atomicAdd(&pv[u], (unsigned long long)s);
  }
  __syncthreads();
  return hits;
}

// Shared-memory layout of the counting kernel.
constexpr int kBlockRowBytes = kBlockRows * 4 * 4 + (kBlockRows + 1) * 4;
constexpr int kBlockSmem = kBlockHashSlotsMax * 4 + kBlockRowBytes;
constexpr int kWarpRowBytes = 32 * 4 * 4 + 33 * 4;
constexpr int kWarpRegion = kWarpHashSlots * 4 + kWarpRowBytes;
constexpr int kWarpSmem = kWarpsPerCTA * kWarpRegion;
constexpr int kCountSmem = kBlockSmem > kWarpSmem ? kBlockSmem : kWarpSmem;

__device__ __forceinline__ Rows rows_at(unsigned char* p, int cap) {
  Rows r;
  r.q0 = reinterpret_cast<uint32_t*>(p);
  r.lo = r.q0 + cap;
  r.hi = r.lo + cap;
  r.v = reinterpret_cast<int32_t*>(r.hi + cap);
  r.P = reinterpret_cast<uint32_t*>(r.v + cap);
  return r;
}

// Count the triangles of one graph, processing its block-bin sources first, then its warp-bin sources.
// cursors[0], cursors[1]: zeroed work counters of this graph.  Returns this thread's count.
template <bool PV>
__device__ __forceinline__ unsigned long long count_graph(const CsrView& g, unsigned long long* pv,
                                                          uint32_t* cursors, unsigned char* smem, uint32_t* ws,
                                                          int* s_idx) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned long long acc = 0;
  if (g.nb > 0) {
    int32_t* tab = reinterpret_cast<int32_t*>(smem);
    const Rows r = rows_at(smem + kBlockHashSlotsMax * 4, kBlockRows);
    for (int i = tid; i < kBlockHashSlotsMax; i += kCountThreads) tab[i] = -1;
    __syncthreads();
    while (true) {
      if (tid == 0) *s_idx = (int)atomicAdd(&cursors[0], 1u);
      __syncthreads();
      const int idx = *s_idx;
      __syncthreads();
      if (idx >= g.nb) break;
      acc += block_source<PV>(g.list[idx], g, tab, r, ws, pv);
    }
  }
  if (g.nw > 0) {
    unsigned char* region = smem + warp * kWarpRegion;
    const Rows r = rows_at(region + kWarpHashSlots * 4, 32);
    uint32_t* words = reinterpret_cast<uint32_t*>(region);
    const uint32_t empty = g.bitmap ? 0u : 0xffffffffu;
    for (int i = lane; i < kWarpHashSlots; i += 32) words[i] = empty;
    __syncwarp();
    const int32_t* wlist = g.list + (g.n - g.nw);
    constexpr int kChunk = 4;
    while (true) {
      int idx = 0;
      if (lane == 0) idx = (int)atomicAdd(&cursors[1], (unsigned)kChunk);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= g.nw) break;
      const int e = min(idx + kChunk, g.nw);
      for (int k = idx; k < e; ++k) {
        const int32_t u = wlist[k];
        if (g.bitmap)
          acc += warp_source<PV>(u, g, BitSet{words}, words, kWarpHashSlots, empty, r, pv);
        else
          acc += warp_source<PV>(u, g, HashSet{reinterpret_cast<int32_t*>(words), kWarpHashSlots - 1, 24}, words,
                                 kWarpHashSlots, empty, r, pv);
      }
    }
  }
  return acc;
}

}  // namespace dev
}  // namespace tc

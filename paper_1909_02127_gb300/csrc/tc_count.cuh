// tc_count.cuh — device side of the fused two-hop traversal with the closing-edge test.
//
// For a source u (Algorithm 1's verification loop, specialised to Q = K3 and fused into one pass):
//   hop 1   v ranges over N+(u)                      (Advance from the candidate set, Sec. III-A/III-B)
//   hop 2   w ranges over N+(v)                      (the second Advance of the spanning path u-v-w)
//   verify  keep u->v->w iff w is in N+(u)           (the stored non-tree edge u-w, Sec. III-A)
// Nothing is materialised: the 2-paths live in registers only, so Algorithm 1's Compute / Write_to_Partial /
// Mask steps, which exist to store and compact intermediate matches, have no counterpart here.
//
// Closing test.  Vertices are numbered by rank in the (input-pair count, id) order, so the ids that occur most
// often as w (targets of hub rows) are the highest ones.  N+(u) is marked in a shared-memory bitmap over the top ids
// [base, n] (4 KB per warp, or 64 KB per CTA for heavy sources); a test is one shared load and a bit extract.
// The entries of N+(u) below base (a prefix of the sorted row) go into a small shared-memory hash (128 slots per
// warp, 2048 per CTA), or, if they do not fit, are found by binary search in the row.  Pad entries (id n) fall
// on bit n - base, which is never set.
//
// Traversal.  Rows are 16-byte aligned and padded to whole quads, so every load is one aligned int4.  In warp mode
// rows of >= kLongQuads quads are walked by the whole warp, two 32-quad steps in flight; shorter rows are
// concatenated and cut into quads, and a warp walks this stream 32 quads at a time.  The row owning a lane's quad
// is found without a search: the lanes holding the next 32 rows OR together one bit per row start inside the
// window, and a lane's owner is the current row plus the number of starts below it (a popcount).  In block mode
// the long rows of a 512-row chunk are handed to warps one at a time from a shared-memory counter, so no warp
// waits at the chunk barrier behind another's long rows, and the short rows' stream is cut into equal shares.
// Dense hub rows are tested 128 ids at a time against the bitmap (dense_walk), and sources with few out-neighbours
// are counted one per lane by pairwise lookups (tiny_source).
#pragma once

#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace dev {

// Hash of a vertex id into 2^bits slots (Fibonacci hashing).
__device__ __forceinline__ uint32_t low_slot(int32_t k, uint32_t mask) {
  return (((uint32_t)k * 2654435761u) >> 16) & mask;
}

// How the entries of N+(u) below the bitmap window are looked up.
enum LowMode { kLowNone = 0, kLowHash = 1, kLowSearch = 2 };

// The closing-edge test against N+(u).
template <int LOW>
struct Closing {
  const uint32_t* bm;    // bit (x - base) set iff x in N+(u), for x in [base, n]
  int32_t base;
  const int32_t* low;    // kLowSearch: N+(u) entries below base (sorted, global); kLowHash: open-addressing table
  int32_t nlow;          // kLowSearch: number of entries; kLowHash: table mask
  uint32_t cap;          // bitmap size in bits: bit `cap` exists and is never set
  int32_t delta;         // quads from this bitmap's base to the warp window's base (dense rows line up there)
  __device__ __forceinline__ uint32_t bit(uint32_t t) const {
    return __funnelshift_r(bm[t >> 5], 0u, t) & 1u;  // shift amount taken mod 32
  }
  __device__ __forceinline__ uint32_t operator()(int32_t w) const {
    // w <= n always, so w - base <= cap; an id below base wraps to a huge value and is clamped to bit `cap`
    if (LOW == kLowNone) return bit(min((uint32_t)(w - base), cap));
    const int32_t t = w - base;
    if (t >= 0) return bit((uint32_t)t);
    if (LOW == kLowHash) {  // linear probing; the table is at most half full, so an empty slot ends the probe
      uint32_t s = low_slot(w, (uint32_t)nlow);
      while (true) {
        const int32_t x = low[s];
        if (x == w) return 1u;
        if (x < 0) return 0u;
        s = (s + 1) & (uint32_t)nlow;
      }
    }
    int a = 0, b = nlow;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (__ldg(&low[mid]) < w)
        a = mid + 1;
      else
        b = mid;
    }
    return (a < nlow && __ldg(&low[a]) == w) ? 1u : 0u;
  }
};

// Insert the low entries row[0..nlow) (distinct ids) into an empty table of mask+1 slots, mask+1 >= 2*nlow.
__device__ __forceinline__ void low_insert(const int32_t* __restrict__ row, int nlow, int32_t* tab, uint32_t mask,
                                           int t, int stride) {
  for (int i = t; i < nlow; i += stride) {
    const int32_t k = __ldg(&row[i]);
    uint32_t s = low_slot(k, mask);
    while (atomicCAS(&tab[s], -1, k) != -1) s = (s + 1) & mask;
  }
}

// What a closed 2-path produces besides the count.  The two per-vertex modes differ only in how they add to the
// per-CTA counters of the top ranks (vertex_add).
enum Mode { kModeCount = 0, kModeVertex = 1, kModeList = 2, kModeVertexChecked = 3 };
__host__ __device__ constexpr bool is_vertex(int mode) { return mode == kModeVertex || mode == kModeVertexChecked; }

struct Sink {
  unsigned long long* pv = nullptr;      // per-vertex modes: t(x) in rank space
  int32_t* tri = nullptr;                // kModeList: triples of original ids, 3 per triangle
  unsigned long long* slot = nullptr;    // kModeList: the next output position of this source (shared memory;
                                         // one per warp, or one per CTA in block mode), advanced atomically
  unsigned long long capacity = 0;       // kModeList: triples that fit in `tri`
  const int32_t* perm = nullptr;         // kModeList: rank -> original id
  int32_t u = 0;                         // kModeList: the current source
  int32_t pu = 0;                        // kModeList: its original id
  uint32_t* hub = nullptr;               // per-vertex modes: this CTA's counters of t(x), x in [hub0, n) (shared
  int32_t hub0 = 0;                      // memory)
};

// Per-vertex modes: per-CTA shared-memory counters for the top kHubRanks ranks.  Ranks follow the input-pair count,
// so these are the vertices in the most triangles, whose global counters would otherwise take most of the atomics
// (on R-MAT 20 the top 5120 ranks take 81% of all t(x) increments).  20 KB per CTA keeps two CTAs on an SM.
constexpr int kHubRanks = 5120;
constexpr uint32_t kHubSpill = 1u << 31;

// t(x) += k for x = v or w of closed 2-paths u->v->w (t(u) goes to pv directly, source_add).  A top rank counts in
// the CTA's shared counter, which the kernel adds to pv when it ends; any other x adds to pv directly.
//
// A source u adds at most d+(u) to any one counter as v (the hits of row v are N+(u) ∩ N+(v)) and at most d+(u) as w
// (the v in N+(u) whose row holds w), so over all sources no counter of any CTA takes more than 2m.  For m < 2^31
// (kModeVertex) a counter therefore never reaches 2^32, and the add needs no read-back: a shared-memory add whose
// old value is not returned is the cheaper instruction (R-MAT 20: per-vertex counting 7.1 -> 5.5 ms).  Otherwise
// (kModeVertexChecked) the add that takes a counter to 2^31 moves 2^31 of it to pv at once, so no counter wraps.
template <int MODE>
__device__ __forceinline__ void vertex_add(const Sink& sk, int32_t x, uint32_t k) {
  const int32_t h = x - sk.hub0;
  if (h < 0) {
    atomicAdd(&sk.pv[x], (unsigned long long)k);
  } else if (MODE == kModeVertex) {
    atomicAdd(&sk.hub[h], k);
  } else {
    const uint32_t old = atomicAdd(&sk.hub[h], k);
    if (old < kHubSpill && old + k >= kHubSpill) {
      atomicSub(&sk.hub[h], kHubSpill);
      atomicAdd(&sk.pv[x], (unsigned long long)kHubSpill);
    }
  }
}

// t(u) += k for a source u (once per source, or once per warp of a CTA's source).
__device__ __forceinline__ void source_add(const Sink& sk, int32_t u, unsigned long long k) { atomicAdd(&sk.pv[u], k); }

// kModeList: triangle (u, v, w) as its sorted original ids at output position pos (nothing past the capacity).
__device__ __forceinline__ void write_triple(const Sink& sk, unsigned long long pos, int32_t a, int32_t b,
                                             int32_t w) {
  if (pos >= sk.capacity) return;
  const int32_t c = __ldg(&sk.perm[w]);
  const int32_t lo = min(a, min(b, c)), hi = max(a, max(b, c));
  int32_t* t = sk.tri + 3 * pos;
  t[0] = lo;
  t[1] = a + b + c - lo - hi;
  t[2] = hi;
}

// Append the closed 2-paths u->v->w of this lane (h_i marks w_i) to the source's own range of the output (known
// from a counting pass): one shared-memory atomic on the source's position reserves the warp's run, and the i-th
// hits of all lanes go to consecutive positions in it (a ballot and a popcount each), so each round of stores
// covers one contiguous run.  Warp-collective: every lane calls it.
__device__ __forceinline__ void list_hits(const int4 q, uint32_t h0, uint32_t h1, uint32_t h2, uint32_t h3,
                                          const Sink& sk, int32_t v) {
  const unsigned b0 = __ballot_sync(kFull, h0), b1 = __ballot_sync(kFull, h1);
  const unsigned b2 = __ballot_sync(kFull, h2), b3 = __ballot_sync(kFull, h3);
  const uint32_t n0 = __popc(b0), n01 = n0 + __popc(b1), n012 = n01 + __popc(b2);
  const uint32_t total = n012 + __popc(b3);
  if (total == 0) return;
  unsigned long long base = 0;
  if ((threadIdx.x & 31) == 0) base = atomicAdd(sk.slot, (unsigned long long)total);
  base = __shfl_sync(kFull, base, 0);
  if (!(h0 | h1 | h2 | h3)) return;
  const unsigned lt = lanemask_lt();
  const int32_t b = __ldg(&sk.perm[v]);
  if (h0) write_triple(sk, base + __popc(b0 & lt), sk.pu, b, q.x);
  if (h1) write_triple(sk, base + n0 + __popc(b1 & lt), sk.pu, b, q.y);
  if (h2) write_triple(sk, base + n01 + __popc(b2 & lt), sk.pu, b, q.z);
  if (h3) write_triple(sk, base + n012 + __popc(b3 & lt), sk.pu, b, q.w);
}

// Position of the k-th (from 0) set bit of x, which has more than k set bits: halve the window five times by the
// population count of its lower half.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t x, uint32_t k) {
  uint32_t pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const uint32_t low = __popc(x & ((1u << w) - 1u));
    if (k >= low) {
      k -= low;
      x >>= w;
      pos += w;
    }
  }
  return pos;
}

// Append the closed 2-paths u->v->w whose w are the set bits of this lane's m0..m3 (bit j of m_i is w = w0 + 32i + j)
// as one run of the source's output, reserved with one shared-memory atomic.  The run is written 32 positions at a
// time, one per lane: lane l takes position t = t0 + l, finds the lane owning it by binary search over the lanes'
// inclusive prefix of bit counts, and the bit within that lane's 128 by population counts, so every pass stores 32
// consecutive triples however unevenly the bits fall across lanes.  Warp-collective.  Returns this lane's number of
// bits.
__device__ __forceinline__ uint32_t list_bits(uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3, int32_t w0,
                                              const Sink& sk, int32_t v) {
  const uint32_t cnt = (__popc(m0) + __popc(m1)) + (__popc(m2) + __popc(m3));
  const uint32_t incl = warp_inclusive_scan(cnt);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return 0;
  const int lane = threadIdx.x & 31;
  const int32_t pv = cnt ? __ldg(&sk.perm[v]) : 0;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(sk.slot, (unsigned long long)total);
  base = __shfl_sync(kFull, base, 0);
  for (uint32_t t0 = 0; t0 < total; t0 += 32) {
    const uint32_t t = t0 + lane;
    int o = 0;  // the owner: the number of lanes whose inclusive prefix is <= t (at most 31, as t < incl[31] or unused)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (__shfl_sync(kFull, incl, o + step - 1) <= t) o += step;
    const uint32_t k = t - (__shfl_sync(kFull, incl, o) - __shfl_sync(kFull, cnt, o));
    const uint32_t a0 = __shfl_sync(kFull, m0, o), a1 = __shfl_sync(kFull, m1, o);
    const uint32_t a2 = __shfl_sync(kFull, m2, o), a3 = __shfl_sync(kFull, m3, o);
    const int32_t ow0 = __shfl_sync(kFull, w0, o), opv = __shfl_sync(kFull, pv, o);
    if (t < total) {
      const uint32_t p0 = __popc(a0), p1 = p0 + __popc(a1), p2 = p1 + __popc(a2);
      int32_t w;
      if (k < p0)
        w = ow0 + (int32_t)nth_set_bit(a0, k);
      else if (k < p1)
        w = ow0 + 32 + (int32_t)nth_set_bit(a1, k - p0);
      else if (k < p2)
        w = ow0 + 64 + (int32_t)nth_set_bit(a2, k - p1);
      else
        w = ow0 + 96 + (int32_t)nth_set_bit(a3, k - p2);
      write_triple(sk, base + t, sk.pu, opv, w);
    }
  }
  return cnt;
}

template <int MODE, class C>
__device__ __forceinline__ uint32_t test_quad(const int4 q, const C& c, const Sink& sk, int32_t v) {
  const uint32_t h0 = c(q.x), h1 = c(q.y), h2 = c(q.z), h3 = c(q.w);
  if (is_vertex(MODE)) {  // t(w) here; the caller adds the row's hits to t(v)
    if (h0) vertex_add<MODE>(sk, q.x, 1u);
    if (h1) vertex_add<MODE>(sk, q.y, 1u);
    if (h2) vertex_add<MODE>(sk, q.z, 1u);
    if (h3) vertex_add<MODE>(sk, q.w, 1u);
    return (h0 + h1) + (h2 + h3);
  }
  if (MODE == kModeList) list_hits(q, h0, h1, h2, h3, sk, v);
  return (h0 + h1) + (h2 + h3);
}

// One long row (quads [q0, q0 + nq)) walked by the calling warp in windows of 64 quads, two independent loads in
// flight per lane (measured faster than four: fewer registers and a cheaper tail).  Trip counts and branches
// depend only on nq, so the warp never diverges; in the last window a lane whose quad lies past the row tests the
// pad id n (never a member) instead of loading.
template <int MODE, class C>
__device__ __forceinline__ uint32_t long_row(const int4* __restrict__ col4, uint32_t q0, uint32_t nq, const C& c,
                                             const Sink& sk, int32_t v, int32_t pad) {
  const uint32_t lane = threadIdx.x & 31;
  const int4* p = col4 + q0 + lane;
  uint32_t hits = 0;
  uint32_t rem = nq;
  for (; rem >= 64; rem -= 64, p += 64) {
    const int4 a = __ldg(p), b = __ldg(p + 32);
    hits += test_quad<MODE>(a, c, sk, v) + test_quad<MODE>(b, c, sk, v);
  }
  if (rem > 0) {
    const int4 none = make_int4(pad, pad, pad, pad);
    const int4 a = lane < rem ? __ldg(p) : none;
    if (rem > 32) {
      const int4 b = lane + 32 < rem ? __ldg(p + 32) : none;
      hits += test_quad<MODE>(a, c, sk, v) + test_quad<MODE>(b, c, sk, v);
    } else {
      hits += test_quad<MODE>(a, c, sk, v);
    }
  }
  if (is_vertex(MODE)) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) vertex_add<MODE>(sk, v, s);
  }
  return hits;
}

// ---- long rows staged through shared memory by cp.async -------------------------------------------------------
// Where the graph does not fit in L2, hop-2 rows come from DRAM, and a warp walking a long row with plain loads has
// one window of loads in flight, then none while it tests them.  The staged walk keeps the next steps' quads in
// flight instead, in a ring of shared memory filled by asynchronous copies, at no cost in registers.
__device__ __forceinline__ void cp_async_quad(int4* smem_dst, const int4* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One long row (quads [q0, q0 + nq)) walked by the calling warp 32 quads per step, with the quads of the next S - 1
// steps in flight: step k's quads go to slot k mod S of `ring` (S x 32 quads of this warp's shared memory, lane l
// using entry l of each slot).  Each lane copies and later reads only its own quads, so the only wait is for the
// lane's own copy group; a slot is refilled one step after it was read and tested.  A lane whose quad lies past
// the row copies nothing and tests the pad id.
template <int MODE, int S, class C>
__device__ __forceinline__ uint32_t long_row_staged(const int4* __restrict__ col4, uint32_t q0, uint32_t nq,
                                                    const C& c, const Sink& sk, int32_t v, int32_t pad, int4* ring) {
  const uint32_t lane = threadIdx.x & 31;
  const int4* p = col4 + q0 + lane;
  int4* slot = ring + lane;
  const uint32_t steps = (nq + 31) >> 5;
#pragma unroll
  for (uint32_t k = 0; k + 1 < (uint32_t)S; ++k) {
    if (32 * k + lane < nq) cp_async_quad(slot + 32 * k, p + 32 * k);
    cp_async_commit();
  }
  uint32_t hits = 0;
  for (uint32_t k = 0; k < steps; ++k) {
    const uint32_t kn = k + S - 1;  // into slot (k - 1) mod S, read and tested at step k - 1
    if (32 * kn + lane < nq) cp_async_quad(slot + 32 * (kn % S), p + 32 * kn);
    cp_async_commit();
    cp_async_wait<S - 1>();  // step k's copy has landed
    const int4 q = 32 * k + lane < nq ? slot[32 * (k % S)] : make_int4(pad, pad, pad, pad);
    hits += test_quad<MODE>(q, c, sk, v);
  }
  // every copy group left pending is empty (its step lies past the row)
  if (is_vertex(MODE)) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) vertex_add<MODE>(sk, v, s);
  }
  return hits;
}

// Short rows in shared memory: row k covers quads [q0[k], q0[k] + P[k+1] - P[k]); P is strictly increasing.
struct Rows {
  uint32_t* q0;
  uint32_t* P;
  int32_t* v;
};

// Walk quads [x0, x1) of the concatenated short rows 0..R-1 with one warp.
template <int MODE, class C>
__device__ __forceinline__ uint32_t walk(const Rows& r, int R, uint32_t x0, uint32_t x1,
                                         const int4* __restrict__ col4, const C& c, const Sink& sk, int32_t pad) {
  uint32_t hits = 0;
  if (x0 >= x1) return 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int a = 0, b = R;  // cur = last row with P <= x0
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
    if (MODE == kModeList) {  // all lanes take part; a lane past x1 tests the pad id
      const int own = x < x1 ? cur + __popc(starts & lt) : cur;
      const int4 q = x < x1 ? __ldg(&col4[r.q0[own] + (x - r.P[own])]) : make_int4(pad, pad, pad, pad);
      hits += test_quad<MODE>(q, c, sk, r.v[own]);
    } else if (x < x1) {
      const int own = cur + __popc(starts & lt);
      const int4 q = __ldg(&col4[r.q0[own] + (x - r.P[own])]);
      const uint32_t h = test_quad<MODE>(q, c, sk, MODE != kModeCount ? r.v[own] : 0);
      if (is_vertex(MODE) && h) vertex_add<MODE>(sk, r.v[own], h);
      hits += h;
    }
    cur += __popc(starts);
  }
  return hits;
}

// Walk quads [x0, x1) of the concatenated dense rows 0..R-1 (row k: r.q0[k] = its first quad in `dense`, r.v[k] =
// the quad of the source bitmap its first quad lines up with) with one warp: each quad is 128 ids, and its closing
// tests are four ANDs with the source's bitmap words and four population counts.
__device__ __forceinline__ uint32_t dense_walk(const Rows& r, int R, uint32_t x0, uint32_t x1,
                                               const int4* __restrict__ dense, const uint4* bm4) {
  uint32_t hits = 0;
  if (x0 >= x1) return 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int a = 0, b = R;  // cur = last row with P <= x0
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (r.P[mid] <= x0)
      a = mid + 1;
    else
      b = mid;
  }
  int cur = a - 1;
  for (uint32_t base = x0; base < x1; base += 32) {
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
      const uint32_t qi = x - r.P[own];
      const int4 q = __ldg(&dense[r.q0[own] + qi]);
      const uint4 w = bm4[r.v[own] + qi];
      hits += (__popc((uint32_t)q.x & w.x) + __popc((uint32_t)q.y & w.y)) +
              (__popc((uint32_t)q.z & w.z) + __popc((uint32_t)q.w & w.w));
    }
    cur += __popc(starts);
  }
  return hits;
}

// kModeList: dense_walk over rows whose r.v[k] holds v itself; each closed 2-path is appended with list_bits.  Quad
// qi of v's row covers ids base_w + 128 * (sq + qi) + [0, 128), sq the warp-window quad of v + 1, and lines up with
// quad sq + qi + delta of the source's bitmap.
__device__ __forceinline__ uint32_t dense_list_walk(const Rows& r, int R, uint32_t x0, uint32_t x1,
                                                    const int4* __restrict__ dense, const uint4* bm4, int32_t base_w,
                                                    int32_t delta, const Sink& sk) {
  uint32_t hits = 0;
  if (x0 >= x1) return 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int a = 0, b = R;
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (r.P[mid] <= x0)
      a = mid + 1;
    else
      b = mid;
  }
  int cur = a - 1;
  for (uint32_t xb = x0; xb < x1; xb += 32) {
    const int j = cur + (lane == 0 ? 32 : lane);
    uint32_t bit = 0;
    if (j < R) {
      const uint32_t pj = r.P[j];
      if (pj <= xb + 32) bit = 1u << (pj - xb - 1);
    }
    const uint32_t starts = __reduce_or_sync(kFull, bit);
    const uint32_t x = xb + lane;
    uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int32_t v = 0, w0 = 0;
    if (x < x1) {
      const int own = cur + __popc(starts & lt);
      const uint32_t qi = x - r.P[own];
      v = r.v[own];
      const int32_t bq = ((v + 1 - base_w) >> 7) + (int32_t)qi;
      const int4 q = __ldg(&dense[r.q0[own] + qi]);
      const uint4 w = bm4[bq + delta];
      m0 = (uint32_t)q.x & w.x;
      m1 = (uint32_t)q.y & w.y;
      m2 = (uint32_t)q.z & w.z;
      m3 = (uint32_t)q.w & w.w;
      w0 = base_w + 128 * bq;
    }
    hits += list_bits(m0, m1, m2, m3, w0, sk, v);
    cur += __popc(starts);
  }
  return hits;
}

// Is v's row also stored as a dense bitmap?  Returns its first quad or -1 (always -1 in the per-vertex modes, which
// walk the id rows: expanding the set bits of each AND into per-vertex adds measured twice as slow, 15.8 vs 7 ms at
// R-MAT 20, and 12.9 vs 5.5 ms with adds that return nothing).
template <int MODE>
__device__ __forceinline__ int32_t dense_row(const CsrView& g, int32_t v) {
  if (is_vertex(MODE) || g.dq0 == nullptr || v < g.base_w || v >= g.n) return -1;
  return __ldg(&g.dq0[v - g.base_w]);
}

// Descriptor of row v (v = n is the pad id: no row).
struct RowOf {
  uint32_t q0, nq;
};
__device__ __forceinline__ RowOf row_of(const int64_t* __restrict__ off, int32_t v, int64_t n) {
  RowOf r{0, 0};
  if (v >= 0 && v < n) {
    const int64_t rs = __ldg(&off[v]), re = __ldg(&off[v + 1]);
    r.q0 = (uint32_t)(rs >> 2);
    r.nq = (uint32_t)((re - rs) >> 2);
  }
  return r;
}

// Mark (set = true) or clear N+(u) ∩ [base, n) in a bitmap, with `stride` cooperating threads at index `t`;
// returns this thread's count of entries below base.
__device__ __forceinline__ uint32_t mark_row(const int32_t* __restrict__ row, int64_t len, int64_t n, int32_t base,
                                             uint32_t* bm, bool set, int t, int stride) {
  uint32_t low = 0;
  for (int64_t i = t; i < len; i += stride) {
    const int32_t x = __ldg(&row[i]);
    if (x >= n) continue;
    if (x >= base) {
      const int32_t b = x - base;
      if (set)
        atomicOr(&bm[b >> 5], 1u << (b & 31));
      else
        bm[b >> 5] = 0u;
    } else {
      ++low;
    }
  }
  return low;
}

// Ring slots of the staged long-row walk: per warp in warp mode, and per warp of the CTA in block mode.
constexpr int kWarpRingSlots = 4;
constexpr int kBlockRingSlots = 2;

// All second hops of source u for the calling warp, given its closing test.  ring: this warp's kWarpRingSlots x 32
// quads for staged long rows, or null for plain loads.
template <int MODE, class C>
__device__ __forceinline__ uint32_t warp_hops(const CsrView& g, int64_t beg, int64_t len, const C& c, const Rows& r,
                                              const Sink& sk, int4* ring = nullptr) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int4* col4 = reinterpret_cast<const int4*>(g.col);
  uint32_t hits = 0;
  for (int64_t vb = 0; vb < len; vb += 32) {
    const int64_t j = vb + lane;
    const int32_t v = j < len ? __ldg(&g.col[beg + j]) : (int32_t)g.n;
    const int32_t dq = dense_row<MODE>(g, v);
    const bool dense = dq >= 0;
    RowOf ro = row_of(g.off, v, g.n);
    if (dense) ro.nq = 0;
    const bool is_long = ro.nq >= (uint32_t)kLongQuads;
    unsigned longs = __ballot_sync(kFull, is_long);
    while (longs) {
      const int k = __ffs(longs) - 1;
      longs &= longs - 1;
      const uint32_t q0 = __shfl_sync(kFull, ro.q0, k), nq = __shfl_sync(kFull, ro.nq, k);
      const int32_t vk = MODE != kModeCount ? __shfl_sync(kFull, v, k) : 0;
      if (ring)
        hits += long_row_staged<MODE, kWarpRingSlots>(col4, q0, nq, c, sk, vk, (int32_t)g.n, ring);
      else
        hits += long_row<MODE>(col4, q0, nq, c, sk, vk, (int32_t)g.n);
    }
    const bool is_short = ro.nq > 0 && !is_long;
    const unsigned shorts = __ballot_sync(kFull, is_short);
    if (shorts) {
      const uint32_t nq = is_short ? ro.nq : 0u;
      const uint32_t incl = warp_inclusive_scan(nq);
      const uint32_t Q = __shfl_sync(kFull, incl, 31);
      if (is_short) {
        const int k = __popc(shorts & lt);
        r.q0[k] = ro.q0;
        r.P[k] = incl - nq;
        if (MODE != kModeCount) r.v[k] = v;
      }
      __syncwarp();
      hits += walk<MODE>(r, __popc(shorts), 0, Q, col4, c, sk, (int32_t)g.n);
      __syncwarp();
    }
    if (MODE == kModeCount) {
      const unsigned dmask = __ballot_sync(kFull, dense);
      if (dmask) {
        const int32_t sq = dense ? (v + 1 - g.base_w) >> 7 : 0;
        const uint32_t nq = dense ? (uint32_t)(g.wtopq - sq) : 0u;
        const uint32_t incl = warp_inclusive_scan(nq);
        const uint32_t Q = __shfl_sync(kFull, incl, 31);
        if (dense) {
          const int k = __popc(dmask & lt);
          r.q0[k] = (uint32_t)dq;
          r.P[k] = incl - nq;
          r.v[k] = sq + c.delta;
        }
        __syncwarp();
        hits += dense_walk(r, __popc(dmask), 0, Q, g.dense, reinterpret_cast<const uint4*>(c.bm));
        __syncwarp();
      }
    } else if (MODE == kModeList) {  // the same rows, r.v = v
      const unsigned dmask = __ballot_sync(kFull, dense);
      if (dmask) {
        const int32_t sq = dense ? (v + 1 - g.base_w) >> 7 : 0;
        const uint32_t nq = dense ? (uint32_t)(g.wtopq - sq) : 0u;
        const uint32_t incl = warp_inclusive_scan(nq);
        const uint32_t Q = __shfl_sync(kFull, incl, 31);
        if (dense) {
          const int k = __popc(dmask & lt);
          r.q0[k] = (uint32_t)dq;
          r.P[k] = incl - nq;
          r.v[k] = v;
        }
        __syncwarp();
        hits += dense_list_walk(r, __popc(dmask), 0, Q, g.dense, reinterpret_cast<const uint4*>(c.bm), g.base_w,
                                c.delta, sk);
        __syncwarp();
      }
    }
  }
  return hits;
}

// One source u, one warp.  bm is the warp's bitmap over [base_w, n] (all zero on entry and on return); ltab its
// low-entry hash (all -1 on entry and on return).
template <int MODE>
__device__ __forceinline__ uint32_t warp_source(int32_t u, const CsrView& g, uint32_t* bm, int32_t* ltab,
                                                const Rows& r, const Sink& sk_in, int4* ring = nullptr) {
  const int lane = threadIdx.x & 31;
  Sink sk = sk_in;
  sk.u = u;
  if (MODE == kModeList) sk.pu = __ldg(&sk.perm[u]);
  const int64_t beg = __ldg(&g.off[u]), len = __ldg(&g.off[u + 1]) - beg;
  const int32_t* row = g.col + beg;
  const uint32_t nlow = warp_sum(mark_row(row, len, g.n, g.base_w, bm, true, lane, 32));
  __syncwarp();
  constexpr uint32_t cap = (uint32_t)kWarpBitmapBits, lmask = (uint32_t)kWarpLowSlots - 1;
  uint32_t hits;
  if (nlow == 0) {
    hits = warp_hops<MODE>(g, beg, len, Closing<kLowNone>{bm, g.base_w, row, 0, cap, 0}, r, sk, ring);
  } else if (nlow <= (uint32_t)kWarpLowSlots / 2) {
    low_insert(row, (int)nlow, ltab, lmask, lane, 32);
    __syncwarp();
    hits = warp_hops<MODE>(g, beg, len, Closing<kLowHash>{bm, g.base_w, ltab, (int32_t)lmask, cap, 0}, r, sk, ring);
    __syncwarp();
    for (int i = lane; i < kWarpLowSlots; i += 32) ltab[i] = -1;
  } else {
    hits = warp_hops<MODE>(g, beg, len, Closing<kLowSearch>{bm, g.base_w, row, (int32_t)nlow, cap, 0}, r, sk, ring);
  }
  __syncwarp();
  mark_row(row, len, g.n, g.base_w, bm, false, lane, 32);
  __syncwarp();
  if (is_vertex(MODE)) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) source_add(sk, u, s);
  }
  return hits;
}

// Block-mode staging of one chunk of rows: long rows (q0, nq, v), short rows as a quad stream, a work counter.
struct BlockRows {
  uint32_t* lq0;
  uint32_t* lnq;
  int32_t* lv;
  Rows sr;
  Rows dr;  // dense rows (count mode)
  uint32_t* next;
  int32_t* ltab;
};

template <int MODE, class C>
__device__ __forceinline__ uint32_t block_hops(const CsrView& g, int64_t beg, int64_t len, const C& c,
                                               const BlockRows& br, uint32_t* ws, const Sink& sk,
                                               int4* ring = nullptr) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4* col4 = reinterpret_cast<const int4*>(g.col);
  uint32_t hits = 0;
  for (int64_t cb = 0; cb < len; cb += kBlockRows) {
    const int64_t j = cb + tid;
    const int32_t v = j < len ? __ldg(&g.col[beg + j]) : (int32_t)g.n;
    const int32_t dq = dense_row<MODE>(g, v);
    const bool dense = dq >= 0;
    RowOf ro = row_of(g.off, v, g.n);
    if (dense) ro.nq = 0;
    const bool is_long = ro.nq >= (uint32_t)kLongQuads;
    const bool is_short = ro.nq > 0 && !is_long;
    uint32_t NL, R, Q, ND = 0, QD = 0;
    const uint32_t lrank = block_exclusive_scan<uint32_t>(is_long ? 1u : 0u, ws, &NL);
    const uint32_t srank = block_exclusive_scan<uint32_t>(is_short ? 1u : 0u, ws, &R);
    const uint32_t pre = block_exclusive_scan<uint32_t>(is_short ? ro.nq : 0u, ws, &Q);
    if (!is_vertex(MODE)) {
      const int32_t sq = dense ? (v + 1 - g.base_w) >> 7 : 0;
      const uint32_t nqd = dense ? (uint32_t)(g.wtopq - sq) : 0u;
      const uint32_t drank = block_exclusive_scan<uint32_t>(dense ? 1u : 0u, ws, &ND);
      const uint32_t dpre = block_exclusive_scan<uint32_t>(nqd, ws, &QD);
      if (dense) {
        br.dr.q0[drank] = (uint32_t)dq;
        br.dr.P[drank] = dpre;
        br.dr.v[drank] = MODE == kModeList ? v : sq + c.delta;
      }
    }
    if (is_long) {
      br.lq0[lrank] = ro.q0;
      br.lnq[lrank] = ro.nq;
      if (MODE != kModeCount) br.lv[lrank] = v;
    }
    if (is_short) {
      br.sr.q0[srank] = ro.q0;
      br.sr.P[srank] = pre;
      if (MODE != kModeCount) br.sr.v[srank] = v;
    }
    if (tid == 0) *br.next = 0;
    __syncthreads();
    // long rows: each warp takes the next untaken row (bounded by NL), so no warp idles behind a long tail
    while (true) {
      uint32_t k = 0;
      if (lane == 0) k = atomicAdd(br.next, 1u);
      k = __shfl_sync(kFull, k, 0);
      if (k >= NL) break;
      if (ring)
        hits += long_row_staged<MODE, kBlockRingSlots>(col4, br.lq0[k], br.lnq[k], c, sk,
                                                       MODE != kModeCount ? br.lv[k] : 0, (int32_t)g.n, ring);
      else
        hits += long_row<MODE>(col4, br.lq0[k], br.lnq[k], c, sk, MODE != kModeCount ? br.lv[k] : 0,
                               (int32_t)g.n);
    }
    // short rows: equal contiguous shares of the quad stream
    const uint32_t per = (Q + kWarpsPerCTA - 1) / kWarpsPerCTA;
    const uint32_t x0 = min(Q, (uint32_t)warp * per), x1 = min(Q, x0 + per);
    hits += walk<MODE>(br.sr, (int)R, x0, x1, col4, c, sk, (int32_t)g.n);
    if (!is_vertex(MODE) && QD > 0) {  // dense rows: equal shares of their quads
      const uint32_t dper = (QD + kWarpsPerCTA - 1) / kWarpsPerCTA;
      const uint32_t d0 = min(QD, (uint32_t)warp * dper), d1 = min(QD, d0 + dper);
      if (MODE == kModeCount)
        hits += dense_walk(br.dr, (int)ND, d0, d1, g.dense, reinterpret_cast<const uint4*>(c.bm));
      else
        hits += dense_list_walk(br.dr, (int)ND, d0, d1, g.dense, reinterpret_cast<const uint4*>(c.bm), g.base_w,
                                c.delta, sk);
    }
    __syncthreads();
  }
  return hits;
}

// One source u, the whole block.  bm is the block's bitmap over [base_b, n] (all zero on entry and on return);
// br.ltab its low-entry hash (all -1 on entry and on return).
template <int MODE>
__device__ __forceinline__ uint32_t block_source(int32_t u, const CsrView& g, uint32_t* bm, const BlockRows& br,
                                                 uint32_t* ws, const Sink& sk_in, int4* ring = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31;
  Sink sk = sk_in;
  sk.u = u;
  if (MODE == kModeList) sk.pu = __ldg(&sk.perm[u]);
  const int64_t beg = __ldg(&g.off[u]), len = __ldg(&g.off[u + 1]) - beg;
  const int32_t* row = g.col + beg;
  uint32_t nlow;
  block_exclusive_scan<uint32_t>(mark_row(row, len, g.n, g.base_b, bm, true, tid, kCountThreads), ws, &nlow);
  // (the scan's barriers also publish the bitmap)
  constexpr uint32_t cap = (uint32_t)kBlockBitmapBits, lmask = (uint32_t)kBlockLowSlots - 1;
  uint32_t hits;
  if (nlow == 0) {
    hits = block_hops<MODE>(g, beg, len, Closing<kLowNone>{bm, g.base_b, row, 0, cap, g.dq_delta}, br, ws, sk,
                            ring);
  } else if (nlow <= (uint32_t)kBlockLowSlots / 2) {
    low_insert(row, (int)nlow, br.ltab, lmask, tid, kCountThreads);
    __syncthreads();
    hits = block_hops<MODE>(g, beg, len, Closing<kLowHash>{bm, g.base_b, br.ltab, (int32_t)lmask, cap, g.dq_delta},
                            br, ws, sk, ring);
    for (int i = tid; i < kBlockLowSlots; i += kCountThreads) br.ltab[i] = -1;  // block_hops ended with a barrier
  } else {
    hits = block_hops<MODE>(g, beg, len, Closing<kLowSearch>{bm, g.base_b, row, (int32_t)nlow, cap, g.dq_delta},
                            br, ws, sk, ring);
  }
  mark_row(row, len, g.n, g.base_b, bm, false, tid, kCountThreads);
  if (is_vertex(MODE)) {
    const uint32_t s = warp_sum(hits);
    if (lane == 0 && s) source_add(sk, u, s);
  }
  __syncthreads();
  return hits;
}

// One thread-bin source u, one lane: N+(u) has at most kTinyMaxDegree entries (one or two padded quads), and the
// triangles u < a < b are the pairs a < b of N+(u) with b in N+(a).  For each a the lane reads its row once: a dense
// row answers each b with one bit; an id row by binary search, whose lower bound only moves forward because the
// b's ascend.  (The per-pair form of the closing test: C(d, 2) lookups instead of walking every N+(a).)  In list
// mode the lane writes u's triangles to consecutive output positions from pos on.
template <int MODE>
__device__ __forceinline__ uint32_t tiny_source(int32_t u, const CsrView& g, const Sink& sk,
                                                unsigned long long pos = 0) {
  const int32_t n = (int32_t)g.n;
  const int64_t beg = __ldg(&g.off[u]);
  const int64_t plen = __ldg(&g.off[u + 1]) - beg;
  const int4* r4 = reinterpret_cast<const int4*>(g.col + beg);
  int32_t x[kTinyMaxDegree];
#pragma unroll
  for (int q = 0; q < kTinyMaxDegree / 4; ++q) {
    const int4 v4 = 4 * q < plen ? __ldg(&r4[q]) : make_int4(n, n, n, n);
    x[4 * q] = v4.x;
    x[4 * q + 1] = v4.y;
    x[4 * q + 2] = v4.z;
    x[4 * q + 3] = v4.w;
  }
  const uint32_t* dense_words = reinterpret_cast<const uint32_t*>(g.dense);
  uint32_t hits = 0;
  const int32_t pu = MODE == kModeList ? __ldg(&sk.perm[u]) : 0;
#pragma unroll
  for (int i = 0; i < kTinyMaxDegree - 1; ++i) {
    const int32_t a = x[i];
    if (a >= n) break;  // pad ids end the row
    const int32_t pa = MODE == kModeList ? __ldg(&sk.perm[a]) : 0;
    int64_t wbase = -1;  // dense row: its word 0 relative to window word 0
    if (g.dq0 != nullptr && a >= g.base_w) {
      const int32_t dq = __ldg(&g.dq0[a - g.base_w]);
      if (dq >= 0) wbase = 4 * ((int64_t)dq - ((a + 1 - g.base_w) >> 7));
    }
    int64_t lo = __ldg(&g.off[a]);
    const int64_t end = __ldg(&g.off[a + 1]);
#pragma unroll
    for (int j = i + 1; j < kTinyMaxDegree; ++j) {
      const int32_t b = x[j];
      if (b >= n) break;
      bool hit;
      if (wbase >= 0) {
        const int32_t t = b - g.base_w;
        hit = (__ldg(&dense_words[wbase + (t >> 5)]) >> (t & 31)) & 1u;
      } else {
        int64_t hi = end;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldg(&g.col[mid]) < b)
            lo = mid + 1;
          else
            hi = mid;
        }
        hit = lo < end && __ldg(&g.col[lo]) == b;
      }
      if (hit) {
        ++hits;
        if (is_vertex(MODE)) {
          vertex_add<MODE>(sk, a, 1u);
          vertex_add<MODE>(sk, b, 1u);
        }
        if (MODE == kModeList) write_triple(sk, pos++, pu, pa, b);
      }
    }
  }
  if (is_vertex(MODE) && hits) source_add(sk, u, hits);
  return hits;
}

// Shared-memory layout of the counting kernels.
constexpr int kWarpBitmapWords = kWarpBitmapBits / 32 + kBitmapSlackWords;
constexpr int kBlockBitmapWords = kBlockBitmapBits / 32 + kBitmapSlackWords;
constexpr int kWarpRowWords = 32 + 33 + 32;                        // q0, P, v
constexpr int kWarpRegionWords = (kWarpBitmapWords + kWarpRowWords + kWarpLowSlots + 3) & ~3;  // 16-byte aligned
constexpr int kWarpSmem = kWarpsPerCTA * kWarpRegionWords * 4;
constexpr int kBlockRowWords = 3 * kBlockRows + 2 * kBlockRows + (kBlockRows + 1) + 1 + 3 * kBlockRows;
// (long, short, counter, dense)
constexpr int kBlockSmem = (kBlockBitmapWords + kBlockRowWords + kBlockLowSlots) * 4;
constexpr int kCountSmem = kBlockSmem > kWarpSmem ? kBlockSmem : kWarpSmem;
// Staged counting (count mode only): a kWarpRingSlots-slot ring after each warp's region in warp mode, and a
// kBlockRingSlots-slot ring per warp after the block-mode layout.  Two CTAs per SM still fit.
constexpr int kWarpRingBytes = kWarpRingSlots * 32 * 16;
constexpr int kBlockRingBytes = kBlockRingSlots * 32 * 16;
constexpr int kWarpStagedSmem = kWarpsPerCTA * (kWarpRegionWords * 4 + kWarpRingBytes);
constexpr int kBlockRingOffset = (kBlockSmem + 15) & ~15;  // 16-byte aligned for the copies
constexpr int kBlockStagedSmem = kBlockRingOffset + kWarpsPerCTA * kBlockRingBytes;
constexpr int kCountStagedSmem = kBlockStagedSmem > kWarpStagedSmem ? kBlockStagedSmem : kWarpStagedSmem;
// two CTAs per SM: dynamic + static (272 bytes in k_count) + the 1 KB the runtime reserves per CTA, within 228 KB
static_assert(2 * (kCountStagedSmem + 512 + 1024) <= 228 * 1024, "staged counting must keep two CTAs per SM");
constexpr int kVertexSmem = kCountSmem + kHubRanks * 4;  // per-vertex modes: the hub counters follow
// two CTAs per SM: dynamic + static (< 1 KB) + the 1 KB the runtime reserves per CTA, within 228 KB
static_assert(2 * (kVertexSmem + 2048) <= 228 * 1024, "vertex-mode counting must keep two CTAs per SM");

__device__ __forceinline__ Rows warp_rows(uint32_t* region) {
  Rows r;
  r.q0 = region + kWarpBitmapWords;
  r.P = r.q0 + 32;
  r.v = reinterpret_cast<int32_t*>(r.P + 33);
  return r;
}

__device__ __forceinline__ int32_t* warp_low(uint32_t* region) {
  return reinterpret_cast<int32_t*>(region + kWarpBitmapWords + kWarpRowWords);
}

__device__ __forceinline__ BlockRows block_rows(uint32_t* smem) {
  BlockRows b;
  uint32_t* p = smem + kBlockBitmapWords;
  b.lq0 = p;
  b.lnq = p + kBlockRows;
  b.lv = reinterpret_cast<int32_t*>(p + 2 * kBlockRows);
  b.sr.q0 = p + 3 * kBlockRows;
  b.sr.v = reinterpret_cast<int32_t*>(p + 4 * kBlockRows);
  b.sr.P = p + 5 * kBlockRows;
  b.next = p + 6 * kBlockRows + 1;
  b.dr.q0 = p + 6 * kBlockRows + 2;
  b.dr.v = reinterpret_cast<int32_t*>(p + 7 * kBlockRows + 2);
  b.dr.P = p + 8 * kBlockRows + 2;
  b.ltab = reinterpret_cast<int32_t*>(p + kBlockRowWords);
  return b;
}

__device__ __forceinline__ void zero_words(uint32_t* p, int nwords, int t, int stride) {
  for (int i = t; i < nwords; i += stride) p[i] = 0u;
}

// Count the triangles of one graph: block-bin sources first (one CTA each), then warp-bin sources, then thread-bin
// sources (one lane each).  cursors[0..2]: zeroed work counters of this graph.  Returns this thread's count.
template <int MODE, bool STAGED = false>
__device__ __forceinline__ unsigned long long count_graph(const CsrView& g, const Sink& sk,
                                                          uint32_t* cursors, uint32_t* smem, uint32_t* ws,
                                                          int* s_idx) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned long long acc = 0;
  // staged layout: warp regions are kWarpRegionWords + the ring apart; block-mode rings follow the block layout
  constexpr int kRegionStride = STAGED ? kWarpRegionWords + kWarpRingBytes / 4 : kWarpRegionWords;
  if (g.nb > 0) {
    const BlockRows br = block_rows(smem);
    int4* bring =
        STAGED ? reinterpret_cast<int4*>(smem + kBlockRingOffset / 4) + warp * (kBlockRingSlots * 32) : nullptr;
    zero_words(smem, kBlockBitmapWords, tid, kCountThreads);
    for (int i = tid; i < kBlockLowSlots; i += kCountThreads) br.ltab[i] = -1;
    __syncthreads();
    while (true) {
      if (tid == 0) *s_idx = (int)atomicAdd(&cursors[0], 1u);
      __syncthreads();
      const int idx = *s_idx;
      __syncthreads();
      if (idx >= g.nb) break;
      acc += block_source<MODE>(g.list[idx], g, smem, br, ws, sk, bring);
    }
  }
  if (g.nw > 0) {
    uint32_t* region = smem + warp * kRegionStride;
    int4* wring = STAGED ? reinterpret_cast<int4*>(region + kWarpRegionWords) : nullptr;
    const Rows r = warp_rows(region);
    int32_t* ltab = warp_low(region);
    zero_words(region, kWarpBitmapWords, lane, 32);
    for (int i = lane; i < kWarpLowSlots; i += 32) ltab[i] = -1;
    __syncwarp();
    const int32_t* wlist = g.list + (g.n - g.nw);
    constexpr int kChunk = 4;
    while (true) {
      int idx = 0;
      if (lane == 0) idx = (int)atomicAdd(&cursors[1], (unsigned)kChunk);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= g.nw) break;
      const int e = min(idx + kChunk, g.nw);
      for (int k = idx; k < e; ++k) acc += warp_source<MODE>(wlist[k], g, region, ltab, r, sk, wring);
    }
  }
  if (g.nt > 0) {  // thread bin: 32 sources per warp, one per lane
    while (true) {
      int idx = 0;
      if (lane == 0) idx = (int)atomicAdd(&cursors[2], 32u);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= g.nt) break;
      if (idx + lane < g.nt) acc += tiny_source<MODE>(g.tlist[idx + lane], g, sk);
    }
  }
  return acc;
}

}  // namespace dev
}  // namespace tc

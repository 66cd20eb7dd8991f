// tc_build.cu — from an edge list to the oriented, relabelled CSR and the source bins.
//
// Steps (all on the caller's stream):
//   pack      validate ids, drop self-loops, key = (min << B) | max; count the input pairs at each vertex
//   rank      sort (count, id) -> rank(x); perm[rank] = x                                 (the visiting order)
//   relabel   pair {a,b} -> (min(rank a, rank b), max(...)): it now points up the order   (UMO, Sec. III-A/III-C)
//   sort      LSD radix sort of the relabelled keys on bits [0, 2B): rows by source, ascending targets
//   unique    keep the first of each run of equal keys                                   (simple graph, Def. 1)
//   csr       row lengths padded to a multiple of 4 (pad id n), int64 offsets by a scan, int32 columns
//   bins      w(u) = padded work of u's second hops; sources with d+(u) >= 2 and a candidate 2-path are kept
//             (the 2-look-ahead of Sec. III-C: a source needs two out-neighbours to close a triangle) and put in
//             the warp bin, or in the block bin when w(u) is large.
//
// The visiting order only has to be a total order for every triangle to be found exactly once (Sec. III-C); it
// is chosen to follow the degree (NE, Sec. III-A) because that bounds d+(u).  The degree used for ranking counts
// the input pairs at each vertex, repeats included, so it is known straight after ingest and the pairs can be
// relabelled before the one sort that also removes the repeats.  Relabelling by rank gives the kernel two things:
// hubs get the highest ids, so a bitmap over the top ids answers most closing-edge tests; and hub rows, which are
// re-read by many sources, sit together in memory.
#include <atomic>
#include <climits>

#include "tc_build.cuh"
#include "tc_internal.cuh"
#include "tc_prims.cuh"

namespace tc {
namespace {

// Warp-aggregated increment: lanes with the same target add once.
__device__ __forceinline__ void agg_inc(int32_t* cnt, uint32_t idx, bool active) {
  const uint32_t key = active ? idx : 0xffffffffu;
  const unsigned peers = __match_any_sync(kFull, key);
  if (active && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[idx], __popc(peers));
}

// Ingest: validate, drop self-loops, pack, and count the input pairs at each vertex.  Counts are first combined over
// tiles of kPackTile pairs in a shared-memory hash (hubs repeat often), then added to global memory once per
// distinct vertex at each flush of the table; a vertex that finds no slot within kPackProbe probes is added
// directly.
constexpr int kPackThreads = 256;
constexpr int kPackItems = 4;
constexpr int kPackTile = kPackThreads * kPackItems;  // 1024 pairs, <= 2048 distinct endpoints
static_assert(kPackItems == 4, "k_pack moves a thread's pairs as one int4 per array");
constexpr int kPackSlots = 4096;
// Tiles hashed between two flushes of the table: two fill it to at most one endpoint per slot (longer probes, half
// the flushes; R-MAT 18 and 20 ingest 3% faster than with one).
constexpr int kPackTilesPerFlush = 2;
constexpr int kPackProbe = 8;

// The slot's claim counts the vertex's first occurrence in the tile (the flush adds it), so a first occurrence costs
// one shared atomic (the claiming CAS) and a repeat one (the add).
__device__ __forceinline__ void pack_count(int32_t* skey, int32_t* scnt, int32_t* indeg, int32_t x) {
  uint32_t s = ((uint32_t)x * 2654435761u) >> 20;  // 12 bits
  for (int p = 0; p < kPackProbe; ++p) {
    const int32_t k = skey[s];
    if (k == x) {
      atomicAdd(&scnt[s], 1);
      return;
    }
    if (k < 0) {
      const int32_t prev = atomicCAS(&skey[s], -1, x);
      if (prev == -1) return;  // claimed: this occurrence is the slot's implicit first count
      if (prev == x) {
        atomicAdd(&scnt[s], 1);
        return;
      }
    }
    s = (s + 1) & (kPackSlots - 1);
  }
  atomicAdd(&indeg[x], 1);
}

// One input pair: its key (the sentinel for a self-loop or an invalid id) and its endpoints counted.
__device__ __forceinline__ uint64_t pack_pair(int32_t a, int32_t b, int64_t n, int B, uint64_t sentinel,
                                              int32_t* skey, int32_t* scnt, int32_t* indeg, bool& bad) {
  if (a < 0 || b < 0 || a >= n || b >= n) {
    bad = true;
    return sentinel;
  }
  if (a == b) return sentinel;
  pack_count(skey, scnt, indeg, a);
  pack_count(skey, scnt, indeg, b);
  return ((uint64_t)(a < b ? a : b) << B) | (uint64_t)(a < b ? b : a);
}

// Tiles of 1024 pairs, four consecutive pairs per thread.  With 16-byte aligned arrays the pairs come in with two
// 16-byte loads, issued for the next tile before the current one is hashed, and the keys leave with 16-byte
// stores; a ragged or unaligned tile takes scalar loads.
__global__ void __launch_bounds__(kPackThreads) k_pack(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                       int64_t len, int64_t n, int B, uint64_t* __restrict__ keys,
                                                       int32_t* __restrict__ indeg, uint32_t* __restrict__ err) {
  __shared__ int32_t skey[kPackSlots];
  __shared__ int32_t scnt[kPackSlots];
  const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
  for (int i = threadIdx.x; i < kPackSlots; i += kPackThreads) {
    skey[i] = -1;
    scnt[i] = 0;
  }
  __syncthreads();
  const bool vec_in = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  const bool vec_out = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
  const int64_t step = (int64_t)gridDim.x * kPackTile;
  bool bad = false;
  int64_t tile = (int64_t)blockIdx.x * kPackTile;
  int4 na = make_int4(0, 0, 0, 0), nb = na;
  if (vec_in && tile + kPackTile <= len) {
    na = __ldg(reinterpret_cast<const int4*>(src + tile) + threadIdx.x);
    nb = __ldg(reinterpret_cast<const int4*>(dst + tile) + threadIdx.x);
  }
  for (; tile < len; tile += step) {
    const int64_t i0 = tile + kPackItems * threadIdx.x;
    if (vec_in && tile + kPackTile <= len) {
      const int4 a4 = na, b4 = nb;
      const int64_t next = tile + step;
      if (next + kPackTile <= len) {
        na = __ldg(reinterpret_cast<const int4*>(src + next) + threadIdx.x);
        nb = __ldg(reinterpret_cast<const int4*>(dst + next) + threadIdx.x);
      }
      const uint64_t k0 = pack_pair(a4.x, b4.x, n, B, sentinel, skey, scnt, indeg, bad);
      const uint64_t k1 = pack_pair(a4.y, b4.y, n, B, sentinel, skey, scnt, indeg, bad);
      const uint64_t k2 = pack_pair(a4.z, b4.z, n, B, sentinel, skey, scnt, indeg, bad);
      const uint64_t k3 = pack_pair(a4.w, b4.w, n, B, sentinel, skey, scnt, indeg, bad);
      if (vec_out) {
        ulonglong2* o = reinterpret_cast<ulonglong2*>(keys + i0);
        o[0] = make_ulonglong2(k0, k1);
        o[1] = make_ulonglong2(k2, k3);
      } else {
        keys[i0] = k0;
        keys[i0 + 1] = k1;
        keys[i0 + 2] = k2;
        keys[i0 + 3] = k3;
      }
    } else {
      for (int j = 0; j < kPackItems; ++j) {
        const int64_t i = i0 + j;
        if (i >= len) break;
        keys[i] = pack_pair(src[i], dst[i], n, B, sentinel, skey, scnt, indeg, bad);
      }
    }
    // the table takes kPackTilesPerFlush tiles between flushes (each flush scans all of it)
    if (((tile - (int64_t)blockIdx.x * kPackTile) / step) % kPackTilesPerFlush != kPackTilesPerFlush - 1 &&
        tile + step < len)
      continue;
    __syncthreads();
    // flush: every occupied slot once (a scan of the table, no shared counter)
    for (int slot = threadIdx.x; slot < kPackSlots; slot += kPackThreads) {
      const int32_t k = skey[slot];
      if (k >= 0) {
        atomicAdd(&indeg[k], scnt[slot] + 1);  // + the claiming occurrence
        skey[slot] = -1;
        scnt[slot] = 0;
      }
    }
    __syncthreads();
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1u);
}

// Ingest of several graphs as their disjoint union: pair i belongs to graph k with eoff[k] <= i < eoff[k + 1], its
// ids are checked against that graph's vertex range [0, voff[k + 1] - voff[k]) and then offset by voff[k].  The
// arrays of graph k are srcs[k], dsts[k] (device-readable).  Tiles of kPackTile pairs, four consecutive pairs per
// thread; the counts are combined per tile as in k_pack.
struct ManyInput {
  const int32_t* const* srcs;
  const int32_t* const* dsts;
  const int64_t* eoff;  // k + 1 pair offsets
  const int64_t* voff;  // k + 1 vertex offsets
  int32_t k;
};

__global__ void __launch_bounds__(kPackThreads) k_pack_many(ManyInput in, int64_t len, int64_t n, int B,
                                                            uint64_t* __restrict__ keys, int32_t* __restrict__ indeg,
                                                            uint32_t* __restrict__ err) {
  __shared__ int32_t skey[kPackSlots];
  __shared__ int32_t scnt[kPackSlots];
  const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
  for (int i = threadIdx.x; i < kPackSlots; i += kPackThreads) {
    skey[i] = -1;
    scnt[i] = 0;
  }
  __syncthreads();
  bool bad = false;
  for (int64_t tile = (int64_t)blockIdx.x * kPackTile; tile < len; tile += (int64_t)gridDim.x * kPackTile) {
    const int64_t i0 = tile + kPackItems * threadIdx.x;
    if (i0 < len) {
      int a = 0, b = in.k;  // graph of pair i0: the last k with eoff[k] <= i0
      while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (__ldg(&in.eoff[mid]) <= i0)
          a = mid;
        else
          b = mid;
      }
      int g = a;
      for (int j = 0; j < kPackItems; ++j) {
        const int64_t i = i0 + j;
        if (i >= len) break;
        while (__ldg(&in.eoff[g + 1]) <= i) ++g;  // graphs without pairs are skipped
        const int64_t e = i - __ldg(&in.eoff[g]);
        const int64_t v0 = __ldg(&in.voff[g]), nv = __ldg(&in.voff[g + 1]) - v0;
        const int32_t x = __ldg(&in.srcs[g][e]), y = __ldg(&in.dsts[g][e]);
        uint64_t key;
        if (x < 0 || y < 0 || x >= nv || y >= nv) {
          bad = true;
          key = sentinel;
        } else {
          key = pack_pair((int32_t)(x + v0), (int32_t)(y + v0), n, B, sentinel, skey, scnt, indeg, bad);
        }
        keys[i] = key;
      }
    }
    __syncthreads();
    for (int slot = threadIdx.x; slot < kPackSlots; slot += kPackThreads) {
      const int32_t key = skey[slot];
      if (key >= 0) {
        atomicAdd(&indeg[key], scnt[slot] + 1);  // + the claiming occurrence
        skey[slot] = -1;
        scnt[slot] = 0;
      }
    }
    __syncthreads();
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1u);
}

// ---- unique: count then scatter the first key of each run (sentinel keys dropped) ----------------------------
constexpr int kUThreads = 256;
constexpr int kUItems = 8;
constexpr int kUTile = kUThreads * kUItems;

__device__ __forceinline__ bool is_first(const uint64_t* keys, int64_t i, uint64_t sentinel) {
  const uint64_t k = keys[i];
  return k != sentinel && (i == 0 || keys[i - 1] != k);
}

__global__ void __launch_bounds__(kUThreads) k_unique_count(const uint64_t* __restrict__ keys, int64_t n,
                                                            uint64_t sentinel, uint32_t* __restrict__ part) {
  __shared__ uint32_t ws[kUThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kUTile;
  uint32_t c = 0;
  for (int i = 0; i < kUItems; ++i) {
    const int64_t idx = base + i * kUThreads + threadIdx.x;
    if (idx < n && is_first(keys, idx, sentinel)) ++c;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kUThreads / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kUThreads) k_unique_scatter(const uint64_t* __restrict__ keys, int64_t n,
                                                              uint64_t sentinel, const uint32_t* __restrict__ part,
                                                              uint64_t* __restrict__ out, int64_t* __restrict__ m) {
  __shared__ uint32_t ws[kUThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kUTile + (int64_t)threadIdx.x * kUItems;  // blocked
  uint32_t f = 0;
  for (int i = 0; i < kUItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n && is_first(keys, idx, sentinel)) f |= 1u << i;
  }
  uint32_t tot;
  uint32_t pos = part[blockIdx.x] + block_exclusive_scan((uint32_t)__popc(f), ws, &tot);
  for (int i = 0; i < kUItems; ++i)
    if (f & (1u << i)) out[pos++] = keys[base + i];
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *m = (int64_t)part[blockIdx.x] + tot;
}

// ---- NE filter to a fixpoint (2-core peeling) ------------------------------------------------------------------
// One round: the degree of every vertex over the live distinct edges, then every edge with an endpoint of degree
// below 2 is replaced by the sentinel (a vertex of degree 1 is in no triangle, so neither is its edge).
__global__ void k_peel_degree(const uint64_t* __restrict__ keys, int64_t m, int B, uint64_t sentinel,
                              int32_t* __restrict__ deg) {
  const uint64_t mask = (1ull << B) - 1ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {  // warp-uniform trip count
    const int64_t i = base + threadIdx.x;
    const uint64_t k = i < m ? keys[i] : sentinel;
    const bool live = k != sentinel;
    agg_inc(deg, (uint32_t)(k >> B), live);
    agg_inc(deg, (uint32_t)(k & mask), live);
  }
}

__global__ void k_peel_kill(uint64_t* __restrict__ keys, int64_t m, int B, uint64_t sentinel,
                            const int32_t* __restrict__ deg, unsigned long long* __restrict__ killed) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const bool kill = k != sentinel && (deg[k >> B] < 2 || deg[k & mask] < 2);
    if (kill) keys[i] = sentinel;
    const unsigned b = __ballot_sync(__activemask(), kill);
    if (kill && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(killed, (unsigned long long)__popc(b));
  }
}

__global__ void k_count_nonzero(const int32_t* __restrict__ deg, int64_t n, unsigned long long* __restrict__ nz) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const bool on = deg[x] > 0;
    const unsigned b = __ballot_sync(__activemask(), on);
    if (on && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(nz, (unsigned long long)__popc(b));
  }
}

// ---- rank, relabel --------------------------------------------------------------------------------------------
// (count << B) | id, in id order: a stable sort on the count bits alone gives the (count, id) order.
__global__ void k_rank_keys(const int32_t* __restrict__ deg, int64_t n, int B, uint64_t* __restrict__ rkeys,
                            int* __restrict__ maxdeg) {
  int mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int d = deg[i];
    rkeys[i] = ((uint64_t)(uint32_t)d << B) | (uint64_t)i;
    mx = max(mx, d);
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (maxdeg && (threadIdx.x & 31) == 0 && mx > 0) atomicMax(maxdeg, mx);
}

// The compact build's rank keys with the count clamped to kRankClamp, so that two 8-bit radix passes order them:
// (min(count, kRankClamp) << B) | id.  The vertices at the clamp (counted in *tail) end up last, in id order, and
// k_rank_tail orders them by their true counts.
constexpr uint32_t kRankClamp = 65535;
constexpr int kRankClampBits = 16;
constexpr int kRankTailMax = 4096;  // the fix-up sort's capacity: 2M / kRankClamp + 1 <= 4096 for M <= 2^27

__global__ void k_rank_keys_clamped(const int32_t* __restrict__ deg, int64_t n, int B, uint64_t* __restrict__ rkeys,
                                    uint32_t* __restrict__ tail) {
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;  // warp-uniform trip count
    uint32_t d = 0;
    if (i < n) {
      d = (uint32_t)deg[i];
      rkeys[i] = ((uint64_t)(d < kRankClamp ? d : kRankClamp) << B) | (uint64_t)i;
    }
    const unsigned at = __ballot_sync(kFull, i < n && d >= kRankClamp);
    if (at && (threadIdx.x & 31) == __ffs(at) - 1) atomicAdd(tail, (uint32_t)__popc(at));
  }
}

// One CTA: the last *tail keys of the sorted array (the vertices at the clamp, in id order) sorted again on their
// true counts, (count << B) | id, by a bitonic sort in shared memory.
__global__ void __launch_bounds__(1024) k_rank_tail(uint64_t* __restrict__ sorted, int64_t n, int B,
                                                    const int32_t* __restrict__ deg, const uint32_t* __restrict__ tail,
                                                    uint32_t* __restrict__ err) {
  __shared__ uint64_t v[kRankTailMax];
  const int t = (int)*tail;
  if (t <= 1) return;
  if (t > kRankTailMax || t > n) {
    if (threadIdx.x == 0) *err = 1u;
    return;
  }
  int p = 1;
  while (p < t) p <<= 1;
  const uint64_t mask = (1ull << B) - 1ull;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    uint64_t k = ~0ull;
    if (i < t) {
      const uint64_t id = sorted[n - t + i] & mask;
      k = ((uint64_t)(uint32_t)deg[id] << B) | id;
    }
    v[i] = k;
  }
  __syncthreads();
  for (int kk = 2; kk <= p; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint64_t a = v[i], b = v[ixj];
          if ((a > b) == ((i & kk) == 0)) {
            v[i] = b;
            v[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < t; i += blockDim.x) sorted[n - t + i] = v[i];
}

// rank[id] = r and perm[r] = id; rcount (may be null) receives the input-pair count of rank r.
__global__ void k_rank(const uint64_t* __restrict__ sorted, int64_t n, int B, int32_t* __restrict__ rank,
                       int32_t* __restrict__ perm, int32_t* __restrict__ rcount) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = sorted[r];
    const int32_t id = (int32_t)(k & mask);
    rank[id] = (int32_t)r;
    perm[r] = id;
    if (rcount) rcount[r] = (int32_t)(k >> B);
  }
}

// k_rank with the bucket starts claimed instead of scanned: each warp's 32 consecutive ranks get adjacent rooms
// (a warp scan of their input-pair counts) at an offset claimed with one atomic add, so rooms follow the claims,
// not the ranks, and no scan or cursor copy is needed.  pstart and cur receive each rank's room.
__global__ void k_rank_buckets(const uint64_t* __restrict__ sorted, int64_t n, int B, int32_t* __restrict__ rank,
                               int32_t* __restrict__ perm, int64_t* __restrict__ pstart, int64_t* __restrict__ cur,
                               unsigned long long* __restrict__ alloc) {
  const uint64_t mask = (1ull << B) - 1ull;
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = base + threadIdx.x;  // warp-uniform trip count
    unsigned long long c = 0;
    int32_t id = 0;
    if (r < n) {
      const uint64_t k = sorted[r];
      id = (int32_t)(k & mask);
      c = k >> B;
      rank[id] = (int32_t)r;
      perm[r] = id;
    }
    const unsigned long long incl = warp_inclusive_scan(c);
    unsigned long long room = 0;
    if (lane == 31 && incl) room = atomicAdd(alloc, incl);
    room = __shfl_sync(kFull, room, 31) + incl - c;
    if (r < n) {
      pstart[r] = (int64_t)room;
      cur[r] = (int64_t)room;
    }
  }
}

// Pair keys (lo << B) | hi (or the sentinel) -> (min rank << B) | max rank (the sentinel stays).
__global__ void k_relabel(const uint64_t* __restrict__ keys, int64_t len, int B, const int32_t* __restrict__ rank,
                          uint64_t* __restrict__ okeys) {
  const uint64_t mask = (1ull << B) - 1ull;
  const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    uint64_t o = sentinel;
    if (k != sentinel) {
      const uint32_t ra = (uint32_t)rank[k >> B], rb = (uint32_t)rank[k & mask];
      o = ((uint64_t)(ra < rb ? ra : rb) << B) | (uint64_t)(ra < rb ? rb : ra);
    }
    okeys[i] = o;
  }
}

// d+(s) from the distinct oriented keys (sorted, so equal sources are adjacent and aggregate within a warp).
__global__ void k_outdeg(const uint64_t* __restrict__ ukeys, int64_t m, int B, int32_t* __restrict__ odeg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < m;
    agg_inc(odeg, ok ? (uint32_t)(ukeys[i] >> B) : 0u, ok);
  }
}

__global__ void k_padded_len(const int32_t* __restrict__ odeg, int64_t n, int32_t* __restrict__ plen) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    plen[i] = (odeg[i] + 3) & ~3;
}

__global__ void k_fill(int32_t* __restrict__ p, int64_t len, int32_t value) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = value;
}

// Entry i of the sorted relabelled keys is the (i - ustart[s])-th out-neighbour of its source s.
__global__ void k_columns(const uint64_t* __restrict__ okeys, int64_t m, int B, const int64_t* __restrict__ ustart,
                          const int64_t* __restrict__ off, int32_t* __restrict__ col) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = okeys[i];
    const int64_t s = (int64_t)(k >> B);
    col[off[s] + (i - ustart[s])] = (int32_t)(k & mask);
  }
}

// ---- bucketed orientation --------------------------------------------------------------------------------------
// The default build groups the relabelled pairs by source without a full sort: count the pairs at each source,
// scan, scatter each target into its source's bucket, then sort and de-duplicate every bucket on chip.  A bucket
// of L pairs belongs to a source with at least L input pairs, and only the vertices ranked above it can be its
// targets; those all have at least L input pairs too, so there are fewer than 2M / L of them.  Long buckets thus
// have a narrow target range, and a shared-memory bitmap over that range sorts and de-duplicates them in one pass.
constexpr int kSmallRow = 32;            // buckets of 2..32 pairs: one warp, bitonic sort in a register
constexpr int kWarpRow = 256;            // up to 256 pairs: one warp, bitonic sort in registers (8 per lane)
constexpr int kWarpBits = 1 << 15;       // target ranges up to 32768 ids: one warp, bitmap (4 KB)
constexpr int kRowThreads = 256;         // block size of k_rows_warp
constexpr int kBigThreads = 1024;        // other buckets: one block, bitmap (<= kBigBits ids) or bitonic sort
constexpr int kBigBits = 1 << 20;        // block bitmap capacity (128 KB)

// Each pair {a, b} goes to the bucket of its lower-ranked endpoint as the higher rank.  Bucket s has room for the
// input-pair count of s (an upper bound on its size) starting at pstart[s]; its cursor cur[s] starts there and ends
// one past its last pair (the order in a bucket is free).
// Each pair is a chain of dependent accesses (its key, two rank lookups, the slot claim, the store), so a thread
// takes four consecutive pairs and runs their chains side by side: four times the accesses in flight.
constexpr int kBucketItems = 4;

__global__ void k_bucket(const uint64_t* __restrict__ keys, int64_t npairs, int B, const int32_t* __restrict__ rank,
                         unsigned long long* __restrict__ cur, int32_t* __restrict__ tgt) {
  const uint64_t mask = (1ull << B) - 1ull;
  const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
  const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kBucketItems; i0 < npairs;
       i0 += (int64_t)gridDim.x * blockDim.x * kBucketItems) {
    uint64_t k[kBucketItems];
    if (vec && i0 + kBucketItems <= npairs) {
      const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(keys + i0);
      const ulonglong2 y = *reinterpret_cast<const ulonglong2*>(keys + i0 + 2);
      k[0] = x.x;
      k[1] = x.y;
      k[2] = y.x;
      k[3] = y.y;
    } else {
#pragma unroll
      for (int j = 0; j < kBucketItems; ++j) k[j] = i0 + j < npairs ? keys[i0 + j] : sentinel;
    }
    int32_t ra[kBucketItems], rb[kBucketItems];
#pragma unroll
    for (int j = 0; j < kBucketItems; ++j) {
      if (k[j] != sentinel) {
        ra[j] = __ldg(&rank[k[j] >> B]);
        rb[j] = __ldg(&rank[k[j] & mask]);
      }
    }
    unsigned long long pos[kBucketItems];
#pragma unroll
    for (int j = 0; j < kBucketItems; ++j)
      if (k[j] != sentinel) pos[j] = atomicAdd(&cur[ra[j] < rb[j] ? ra[j] : rb[j]], 1ull);
#pragma unroll
    for (int j = 0; j < kBucketItems; ++j)
      if (k[j] != sentinel) tgt[pos[j]] = ra[j] < rb[j] ? rb[j] : ra[j];
  }
}

// Buckets of up to kSmallRow pairs, sorted and de-duplicated in place by one warp each (32 consecutive sources per
// warp).  Longer buckets are listed for k_rows_warp (front of `lists`) when their target range fits a warp's bitmap
// or they fit a warp's registers, and for k_rows_block (back of `lists`) otherwise.  d[s] = distinct targets of s.
__global__ void k_rows_small(const int64_t* __restrict__ pstart, const int64_t* __restrict__ cur, int64_t n,
                             int32_t* __restrict__ tgt, int32_t* __restrict__ d, int32_t* __restrict__ lists,
                             RowCounters* __restrict__ rc) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long msum = 0;
  for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {
    const int64_t sidx = base + lane;
    int64_t ps = 0;
    int32_t L = 0;
    if (sidx < n) {
      ps = pstart[sidx];
      L = (int32_t)(cur[sidx] - ps);
    }
    const int64_t range = n - 1 - sidx;
    const bool to_warp = L > kSmallRow && (range <= kWarpBits || L <= kWarpRow);
    const bool to_block = L > kSmallRow && !to_warp;
    const unsigned mw = __ballot_sync(kFull, to_warp), mb = __ballot_sync(kFull, to_block);
    unsigned pw = 0, pb = 0;
    if (lane == 0) {
      if (mw) pw = atomicAdd(&rc->nwarp, (unsigned)__popc(mw));
      if (mb) pb = atomicAdd(&rc->nblock, (unsigned)__popc(mb));
    }
    pw = __shfl_sync(kFull, pw, 0);
    pb = __shfl_sync(kFull, pb, 0);
    if (to_warp) lists[pw + __popc(mw & lt)] = (int32_t)sidx;
    if (to_block) lists[n - 1 - (pb + __popc(mb & lt))] = (int32_t)sidx;
    int32_t dd = L <= 1 ? L : 0;  // a bucket of one pair is sorted and distinct
    // buckets of 2..32 pairs, four at a time: their loads issued together, their sorting networks interleaved
    unsigned todo = __ballot_sync(kFull, L >= 2 && L <= kSmallRow);
    while (todo) {
      int32_t x[4], rl[4], rk[4];
      int64_t rps[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        rl[r] = 0;
        rk[r] = -1;
        rps[r] = 0;
        x[r] = INT_MAX;
        if (todo) {
          rk[r] = __ffs(todo) - 1;
          todo &= todo - 1;
          rps[r] = __shfl_sync(kFull, ps, rk[r]);
          rl[r] = __shfl_sync(kFull, L, rk[r]);
          if (lane < rl[r]) x[r] = tgt[rps[r] + lane];
        }
      }
#pragma unroll
      for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
          const bool lower = ((lane & j) == 0) == ((lane & kk) == 0);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int32_t y = __shfl_xor_sync(kFull, x[r], j);
            x[r] = lower ? min(x[r], y) : max(x[r], y);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int32_t prev = __shfl_up_sync(kFull, x[r], 1);
        const bool keep = x[r] != INT_MAX && (lane == 0 || x[r] != prev);
        const unsigned km = __ballot_sync(kFull, keep);
        if (rl[r] > 0) {
          if (keep) tgt[rps[r] + __popc(km & lt)] = x[r];
          if (lane == rk[r]) dd = __popc(km);
        }
      }
    }
    if (sidx < n && L <= kSmallRow) {
      d[sidx] = dd;
      msum += (unsigned long long)dd;
    }
  }
  msum = warp_sum(msum);
  if (lane == 0 && msum) atomicAdd(&rc->m, msum);
}

// Bitonic sort of p (a power of two) values in shared memory by `stride` cooperating threads at index t; sync()
// separates the stages.
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <class Sync>
__device__ __forceinline__ void bitonic_smem(int32_t* v, int p, int t, int stride, Sync sync) {
  for (int kk = 2; kk <= p; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = t; i < p; i += stride) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = v[i], b = v[ixj];
          if ((a > b) == ((i & kk) == 0)) {
            v[i] = b;
            v[ixj] = a;
          }
        }
      }
      sync();
    }
  }
}

// Bitonic sort of 32*T values held by a warp, value t of lane l at position 32t + l; then the distinct values are
// written in order to out[0..) and their number returned (INT_MAX marks an empty position).
template <int T>
__device__ __forceinline__ uint32_t warp_sort_unique(int32_t (&x)[T], int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int kk = 2; kk <= 32 * T; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int jt = j >> 5;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          if (t & jt) continue;
          const bool asc = ((t * 32 + lane) & kk) == 0;
          const int32_t a = x[t], b = x[t + jt];
          if ((a > b) == asc) {
            x[t] = b;
            x[t + jt] = a;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int32_t y = __shfl_xor_sync(kFull, x[t], j);
          const bool asc = ((t * 32 + lane) & kk) == 0;
          x[t] = (((lane & j) == 0) == asc) ? min(x[t], y) : max(x[t], y);
        }
      }
    }
  }
  uint32_t run = 0;
  int32_t last = __shfl_sync(kFull, x[0], 0) - 1;  // differs from the first value
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int32_t up = __shfl_up_sync(kFull, x[t], 1);
    const int32_t prev = lane == 0 ? last : up;
    const bool keep = x[t] != INT_MAX && x[t] != prev;
    const unsigned km = __ballot_sync(kFull, keep);
    if (keep) out[run + __popc(km & lt)] = x[t];
    run += __popc(km);
    last = __shfl_sync(kFull, x[t], 31);
  }
  return run;
}

// Buckets listed for one warp each: a bitmap over the target range (s, n) in the warp's shared memory when the range
// has at most kWarpBits ids, else (at most kWarpRow pairs) a bitonic sort in registers.
__global__ void __launch_bounds__(kRowThreads) k_rows_warp(const int64_t* __restrict__ pstart,
                                                           const int64_t* __restrict__ cur, int64_t n,
                                                           int32_t* __restrict__ tgt, int32_t* __restrict__ d,
                                                           const int32_t* __restrict__ list,
                                                           RowCounters* __restrict__ rc) {
  __shared__ uint32_t bm_all[kRowThreads / 32][kWarpBits / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned rows = rc->nwarp;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  uint32_t* bm = bm_all[warp];
  unsigned long long msum = 0;
  for (unsigned r = gw; r < rows; r += nw) {
    const int32_t sidx = list[r];
    const int64_t ps = pstart[sidx];
    const int32_t L = (int32_t)(cur[sidx] - ps);
    const int64_t range = n - 1 - sidx;
    uint32_t run;
    if (range <= kWarpBits) {
      const int words = (int)((range + 31) >> 5);
      for (int w = lane; w < words; w += 32) bm[w] = 0u;
      __syncwarp();
      for (int32_t i = lane; i < L; i += 32) {
        const int32_t b = tgt[ps + i] - sidx - 1;
        atomicOr(&bm[b >> 5], 1u << (b & 31));
      }
      __syncwarp();
      // lane l emits words [l*per, (l+1)*per) in order
      const int per = (words + 31) >> 5;
      const int w0 = min(words, lane * per), w1 = min(words, w0 + per);
      uint32_t c = 0;
      for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
      const uint32_t incl = warp_inclusive_scan(c);
      uint32_t pos = incl - c;
      run = __shfl_sync(kFull, incl, 31);
      for (int w = w0; w < w1; ++w) {
        uint32_t bits = bm[w];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          tgt[ps + pos++] = sidx + 1 + w * 32 + b;
        }
      }
      __syncwarp();
    } else if (L <= 64) {
      int32_t x[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) x[t] = t * 32 + lane < L ? tgt[ps + t * 32 + lane] : INT_MAX;
      run = warp_sort_unique<2>(x, tgt + ps);
    } else if (L <= 128) {
      int32_t x[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) x[t] = t * 32 + lane < L ? tgt[ps + t * 32 + lane] : INT_MAX;
      run = warp_sort_unique<4>(x, tgt + ps);
    } else {
      int32_t x[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) x[t] = t * 32 + lane < L ? tgt[ps + t * 32 + lane] : INT_MAX;
      run = warp_sort_unique<8>(x, tgt + ps);
    }
    if (lane == 0) d[sidx] = (int32_t)run;
    msum += run;
  }
  if (lane == 0 && msum) atomicAdd(&rc->m, msum);
}

// Buckets listed for one block each (more than kWarpRow pairs, target range above kWarpBits): a bitmap over the
// range when it has at most kBigBits ids, else a bitonic sort in shared memory (such a bucket has fewer than
// 2M / kBigBits <= mid_max pairs).
__global__ void __launch_bounds__(kBigThreads) k_rows_block(const int64_t* __restrict__ pstart,
                                                            const int64_t* __restrict__ cur, int64_t n,
                                                            int32_t mid_max, int32_t* __restrict__ tgt,
                                                            int32_t* __restrict__ d,
                                                            const int32_t* __restrict__ lists,
                                                            RowCounters* __restrict__ rc) {
  extern __shared__ __align__(16) uint32_t blk_smem[];  // kBigBits / 32 words (>= mid_max ints)
  __shared__ uint32_t ws[kBigThreads / 32];
  const int tid = threadIdx.x;
  const unsigned rows = rc->nblock;
  for (unsigned r = blockIdx.x; r < rows; r += gridDim.x) {
    const int32_t sidx = lists[n - 1 - r];
    const int64_t ps = pstart[sidx];
    const int64_t L = cur[sidx] - ps;
    const int64_t range = n - 1 - sidx;
    uint32_t total = 0;
    if (range <= kBigBits) {
      const int words = (int)((range + 31) >> 5);
      for (int w = tid; w < words; w += kBigThreads) blk_smem[w] = 0u;
      __syncthreads();
      for (int64_t i = tid; i < L; i += kBigThreads) {
        const int32_t b = tgt[ps + i] - sidx - 1;
        atomicOr(&blk_smem[b >> 5], 1u << (b & 31));
      }
      __syncthreads();
      const int per = (words + kBigThreads - 1) / kBigThreads;
      const int w0 = min(words, tid * per), w1 = min(words, w0 + per);
      uint32_t c = 0;
      for (int w = w0; w < w1; ++w) c += __popc(blk_smem[w]);
      uint32_t pos = block_exclusive_scan<uint32_t>(c, ws, &total);
      for (int w = w0; w < w1; ++w) {
        uint32_t bits = blk_smem[w];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          tgt[ps + pos++] = sidx + 1 + w * 32 + b;
        }
      }
    } else if (L <= mid_max) {
      int32_t* v = reinterpret_cast<int32_t*>(blk_smem);
      int p = 2 * kWarpRow;
      while (p < L) p <<= 1;
      for (int i = tid; i < p; i += kBigThreads) v[i] = i < L ? tgt[ps + i] : INT_MAX;
      __syncthreads();
      bitonic_smem(v, p, tid, kBigThreads, BlockSync{});
      for (int64_t c = 0; c < L; c += kBigThreads) {
        const int64_t i = c + tid;
        const bool keep = i < L && (i == 0 || v[i] != v[i - 1]);
        uint32_t tot;
        const uint32_t pos = total + block_exclusive_scan<uint32_t>(keep ? 1u : 0u, ws, &tot);
        if (keep) tgt[ps + pos] = v[i];
        total += tot;
      }
    } else if (tid == 0) {  // cannot happen for consistent counts: report and leave the bucket alone
      atomicOr(&rc->err, 1u);
    }
    if (tid == 0) {
      d[sidx] = (int32_t)total;
      atomicAdd(&rc->m, (unsigned long long)total);
    }
    __syncthreads();
  }
}

// Rows into the CSR: row s takes its d[s] sorted distinct targets, then pad ids up to its padded length.  A row of
// one quad is written by its own lane with one 16-byte store; longer rows by the whole warp.
__global__ void k_rows_copy(const int64_t* __restrict__ pstart, const int32_t* __restrict__ tgt,
                            const int32_t* __restrict__ d, const int64_t* __restrict__ off, int64_t n,
                            int32_t* __restrict__ col, int32_t pad, int64_t* __restrict__ entries_out) {
  const int lane = threadIdx.x & 31;
  if (entries_out && blockIdx.x == 0 && threadIdx.x < 4) {  // the spare quad after the last row, and off[n]
    const int64_t e = off[n];
    col[e + threadIdx.x] = pad;
    if (threadIdx.x == 0) *entries_out = e;
  }
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {
    const int64_t sidx = base + lane;
    int64_t ps = 0, o = 0;
    int32_t dd = 0, pl = 0;
    if (sidx < n) {
      ps = pstart[sidx];
      o = off[sidx];
      dd = d[sidx];
      pl = (int32_t)(off[sidx + 1] - o);
    }
    if (pl == 4) {
      int4 q = make_int4(pad, pad, pad, pad);
      q.x = tgt[ps];
      if (dd > 1) q.y = tgt[ps + 1];
      if (dd > 2) q.z = tgt[ps + 2];
      if (dd > 3) q.w = tgt[ps + 3];
      *reinterpret_cast<int4*>(col + o) = q;
    }
    // rows of two to eight quads, four at a time: their loads are issued together before any store waits on them
    unsigned todo = __ballot_sync(kFull, pl > 4 && pl <= 32);
    while (todo) {
      int32_t v[4], rpl[4];
      int64_t ro[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        rpl[r] = 0;
        ro[r] = 0;
        v[r] = pad;
        if (todo) {
          const int k = __ffs(todo) - 1;
          todo &= todo - 1;
          const int64_t rps = __shfl_sync(kFull, ps, k);
          ro[r] = __shfl_sync(kFull, o, k);
          const int32_t rd = __shfl_sync(kFull, dd, k);
          rpl[r] = __shfl_sync(kFull, pl, k);
          if (lane < rd) v[r] = tgt[rps + lane];
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (lane < rpl[r]) col[ro[r] + lane] = v[r];
    }
    todo = __ballot_sync(kFull, pl > 32);
    while (todo) {
      const int k = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t rps = __shfl_sync(kFull, ps, k), ro = __shfl_sync(kFull, o, k);
      const int32_t rd = __shfl_sync(kFull, dd, k), rpl = __shfl_sync(kFull, pl, k);
      for (int32_t j = lane; j < rpl; j += 32) col[ro + j] = j < rd ? tgt[rps + j] : pad;
    }
  }
}

// ---- work estimate and binning ----------------------------------------------------------------------------------

// w(u) = the hop-2 work of source u: the padded length of each id row of N+(u), and four ids' worth per quad of
// each dense row (see k_dense_select); plus the true 2-path count.  Sources with d+(u) >= 2 and a 2-path go to
// the block bin (w above the threshold) or the warp bin.  Rows of up to 32 entries are summed by their own lane,
// longer ones by the whole warp.  rowinfo[v] = {d+(v), padded length or minus dense quads}.
__global__ void k_bins(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                       const int2* __restrict__ rowinfo, int64_t n, int64_t block_min_work,
                       int32_t* __restrict__ list, int32_t* __restrict__ tlist, BinCounters* __restrict__ bc) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long wsum = 0, act = 0, dw = 0, dv = 0;
  int dmax = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t u = base + threadIdx.x;
    int64_t b = 0;
    int32_t d = 0;
    if (u < n) {
      d = rowinfo[u].x;
      b = off[u];
    }
    RowWork w;
    if (d <= 32) {  // the row as 16-byte quads (rows start on 16-byte boundaries), four row-info loads at a time,
                    // the next quad's load in flight with them
      const int4* r4 = reinterpret_cast<const int4*>(col + b);
      const int32_t nq = (d + 3) >> 2;
      const int4 none = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
      int4 q = nq > 0 ? __ldg(&r4[0]) : none;
      for (int32_t k = 0; k < nq; ++k) {
        const int4 qn = k + 1 < nq ? __ldg(&r4[k + 1]) : none;
        const int2 zero = make_int2(0, 0);
        const int2 i0 = q.x < n ? __ldg(&rowinfo[q.x]) : zero, i1 = q.y < n ? __ldg(&rowinfo[q.y]) : zero;
        const int2 i2 = q.z < n ? __ldg(&rowinfo[q.z]) : zero, i3 = q.w < n ? __ldg(&rowinfo[q.w]) : zero;
        w.add(i0);
        w.add(i1);
        w.add(i2);
        w.add(i3);
        q = qn;
      }
    }
    unsigned longs = __ballot_sync(kFull, d > 32);
    while (longs) {
      const int k = __ffs(longs) - 1;
      longs &= longs - 1;
      const int64_t rb = __shfl_sync(kFull, b, k);
      const int32_t rd = __shfl_sync(kFull, d, k);
      RowWork p;
      for (int32_t j = lane; j < rd; j += 32) p.add(rowinfo[col[rb + j]]);
      p.pad = warp_sum(p.pad);
      p.wtrue = warp_sum(p.wtrue);
      p.wdense = warp_sum(p.wdense);
      p.qdense = warp_sum(p.qdense);
      if (lane == k) w = p;
    }
    const int64_t wpad = w.pad, wtrue = w.wtrue;
    wsum += (unsigned long long)wtrue;
    dw += (unsigned long long)w.wdense;
    dv += (unsigned long long)w.qdense;
    if (d > dmax) dmax = d;
    const bool keep = d >= 2 && wtrue > 0;
    // thread bin: few out-neighbours whose pairs cost far less to look up than the hop-2 rows cost to walk
    // (4 C(d, 2) lookups' worth of entries or more; measured on GB300 against factors 2, 8 and 16 of C(d, 2))
    const bool tny = keep && d <= kTinyMaxDegree && 8 * (int64_t)d * (d - 1) <= wpad;
    const bool blk = keep && !tny && wpad > block_min_work;
    const bool wrp = keep && !tny && !blk;
    act += keep ? 1 : 0;
    const unsigned mb = __ballot_sync(kFull, blk);
    const unsigned mw = __ballot_sync(kFull, wrp);
    const unsigned mt = __ballot_sync(kFull, tny);
    unsigned pb = 0, pw = 0, pt = 0;
    if (lane == 0) {
      if (mb) pb = atomicAdd(&bc->nb, (unsigned)__popc(mb));
      if (mw) pw = atomicAdd(&bc->nw, (unsigned)__popc(mw));
      if (mt) pt = atomicAdd(&bc->nt, (unsigned)__popc(mt));
    }
    pb = __shfl_sync(kFull, pb, 0);
    pw = __shfl_sync(kFull, pw, 0);
    pt = __shfl_sync(kFull, pt, 0);
    if (blk) list[pb + __popc(mb & lt)] = (int32_t)u;
    if (wrp) list[n - 1 - (pw + __popc(mw & lt))] = (int32_t)u;
    if (tny) tlist[pt + __popc(mt & lt)] = (int32_t)u;
  }
  wsum = warp_sum(wsum);
  act = warp_sum(act);
  dw = warp_sum(dw);
  dv = warp_sum(dv);
  for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(kFull, dmax, o));
  if (lane == 0) {
    atomicAdd(&bc->wedges, wsum);
    atomicAdd(&bc->active, act);
    if (dw) atomicAdd(&bc->dense_wedges, dw);
    if (dv) atomicAdd(&bc->dense_visits, dv);
    atomicMax(&bc->max_out, dmax);
  }
}

// ---- dense rows -------------------------------------------------------------------------------------------------
// Row v (in the warp window) is kept as a bitmap too when its bitmap quads cover no more words than it has entries.
// For every vertex, rowinfo[v] = {d+(v), its hop-2 cost code}: the padded row length, or minus the quads of its
// dense row; nq[v - base_w] = those quads (0: id list only) for the window.
__global__ void k_dense_select(const int32_t* __restrict__ dplus, int64_t n, int32_t base_w, int32_t wtopq,
                               int32_t* __restrict__ nq, int2* __restrict__ rowinfo) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = dplus[v];
    int32_t code = (d + 3) & ~3;
    if (v >= base_w) {
      const int32_t q = wtopq - (int32_t)((v + 1 - base_w) >> 7);
      const bool dense = d >= kDenseMinDegree && 4 * (int64_t)q <= d;
      nq[v - base_w] = dense ? q : 0;
      if (dense) code = -q;
    }
    rowinfo[v] = make_int2(d, code);
  }
}

// dq0[i] = first quad of the dense row of base_w + i, or -1; qoff is the exclusive scan of the quad counts.
__global__ void k_dense_index(const int32_t* __restrict__ nq, const int64_t* __restrict__ qoff, int64_t wn,
                              int32_t* __restrict__ dq0, unsigned long long* __restrict__ rows,
                              int64_t* __restrict__ quads_out) {
  if (quads_out && blockIdx.x == 0 && threadIdx.x == 0) *quads_out = qoff[wn];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < wn; i += (int64_t)gridDim.x * blockDim.x) {
    const bool on = nq[i] > 0;
    dq0[i] = on ? (int32_t)qoff[i] : -1;
    const unsigned b = __ballot_sync(__activemask(), on);
    if (on && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(rows, (unsigned long long)__popc(b));
  }
}

// One warp per window vertex: the bits of N+(v) into its dense row, which is zero beforehand, or is zeroed here
// first when nq (its quad count per window vertex) is given.
__global__ void k_dense_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ dplus, int64_t n, int32_t base_w,
                             const int32_t* __restrict__ dq0, uint32_t* __restrict__ words,
                             const int32_t* __restrict__ nq) {
  const int lane = threadIdx.x & 31;
  const int64_t wn = n - base_w;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp0; i < wn; i += nwarps) {
    const int32_t q0 = dq0[i];
    if (q0 < 0) continue;
    const int64_t v = base_w + i;
    const int64_t beg = off[v];
    const int32_t d = dplus[v];
    const int64_t w0 = 4 * (int64_t)q0 - 4 * ((v + 1 - base_w) >> 7);  // word of window word 0, relative
    if (nq) {
      uint4* q = reinterpret_cast<uint4*>(words) + q0;
      for (int32_t j = lane; j < nq[i]; j += 32) q[j] = make_uint4(0u, 0u, 0u, 0u);
      __syncwarp();
    }
    for (int32_t j = lane; j < d; j += 32) {
      const int32_t b = col[beg + j] - base_w;
      atomicOr(&words[w0 + (b >> 5)], 1u << (b & 31));
    }
  }
}

// ---- the CSR's tail with one scan (compact builds) --------------------------------------------------------------
// Per vertex from d+(v): sizes[v] = (padded length << 32) | dense quads, its row code (the rules of k_padded_len and
// k_dense_select), and its dense quads by window position.  Summed over the vertices, the low half stays below 2^32
// and never carries into the high one, so one scan gives both the offsets and the dense rows' first quads.
__global__ void k_row_codes(const int32_t* __restrict__ dplus, int64_t n, int32_t base_w, int32_t wtopq,
                            uint64_t* __restrict__ sizes, int32_t* __restrict__ nq, int2* __restrict__ rowinfo) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = dplus[v];
    const int32_t pl = (d + 3) & ~3;
    int32_t code = pl, q = 0;
    if (v >= base_w) {
      const int32_t wq = wtopq - (int32_t)((v + 1 - base_w) >> 7);
      if (d >= kDenseMinDegree && 4 * (int64_t)wq <= d) q = wq;
      nq[v - base_w] = q;
      if (q) code = -q;
    }
    sizes[v] = ((uint64_t)(uint32_t)pl << 32) | (uint32_t)q;
    rowinfo[v] = make_int2(d, code);
  }
}

// k_rows_copy from the scanned sizes: each source's offset and dense-row start are unpacked (off, dq0) as its row is
// copied; the first thread also writes off[n], the spare quad and the totals.
__global__ void k_rows_copy_scanned(const int64_t* __restrict__ pstart, const int32_t* __restrict__ tgt,
                                    const int32_t* __restrict__ d, const uint64_t* __restrict__ psz, int64_t n,
                                    int32_t base_w, int64_t* __restrict__ off, int32_t* __restrict__ col,
                                    int32_t* __restrict__ dq0, CompactSizes* __restrict__ sizes) {
  const int lane = threadIdx.x & 31;
  const int32_t pad = (int32_t)n;
  if (blockIdx.x == 0 && threadIdx.x < 4) {
    const uint64_t t = psz[n];
    const int64_t e = (int64_t)(t >> 32);
    col[e + threadIdx.x] = pad;
    if (threadIdx.x == 0) {
      off[n] = e;
      sizes->entries = e;
      sizes->dquads = (int64_t)(uint32_t)t;
    }
  }
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long drows = 0;
  for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {
    const int64_t sidx = base + lane;
    int64_t ps = 0, o = 0;
    int32_t dd = 0, pl = 0;
    if (sidx < n) {
      const uint64_t a = psz[sidx], b = psz[sidx + 1];
      ps = pstart[sidx];
      o = (int64_t)(a >> 32);
      dd = d[sidx];
      pl = (int32_t)((b >> 32) - (a >> 32));
      off[sidx] = o;
      if (sidx >= base_w) {
        const bool dense = (uint32_t)b != (uint32_t)a;
        dq0[sidx - base_w] = dense ? (int32_t)(uint32_t)a : -1;
        drows += dense ? 1 : 0;
      }
    }
    if (pl == 4) {
      int4 q = make_int4(pad, pad, pad, pad);
      q.x = tgt[ps];
      if (dd > 1) q.y = tgt[ps + 1];
      if (dd > 2) q.z = tgt[ps + 2];
      if (dd > 3) q.w = tgt[ps + 3];
      *reinterpret_cast<int4*>(col + o) = q;
    }
    // rows of two to eight quads, four at a time: their loads are issued together before any store waits on them
    unsigned todo = __ballot_sync(kFull, pl > 4 && pl <= 32);
    while (todo) {
      int32_t v[4], rpl[4];
      int64_t ro[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        rpl[r] = 0;
        ro[r] = 0;
        v[r] = pad;
        if (todo) {
          const int k = __ffs(todo) - 1;
          todo &= todo - 1;
          const int64_t rps = __shfl_sync(kFull, ps, k);
          ro[r] = __shfl_sync(kFull, o, k);
          const int32_t rd = __shfl_sync(kFull, dd, k);
          rpl[r] = __shfl_sync(kFull, pl, k);
          if (lane < rd) v[r] = tgt[rps + lane];
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (lane < rpl[r]) col[ro[r] + lane] = v[r];
    }
    todo = __ballot_sync(kFull, pl > 32);
    while (todo) {
      const int k = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t rps = __shfl_sync(kFull, ps, k), ro = __shfl_sync(kFull, o, k);
      const int32_t rd = __shfl_sync(kFull, dd, k), rpl = __shfl_sync(kFull, pl, k);
      for (int32_t j = lane; j < rpl; j += 32) col[ro + j] = j < rd ? tgt[rps + j] : pad;
    }
  }
  drows = warp_sum(drows);
  if (lane == 0 && drows) atomicAdd(&sizes->dense_rows, drows);
}

// Scatter of counts from rank space back to original ids.
__global__ void k_unpermute(const unsigned long long* __restrict__ by_rank, const int32_t* __restrict__ perm,
                            int64_t n, unsigned long long* __restrict__ by_id) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    by_id[perm[r]] = by_rank[r];
}

}  // namespace

tc_status pack_edges(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t len, int64_t offset,
                     uint32_t* d_err, cudaStream_t s) {
  if (len <= 0) return TC_OK;
  const int64_t tiles = (len + kPackTile - 1) / kPackTile;
  const int grid = (int)(tiles < 4 * num_sms() ? tiles : 4 * num_sms());
  k_pack<<<grid, kPackThreads, 0, s>>>(src, dst, len, g->n, g->key_bits, g->keys.as<uint64_t>() + offset,
                                       g->indeg.as<int32_t>(), d_err);
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status pack_edges_many(tc_graph* g, const int32_t* const* d_srcs, const int32_t* const* d_dsts,
                          const int64_t* d_eoff, const int64_t* d_voff, int32_t k, uint32_t* d_err, cudaStream_t s) {
  const int64_t len = g->num_pairs;
  if (len <= 0) return TC_OK;
  const int64_t tiles = (len + kPackTile - 1) / kPackTile;
  const int grid = (int)(tiles < 4 * num_sms() ? tiles : 4 * num_sms());
  k_pack_many<<<grid, kPackThreads, 0, s>>>(ManyInput{d_srcs, d_dsts, d_eoff, d_voff, k}, len, g->n, g->key_bits,
                                            g->keys.as<uint64_t>(), g->indeg.as<int32_t>(), d_err);
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

tc_status unpermute_counts(const tc_graph* g, const uint64_t* by_rank, uint64_t* by_id, cudaStream_t s) {
  if (g->n <= 0) return TC_OK;
  k_unpermute<<<grid_for(g->n, 256), 256, 0, s>>>((const unsigned long long*)by_rank, g->perm.as<int32_t>(), g->n,
                                                  (unsigned long long*)by_id);
  note_launch();
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// Peels the m distinct keys in *ukeys to the 2-core (at most max_rounds rounds; <= 0: until a round removes
// nothing, capped at kPeelMaxRounds) and compacts them; *m becomes the number left.
constexpr int32_t kPeelMaxRounds = 1 << 16;

tc_status peel_keys(const Allocator& a, Buf& ukeys, int64_t* m, int64_t n, int B, uint64_t sentinel,
                    int32_t max_rounds, tc_prune_stats* ps, cudaStream_t s) {
  const int32_t limit = max_rounds > 0 ? max_rounds : kPeelMaxRounds;
  Buf deg, words, out, part;
  tc_status st = TC_OK;
  unsigned long long hw[2] = {0, 0};
  int64_t nz_first = 0, nz_last = 0;
  int32_t rounds = 0;
  auto launched = [&](const char* what) {
    note_launch();
    return cuda_status(cudaGetLastError(), what);
  };
  do {
    if ((st = buf_alloc(a, deg, (size_t)n * 4, s))) break;
    if ((st = buf_alloc(a, words, 16, s))) break;
    // pass: degrees over the live keys and how many vertices have one ([1]); with kill, the edges removed ([0])
    auto pass = [&](bool kill) -> tc_status {
      TC_CUDA(cudaMemsetAsync(deg.p, 0, (size_t)n * 4, s));
      TC_CUDA(cudaMemsetAsync(words.p, 0, 16, s));
      k_peel_degree<<<grid_for(*m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), *m, B, sentinel, deg.as<int32_t>());
      TC_TRY(launched("k_peel_degree"));
      k_count_nonzero<<<grid_for(n, 256), 256, 0, s>>>(deg.as<int32_t>(), n, words.as<unsigned long long>() + 1);
      TC_TRY(launched("k_count_nonzero"));
      if (kill) {
        k_peel_kill<<<grid_for(*m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), *m, B, sentinel, deg.as<int32_t>(),
                                                      words.as<unsigned long long>());
        TC_TRY(launched("k_peel_kill"));
      }
      TC_CUDA(cudaMemcpyAsync(hw, words.p, 16, cudaMemcpyDeviceToHost, s));
      TC_CUDA(cudaStreamSynchronize(s));
      return TC_OK;
    };
    bool removed = true;
    int32_t passes = 0;
    while (removed && passes < limit) {
      if ((st = pass(true))) break;
      if (passes == 0) nz_first = (int64_t)hw[1];
      nz_last = (int64_t)hw[1];  // vertices with an edge at the start of this round
      ++passes;
      removed = hw[0] > 0;
    }
    if (st) break;
    rounds = removed ? passes : passes - 1;  // rounds that removed something
    if (removed) {  // stopped by the limit: the degrees of what is left
      if ((st = pass(false))) break;
      nz_last = (int64_t)hw[1];
    }
    // compaction of the live keys (they stay sorted and distinct)
    const int64_t tiles = (*m + kUTile - 1) / kUTile;
    if ((st = buf_alloc(a, out, (size_t)*m * 8, s))) break;
    if ((st = buf_alloc(a, part, (size_t)tiles * 4, s))) break;
    k_unique_count<<<(unsigned)tiles, kUThreads, 0, s>>>(ukeys.as<uint64_t>(), *m, sentinel, part.as<uint32_t>());
    if ((st = launched("k_unique_count"))) break;
    if ((st = exclusive_scan_u32(a, part.as<uint32_t>(), tiles, s))) break;
    k_unique_scatter<<<(unsigned)tiles, kUThreads, 0, s>>>(ukeys.as<uint64_t>(), *m, sentinel, part.as<uint32_t>(),
                                                            out.as<uint64_t>(), words.as<int64_t>());
    if ((st = launched("k_unique_scatter"))) break;
    int64_t left = 0;
    if ((st = cuda_status(cudaMemcpyAsync(&left, words.p, 8, cudaMemcpyDeviceToHost, s), "copy kept"))) break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "sync kept"))) break;
    if (ps) {
      ps->rounds = rounds;
      ps->edges_removed = *m - left;
      ps->vertices_removed = nz_first - nz_last;
    }
    *m = left;
    buf_release(a, ukeys, s);
    ukeys = out;
    out = Buf{};
  } while (0);
  for (Buf* b : {&deg, &words, &out, &part}) buf_release(a, *b, s);
  return st;
}

// The bucketed orientation: from the pair keys, the ranks and each rank's input-pair count to g->off, g->col;
// dplus (n entries, allocated here) receives d+(s); *m the distinct edges and *entries the padded column entries.
tc_status bucket_csr(tc_graph* g, const int32_t* rank, const int32_t* rcount, Buf& dplus, int64_t* m,
                     int64_t* entries, cudaStream_t s) {
  const Allocator& a = g->alloc;
  const int B = g->key_bits;
  const int64_t M = g->num_pairs;
  const int64_t n = g->n;
  const int64_t n1 = n > 0 ? n : 1;
  Buf pstart, cur, tgt, lists, rcb, plen;
  tc_status st = TC_OK;
  auto launched = [&](const char* what) {
    note_launch();
    return cuda_status(cudaGetLastError(), what);
  };
  // a bucket whose targets span more than kBigBits ids has fewer than 2M / kBigBits <= mid_max pairs
  int32_t mid_max = 2048;
  while ((2 * M) / mid_max > (int64_t)kBigBits) mid_max <<= 1;
  RowCounters hrc{};
  do {
    // bucket s has room for the input-pair count of s: 2 slots per pair in all
    if ((st = buf_alloc(a, pstart, (size_t)(n + 1) * 8, s))) break;
    if ((st = buf_alloc(a, cur, (size_t)n1 * 8, s))) break;
    if ((st = buf_alloc(a, tgt, (size_t)(M > 0 ? 2 * M : 1) * 4, s))) break;
    if ((st = buf_alloc(a, dplus, (size_t)n1 * 4, s))) break;
    if ((st = buf_alloc(a, lists, (size_t)n1 * 4, s))) break;
    if ((st = buf_alloc(a, rcb, sizeof(RowCounters), s))) break;
    if ((st = cuda_status(cudaMemsetAsync(rcb.p, 0, sizeof(RowCounters), s), "memset rows"))) break;
    if (n > 0) {
      if ((st = exclusive_scan_i32_to_i64(a, rcount, pstart.as<int64_t>(), n, s))) break;
    } else if ((st = cuda_status(cudaMemsetAsync(pstart.p, 0, 8, s), "memset pstart"))) {
      break;
    }
    if ((st = cuda_status(cudaMemcpyAsync(cur.p, pstart.p, (size_t)n1 * 8, cudaMemcpyDeviceToDevice, s),
                          "copy cursors")))
      break;
    if (M > 0) {
      k_bucket<<<grid_for((M + kBucketItems - 1) / kBucketItems, 256), 256, 0, s>>>(
          g->keys.as<uint64_t>(), M, B, rank, cur.as<unsigned long long>(), tgt.as<int32_t>());
      if ((st = launched("k_bucket"))) break;
    }
    buf_release(a, g->keys, s);
    RowCounters* rc = rcb.as<RowCounters>();
    int32_t* rlist = lists.as<int32_t>();
    if (n > 0) {
      k_rows_small<<<grid_for(n, 256), 256, 0, s>>>(pstart.as<int64_t>(), cur.as<int64_t>(), n, tgt.as<int32_t>(),
                                                    dplus.as<int32_t>(), rlist, rc);
      if ((st = launched("k_rows_small"))) break;
      k_rows_warp<<<4 * num_sms(), kRowThreads, 0, s>>>(pstart.as<int64_t>(), cur.as<int64_t>(), n,
                                                      tgt.as<int32_t>(), dplus.as<int32_t>(), rlist, rc);
      if ((st = launched("k_rows_warp"))) break;
      const size_t blk_smem = (size_t)kBigBits / 8;
      if ((st = cuda_status(cudaFuncSetAttribute(k_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)blk_smem), "k_rows_block attribute")))
        break;
      k_rows_block<<<num_sms(), kBigThreads, blk_smem, s>>>(pstart.as<int64_t>(), cur.as<int64_t>(), n, mid_max,
                                                          tgt.as<int32_t>(), dplus.as<int32_t>(), rlist, rc);
      if ((st = launched("k_rows_block"))) break;
    }
    buf_release(a, cur, s);
    // padded offsets
    if ((st = buf_alloc(a, g->off, (size_t)(n + 1) * 8, s))) break;
    if ((st = buf_alloc(a, plen, (size_t)n1 * 4, s))) break;
    if (n > 0) {
      k_padded_len<<<grid_for(n, 256), 256, 0, s>>>(dplus.as<int32_t>(), n, plen.as<int32_t>());
      if ((st = launched("k_padded_len"))) break;
      if ((st = exclusive_scan_i32_to_i64(a, plen.as<int32_t>(), g->off.as<int64_t>(), n, s))) break;
    } else if ((st = cuda_status(cudaMemsetAsync(g->off.p, 0, 8, s), "memset off"))) {
      break;
    }
    buf_release(a, plen, s);
    if ((st = cuda_status(cudaMemcpyAsync(entries, g->off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s),
                          "copy entries")))
      break;
    if ((st = cuda_status(cudaMemcpyAsync(&hrc, rc, sizeof(RowCounters), cudaMemcpyDeviceToHost, s), "copy rows")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "sync entries"))) break;
    if (hrc.err) {
      set_error("tc_build: a bucket's targets exceeded the range bound (inconsistent pair counts)");
      st = TC_ERR_INTERNAL;
      break;
    }
    *m = (int64_t)hrc.m;
    // columns: rows then pad ids, and one spare quad of pad ids at the end
    const int64_t ncol = *entries + 4;
    if ((st = buf_alloc(a, g->col, (size_t)ncol * 4, s))) break;
    k_fill<<<1, 32, 0, s>>>(g->col.as<int32_t>() + *entries, 4, (int32_t)n);
    if ((st = launched("k_fill"))) break;
    if (n > 0 && *entries > 0) {
      k_rows_copy<<<grid_for(n, 256), 256, 0, s>>>(pstart.as<int64_t>(), tgt.as<int32_t>(), dplus.as<int32_t>(),
                                                   g->off.as<int64_t>(), n, g->col.as<int32_t>(), (int32_t)n,
                                                   nullptr);
      if ((st = launched("k_rows_copy"))) break;
    }
  } while (0);
  for (Buf* b : {&pstart, &cur, &tgt, &lists, &rcb, &plen}) buf_release(a, *b, s);
  return st;
}

tc_status build_graph(tc_graph* g, cudaStream_t s) {
  if (g->tiny || (use_buckets(g->num_pairs) && tiny_eligible(g->n, g->num_pairs))) return build_graph_tiny(g, s);
  if (g->n > 0 && g->num_pairs > 0 && g->num_pairs <= compact_max_pairs() && use_buckets(g->num_pairs))
    return build_graph_compact(g, s);
  return build_graph_pruned(g, -1, nullptr, s);
}

tc_status build_graph_pruned(tc_graph* g, int32_t peel_rounds, tc_prune_stats* ps, cudaStream_t s) {
  const Allocator& a = g->alloc;
  const int B = g->key_bits;
  const int64_t M = g->num_pairs;
  const int64_t n = g->n;
  const int64_t n1 = n > 0 ? n : 1;
  const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
  tc_status st = TC_OK;
  const bool buckets = peel_rounds < 0 && use_buckets(M);
  Buf alt, part, counters, odeg, ukeys, rkeys, rkeys_alt, rank, rcount, ustart, plen, dnq, dqoff, rowinfo;
  int64_t m = 0;
  BinCounters hb{};
  int64_t total_padded = 0;
  int32_t maxdeg = 0;
  auto launched = [&](const char* what) {
    note_launch();
    return cuda_status(cudaGetLastError(), what);
  };

  do {
    if ((st = buf_alloc(a, counters, 64, s))) break;
    // ---- rank: stable sort of (count << B) | id on the count bits ----
    if ((st = buf_alloc(a, rank, (size_t)n1 * 4, s))) break;
    if ((st = buf_alloc(a, g->perm, (size_t)n1 * 4, s))) break;
    if (n > 0) {
      if ((st = buf_alloc(a, rkeys, (size_t)n * 8, s))) break;
      if ((st = buf_alloc(a, rkeys_alt, (size_t)n * 8, s))) break;
      if ((st = cuda_status(cudaMemsetAsync(counters.p, 0, 8, s), "memset maxdeg"))) break;
      k_rank_keys<<<grid_for(n, 256), 256, 0, s>>>(g->indeg.as<int32_t>(), n, B, rkeys.as<uint64_t>(),
                                                   counters.as<int>());
      if ((st = launched("k_rank_keys"))) break;
      if ((st = cuda_status(cudaMemcpyAsync(&maxdeg, counters.p, 4, cudaMemcpyDeviceToHost, s), "copy maxdeg")))
        break;
      if ((st = cuda_status(cudaStreamSynchronize(s), "sync maxdeg"))) break;
      int dbits = 0;
      while (dbits < 32 && (1ll << dbits) <= (int64_t)maxdeg) ++dbits;
      uint64_t* rs = nullptr;
      if ((st = radix_sort_u64(a, rkeys.as<uint64_t>(), rkeys_alt.as<uint64_t>(), n, B, B + dbits, &rs, s))) break;
      if (buckets && (st = buf_alloc(a, rcount, (size_t)n * 4, s))) break;
      k_rank<<<grid_for(n, 256), 256, 0, s>>>(rs, n, B, rank.as<int32_t>(), g->perm.as<int32_t>(),
                                              rcount.as<int32_t>());
      if ((st = launched("k_rank"))) break;
      buf_release(a, rkeys, s);
      buf_release(a, rkeys_alt, s);
    }
    buf_release(a, g->indeg, s);

    if (buckets) {  // the default: bucketed orientation
      if ((st = bucket_csr(g, rank.as<int32_t>(), rcount.as<int32_t>(), odeg, &m, &total_padded, s))) break;
      buf_release(a, rank, s);
      buf_release(a, rcount, s);
      g->m = m;
      g->csr_entries = total_padded;
    } else {  // the sort path (for very large inputs, and for pruning, which works on the sorted distinct keys)
      // ---- relabel, sort, unique: ukeys = distinct (rank s << B) | rank d with s < d, sorted ----
      if (M > 0) {
        uint64_t* sorted = nullptr;
        if ((st = buf_alloc(a, alt, (size_t)M * 8, s))) break;
        k_relabel<<<grid_for(M, 256), 256, 0, s>>>(g->keys.as<uint64_t>(), M, B, rank.as<int32_t>(),
                                                   alt.as<uint64_t>());
        if ((st = launched("k_relabel"))) break;
        if ((st = radix_sort_u64(a, alt.as<uint64_t>(), g->keys.as<uint64_t>(), M, 0, 2 * B, &sorted, s))) break;
        const bool in_alt = sorted == alt.as<uint64_t>();
        uint64_t* uout = in_alt ? g->keys.as<uint64_t>() : alt.as<uint64_t>();
        const int64_t tiles = (M + kUTile - 1) / kUTile;
        if ((st = buf_alloc(a, part, (size_t)tiles * 4, s))) break;
        k_unique_count<<<(unsigned)tiles, kUThreads, 0, s>>>(sorted, M, sentinel, part.as<uint32_t>());
        if ((st = launched("k_unique_count"))) break;
        if ((st = exclusive_scan_u32(a, part.as<uint32_t>(), tiles, s))) break;
        k_unique_scatter<<<(unsigned)tiles, kUThreads, 0, s>>>(sorted, M, sentinel, part.as<uint32_t>(), uout,
                                                                counters.as<int64_t>());
        if ((st = launched("k_unique_scatter"))) break;
        if ((st = cuda_status(cudaMemcpyAsync(&m, counters.p, 8, cudaMemcpyDeviceToHost, s), "copy m"))) break;
        if ((st = cuda_status(cudaStreamSynchronize(s), "sync m"))) break;
        buf_release(a, part, s);
        if (in_alt) {
          ukeys = g->keys;
          g->keys = Buf{};
        } else {
          ukeys = alt;
          alt = Buf{};
        }
        buf_release(a, alt, s);
        buf_release(a, g->keys, s);
      }
      buf_release(a, rank, s);
      if (peel_rounds >= 0 && m > 0 && (st = peel_keys(a, ukeys, &m, n, B, sentinel, peel_rounds, ps, s))) break;
      g->m = m;

      // ---- offsets: unpadded starts (ustart) and padded offsets (off) ----
      if ((st = buf_alloc(a, odeg, (size_t)n1 * 4, s))) break;
      if ((st = cuda_status(cudaMemsetAsync(odeg.p, 0, (size_t)n1 * 4, s), "memset odeg"))) break;
      if (m > 0) {
        k_outdeg<<<grid_for(m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), m, B, odeg.as<int32_t>());
        if ((st = launched("k_outdeg"))) break;
      }
      if ((st = buf_alloc(a, ustart, (size_t)(n + 1) * 8, s))) break;
      if ((st = buf_alloc(a, g->off, (size_t)(n + 1) * 8, s))) break;
      if ((st = buf_alloc(a, plen, (size_t)n1 * 4, s))) break;
      if (n > 0) {
        if ((st = exclusive_scan_i32_to_i64(a, odeg.as<int32_t>(), ustart.as<int64_t>(), n, s))) break;
        k_padded_len<<<grid_for(n, 256), 256, 0, s>>>(odeg.as<int32_t>(), n, plen.as<int32_t>());
        if ((st = launched("k_padded_len"))) break;
        if ((st = exclusive_scan_i32_to_i64(a, plen.as<int32_t>(), g->off.as<int64_t>(), n, s))) break;
      } else {
        if ((st = cuda_status(cudaMemsetAsync(ustart.p, 0, 8, s), "memset ustart"))) break;
        if ((st = cuda_status(cudaMemsetAsync(g->off.p, 0, 8, s), "memset off"))) break;
      }
      buf_release(a, plen, s);
      if ((st = cuda_status(cudaMemcpyAsync(&total_padded, g->off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s),
                            "copy entries")))
        break;
      if ((st = cuda_status(cudaStreamSynchronize(s), "sync entries"))) break;
      g->csr_entries = total_padded;

      // ---- columns: fill with the pad id n, then scatter ----
      const int64_t ncol = total_padded + 4;
      if ((st = buf_alloc(a, g->col, (size_t)ncol * 4, s))) break;
      k_fill<<<grid_for(ncol, 256), 256, 0, s>>>(g->col.as<int32_t>(), ncol, (int32_t)n);
      if ((st = launched("k_fill"))) break;
      if (m > 0) {
        k_columns<<<grid_for(m, 256), 256, 0, s>>>(ukeys.as<uint64_t>(), m, B, ustart.as<int64_t>(),
                                                   g->off.as<int64_t>(), g->col.as<int32_t>());
        if ((st = launched("k_columns"))) break;
      }
      buf_release(a, ukeys, s);
    }

    // ---- dense rows: selection and quad offsets (before the bins, which charge their cost) ----
    const CsrView vw = g->view();
    const int64_t wn = n - vw.base_w;
    unsigned long long* drows = reinterpret_cast<unsigned long long*>(counters.as<char>() + 48);
    int64_t dquads = 0;
    unsigned long long hrows = 0;
    if ((st = buf_alloc(a, rowinfo, (size_t)n1 * 8, s))) break;
    if (n > 0) {
      if ((st = buf_alloc(a, dnq, (size_t)(wn > 0 ? wn : 1) * 4, s))) break;
      if ((st = buf_alloc(a, dqoff, (size_t)(wn + 1) * 8, s))) break;
      if ((st = buf_alloc(a, g->dq0, (size_t)wn * 4, s))) break;
      if ((st = cuda_status(cudaMemsetAsync(drows, 0, 8, s), "memset dense rows"))) break;
      k_dense_select<<<grid_for(n, 256), 256, 0, s>>>(odeg.as<int32_t>(), n, vw.base_w, vw.wtopq,
                                                      dnq.as<int32_t>(), rowinfo.as<int2>());
      if ((st = launched("k_dense_select"))) break;
      if ((st = exclusive_scan_i32_to_i64(a, dnq.as<int32_t>(), dqoff.as<int64_t>(), wn, s))) break;
      k_dense_index<<<grid_for(wn, 256), 256, 0, s>>>(dnq.as<int32_t>(), dqoff.as<int64_t>(), wn,
                                                      g->dq0.as<int32_t>(), drows, nullptr);
      if ((st = launched("k_dense_index"))) break;
      if ((st = cuda_status(cudaMemcpyAsync(&dquads, dqoff.as<int64_t>() + wn, 8, cudaMemcpyDeviceToHost, s),
                            "copy dense quads")))
        break;
      if ((st = cuda_status(cudaMemcpyAsync(&hrows, drows, 8, cudaMemcpyDeviceToHost, s), "copy dense rows")))
        break;
    }

    // ---- bins ----
    if ((st = buf_alloc(a, g->list, (size_t)n1 * 4, s))) break;
    if ((st = buf_alloc(a, g->tlist, (size_t)n1 * 4, s))) break;
    if ((st = cuda_status(cudaMemsetAsync(counters.p, 0, sizeof(BinCounters), s), "memset bins"))) break;
    if (n > 0) {
      k_bins<<<grid_for(n, 256), 256, 0, s>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), rowinfo.as<int2>(), n,
                                              block_min_work_for(m), g->list.as<int32_t>(), g->tlist.as<int32_t>(),
                                              counters.as<BinCounters>());
      if ((st = launched("k_bins"))) break;
    }
    if ((st = cuda_status(cudaMemcpyAsync(&hb, counters.p, sizeof(BinCounters), cudaMemcpyDeviceToHost, s),
                          "copy bins")))
      break;
    if ((st = cuda_status(cudaStreamSynchronize(s), "sync bins"))) break;
    if (hrows > 0) {
      if ((st = buf_alloc(a, g->dense, (size_t)dquads * 16, s))) break;
      if ((st = cuda_status(cudaMemsetAsync(g->dense.p, 0, (size_t)dquads * 16, s), "memset dense"))) break;
      k_dense_fill<<<grid_for(wn * 32, 256), 256, 0, s>>>(g->off.as<int64_t>(), g->col.as<int32_t>(),
                                                           odeg.as<int32_t>(), n, vw.base_w, g->dq0.as<int32_t>(),
                                                           g->dense.as<uint32_t>(), nullptr);
      if ((st = launched("k_dense_fill"))) break;
      // the graph is complete when tc_build returns: another stream may count it next
      if ((st = cuda_status(cudaStreamSynchronize(s), "sync dense rows"))) break;
      g->dense_rows = (int64_t)hrows;
      g->dense_quads = dquads;
    } else {
      buf_release(a, g->dq0, s);
    }
  } while (0);

  for (Buf* b : {&alt, &part, &counters, &odeg, &ukeys, &rkeys, &rkeys_alt, &rank, &rcount, &ustart, &plen, &dnq,
                 &dqoff, &rowinfo})
    buf_release(a, *b, s);
  buf_release(a, g->keys, s);
  buf_release(a, g->indeg, s);
  buf_release(a, g->ingest, s);
  if (st != TC_OK) return st;
  g->wedges = (int64_t)hb.wedges;
  g->dense_wedges = g->dense_rows > 0 ? (int64_t)hb.dense_wedges : 0;
  g->dense_visits = g->dense_rows > 0 ? (int64_t)hb.dense_visits : 0;
  g->active = (int64_t)hb.active;
  g->nb = hb.nb;
  g->nw = hb.nw;
  g->nt = hb.nt;
  g->max_out_degree = hb.max_out;
  return TC_OK;
}

}  // namespace tc

namespace tc {

int bits_of(int64_t x) {
  int b = 0;
  while (b < 63 && (int64_t(1) << b) <= x) ++b;
  return b;
}

void apply_sizes(tc_graph* g, const CompactSizes& hs) {
  g->m = (int64_t)hs.rc.m;
  g->csr_entries = hs.entries;
  g->dense_rows = (int64_t)hs.dense_rows;
  g->dense_quads = hs.dquads;
  g->wedges = (int64_t)hs.bc.wedges;
  g->dense_wedges = g->dense_rows > 0 ? (int64_t)hs.bc.dense_wedges : 0;
  g->dense_visits = g->dense_rows > 0 ? (int64_t)hs.bc.dense_visits : 0;
  g->active = (int64_t)hs.bc.active;
  g->nb = hs.bc.nb;
  g->nw = hs.bc.nw;
  g->nt = hs.bc.nt;
  g->max_out_degree = hs.bc.max_out;
}

namespace {

// Scratch of a compact build, all pieces of one allocation.
struct CompactScratch {
  CompactSizes* sizes;
  uint64_t *rkeys, *rkeys_alt;
  int32_t *rank, *tgt, *odeg, *lists, *dnq;
  int64_t *pstart, *cur;
  uint64_t* psz;  // [n + 1] (padded length << 32) | dense quads, scanned in place
  int2* rowinfo;
  void *scan_tmp, *sort_tmp;
};

CompactScratch compact_scratch(Arena& ar, int64_t n, int64_t M, int64_t wn) {
  CompactScratch c;
  c.sizes = ar.take<CompactSizes>(1);
  c.rkeys = ar.take<uint64_t>(n);
  c.rkeys_alt = ar.take<uint64_t>(n);
  c.rank = ar.take<int32_t>(n);
  c.pstart = ar.take<int64_t>(n + 1);
  c.cur = ar.take<int64_t>(n);
  c.tgt = ar.take<int32_t>(2 * M);
  c.odeg = ar.take<int32_t>(n);
  c.lists = ar.take<int32_t>(n);
  c.psz = ar.take<uint64_t>(n + 1);
  c.rowinfo = ar.take<int2>(n);
  c.dnq = ar.take<int32_t>(wn > 0 ? wn : 1);
  c.scan_tmp = ar.take<char>(scan_temp_bytes(n > wn ? n : wn));
  c.sort_tmp = ar.take<char>(radix_temp_bytes(n));
  return c;
}

}  // namespace

void csr_views(Arena& ar, tc_graph* g, int64_t n, int64_t bound_entries, int64_t wn, int64_t dense_quads) {
  g->off = ar.view((size_t)(n + 1) * 8);
  g->col = ar.view((size_t)(bound_entries + 4) * 4);
  g->perm = ar.view((size_t)n * 4);
  g->list = ar.view((size_t)n * 4);
  g->tlist = ar.view((size_t)n * 4);
  g->dq0 = ar.view((size_t)(wn > 0 ? wn : 1) * 4);
  g->dense = ar.view((size_t)dense_quads * 16);
}

// tc_build for inputs of up to compact_max_pairs() pairs, on the bucketed path, with one host synchronisation and
// few host calls: the same kernels as build_graph_pruned, launched back to back; every buffer whose size depends on
// the data is allocated at a bound known from n and the pair count M, and every size is read back once at the end.
//   rank sort   on bits(M) count bits (an input-pair count is at most M) instead of the measured maximum
//   columns     at most M + 3 min(n, M) padded entries (m <= M; padding adds at most 3 per non-empty row)
//   dense rows  at most M / 4 quads (a row is dense only when it has at least 4 entries per quad); each row is
//               zeroed by the warp that fills it
// All scratch is one allocation, and the graph's arrays are views into one block, so a build makes two allocation
// calls: for small graphs the host calls, not the kernels, took most of the build.
tc_status build_graph_compact(tc_graph* g, cudaStream_t s) {
  const Allocator& a = g->alloc;
  const int B = g->key_bits;
  const int64_t M = g->num_pairs;
  const int64_t n = g->n;
  tc_status st = TC_OK;
  auto launched = [&](const char* what) {
    note_launch();
    return cuda_status(cudaGetLastError(), what);
  };
  int32_t mid_max = 2048;
  while ((2 * M) / mid_max > (int64_t)kBigBits) mid_max <<= 1;
  const int64_t bound_entries = M + 3 * (n < M ? n : M);
  const int64_t bound_quads = M / 4 + 1;
  // the offsets and dense quads are scanned as the two 32-bit halves of one word
  if (bound_entries + 4 >= (int64_t(1) << 32) || bound_quads >= (int64_t(1) << 32))
    return build_graph_pruned(g, -1, nullptr, s);
  const int64_t base_w = tc_graph::window_base(n, kWarpBitmapBits);
  const int64_t wn = n - base_w;
  Buf scratch;
  do {
    // ---- the two allocations ----
    Arena sizing;
    compact_scratch(sizing, n, M, wn);
    if ((st = buf_alloc(a, scratch, sizing.used, s))) break;
    Arena sa{scratch.as<char>()};
    const CompactScratch c = compact_scratch(sa, n, M, wn);
    Arena bsizing;
    csr_views(bsizing, g, n, bound_entries, wn, bound_quads);
    if ((st = buf_alloc(a, g->block, bsizing.used, s))) break;
    Arena ba{g->block.as<char>()};
    csr_views(ba, g, n, bound_entries, wn, bound_quads);
    if ((st = cuda_status(cudaMemsetAsync(c.sizes, 0, sizeof(CompactSizes), s), "memset sizes"))) break;
    CompactSizes* ds = c.sizes;
    // ---- rank: stable sort of (count << B) | id on the count bits ----
    uint64_t* rs = nullptr;
    const int count_bits = bits_of(M);
    if (count_bits > kRankClampBits && (2 * M) / kRankClamp + 1 <= kRankTailMax) {
      // two radix passes on the clamped counts, then the few vertices at the clamp ordered by their true counts
      k_rank_keys_clamped<<<grid_for(n, 256), 256, 0, s>>>(g->indeg.as<int32_t>(), n, B, c.rkeys, &ds->rank_tail);
      if ((st = launched("k_rank_keys_clamped"))) break;
      if ((st = radix_sort_u64(a, c.rkeys, c.rkeys_alt, n, B, B + kRankClampBits, &rs, s, c.sort_tmp))) break;
      k_rank_tail<<<1, 1024, 0, s>>>(rs, n, B, g->indeg.as<int32_t>(), &ds->rank_tail, &ds->rank_err);
      if ((st = launched("k_rank_tail"))) break;
    } else {
      k_rank_keys<<<grid_for(n, 256), 256, 0, s>>>(g->indeg.as<int32_t>(), n, B, c.rkeys, nullptr);
      if ((st = launched("k_rank_keys"))) break;
      if ((st = radix_sort_u64(a, c.rkeys, c.rkeys_alt, n, B, B + count_bits, &rs, s, c.sort_tmp))) break;
    }
    // ranks, and each rank's bucket room (claimed, so no scan)
    k_rank_buckets<<<grid_for(n, 256), 256, 0, s>>>(rs, n, B, c.rank, g->perm.as<int32_t>(), c.pstart, c.cur,
                                                    &ds->bucket_alloc);
    if ((st = launched("k_rank_buckets"))) break;
    // ---- buckets: group by the lower-ranked endpoint, sort and de-duplicate each ----
    k_bucket<<<grid_for((M + kBucketItems - 1) / kBucketItems, 256), 256, 0, s>>>(
        g->keys.as<uint64_t>(), M, B, c.rank, reinterpret_cast<unsigned long long*>(c.cur), c.tgt);
    if ((st = launched("k_bucket"))) break;
    RowCounters* rc = &ds->rc;
    k_rows_small<<<grid_for(n, 256), 256, 0, s>>>(c.pstart, c.cur, n, c.tgt, c.odeg, c.lists, rc);
    if ((st = launched("k_rows_small"))) break;
    k_rows_warp<<<4 * num_sms(), kRowThreads, 0, s>>>(c.pstart, c.cur, n, c.tgt, c.odeg, c.lists, rc);
    if ((st = launched("k_rows_warp"))) break;
    const size_t blk_smem = (size_t)kBigBits / 8;
    if ((st = smem_attribute_once<k_rows_block>((int)blk_smem))) break;
    k_rows_block<<<num_sms(), kBigThreads, blk_smem, s>>>(c.pstart, c.cur, n, mid_max, c.tgt, c.odeg, c.lists, rc);
    if ((st = launched("k_rows_block"))) break;
    // ---- row codes, then one scan of (padded length << 32) | dense quads, then the rows with their offsets ----
    const int32_t wtopq = n > base_w ? (int32_t)(((n - 1 - base_w) >> 7) + 1) : 0;
    k_row_codes<<<grid_for(n, 256), 256, 0, s>>>(c.odeg, n, (int32_t)base_w, wtopq, c.psz, c.dnq, c.rowinfo);
    if ((st = launched("k_row_codes"))) break;
    if ((st = exclusive_scan_u64(a, c.psz, c.psz, n, s, c.scan_tmp))) break;
    k_rows_copy_scanned<<<grid_for(n, 256), 256, 0, s>>>(c.pstart, c.tgt, c.odeg, c.psz, n, (int32_t)base_w,
                                                         g->off.as<int64_t>(), g->col.as<int32_t>(),
                                                         g->dq0.as<int32_t>(), ds);
    if ((st = launched("k_rows_copy_scanned"))) break;
    // ---- bins ----
    k_bins<<<grid_for(n, 256), 256, 0, s>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), c.rowinfo, n,
                                            block_min_work_for(M), g->list.as<int32_t>(), g->tlist.as<int32_t>(),
                                            &ds->bc);
    if ((st = launched("k_bins"))) break;
    // ---- dense rows: the bitmaps (each row zeroed by its own warp) ----
    k_dense_fill<<<grid_for(wn * 32, 256), 256, 0, s>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), c.odeg, n,
                                                         (int32_t)base_w, g->dq0.as<int32_t>(),
                                                         g->dense.as<uint32_t>(), c.dnq);
    if ((st = launched("k_dense_fill"))) break;
    // ---- every size at once, then the one synchronisation ----
    CompactSizes* hs = reinterpret_cast<CompactSizes*>(g->host_total + 1);
    if ((st = cuda_status(cudaMemcpyAsync(hs, ds, sizeof(CompactSizes), cudaMemcpyDeviceToHost, s), "copy sizes")))
      break;
    // the graph is complete when tc_build returns: another stream may count it next
    if ((st = cuda_status(cudaStreamSynchronize(s), "tc_build sync"))) break;
    if (hs->rc.err) {
      set_error("tc_build: a bucket's targets exceeded the range bound (inconsistent pair counts)");
      st = TC_ERR_INTERNAL;
      break;
    }
    if (hs->rank_err) {
      set_error("tc_build: more vertices at the rank sort's count clamp than its fix-up sort holds");
      st = TC_ERR_INTERNAL;
      break;
    }
    if (hs->entries > bound_entries || hs->dquads > bound_quads) {
      set_error("tc_build: the compact build's size bounds were exceeded");
      st = TC_ERR_INTERNAL;
      break;
    }
    apply_sizes(g, *hs);
  } while (0);
  buf_release(a, scratch, s);
  buf_release(a, g->keys, s);
  buf_release(a, g->indeg, s);
  buf_release(a, g->ingest, s);
  return st;
}

}  // namespace tc

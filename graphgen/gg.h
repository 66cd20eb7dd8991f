/*
 * gg.h — seeded synthetic graph inputs, identical on host and device.
 *
 * This header holds the input generators only: it contains none of the triangle-counting arithmetic, and both
 * the CPU oracle's tests and the CUDA library's tests and benchmark draw their edge lists from it.  Every edge is
 * a pure function of (seed, edge index), so a host thread and a CUDA thread that evaluate the same edge produce the
 * same bits, and a graph of any size can be generated in parallel without sharing state.
 *
 * Random numbers: a counter-based use of the SplitMix64 output function (Steele, Lea & Flood, "Fast Splittable
 * Pseudorandom Number Generators", OOPSLA 2014).  The i-th draw of stream key k is mix64(k + (i+1)*GAMMA), GAMMA the
 * 64-bit golden-ratio constant; mix64 is the published variant-13 finaliser of MurmurHash3's fmix64.
 *
 * Generators:
 *  - Uniform edge sampling ("ER"): edge e draws one 64-bit word; its high and low 32-bit halves pick the two
 *    endpoints uniformly from [0,n) by multiply-shift (Lemire, "Fast Random Integer Generation in an Interval",
 *    TOMACS 2019, without the rejection step; the bias is below n/2^32).  Self-loops and duplicate pairs can occur
 *    and are left for the graph builder to remove, as the workloads prescribe.
 *  - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004): each edge descends `scale` levels of the 2x2 quadrant
 *    recursion; level l compares one 32-bit draw with the cumulative thresholds of (a_l, b_l, c_l, d_l).  The
 *    per-level thresholds are inputs (computed once on the host from the seed), so host and device agree bit for
 *    bit.  When n is not a power of two an edge whose endpoint falls at or above n is redrawn with the next attempt
 *    counter, up to GG_RMAT_MAX_ATTEMPTS attempts, after which both endpoints are reduced modulo n.
 *  - Vertex relabelling: a 4-round balanced Feistel network on 2h bits (Luby & Rackoff 1988) with cycle-walking
 *    (Black & Rogaway, "Ciphers with Arbitrary Finite Domains", CT-RSA 2002) gives a seeded bijection on [0,n).
 *  - Erdos-Renyi G(n, p) (every pair {i, j} present independently with probability p; no self-loops, no repeats)
 *    by geometric skipping (Batagelj & Brandes, "Efficient generation of large random networks", Phys. Rev. E 71,
 *    2005): row i walks the candidates j = i+1 .. n-1 and jumps over a Geometric(p) number of absent pairs before
 *    each present one.  Rows are independent (row i's draws use counters (i << 32) | t), so rows run in parallel.
 *    The gap is drawn by inversion, floor(log2(U) / log2(1-p)) with U uniform on (0, 1], both logarithms in
 *    Q.40 fixed point from the bit-by-bit squaring method for the binary logarithm, so the host and the device
 *    take the same integer steps.  -log2(1-p) is an input (lq), computed once by the caller with the same method.
 *    The gap law is exact up to the 2^-40 truncation of the logarithms.
 */
#ifndef GRAPHGEN_GG_H
#define GRAPHGEN_GG_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GG_HD __host__ __device__ __forceinline__
#else
#define GG_HD static inline
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL
#define GG_RMAT_MAX_ATTEMPTS 64

/* SplitMix64 finaliser (Steele, Lea & Flood 2014, "mix64"). */
GG_HD uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Stream key for (seed, stream id): separates the draws of different generators that share a seed. */
GG_HD uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix64(seed + GG_GAMMA * (2 * stream + 1)) ^ gg_mix64(stream + 0x632BE59BD9B4E019ULL);
}

/* ctr-th draw of stream key k. */
GG_HD uint64_t gg_draw(uint64_t key, uint64_t ctr) { return gg_mix64(key + (ctr + 1) * GG_GAMMA); }

/* Uniform integer in [0, n) from 32 random bits (multiply-shift). */
GG_HD uint32_t gg_below(uint32_t r32, uint32_t n) { return (uint32_t)(((uint64_t)r32 * (uint64_t)n) >> 32); }

/* Stream ids used by the generators (4 and 5 are drawn by the Python workload definitions). */
enum { GG_STREAM_ER = 1, GG_STREAM_RMAT = 2, GG_STREAM_PERM = 3, GG_STREAM_GNP = 6 };

/* 64 x 64 -> 128-bit unsigned product. */
GG_HD void gg_mul64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
#if defined(__CUDA_ARCH__)
  *hi = __umul64hi(a, b);
  *lo = a * b;
#else
  const unsigned __int128 p = (unsigned __int128)a * b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
#endif
}

/* Number of leading zero bits of x != 0. */
GG_HD int gg_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

#define GG_LOG_FRAC_BITS 40

/* log2(x) for x >= 1 in Q.40 fixed point (truncated).  The integer part is the position of the top bit; the
 * fraction comes one bit at a time from the mantissa m in [1, 2): square it, and a square of 2 or more is a 1 bit
 * and is halved, else a 0 bit. */
GG_HD uint64_t gg_log2_q40(uint64_t x) {
  const int e = 63 - gg_clz64(x);
  uint64_t m = x << (63 - e); /* mantissa, Q1.63 */
  uint64_t r = (uint64_t)e << GG_LOG_FRAC_BITS;
  for (int b = GG_LOG_FRAC_BITS - 1; b >= 0; --b) {
    uint64_t hi, lo;
    gg_mul64(m, m, &hi, &lo); /* m^2 in Q2.126 */
    if (hi >> 63) {           /* m^2 >= 2: bit set, keep m^2 / 2 */
      r |= (uint64_t)1 << b;
      m = hi;
    } else {
      m = (hi << 1) | (lo >> 63);
    }
  }
  return r;
}

/* A Geometric(p) variate (absent pairs before the next present one) from the 64-bit draw r, with
 * lq = -log2(1 - p) in Q.40 (lq > 0).  U = ((r >> 1) + 1) / 2^63 lies in (0, 1]; the variate is
 * floor(-log2(U) / lq), and P(variate >= k) = P(U <= (1-p)^k) = (1-p)^k. */
GG_HD uint64_t gg_geometric(uint64_t r, uint64_t lq) {
  const uint64_t x = (r >> 1) + 1;
  const uint64_t neg_log2_u = ((uint64_t)63 << GG_LOG_FRAC_BITS) - gg_log2_q40(x);
  return neg_log2_u / lq;
}

/* Row i of G(n, p): the present pairs {i, j}, j = i+1 .. n-1, in ascending j.  Writes them to src/dst when src is
 * not null and returns how many there are.  lq = 0 stands for p = 0 (no pairs). */
GG_HD int64_t gg_gnp_row(uint64_t seed, uint32_t n, uint64_t lq, uint32_t i, int32_t* src, int32_t* dst) {
  if (lq == 0 || (uint64_t)i + 1 >= (uint64_t)n) return 0;
  const uint64_t key = gg_key(seed, GG_STREAM_GNP);
  const uint64_t len = (uint64_t)n - 1 - i; /* candidates */
  uint64_t k = 0;                           /* first candidate not yet decided */
  int64_t c = 0;
  for (uint64_t t = 0; k < len; ++t) {
    const uint64_t gap = gg_geometric(gg_draw(key, ((uint64_t)i << 32) | t), lq);
    if (gap >= len - k) break;
    k += gap;
    if (src) {
      src[c] = (int32_t)i;
      dst[c] = (int32_t)(i + 1 + k);
    }
    ++c;
    ++k;
  }
  return c;
}

/* Edge e of the uniform edge sampler on n vertices. */
GG_HD void gg_er_edge(uint64_t seed, uint32_t n, uint64_t e, int32_t* s, int32_t* d) {
  uint64_t r = gg_draw(gg_key(seed, GG_STREAM_ER), e);
  *s = (int32_t)gg_below((uint32_t)(r >> 32), n);
  *d = (int32_t)gg_below((uint32_t)r, n);
}

/* Edge e of an R-MAT graph with 2^scale >= n vertices.  thr[3*l + 0..2] are the cumulative thresholds
 * (a_l, a_l+b_l, a_l+b_l+c_l) * 2^32 of level l (level 0 picks the most significant bit). */
GG_HD void gg_rmat_edge(uint64_t seed, int scale, uint32_t n, const uint32_t* thr, uint64_t e, int32_t* s,
                        int32_t* d) {
  const uint64_t key = gg_key(seed, GG_STREAM_RMAT);
  const int pairs = (scale + 1) / 2; /* one 64-bit draw serves two levels */
  uint32_t src = 0, dst = 0;
  for (int att = 0; att < GG_RMAT_MAX_ATTEMPTS; ++att) {
    const uint64_t base = (e * GG_RMAT_MAX_ATTEMPTS + (uint64_t)att) * (uint64_t)pairs;
    src = 0;
    dst = 0;
    uint64_t r = 0;
    for (int l = 0; l < scale; ++l) {
      uint32_t r32;
      if ((l & 1) == 0) {
        r = gg_draw(key, base + (uint64_t)(l >> 1));
        r32 = (uint32_t)(r >> 32);
      } else {
        r32 = (uint32_t)r;
      }
      const uint32_t t1 = thr[3 * l + 0], t2 = thr[3 * l + 1], t3 = thr[3 * l + 2];
      const uint32_t sbit = (r32 >= t2) ? 1u : 0u;                          /* quadrants c, d: lower half */
      const uint32_t dbit = ((r32 >= t1 && r32 < t2) || r32 >= t3) ? 1u : 0u; /* quadrants b, d: right half */
      src = (src << 1) | sbit;
      dst = (dst << 1) | dbit;
    }
    if (src < n && dst < n) {
      *s = (int32_t)src;
      *d = (int32_t)dst;
      return;
    }
  }
  *s = (int32_t)(src % n);
  *d = (int32_t)(dst % n);
}

/* Seeded bijection on [0, n): Feistel on 2h bits (2^(2h) >= n) with cycle-walking. */
GG_HD uint32_t gg_permute(uint64_t seed, uint32_t n, uint32_t x) {
  int h = 1;
  while ((1ULL << (2 * h)) < (uint64_t)n) ++h;
  const uint32_t mask = (uint32_t)((1ULL << h) - 1);
  const uint64_t key = gg_key(seed, GG_STREAM_PERM);
  uint32_t y = x;
  do {
    uint32_t L = y >> h, R = y & mask;
    for (int round = 0; round < 4; ++round) {
      const uint32_t F = (uint32_t)gg_draw(key, ((uint64_t)round << 32) | R) & mask;
      const uint32_t nL = R;
      R = L ^ F;
      L = nL;
    }
    y = (L << h) | R;
  } while (y >= n);
  return y;
}

#endif /* GRAPHGEN_GG_H */

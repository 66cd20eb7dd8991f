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

/* Stream ids used by the generators. */
enum { GG_STREAM_ER = 1, GG_STREAM_RMAT = 2, GG_STREAM_PERM = 3 };

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

/*
 * gg_core.h - seeded, counter-based synthetic graph generators.
 *
 * This header is the one source of the synthetic inputs used by the tests,
 * the benchmark and the stored expected values. It is compiled twice: into
 * the host library (plain C + OpenMP, gg_host.c) and into the device library
 * (CUDA, gg_device.cu). Every function is pure 64-bit integer arithmetic, so
 * x86-64, aarch64 and the GPU produce the same bits for the same arguments.
 * Nothing here computes connected components.
 *
 * Random numbers: splitmix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). The i-th output of a
 * splitmix64 stream whose state starts at k is mix64(k + (i + 1) * gamma);
 * gg_draw(key, i) evaluates exactly that, so any output can be computed
 * without the ones before it (counter-based use).
 *
 * Generators (each emits uint32 (u, v) pairs interleaved u0, v0, u1, v1, ...):
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004) with the Graph500
 *     quadrant probabilities a = 0.57, b = 0.19, c = 0.19, d = 0.05 and no
 *     parameter noise; one 32-bit draw per recursion level; an optional seeded
 *     bijective scramble of vertex ids on [0, 2^scale).
 *   - 2D grid W x H with 4-neighbour candidate edges, each kept with
 *     probability p; candidates in row-major order, "right" before "down".
 *   - Erdos-Renyi G(n, m): m independent uniform pairs (self-loops and
 *     duplicates kept).
 *   - the mixed batch of many small graphs and uniform-random pair batches.
 */
#ifndef GG_CORE_H
#define GG_CORE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GG_HD static __host__ __device__ __forceinline__
#else
#define GG_HD static inline
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

/* Stream ids: independent splitmix64 streams for each use of randomness. */
#define GG_STREAM_RMAT 1ULL
#define GG_STREAM_SCRAMBLE 2ULL
#define GG_STREAM_GRID 3ULL
#define GG_STREAM_ER 4ULL
#define GG_STREAM_PAIRS 5ULL
#define GG_STREAM_BATCH_PLAN 6ULL
#define GG_STREAM_BATCH_GRAPH 0x100000000ULL /* + graph index */

/* R-MAT quadrant thresholds on a uniform 32-bit draw r:
 *   r <  round(0.57 * 2^32)  -> quadrant a (u bit 0, v bit 0)
 *   r <  round(0.76 * 2^32)  -> quadrant b (u bit 0, v bit 1)
 *   r <  round(0.95 * 2^32)  -> quadrant c (u bit 1, v bit 0)
 *   otherwise                -> quadrant d (u bit 1, v bit 1)          */
#define GG_RMAT_TA 2448131359u
#define GG_RMAT_TAB 3264175145u
#define GG_RMAT_TABC 4080218931u

/* Keep threshold for the grid: round(0.9 * 2^32). */
#define GG_P90 3865470566u

/* splitmix64 output function. */
GG_HD uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Starting state of the stream (seed, stream). */
GG_HD uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix64(seed * GG_GAMMA + gg_mix64(stream ^ 0x632BE59BD9B4E019ULL));
}

/* Output number idx of the stream that starts at state key. */
GG_HD uint64_t gg_draw(uint64_t key, uint64_t idx) {
  return gg_mix64(key + (idx + 1ULL) * GG_GAMMA);
}

/* floor(r * n / 2^32): a uniform value in [0, n) from a 32-bit draw. */
GG_HD uint32_t gg_range32(uint32_t r, uint64_t n) {
  return (uint32_t)(((uint64_t)r * n) >> 32);
}

/* ---------------------------------------------------------------- R-MAT */

/* Edge number e of an unscrambled R-MAT graph with 2^scale vertices
 * (1 <= scale <= 32). Level l (most significant bit first) uses the low
 * 32 bits of draw e*ceil(scale/2) + l/2 for even l and the high 32 bits for
 * odd l. */
GG_HD void gg_rmat_edge_raw(uint64_t key, int scale, uint64_t e, uint32_t *u,
                            uint32_t *v) {
  uint64_t a = 0, b = 0;
  uint64_t base = e * (uint64_t)((scale + 1) / 2);
  for (int l = 0; l < scale; l += 2) {
    uint64_t r = gg_draw(key, base + (uint64_t)(l / 2));
    for (int h = 0; h < 2; ++h) {
      if (l + h >= scale) break;
      uint32_t r32 = h ? (uint32_t)(r >> 32) : (uint32_t)r;
      uint64_t bu = r32 >= GG_RMAT_TAB;
      uint64_t bv = (r32 >= GG_RMAT_TA && r32 < GG_RMAT_TAB) || r32 >= GG_RMAT_TABC;
      a = (a << 1) | bu;
      b = (b << 1) | bv;
    }
  }
  *u = (uint32_t)a;
  *v = (uint32_t)b;
}

/* Seeded bijection on [0, 2^scale): two rounds of
 *   x <- (x * odd + add) mod 2^scale;  x <- x xor (x >> ceil(scale/2)).
 * Multiplication by an odd number, addition and a right xorshift are each
 * invertible modulo 2^scale, so the composition is a permutation. */
GG_HD uint32_t gg_scramble(uint64_t skey, int scale, uint32_t x) {
  uint64_t mask = (scale >= 32) ? 0xFFFFFFFFULL : ((1ULL << scale) - 1ULL);
  uint64_t y = x;
  int sh = (scale + 1) / 2;
  for (uint64_t r = 0; r < 2; ++r) {
    uint64_t k = gg_draw(skey, r);
    uint64_t mul = (k | 1ULL) & mask;
    uint64_t add = (k >> 32) & mask;
    y = (y * mul + add) & mask;
    y ^= y >> sh;
  }
  return (uint32_t)y;
}

/* Edge e of R-MAT(scale, seed), scrambled when scramble != 0. */
GG_HD void gg_rmat_edge(uint64_t seed, int scale, int scramble, uint64_t e,
                        uint32_t *u, uint32_t *v) {
  uint32_t a, b;
  gg_rmat_edge_raw(gg_key(seed, GG_STREAM_RMAT), scale, e, &a, &b);
  if (scramble) {
    uint64_t sk = gg_key(seed, GG_STREAM_SCRAMBLE);
    a = gg_scramble(sk, scale, a);
    b = gg_scramble(sk, scale, b);
  }
  *u = a;
  *v = b;
}

/* ---------------------------------------------------------------- grid */

/* Candidate slot s = 2*(r*W + c) + dir of a W x H grid: dir 0 joins (r,c) to
 * (r,c+1) and exists for c+1 < W; dir 1 joins (r,c) to (r+1,c) and exists for
 * r+1 < H. A candidate is kept when the low 32 bits of draw s are below
 * p_thresh and both endpoint ids (r*W + c) are below n_limit. Returns 1 and
 * writes the pair when slot s yields an edge, else 0. */
GG_HD int gg_grid_slot(uint64_t gkey, uint32_t W, uint32_t H, uint64_t n_limit,
                       uint32_t p_thresh, uint64_t s, uint32_t *u, uint32_t *v) {
  uint64_t cell = s >> 1;
  uint32_t dir = (uint32_t)(s & 1ULL);
  uint64_t r = cell / W, c = cell % W;
  uint64_t a = cell, b;
  if (dir == 0) {
    if (c + 1 >= W) return 0;
    b = cell + 1;
  } else {
    if (r + 1 >= H) return 0;
    b = cell + W;
  }
  if (a >= n_limit || b >= n_limit) return 0;
  if ((uint32_t)gg_draw(gkey, s) >= p_thresh) return 0;
  *u = (uint32_t)a;
  *v = (uint32_t)b;
  return 1;
}

/* ---------------------------------------------------------------- G(n,m) */

/* Pair e of G(n, m): u from the low, v from the high 32 bits of draw e. */
GG_HD void gg_er_edge(uint64_t ekey, uint64_t n, uint64_t e, uint32_t *u,
                      uint32_t *v) {
  uint64_t r = gg_draw(ekey, e);
  *u = gg_range32((uint32_t)r, n);
  *v = gg_range32((uint32_t)(r >> 32), n);
}

/* ---------------------------------------------------------------- batch */

/* Kinds of graphs in the mixed batch. */
#define GG_KIND_ER 0
#define GG_KIND_RMAT 1
#define GG_KIND_GRID 2

/* Integer square root: largest w with w*w <= x. */
GG_HD uint64_t gg_isqrt(uint64_t x) {
  uint64_t r = 0, bit = 1ULL << 62;
  while (bit > x) bit >>= 2;
  while (bit) {
    if (x >= r + bit) {
      x -= r + bit;
      r = (r >> 1) + bit;
    } else {
      r >>= 1;
    }
    bit >>= 2;
  }
  return r;
}

/* Smallest s with 2^s >= x (x >= 1). */
GG_HD int gg_ceil_log2(uint64_t x) {
  int s = 0;
  while ((1ULL << s) < x) ++s;
  return s;
}

/* Shape of graph g of the mixed batch:
 *   kind: draw0 mod 100 < 40 -> G(n,m); < 80 -> R-MAT; else grid (p = 0.9);
 *   |V|:  octave e uniform in 8..17, then |V| uniform in [2^e, 2^(e+1)),
 *         a piecewise log-uniform law on [2^8, 2^18);
 *   average degree d = d2 / 2 with d2 uniform in 4..64 (d in [2, 32] in
 *   steps of 0.5) and |E| = round(|V| * d / 2) = floor((|V| * d2 + 2) / 4)
 *   for G(n,m) and R-MAT; the grid ignores d (w = isqrt(|V|),
 *   h = ceil(|V| / w), ids >= |V| cut). */
typedef struct gg_batch_shape {
  uint32_t kind;
  uint32_t n_vertices;
  uint64_t n_edges_target; /* exact for G(n,m) and R-MAT; grid: see gg_grid_* */
  uint32_t grid_w, grid_h;
} gg_batch_shape;

GG_HD gg_batch_shape gg_batch_graph_shape(uint64_t seed, uint64_t g) {
  gg_batch_shape s;
  uint64_t pk = gg_key(seed, GG_STREAM_BATCH_PLAN);
  uint64_t r0 = gg_draw(pk, 3 * g + 0);
  uint64_t r1 = gg_draw(pk, 3 * g + 1);
  uint64_t r2 = gg_draw(pk, 3 * g + 2);
  uint32_t k = (uint32_t)(r0 % 100ULL);
  s.kind = k < 40 ? GG_KIND_ER : (k < 80 ? GG_KIND_RMAT : GG_KIND_GRID);
  uint32_t e = 8u + (uint32_t)((r0 >> 32) % 10ULL);
  s.n_vertices = (1u << e) + (uint32_t)(r1 % (1ULL << e));
  uint64_t d2 = 4ULL + (r2 % 61ULL);
  s.n_edges_target = ((uint64_t)s.n_vertices * d2 + 2ULL) / 4ULL;
  s.grid_w = (uint32_t)gg_isqrt(s.n_vertices);
  s.grid_h = (s.n_vertices + s.grid_w - 1) / s.grid_w;
  return s;
}

/* Edge e of an R-MAT batch graph on n vertices at scale ceil(log2 n): draw
 * attempt a = 0..63 uses R-MAT edge index e*64 + a (unscrambled) and the first
 * attempt with both ids < n is kept; if all 64 fail, ids are reduced mod n. */
GG_HD void gg_batch_rmat_edge(uint64_t gkey, uint32_t n, uint64_t e, uint32_t *u,
                              uint32_t *v) {
  int scale = gg_ceil_log2(n);
  if (scale < 1) scale = 1;
  uint32_t a = 0, b = 0;
  for (uint64_t t = 0; t < 64; ++t) {
    gg_rmat_edge_raw(gkey, scale, e * 64ULL + t, &a, &b);
    if (a < n && b < n) {
      *u = a;
      *v = b;
      return;
    }
  }
  *u = a % n;
  *v = b % n;
}

#endif /* GG_CORE_H */

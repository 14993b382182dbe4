/*
 * gg_host.c - host (CPU, OpenMP) build of the seeded generators in gg_core.h.
 * Output is bit-identical to the device build (gg_device.cu) and independent
 * of the thread count: every edge is a pure function of its index.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gg_core.h"

#define GG_EXPORT __attribute__((visibility("default")))

/* Edges [e_begin, e_end) of R-MAT(scale, seed) into out[0 .. 2*(e_end-e_begin)). */
GG_EXPORT void gg_rmat(uint64_t seed, int scale, int scramble, uint64_t e_begin,
                       uint64_t e_end, uint32_t *out) {
  int64_t cnt = (int64_t)(e_end - e_begin);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < cnt; ++i) {
    uint32_t u, v;
    gg_rmat_edge(seed, scale, scramble, e_begin + (uint64_t)i, &u, &v);
    out[2 * i] = u;
    out[2 * i + 1] = v;
  }
}

/* Pairs [e_begin, e_end) of G(n, m) with the given seed. */
GG_EXPORT void gg_er(uint64_t seed, uint64_t n, uint64_t e_begin, uint64_t e_end,
                     uint32_t *out) {
  uint64_t k = gg_key(seed, GG_STREAM_ER);
  int64_t cnt = (int64_t)(e_end - e_begin);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < cnt; ++i) {
    uint32_t u, v;
    gg_er_edge(k, n, e_begin + (uint64_t)i, &u, &v);
    out[2 * i] = u;
    out[2 * i + 1] = v;
  }
}

/* count uniform pairs on [0, n) from stream (seed, GG_STREAM_PAIRS, tag):
 * insert and query batches. */
GG_EXPORT void gg_pairs(uint64_t seed, uint64_t tag, uint64_t n, uint64_t count,
                        uint32_t *out) {
  uint64_t k = gg_key(seed ^ gg_mix64(tag + 0x5851F42D4C957F2DULL), GG_STREAM_PAIRS);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)count; ++i) {
    uint32_t u, v;
    gg_er_edge(k, n, (uint64_t)i, &u, &v);
    out[2 * i] = u;
    out[2 * i + 1] = v;
  }
}

#define GG_GRID_CHUNK (1ULL << 20)

static uint64_t grid_chunk_count(uint64_t gkey, uint32_t W, uint32_t H,
                                 uint64_t n_limit, uint32_t p, uint64_t s0,
                                 uint64_t s1) {
  uint64_t c = 0;
  for (uint64_t s = s0; s < s1; ++s) {
    uint32_t u, v;
    c += (uint64_t)gg_grid_slot(gkey, W, H, n_limit, p, s, &u, &v);
  }
  return c;
}

/* Number of edges the W x H grid keeps (see gg_grid_slot). */
GG_EXPORT uint64_t gg_grid_count(uint64_t seed, uint32_t W, uint32_t H,
                                 uint64_t n_limit, uint32_t p_thresh) {
  uint64_t gkey = gg_key(seed, GG_STREAM_GRID);
  uint64_t slots = 2ULL * (uint64_t)W * (uint64_t)H;
  int64_t nch = (int64_t)((slots + GG_GRID_CHUNK - 1) / GG_GRID_CHUNK);
  uint64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
  for (int64_t ch = 0; ch < nch; ++ch) {
    uint64_t s0 = (uint64_t)ch * GG_GRID_CHUNK;
    uint64_t s1 = s0 + GG_GRID_CHUNK < slots ? s0 + GG_GRID_CHUNK : slots;
    total += grid_chunk_count(gkey, W, H, n_limit, p_thresh, s0, s1);
  }
  return total;
}

/* The kept grid edges, in slot order, into out; returns how many. out must
 * hold 2 * gg_grid_count(...) uint32. */
GG_EXPORT uint64_t gg_grid(uint64_t seed, uint32_t W, uint32_t H, uint64_t n_limit,
                           uint32_t p_thresh, uint32_t *out) {
  uint64_t gkey = gg_key(seed, GG_STREAM_GRID);
  uint64_t slots = 2ULL * (uint64_t)W * (uint64_t)H;
  int64_t nch = (int64_t)((slots + GG_GRID_CHUNK - 1) / GG_GRID_CHUNK);
  uint64_t *off = (uint64_t *)calloc((size_t)nch + 1, sizeof(uint64_t));
  if (!off) return 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ch = 0; ch < nch; ++ch) {
    uint64_t s0 = (uint64_t)ch * GG_GRID_CHUNK;
    uint64_t s1 = s0 + GG_GRID_CHUNK < slots ? s0 + GG_GRID_CHUNK : slots;
    off[ch + 1] = grid_chunk_count(gkey, W, H, n_limit, p_thresh, s0, s1);
  }
  for (int64_t ch = 0; ch < nch; ++ch) off[ch + 1] += off[ch];
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ch = 0; ch < nch; ++ch) {
    uint64_t s0 = (uint64_t)ch * GG_GRID_CHUNK;
    uint64_t s1 = s0 + GG_GRID_CHUNK < slots ? s0 + GG_GRID_CHUNK : slots;
    uint64_t w = off[ch];
    for (uint64_t s = s0; s < s1; ++s) {
      uint32_t u, v;
      if (gg_grid_slot(gkey, W, H, n_limit, p_thresh, s, &u, &v)) {
        out[2 * w] = u;
        out[2 * w + 1] = v;
        ++w;
      }
    }
  }
  uint64_t total = off[nch];
  free(off);
  return total;
}

/* Shapes of the mixed batch: kinds[g], vtx_off[0..G], edge_off[0..G]. */
GG_EXPORT void gg_batch_plan(uint64_t seed, uint32_t n_graphs, uint32_t *kinds,
                             uint64_t *vtx_off, uint64_t *edge_off) {
  uint64_t *ne = (uint64_t *)malloc(sizeof(uint64_t) * (n_graphs ? n_graphs : 1));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t g = 0; g < (int64_t)n_graphs; ++g) {
    gg_batch_shape s = gg_batch_graph_shape(seed, (uint64_t)g);
    kinds[g] = s.kind;
    if (s.kind == GG_KIND_GRID) {
      uint64_t gk = gg_key(seed, GG_STREAM_BATCH_GRAPH + (uint64_t)g);
      uint64_t slots = 2ULL * s.grid_w * s.grid_h;
      ne[g] = grid_chunk_count(gk, s.grid_w, s.grid_h, s.n_vertices, GG_P90, 0, slots);
    } else {
      ne[g] = s.n_edges_target;
    }
  }
  vtx_off[0] = 0;
  edge_off[0] = 0;
  for (uint32_t g = 0; g < n_graphs; ++g) {
    gg_batch_shape s = gg_batch_graph_shape(seed, g);
    vtx_off[g + 1] = vtx_off[g] + s.n_vertices;
    edge_off[g + 1] = edge_off[g] + ne[g];
  }
  free(ne);
}

/* Edges of the mixed batch (graph-local ids), concatenated in graph order. */
GG_EXPORT void gg_batch_fill(uint64_t seed, uint32_t n_graphs, const uint64_t *edge_off,
                             uint32_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t g = 0; g < (int64_t)n_graphs; ++g) {
    gg_batch_shape s = gg_batch_graph_shape(seed, (uint64_t)g);
    uint64_t gk = gg_key(seed, GG_STREAM_BATCH_GRAPH + (uint64_t)g);
    uint32_t *o = out + 2 * edge_off[g];
    uint64_t ne = edge_off[g + 1] - edge_off[g];
    if (s.kind == GG_KIND_GRID) {
      uint64_t slots = 2ULL * s.grid_w * s.grid_h, w = 0;
      for (uint64_t t = 0; t < slots && w < ne; ++t) {
        uint32_t u, v;
        if (gg_grid_slot(gk, s.grid_w, s.grid_h, s.n_vertices, GG_P90, t, &u, &v)) {
          o[2 * w] = u;
          o[2 * w + 1] = v;
          ++w;
        }
      }
    } else if (s.kind == GG_KIND_RMAT) {
      for (uint64_t e = 0; e < ne; ++e) gg_batch_rmat_edge(gk, s.n_vertices, e, &o[2 * e], &o[2 * e + 1]);
    } else {
      for (uint64_t e = 0; e < ne; ++e) gg_er_edge(gk, s.n_vertices, e, &o[2 * e], &o[2 * e + 1]);
    }
  }
}

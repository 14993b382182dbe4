// cc_csr.cu - the edge pass and the root selection on CSR input
// (cc_run_csr): offsets[n + 1] (64-bit) and neighbors[offsets[n]], the
// in-memory layout of the paper's implementation (Section V). The edges are
// (u, neighbors[j]) for offsets[u] <= j < offsets[u + 1]; direction does not
// matter (Section II).
//
// What CSR changes on the GPU: every edge of row u shares the endpoint u, so
// the lanes of a warp that hold entries of one row load P[u] in one
// transaction, and a skewed graph pays about one random parent read per edge
// instead of two. max_degree() of Algorithm 4 is read from the offsets (the
// row length), as the paper does.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {

namespace {

// 32-bit streaming load of a neighbour id: non-coherent path, no L1 allocation.
__device__ __forceinline__ uint32_t ld_nc_u32(const uint32_t *a, uint64_t pol) {
  uint32_t r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
  return r;
}

// Row length of vertex v (0 when the offsets are not monotone there).
__device__ __forceinline__ uint64_t row_len(const uint64_t *off, uint32_t v) {
  const uint64_t a = off[v], b = off[v + 1];
  return b > a ? b - a : 0u;
}

// Longest row, and a check of the offsets: off[0] == 0, off[n] == n_entries,
// never decreasing (violations set kErrFormat). One pass also keeps the
// argmax key (min(length, 2^32 - 1) << 32) | ~v, which is exact unless a row
// reaches 2^32 - 1 entries (then k_csr_minid settles the smallest id).
__global__ void __launch_bounds__(256) k_csr_maxlen(const uint64_t *__restrict__ off, uint32_t n,
                                                    uint64_t n_entries, Ctrl *ctrl) {
  unsigned long long best = 0, key = 0;
  bool bad = false;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = off[v], b = off[v + 1];
    bad |= b < a;
    const uint64_t len = b > a ? b - a : 0u;
    best = len > best ? len : best;
    const uint64_t l32 = len < 0xFFFFFFFFull ? len : 0xFFFFFFFFull;
    const unsigned long long k = (l32 << 32) | (uint32_t)~(uint32_t)v;
    key = k > key ? k : key;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) bad |= off[0] != 0u || off[n] != n_entries;
  if (bad) set_err(ctrl, kErrFormat);
  best = warp_max_u64(best);
  key = warp_max_u64(key);
  if ((threadIdx.x & 31) == 0) {
    if (best) atomicMax(&ctrl->maxcnt, best);
    if (key) atomicMax(&ctrl->maxkey, key);
  }
}

// Smallest vertex with the longest row, when that row has 2^32 - 1 entries
// or more (the packed key cannot order such lengths); otherwise nothing.
__global__ void __launch_bounds__(256) k_csr_minid(const uint64_t *__restrict__ off, uint32_t n, Ctrl *ctrl) {
  const unsigned long long mx = *(volatile unsigned long long *)&ctrl->maxcnt;
  if (mx < 0xFFFFFFFFull) return;
  uint32_t best = 0xFFFFFFFFu;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    if (row_len(off, (uint32_t)v) == mx && (uint32_t)v < best) best = (uint32_t)v;
  best = __reduce_min_sync(0xFFFFFFFFu, best);
  if ((threadIdx.x & 31) == 0 && best != 0xFFFFFFFFu) atomicMin(&ctrl->m_sel, best);
}

__global__ void k_csr_finalize_m(Ctrl *ctrl) {
  if (ctrl->maxcnt >= 0xFFFFFFFFull) ctrl->maxkey = (unsigned long long)(uint32_t)~ctrl->m_sel;
}

// The row that holds entry t * tile: the largest r with off[r] <= t * tile
// (one binary search per tile, all tiles in parallel).
__global__ void __launch_bounds__(256) k_csr_tile_rows(const uint64_t *__restrict__ off, uint32_t n,
                                                       uint64_t n_tiles, uint32_t tile, uint32_t *tile_row) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_tiles;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = t * tile;
    uint32_t lo = 0, hi = n;  // off[lo] <= j (off[0] = 0) ... answer in [lo, hi)
    while (hi - lo > 1u) {
      const uint32_t mid = lo + (hi - lo) / 2u;
      if (off[mid] <= j)
        lo = mid;
      else
        hi = mid;
    }
    tile_row[t] = lo;
  }
}

// Chunks of 32 entries a warp handles per iteration: their neighbour loads,
// then their row searches, then all their parent loads are issued before any
// of them is used, so that a warp keeps 2 * kCsrChunks parent loads in flight.
// Edge pass, ms, for 1 / 2 / 4 / 8 chunks: R-MAT 24 1.40 / 1.35 / 1.40 / 1.70,
// the 8192^2 grid 1.44 / 1.44 / 1.46 / 2.36, R-MAT 26 (P larger than L2)
// 11.0 / 10.6 / 10.9 / 9.9. More loads in flight per warp barely help: the
// pass is bound by its random parent requests, which the COO pass cuts with
// the zero-tree bitmap and the hot-vertex table.
#ifndef CC_CSR_CHUNKS
#define CC_CSR_CHUNKS 2
#endif
constexpr int kCsrChunks = CC_CSR_CHUNKS;

// The edge pass over CSR: warp-sized chunks of consecutive entries, the row
// of each lane found by walking the offsets forward from the warp's current
// row (bounded by n), the filter and the warp ring as in the COO pass. Warps
// claim tiles one at a time from *work (the dynamic schedule of the COO pass).
// The filter may read parent values older than the pushes of earlier chunks
// of the same iteration: equal values still mean that the endpoints were
// already joined, and different ones only send the edge to the union.
template <class F>
__global__ void __launch_bounds__(512) k_edge_pass_csr(const uint64_t *__restrict__ off,
                                                       const uint32_t *__restrict__ nb, uint64_t n_entries,
                                                       uint32_t n, uint32_t tile, const uint32_t *tile_row,
                                                       uint32_t *P, Ctrl *ctrl, unsigned long long *work) {
  constexpr int K = kCsrChunks;
  extern __shared__ uint32_t ring_smem[];
  const F fn = F::load(ctrl);
  uint32_t *const S = slots<F>(P);
  const uint64_t pol = policy_evict_first();
  WarpRing ring;
  // always through the queue: the lanes of a chunk share row endpoints, and
  // resolving them in place measured slower (R-MAT 24 and the grid)
  ring.init(ring_smem, nullptr, nullptr, kNeverDirect);
  const uint64_t n_tiles = (n_entries + tile - 1) / tile;
  for (;;) {
    unsigned long long t = 0;
    if (ring.lane == 0) t = atomicAdd(work, 1ULL);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= n_tiles) break;
    uint32_t r = tile_row[t];  // warp-uniform: the row of the tile's first entry
    const uint64_t end = (t + 1) * tile < n_entries ? (t + 1) * tile : n_entries;
    for (uint64_t base = t * tile; base < end; base += 32u * K) {
      uint32_t u[K], v[K];
      bool live[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const uint64_t j = base + 32u * c + ring.lane;
        live[c] = j < end;
        v[c] = live[c] ? ld_nc_u32(nb + j, pol) : 0u;
      }
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const uint64_t cb = base + 32u * c;  // the chunk's first entry
        u[c] = r;
        if (cb >= end) continue;  // warp-uniform: the tile ended in an earlier chunk
        const uint64_t j = cb + ring.lane;
        // The row of entry j: lane k holds the boundary off[r + 1 + k], and
        // each lane counts, by a binary search over the 32 boundaries in
        // registers, the rows that end at or before its entry.
        const uint64_t bnd = r + 1u + ring.lane <= n ? off[r + 1u + ring.lane] : ~0ull;
        uint32_t lo = 0, hi = 32;  // answer in [0, 32]: six halvings settle it
        const uint64_t last_j = (end - cb < 32u ? end : cb + 32u) - 1u;
        if (__shfl_sync(0xFFFFFFFFu, bnd, 0) <= last_j) {  // else the whole chunk lies in row r
#pragma unroll
          for (int step = 0; step < 6; ++step) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint64_t b = __shfl_sync(0xFFFFFFFFu, bnd, (int)(mid < 32u ? mid : 31u));
            if (live[c] && mid < 32u && b <= j)
              lo = mid + 1u;
            else
              hi = mid;
          }
        }
        uint32_t uu = r + lo < n ? r + lo : n - 1u;
        // more than 32 rows (empty ones) end inside this chunk: walk on
        if (live[c])
          while (uu + 1u < n && off[uu + 1] <= j) ++uu;
        u[c] = uu;
        // the next chunk starts in the row of this chunk's last entry
        const int last = (int)((end - cb < 32u ? end - cb : 32u) - 1u);
        r = __shfl_sync(0xFFFFFFFFu, uu, last);
      }
      uint32_t pu[K], pv[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (live[c] && v[c] >= n) {
          set_err(ctrl, kErrRange);
          v[c] = u[c];  // a self-loop: no effect
        }
        pu[c] = live[c] ? ldP(P + u[c]) : 0u;
        pv[c] = live[c] ? ldP(P + v[c]) : 0u;
      }
#pragma unroll
      for (int c = 0; c < K; ++c)
        ring.push(S, live[c] && pu[c] != pv[c], fn.f(u[c]), pu[c], fn.f(v[c]), pv[c]);
    }
  }
  ring.drain(S);
}

}  // namespace

constexpr uint32_t kCsrTile = 1024;

uint64_t csr_tiles(uint64_t n_entries) { return (n_entries + kCsrTile - 1) / kCsrTile; }

cudaError_t launch_csr_root_select(const uint64_t *off, uint32_t n, uint64_t n_entries, Ctrl *ctrl, cudaStream_t s) {
  cudaError_t err;
  static_assert(offsetof(Ctrl, maxcnt) == offsetof(Ctrl, maxkey) + sizeof(unsigned long long), "reset together");
  if ((err = cudaMemsetAsync(&ctrl->maxkey, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->m_sel, 0xFF, sizeof(uint32_t), s)) != cudaSuccess) return err;
  const unsigned g = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_csr_maxlen, 256, 0));
  k_csr_maxlen<<<g, 256, 0, s>>>(off, n, n_entries, ctrl);
  note_launch();
  k_csr_minid<<<g, 256, 0, s>>>(off, n, ctrl);
  note_launch();
  k_csr_finalize_m<<<1, 1, 0, s>>>(ctrl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_csr_check(const uint64_t *off, uint32_t n, uint64_t n_entries, Ctrl *ctrl, cudaStream_t s) {
  // the offsets check alone (the longest row goes to maxcnt and maxkey, unused)
  const unsigned g = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_csr_maxlen, 256, 0));
  k_csr_maxlen<<<g, 256, 0, s>>>(off, n, n_entries, ctrl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_edge_pass_csr(bool rf, const uint64_t *off, const uint32_t *nb, uint64_t n_entries, uint32_t n,
                                 uint32_t *tile_row, uint32_t *P, Ctrl *ctrl, cudaStream_t s) {
  if (n_entries == 0 || n == 0) return cudaSuccess;
  const uint64_t n_tiles = csr_tiles(n_entries);
  const unsigned gt = clamp_grid((n_tiles + 255) / 256, persistent_cap((const void *)k_csr_tile_rows, 256, 0));
  k_csr_tile_rows<<<gt, 256, 0, s>>>(off, n, n_tiles, kCsrTile, tile_row);
  note_launch();
  cudaError_t err = cudaMemsetAsync(&ctrl->work, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess) return err;
  const int block = 256;
  const size_t smem = (size_t)(block / 32) * 4 * kRing * sizeof(uint32_t);
  // at least eight tiles per warp (as the COO pass keeps eight waves)
  const uint64_t want = (n_tiles + (block / 32) * 8 - 1) / ((block / 32) * 8);
  if (rf) {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_edge_pass_csr<RootR>, block, smem));
    k_edge_pass_csr<RootR><<<g, block, smem, s>>>(off, nb, n_entries, n, kCsrTile, tile_row, P, ctrl,
                                                   &ctrl->work);
  } else {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_edge_pass_csr<RootId>, block, smem));
    k_edge_pass_csr<RootId><<<g, block, smem, s>>>(off, nb, n_entries, n, kCsrTile, tile_row, P, ctrl,
                                                    &ctrl->work);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace cc

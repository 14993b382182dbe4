/*
 * gg_device.cu - device (CUDA) build of the seeded generators in gg_core.h.
 * Each kernel writes the same bits as the host build for the same arguments,
 * so large inputs can be produced in HBM without a host copy.
 * All entry points return a cudaError_t value (0 = success).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "gg_core.h"

#define GG_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

__global__ void k_rmat(uint64_t seed, int scale, int scramble, uint64_t e_begin,
                       uint64_t cnt, uint2 *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gg_rmat_edge(seed, scale, scramble, e_begin + i, &u, &v);
    out[i] = make_uint2(u, v);
  }
}

__global__ void k_er(uint64_t key, uint64_t n, uint64_t e_begin, uint64_t cnt,
                     uint2 *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gg_er_edge(key, n, e_begin + i, &u, &v);
    out[i] = make_uint2(u, v);
  }
}

constexpr uint64_t kGridChunk = 1ULL << 12;

/* One thread per chunk of kGridChunk slots: count kept candidates. */
__global__ void k_grid_count(uint64_t gkey, uint32_t W, uint32_t H, uint64_t n_limit,
                             uint32_t p, uint64_t slots, uint64_t nch,
                             unsigned long long *cnt) {
  uint64_t ch = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (ch >= nch) return;
  uint64_t s0 = ch * kGridChunk, s1 = s0 + kGridChunk < slots ? s0 + kGridChunk : slots;
  unsigned long long c = 0;
  for (uint64_t s = s0; s < s1; ++s) {
    uint32_t u, v;
    c += (unsigned long long)gg_grid_slot(gkey, W, H, n_limit, p, s, &u, &v);
  }
  cnt[ch] = c;
}

/* Exclusive prefix over the chunk counts by one block (nch is modest). */
__global__ void k_grid_scan(unsigned long long *cnt, uint64_t nch, unsigned long long *total) {
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nch; base += blockDim.x) {
    uint64_t i = base + threadIdx.x;
    unsigned long long x = i < nch ? cnt[i] : 0ULL;
    /* inclusive scan inside the block (Hillis-Steele in shared memory) */
    __shared__ unsigned long long buf[1024];
    buf[threadIdx.x] = x;
    __syncthreads();
    for (unsigned off = 1; off < blockDim.x; off <<= 1) {
      unsigned long long y = threadIdx.x >= off ? buf[threadIdx.x - off] : 0ULL;
      __syncthreads();
      buf[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < nch) cnt[i] = carry + buf[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_grid_fill(uint64_t gkey, uint32_t W, uint32_t H, uint64_t n_limit,
                            uint32_t p, uint64_t slots, uint64_t nch,
                            const unsigned long long *off, uint2 *out) {
  uint64_t ch = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (ch >= nch) return;
  uint64_t s0 = ch * kGridChunk, s1 = s0 + kGridChunk < slots ? s0 + kGridChunk : slots;
  uint64_t w = off[ch];
  for (uint64_t s = s0; s < s1; ++s) {
    uint32_t u, v;
    if (gg_grid_slot(gkey, W, H, n_limit, p, s, &u, &v)) out[w++] = make_uint2(u, v);
  }
}

// Mixed batch, G(n,m) and R-MAT graphs: one thread per edge of the
// concatenated list; grid graphs are left to k_batch_grid.
__global__ void k_batch_edges(uint64_t seed, uint32_t n_graphs, const uint64_t *edge_off, uint64_t total,
                              uint2 *out) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_graphs;  // largest g with edge_off[g] <= e
    while (hi - lo > 1u) {
      const uint32_t mid = (lo + hi) >> 1;
      if (edge_off[mid] <= e) lo = mid; else hi = mid;
    }
    const gg_batch_shape sh = gg_batch_graph_shape(seed, lo);
    if (sh.kind == GG_KIND_GRID) continue;
    const uint64_t gk = gg_key(seed, GG_STREAM_BATCH_GRAPH + lo);
    uint32_t u, v;
    if (sh.kind == GG_KIND_RMAT)
      gg_batch_rmat_edge(gk, sh.n_vertices, e - edge_off[lo], &u, &v);
    else
      gg_er_edge(gk, sh.n_vertices, e - edge_off[lo], &u, &v);
    out[e] = make_uint2(u, v);
  }
}

// Mixed batch, grid graphs: one block per graph scans the candidate slots in
// order and writes the kept edges in that order.
__global__ void k_batch_grid(uint64_t seed, uint32_t n_graphs, const uint64_t *edge_off, uint2 *out) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint64_t s_run;
  for (uint32_t g = blockIdx.x; g < n_graphs; g += gridDim.x) {
    const gg_batch_shape sh = gg_batch_graph_shape(seed, g);
    if (sh.kind != GG_KIND_GRID) continue;
    const uint64_t gk = gg_key(seed, GG_STREAM_BATCH_GRAPH + g);
    const uint64_t slots = 2ULL * sh.grid_w * sh.grid_h;
    if (threadIdx.x == 0) s_run = edge_off[g];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint64_t base = 0; base < slots; base += blockDim.x) {
      const uint64_t sl = base + threadIdx.x;
      uint32_t u = 0, v = 0;
      const int keep = sl < slots && gg_grid_slot(gk, sh.grid_w, sh.grid_h, sh.n_vertices, GG_P90, sl, &u, &v);
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
      if (lane == 0) s_warp[wid] = __popc(bal);
      __syncthreads();
      uint32_t before = 0, total = 0;
      for (uint32_t w = 0; w < nw; ++w) {
        if (w < wid) before += s_warp[w];
        total += s_warp[w];
      }
      if (keep) out[s_run + before + __popc(bal & ((1u << lane) - 1u))] = make_uint2(u, v);
      __syncthreads();
      if (threadIdx.x == 0) s_run += total;
      __syncthreads();
    }
  }
}

inline unsigned grid_for(uint64_t cnt) {
  uint64_t b = (cnt + 255) / 256;
  if (b > 152ULL * 64ULL) b = 152ULL * 64ULL;
  if (b == 0) b = 1;
  return (unsigned)b;
}

}  // namespace

/* Edges [e_begin, e_end) of R-MAT(scale, seed) into out_dev (8-byte aligned). */
GG_EXPORT int gg_rmat_dev(uint64_t seed, int scale, int scramble, uint64_t e_begin,
                          uint64_t e_end, uint32_t *out_dev, cudaStream_t stream) {
  uint64_t cnt = e_end - e_begin;
  if (cnt == 0) return 0;
  k_rmat<<<grid_for(cnt), 256, 0, stream>>>(seed, scale, scramble, e_begin, cnt,
                                            reinterpret_cast<uint2 *>(out_dev));
  return (int)cudaGetLastError();
}

/* Pairs [e_begin, e_end) of G(n, m) with the given seed. */
GG_EXPORT int gg_er_dev(uint64_t seed, uint64_t n, uint64_t e_begin, uint64_t e_end,
                        uint32_t *out_dev, cudaStream_t stream) {
  uint64_t cnt = e_end - e_begin;
  if (cnt == 0) return 0;
  k_er<<<grid_for(cnt), 256, 0, stream>>>(gg_key(seed, GG_STREAM_ER), n, e_begin, cnt,
                                          reinterpret_cast<uint2 *>(out_dev));
  return (int)cudaGetLastError();
}

/* Uniform pairs with the same stream as the host gg_pairs. */
GG_EXPORT int gg_pairs_dev(uint64_t seed, uint64_t tag, uint64_t n, uint64_t count,
                           uint32_t *out_dev, cudaStream_t stream) {
  if (count == 0) return 0;
  uint64_t k = gg_key(seed ^ gg_mix64(tag + 0x5851F42D4C957F2DULL), GG_STREAM_PAIRS);
  k_er<<<grid_for(count), 256, 0, stream>>>(k, n, 0, count,
                                            reinterpret_cast<uint2 *>(out_dev));
  return (int)cudaGetLastError();
}

/* Grid edges into out_dev (capacity >= 2 * count uint32); writes the count to
 * *count_out. Synchronises the stream. */
GG_EXPORT int gg_grid_dev(uint64_t seed, uint32_t W, uint32_t H, uint64_t n_limit,
                          uint32_t p_thresh, uint32_t *out_dev, uint64_t *count_out,
                          cudaStream_t stream) {
  uint64_t slots = 2ULL * W * H;
  uint64_t nch = (slots + kGridChunk - 1) / kGridChunk;
  unsigned long long *buf = nullptr;
  cudaError_t err = cudaMalloc(&buf, (nch + 1) * sizeof(unsigned long long));
  if (err != cudaSuccess) return (int)err;
  uint64_t gkey = gg_key(seed, GG_STREAM_GRID);
  unsigned nb = (unsigned)((nch + 255) / 256);
  if (nb == 0) nb = 1;
  k_grid_count<<<nb, 256, 0, stream>>>(gkey, W, H, n_limit, p_thresh, slots, nch, buf);
  k_grid_scan<<<1, 1024, 0, stream>>>(buf, nch, buf + nch);
  k_grid_fill<<<nb, 256, 0, stream>>>(gkey, W, H, n_limit, p_thresh, slots, nch, buf,
                                      reinterpret_cast<uint2 *>(out_dev));
  unsigned long long total = 0;
  err = cudaMemcpyAsync(&total, buf + nch, sizeof(total), cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  cudaFree(buf);
  if (err == cudaSuccess) err = cudaGetLastError();
  *count_out = total;
  return (int)err;
}

/* Edges of the mixed batch (graph-local ids) into out_dev, given the device
 * copy of its edge offsets (uint64[n_graphs + 1], from gg_batch_plan). */
GG_EXPORT int gg_batch_fill_dev(uint64_t seed, uint32_t n_graphs, const uint64_t *edge_off_dev,
                                uint64_t total_edges, uint32_t *out_dev, cudaStream_t stream) {
  if (n_graphs == 0) return 0;
  uint2 *o = reinterpret_cast<uint2 *>(out_dev);
  if (total_edges) k_batch_edges<<<grid_for(total_edges), 256, 0, stream>>>(seed, n_graphs, edge_off_dev, total_edges, o);
  k_batch_grid<<<n_graphs < 4096u ? n_graphs : 4096u, 256, 0, stream>>>(seed, n_graphs, edge_off_dev, o);
  return (int)cudaGetLastError();
}


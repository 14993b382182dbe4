// cc_pack.cu - compact edge encoding for host input (cc_run_host_packed).
//
// Section V sends vertex ids in the fewest whole bytes that hold them (3
// bytes below 2^24 vertices) to cut communication. Here the costly link is
// the one between host memory and the GPU, so host edges may come in that
// form: edge i is bytes [6i, 6i + 6): u then v, each 3 bytes little-endian.
// Each chunk crosses the link packed and is unpacked on the device into the
// uint32 pairs the edge pass reads.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cc_internal.h"

namespace cc {

namespace {

// Id k (0..15) of a group of 8 edges held in 12 little-endian words: it
// starts at byte 3k.
__device__ __forceinline__ uint32_t id3(const uint32_t (&w)[13], int k) {
  const int byte = 3 * k;
  return __funnelshift_r(w[byte >> 2], w[(byte >> 2) + 1], 8 * (byte & 3)) & 0xFFFFFFu;
}

// Groups of 8 edges (48 bytes in, 64 bytes out) per thread and iteration;
// src must be 16-byte aligned. The last n_edges % 8 edges are done one by one.
__global__ void __launch_bounds__(256) k_unpack3(const uint8_t *__restrict__ src, uint64_t n_edges,
                                                 uint32_t *__restrict__ dst) {
  const uint64_t groups = n_edges / 8u;
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint4 *in = reinterpret_cast<const uint4 *>(src);
  uint4 *out = reinterpret_cast<uint4 *>(dst);
  for (uint64_t g = t; g < groups; g += T) {
    uint32_t w[13];
    const uint4 a = __ldcs(in + 3 * g), b = __ldcs(in + 3 * g + 1), c = __ldcs(in + 3 * g + 2);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
    w[12] = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      out[4 * g + q] = make_uint4(id3(w, 4 * q), id3(w, 4 * q + 1), id3(w, 4 * q + 2), id3(w, 4 * q + 3));
  }
  const uint64_t rest = n_edges - 8u * groups;
  if (t < 2u * rest) {  // one id per thread
    const uint64_t i = 16u * groups + t;
    const uint8_t *p = src + 3u * i;
    dst[i] = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
  }
}

}  // namespace

cudaError_t launch_unpack3(const uint8_t *src, uint64_t n_edges, uint32_t *dst, cudaStream_t s) {
  if (n_edges == 0) return cudaSuccess;
  const uint64_t groups = n_edges / 8u;
  const unsigned g = clamp_grid((groups + 255) / 256 + 1, persistent_cap((const void *)k_unpack3, 256, 0));
  k_unpack3<<<g, 256, 0, s>>>(src, n_edges, dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cc

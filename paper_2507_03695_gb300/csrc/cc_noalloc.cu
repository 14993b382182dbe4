// cc_noalloc.cu - the maximum-degree vertex without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's allocator or memory-pool callbacks, services whose device
// memory is fixed when they start, and code that must not risk the implicit
// device synchronisation that cudaMalloc and cudaFree can cause. For them,
// cc_max_degree_vertex_noalloc runs the library's root-selection kernels (the
// degree histogram and its argmax) on a scratch array that lives in this
// file as a static __device__ array of fixed size, so it allocates nothing.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (CC_NOALLOC_MAX_VERTICES counters plus a 256-byte header,
// about 16 MiB) until the process exits. Host code cannot use the array's
// name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current and
// caches it; that first call should therefore come before any stream
// capture. Every call shares the one array and leaves its contents behind,
// so each call clears the counters it uses first, and calls whose work
// overlaps on the GPU (different streams, or several host threads) race.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cc.h"
#include "cc_internal.h"

namespace {

constexpr uint64_t kHeaderWords = 64;  // 256 bytes: room for the argmax key
constexpr uint64_t kScratchWords = kHeaderWords + CC_NOALLOC_MAX_VERTICES;

// Words [0, 64): header, read by the argmax as a cc::Ctrl (only maxkey used).
// Words [64, 64 + n): one degree counter per vertex.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

static_assert(sizeof(cc::Ctrl) <= kHeaderWords * sizeof(uint32_t), "header too small");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).
cudaError_t scratch_address(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

// m = the vertex encoded in the packed argmax key (degree << 32 | ~v).
__global__ void k_noalloc_finish(const cc::Ctrl *hdr, uint32_t n, uint32_t *m_out) {
  uint32_t m = ~(uint32_t)hdr->maxkey;
  *m_out = m < n ? m : 0u;
}

}  // namespace

extern "C" cc_status cc_max_degree_vertex_noalloc(const uint32_t *edges_dev, uint64_t n_edges,
                                                   uint64_t n_vertices, uint32_t *m_out_dev,
                                                   cc_stream_t stream) {
  if (n_vertices == 0 || !m_out_dev || ((uintptr_t)m_out_dev & 3u)) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges && (!edges_dev || ((uintptr_t)edges_dev & 7u))) return CC_ERR_INVALID_ARGUMENT;
  if (n_vertices > CC_NOALLOC_MAX_VERTICES) return CC_ERR_TOO_LARGE;
  if (n_edges >= (1ULL << 31)) return CC_ERR_TOO_LARGE;  // 32-bit counters stay exact
  uint32_t *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return CC_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cc::Ctrl *hdr = reinterpret_cast<cc::Ctrl *>(scratch);
  uint32_t *cnt = scratch + kHeaderWords;
  const uint32_t n = (uint32_t)n_vertices;
  // clear the header and the n counters this call uses
  if (cudaMemsetAsync(scratch, 0, (kHeaderWords + n) * sizeof(uint32_t), s) != cudaSuccess)
    return CC_ERR_CUDA;
  if (n_edges) {
    const cc::EdgeSpan span = cc::split_edges(edges_dev, n_edges);
    if (cc::launch_degree_u32(span, cnt, n, s) != cudaSuccess) return CC_ERR_CUDA;
  }
  if (cc::launch_argmax_u32(cnt, n, hdr, s) != cudaSuccess) return CC_ERR_CUDA;
  k_noalloc_finish<<<1, 1, 0, s>>>(hdr, n, m_out_dev);
  cc::note_launch();
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

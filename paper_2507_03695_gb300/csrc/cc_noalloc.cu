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
// caches it together with the id of the device's current context; that
// first call should therefore come before any stream capture. A later call
// in another context (after cudaDeviceReset, which reloads the module at a
// possibly different address) looks the address up again. Every call shares
// the one array and leaves its contents behind, so each call clears the
// counters it uses first, and calls whose work overlaps on the GPU
// (different streams, or several host threads) race.
#include <cuda.h>  // CUcontext and CUresult, for the context id (no libcuda link)
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
unsigned long long g_ctx[kMaxDevices] = {};  // context id the cached address belongs to

// Id of the calling thread's current context (unique for the process's
// lifetime), or 0 when there is none or the driver does not say. The two
// driver calls are reached through the runtime's entry-point query, so the
// library needs no link to libcuda.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device: looked up once
// per device and context (every call, if the context id is unknown).
cudaError_t scratch_address(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx = current_ctx_id();
  if (g_ptr[dev] && ctx != 0 && ctx == g_ctx[dev]) {
    *out = g_ptr[dev];
    return cudaSuccess;
  }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the context current if it was not
  if (e != cudaSuccess) return e;
  g_ptr[dev] = static_cast<uint32_t *>(p);
  g_ctx[dev] = ctx != 0 ? ctx : current_ctx_id();
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

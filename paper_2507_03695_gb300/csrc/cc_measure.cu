// cc_measure.cu - the random-load rate that bounds the edge pass's lookups.
//
// Each thread walks ILP independent linear congruential sequences
// (x <- 1664525 x + 1013904223 mod 2^32, the constants of Numerical Recipes'
// quick generator) and reads the array at the top bits of each state, so
// that every load is its own L2 request at a uniformly random word. The sum
// of the loaded words is consumed by a store that never happens (the array is
// zero), so no load can be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cc_internal.h"
#include "cc_measure.h"

namespace {

template <int ILP, bool kCG>
__global__ void __launch_bounds__(512) k_random_loads(const uint32_t *__restrict__ a, uint32_t shift,
                                                      uint32_t rounds, uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[ILP];
#pragma unroll
  for (int j = 0; j < ILP; ++j) x[j] = (t * ILP + j) * 2654435761u + 12345u;
  uint32_t acc = 0;
  for (uint32_t r = 0; r < rounds; ++r) {
    uint32_t v[ILP];
#pragma unroll
    for (int j = 0; j < ILP; ++j) {
      x[j] = x[j] * 1664525u + 1013904223u;
      const uint32_t *p = a + (x[j] >> shift);
      v[j] = kCG ? __ldcg(p) : *p;
    }
#pragma unroll
    for (int j = 0; j < ILP; ++j) acc += v[j];
  }
  if (acc == 0xFFFFFFFFu) *sink = t;
}

template <int ILP, bool kCG>
cudaError_t time_shape(const uint32_t *a, uint32_t shift, uint32_t *sink, cudaStream_t s, cudaEvent_t e0,
                       cudaEvent_t e1, double *rate) {
  const void *k = (const void *)k_random_loads<ILP, kCG>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 512, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const unsigned grid = (unsigned)(cc::num_sms() * per_sm);
  // about 2^28 loads per launch (a millisecond or so)
  const uint64_t threads = (uint64_t)grid * 512;
  uint32_t rounds = (uint32_t)((1ull << 28) / (threads * ILP));
  if (rounds < 16) rounds = 16;
  k_random_loads<ILP, kCG><<<grid, 512, 0, s>>>(a, shift, rounds, sink);
  err = cudaEventRecord(e0, s);
  for (int i = 0; i < 3 && err == cudaSuccess; ++i) {
    k_random_loads<ILP, kCG><<<grid, 512, 0, s>>>(a, shift, rounds, sink);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess && ms > 0.f) *rate = 3.0 * (double)threads * ILP * rounds / (ms * 1e-3);
  return err;
}

}  // namespace

extern "C" cc_status cc_measure_random_loads(uint64_t array_bytes, double *loads_per_second) {
  if (!loads_per_second) return CC_ERR_INVALID_ARGUMENT;
  if (array_bytes < (1ull << 16) || array_bytes > (1ull << 32) || (array_bytes & (array_bytes - 1)))
    return CC_ERR_INVALID_ARGUMENT;
  uint32_t log2w = 0;  // log2 of the word count
  while ((4ull << log2w) < array_bytes) ++log2w;
  const uint32_t shift = 32u - log2w;  // top log2w bits of a state index the array
  uint32_t *a = nullptr, *sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc((void **)&a, array_bytes);
  if (err == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return CC_ERR_OOM;
  }
  if (err == cudaSuccess) err = cudaMalloc((void **)&sink, sizeof(uint32_t));
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaMemsetAsync(a, 0, array_bytes, s);
  double best = 0.0, r = 0.0;
  if (err == cudaSuccess && (err = time_shape<4, false>(a, shift, sink, s, e0, e1, &r)) == cudaSuccess && r > best) best = r;
  if (err == cudaSuccess && (err = time_shape<8, false>(a, shift, sink, s, e0, e1, &r)) == cudaSuccess && r > best) best = r;
  if (err == cudaSuccess && (err = time_shape<4, true>(a, shift, sink, s, e0, e1, &r)) == cudaSuccess && r > best) best = r;
  if (err == cudaSuccess && (err = time_shape<8, true>(a, shift, sink, s, e0, e1, &r)) == cudaSuccess && r > best) best = r;
  if (s) cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(sink);
  cudaFree(a);
  if (err != cudaSuccess) return CC_ERR_CUDA;
  *loads_per_second = best;
  return CC_OK;
}

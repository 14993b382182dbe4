// cc_batched.cu - connected components of many independent graphs in one
// cooperative persistent launch (include/cc_batch.h).
//
// All graphs share one name space: vertex i of graph g is named
// vtx_off[g] + i and f is the identity (Algorithm 1), so each graph's forest
// lives in its own range and the root of a component is its smallest global
// name; minus vtx_off[g] that is the graph-local min-id label. The label array
// is the parent array during the run. Phases, separated by grid barriers:
//   0. block 0 checks the offsets and turns them into tile offsets;
//   1. P[x] = x for every vertex;
//   2. hooking: edge tiles (each inside one graph) with rebased ids, through
//      the warp ring or per lane;
//   3. compression: every vertex stores its root's name (read-only walks with
//      L2-coherent loads, so each entry is written only by its owner);
//   4. labels: vertex tiles turn root names into graph-local ids in place.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "cc_batch.h"
#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {

struct alignas(128) BatchCtrl {
  unsigned int bar_count;    // cumulative arrivals at grid barriers   } reset
  unsigned int bar_gen;      // barriers completed                     } before
  unsigned int abort;        // nonzero: every block leaves at the next barrier } each run
  unsigned int err;          // kErr* bits (sticky until cc_batch_sync)
  unsigned int bad_offsets;  // malformed offsets (sticky until cc_batch_sync)
  unsigned int pad[3];
};

struct BatchArgs {
  uint32_t n_graphs;
  const uint64_t *vtx_off;
  const uint64_t *edge_off;
  const uint2 *edges;
  uint32_t *P;  // the label array
  uint64_t *etile_off;  // n_graphs + 1
  uint64_t *vtile_off;  // n_graphs + 1
  uint32_t tile_edges, tile_vertices;
  unsigned long long barrier_ns;  // bounded wait of every grid barrier
  BatchCtrl *ctrl;
};

namespace {

constexpr unsigned long long kBarrierTimeoutNs = 4000000000ULL;  // 4 s: default barrier wait

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Built with -DCC_BATCH_CLOCK, block 0 records the global timer at the
// kernel's start, after each grid barrier and at its end (diagnostics of the
// phase times only, off in normal builds).
#ifdef CC_BATCH_CLOCK
__device__ unsigned long long g_batch_clock[8];
#define CC_BATCH_TICK(i)                                                     \
  do {                                                                       \
    if (blockIdx.x == 0 && threadIdx.x == 0) g_batch_clock[(i)] = globaltimer(); \
  } while (0)
#else
#define CC_BATCH_TICK(i) ((void)0)
#endif

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier for a cooperative launch (all blocks co-resident). Arrivals
// are counted cumulatively, so barrier k completes when the count reaches
// k * gridDim.x. Every wait gives up after limit_ns, flags kErrTimeout and
// aborts the run (every block then leaves at its next barrier). Returns false
// when the run must stop.
__device__ bool grid_barrier(BatchCtrl *c, unsigned int &gen, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = gen + 1u;
    int ok = 1;
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == gridDim.x * target) {
      __threadfence();
      atomicExch(&c->bar_gen, target);
    } else {
      const unsigned long long t0 = globaltimer();
      while (ld_acquire_u32(&c->bar_gen) < target) {
        if (globaltimer() - t0 > limit_ns) {
          atomicOr(&c->err, kErrTimeout);
          atomicExch(&c->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (*(volatile unsigned int *)&c->abort) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  CC_BATCH_TICK(gen);
  return s_ok != 0;
}

// Largest g in [0, n) with off[g] <= t (off nondecreasing, off[0] == 0).
__device__ __forceinline__ uint32_t owner(const uint64_t *off, uint32_t n, uint64_t t) {
  uint32_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Phase 0 (one block): validate the offsets and write exclusive prefix sums
// of the per-graph tile counts.
__device__ void scan_tiles(const BatchArgs &a) {
  __shared__ unsigned long long s_carry_e, s_carry_v;
  __shared__ unsigned long long s_we[32], s_wv[32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) {
    s_carry_e = s_carry_v = 0ULL;
    s_bad = (a.vtx_off[0] != 0ULL || a.edge_off[0] != 0ULL);
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = 0; base < a.n_graphs; base += blockDim.x) {
    const uint32_t g = base + threadIdx.x;
    unsigned long long te = 0, tv = 0;
    if (g < a.n_graphs) {
      const uint64_t v0 = a.vtx_off[g], v1 = a.vtx_off[g + 1];
      const uint64_t e0 = a.edge_off[g], e1 = a.edge_off[g + 1];
      if (v1 < v0 || e1 < e0) s_bad = 1;
      else {
        te = (e1 - e0 + a.tile_edges - 1) / a.tile_edges;
        tv = (v1 - v0 + a.tile_vertices - 1) / a.tile_vertices;
      }
    }
    // inclusive warp scans
    unsigned long long ie = te, iv = tv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long ye = __shfl_up_sync(0xFFFFFFFFu, ie, o);
      const unsigned long long yv = __shfl_up_sync(0xFFFFFFFFu, iv, o);
      if (lane >= (uint32_t)o) {
        ie += ye;
        iv += yv;
      }
    }
    if (lane == 31) {
      s_we[wid] = ie;
      s_wv[wid] = iv;
    }
    __syncthreads();
    if (wid == 0) {
      unsigned long long xe = lane < nw ? s_we[lane] : 0ULL, xv = lane < nw ? s_wv[lane] : 0ULL;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ye = __shfl_up_sync(0xFFFFFFFFu, xe, o);
        const unsigned long long yv = __shfl_up_sync(0xFFFFFFFFu, xv, o);
        if (lane >= (uint32_t)o) {
          xe += ye;
          xv += yv;
        }
      }
      if (lane < nw) {
        s_we[lane] = xe;  // inclusive prefix over warps
        s_wv[lane] = xv;
      }
    }
    __syncthreads();
    const unsigned long long off_e = s_carry_e + (wid ? s_we[wid - 1] : 0ULL) + ie - te;
    const unsigned long long off_v = s_carry_v + (wid ? s_wv[wid - 1] : 0ULL) + iv - tv;
    if (g < a.n_graphs) {
      a.etile_off[g] = off_e;
      a.vtile_off[g] = off_v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_carry_e += s_we[nw - 1];
      s_carry_v += s_wv[nw - 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.etile_off[a.n_graphs] = s_carry_e;
    a.vtile_off[a.n_graphs] = s_carry_v;
    if (a.vtx_off[a.n_graphs] > 0x7FFFFFFFULL) s_bad = 1;
    if (s_bad) {
      a.ctrl->bad_offsets = 1u;
      atomicExch(&a.ctrl->abort, 1u);
    }
  }
}

template <int EPT, bool FILTER>
__global__ void __launch_bounds__(512) k_batched(BatchArgs a) {
  extern __shared__ uint32_t ring_smem[];
  __shared__ uint64_t s_tile[4];  // graph, first edge / vertex, end, name base
  BatchCtrl *c = a.ctrl;
  unsigned int gen = 0;
  CC_BATCH_TICK(0);
  if (blockIdx.x == 0) scan_tiles(a);
  if (!grid_barrier(c, gen, a.barrier_ns)) return;

  // 1. initialisation: P[x] = x
  const uint64_t V = a.vtx_off[a.n_graphs];
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (uint64_t x = tid; x < V; x += T) a.P[x] = (uint32_t)x;
  if (!grid_barrier(c, gen, a.barrier_ns)) return;

  // 2. hooking over edge tiles, one warp per tile: lane 0 finds the tile's
  // graph and broadcasts it, so no block barrier is taken per tile (a block
  // would wait for its slowest warp's searches). Tile t goes to warp
  // t % warps of block t / warps % gridDim.x: consecutive tiles, often of one
  // graph, stay on one SM and share its L1.
  uint32_t *const P = a.P;  // names are global ids: the slot of name x is P[x]
  WarpRing ring;
  if (FILTER) ring.init(ring_smem);
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t wpb = blockDim.x >> 5;
  const uint64_t wid = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5);  // block-major
  const uint64_t n_warps = wpb * gridDim.x;
  const uint64_t n_etiles = a.etile_off[a.n_graphs];
  for (uint64_t t = wid; t < n_etiles; t += n_warps) {
    uint64_t nv = 0, e0 = 0, e1 = 0, base64 = 0;
    if (lane == 0) {
      const uint32_t g = owner(a.etile_off, a.n_graphs, t);
      e0 = a.edge_off[g] + (t - a.etile_off[g]) * a.tile_edges;
      const uint64_t ge = a.edge_off[g + 1];
      e1 = e0 + a.tile_edges < ge ? e0 + a.tile_edges : ge;
      nv = a.vtx_off[g + 1] - a.vtx_off[g];
      base64 = a.vtx_off[g];
    }
    nv = __shfl_sync(0xFFFFFFFFu, nv, 0);
    e0 = __shfl_sync(0xFFFFFFFFu, e0, 0);
    e1 = __shfl_sync(0xFFFFFFFFu, e1, 0);
    const uint32_t base = (uint32_t)__shfl_sync(0xFFFFFFFFu, base64, 0);
    for (uint64_t r0 = e0; r0 < e1; r0 += 32u * EPT) {
      uint32_t u[EPT], v[EPT], pu[EPT], pv[EPT];
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const uint64_t i = r0 + (uint64_t)j * 32u + lane;
        uint2 ed = make_uint2(0u, 0u);
        bool ok = false;
        if (i < e1) {
          ed = ld_edge(a.edges + i);
          ok = ed.x < nv && ed.y < nv;
          if (!ok) atomicOr(&c->err, kErrRange);
        }
        // an empty or invalid slot touches no memory: equal parents drop it
        u[j] = ok ? base + ed.x : 0u;
        v[j] = ok ? base + ed.y : 0u;
        pu[j] = ok ? 1u : 0u;
        pv[j] = pu[j];
      }
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (pu[j]) {
          pu[j] = ldP(P + u[j]);
          pv[j] = ldP(P + v[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (FILTER)
          ring.push(P, pu[j] != pv[j], u[j], pu[j], v[j], pv[j]);
        else
          unite(P, u[j], pu[j], v[j], pv[j]);
      }
    }
  }
  if (FILTER) ring.drain(P);
  if (!grid_barrier(c, gen, a.barrier_ns)) return;

  // 3. compression: each vertex stores its root's name (read-only walks)
  for (uint64_t x = tid; x < V; x += T) {
    const uint32_t px = ldP_strong(P + x);
    if (px == (uint32_t)x) continue;
    uint32_t r = px, pr = ldP_strong(P + r);
    while (pr != r) {
      r = pr;
      pr = ldP_strong(P + r);
    }
    if (r != px) stP(P + x, r);
  }
  if (!grid_barrier(c, gen, a.barrier_ns)) return;

  // 4. graph-local labels, in place
  const uint64_t n_vtiles = a.vtile_off[a.n_graphs];
  for (uint64_t t = blockIdx.x; t < n_vtiles; t += gridDim.x) {
    if (threadIdx.x == 0) {
      const uint32_t g = owner(a.vtile_off, a.n_graphs, t);
      const uint64_t x0 = a.vtx_off[g] + (t - a.vtile_off[g]) * a.tile_vertices;
      const uint64_t x1 = a.vtx_off[g + 1];
      s_tile[1] = x0;
      s_tile[2] = x0 + a.tile_vertices < x1 ? x0 + a.tile_vertices : x1;
      s_tile[3] = a.vtx_off[g];
    }
    __syncthreads();
    const uint64_t x0 = s_tile[1], x1 = s_tile[2];
    const uint32_t base = (uint32_t)s_tile[3];
    __syncthreads();
    for (uint64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) P[x] = ldP_strong(P + x) - base;
  }
  CC_BATCH_TICK(5);
}

}  // namespace
}  // namespace cc

#ifdef CC_BATCH_CLOCK
// Diagnostics builds only: the timer readings of the last batched run.
extern "C" __attribute__((visibility("default"))) int cc_batch_clock_read(unsigned long long out[8]) {
  return (int)cudaMemcpyFromSymbol(out, cc::g_batch_clock, 8 * sizeof(unsigned long long));
}
#endif

using cc::BatchArgs;
using cc::BatchCtrl;

struct cc_batch {
  int device = 0;
  uint32_t max_graphs = 0;
  cc_batch_config cfg{};
  BatchCtrl *ctrl = nullptr;
  BatchCtrl *host_ctrl = nullptr;
  uint64_t *tile_off = nullptr;  // 2 * (max_graphs + 1)
  cudaStream_t last = nullptr;
  // the last cc_batch_tune: every candidate with its best time
  cc_batch_config tuned[64];
  float tuned_ms[64];
  uint32_t n_tuned = 0;
};

namespace {

bool cfg_valid(const cc_batch_config &c) {
  if (c.block_size != 256 && c.block_size != 512) return false;
  if (c.edges_per_thread != 1 && c.edges_per_thread != 2 && c.edges_per_thread != 4) return false;
  if (c.filter != 0 && c.filter != 1) return false;
  if (c.tile_edges < 256 || c.tile_edges % 256 || c.tile_vertices < 256) return false;
  if (c.barrier_wait_us > 60u * 1000u * 1000u) return false;
  for (int r : c.reserved)
    if (r) return false;
  return true;
}

// The best configuration measured on the 4096-graph mixed batch (11.1 ms),
// used until cc_batch_tune or cc_batch_set_config chooses another.
cc_batch_config default_cfg() {
  cc_batch_config c{};
  c.block_size = 512;
  c.edges_per_thread = 1;
  c.filter = 1;
  c.tile_edges = 8192;
  c.tile_vertices = 4096;
  return c;
}

template <int EPT, bool FILTER>
cudaError_t launch_batched_t(const cc_batch_config &cfg, BatchArgs &a, cudaStream_t s) {
  const void *k = (const void *)cc::k_batched<EPT, FILTER>;
  const size_t smem = FILTER ? (size_t)(cfg.block_size / 32) * 4 * cc::kRing * sizeof(uint32_t) : 0;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, cfg.block_size, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const unsigned grid = (unsigned)(cc::num_sms() * occ);
  void *args[] = {&a};
  e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(cfg.block_size), args, smem, s);
  cc::note_launch();
  return e;
}

cudaError_t launch_batched(const cc_batch_config &cfg, BatchArgs &a, cudaStream_t s) {
  switch (cfg.edges_per_thread * 2 + cfg.filter) {
    case 2: return launch_batched_t<1, false>(cfg, a, s);
    case 3: return launch_batched_t<1, true>(cfg, a, s);
    case 4: return launch_batched_t<2, false>(cfg, a, s);
    case 5: return launch_batched_t<2, true>(cfg, a, s);
    case 8: return launch_batched_t<4, false>(cfg, a, s);
    default: return launch_batched_t<4, true>(cfg, a, s);
  }
}

cc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  if (e == cudaErrorMemoryAllocation) return CC_ERR_OOM;
  return CC_ERR_CUDA;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != d) {
      prev = cur;
      cudaSetDevice(d);
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cc_status enqueue(cc_batch *b, const cc_batch_config &cfg, uint32_t n_graphs, const uint64_t *vtx_off,
                  const uint64_t *edge_off, const uint32_t *edges, uint32_t *L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->ctrl, 0, 3 * sizeof(unsigned int), s);  // barrier state and abort
  if (e != cudaSuccess) return from_cuda(e);
  BatchArgs a;
  a.n_graphs = n_graphs;
  a.vtx_off = vtx_off;
  a.edge_off = edge_off;
  a.edges = reinterpret_cast<const uint2 *>(edges);
  a.P = L;
  a.etile_off = b->tile_off;
  a.vtile_off = b->tile_off + (b->max_graphs + 1);
  a.tile_edges = cfg.tile_edges;
  a.tile_vertices = cfg.tile_vertices;
  a.barrier_ns = cfg.barrier_wait_us ? (unsigned long long)cfg.barrier_wait_us * 1000ULL : cc::kBarrierTimeoutNs;
  a.ctrl = b->ctrl;
  return from_cuda(launch_batched(cfg, a, s));
}

cc_status check_args(cc_batch *b, uint32_t n_graphs, const uint64_t *vtx_off, const uint64_t *edge_off,
                     const uint32_t *edges, uint32_t *L) {
  if (!b) return CC_ERR_INVALID_ARGUMENT;
  if (n_graphs > b->max_graphs) return CC_ERR_TOO_LARGE;
  if (n_graphs == 0) return CC_OK;
  if (!vtx_off || !edge_off || !L || ((uintptr_t)vtx_off & 7u) || ((uintptr_t)edge_off & 7u) ||
      ((uintptr_t)L & 3u) || (edges && ((uintptr_t)edges & 7u)))
    return CC_ERR_INVALID_ARGUMENT;
  return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_batch_create(uint32_t max_graphs, cc_batch **out) {
  if (!out) return CC_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (max_graphs == 0 || max_graphs > (1u << 28)) return CC_ERR_INVALID_ARGUMENT;
  cc_batch *b = new (std::nothrow) cc_batch();
  if (!b) return CC_ERR_OOM;
  b->max_graphs = max_graphs;
  b->cfg = default_cfg();
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->ctrl, sizeof(BatchCtrl));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->host_ctrl, sizeof(BatchCtrl));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->tile_off, 2 * ((size_t)max_graphs + 1) * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMemset(b->ctrl, 0, sizeof(BatchCtrl));
  if (e != cudaSuccess) {
    cc_batch_destroy(b);
    return from_cuda(e);
  }
  *out = b;
  return CC_OK;
}

void cc_batch_destroy(cc_batch *b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaDeviceSynchronize();
  if (b->ctrl) cudaFree(b->ctrl);
  if (b->host_ctrl) cudaFreeHost(b->host_ctrl);
  if (b->tile_off) cudaFree(b->tile_off);
  delete b;
}

cc_status cc_run_batched(cc_batch *b, uint32_t n_graphs, const uint64_t *vtx_off_dev,
                         const uint64_t *edge_off_dev, const uint32_t *edges_dev, uint32_t *L_out_dev,
                         cc_stream_t stream) {
  cc_status st = check_args(b, n_graphs, vtx_off_dev, edge_off_dev, edges_dev, L_out_dev);
  if (st != CC_OK || n_graphs == 0) return st;
  DeviceGuard dg(b->device);
  b->last = (cudaStream_t)stream;
  return enqueue(b, b->cfg, n_graphs, vtx_off_dev, edge_off_dev, edges_dev, L_out_dev, b->last);
}

cc_status cc_batch_tune_results(const cc_batch *b, cc_batch_config *cfgs, float *ms, uint32_t cap,
                                uint32_t *count) {
  if (!b || !count || (cap && (!cfgs || !ms))) return CC_ERR_INVALID_ARGUMENT;
  const uint32_t k = b->n_tuned < cap ? b->n_tuned : cap;
  for (uint32_t i = 0; i < k; ++i) {
    cfgs[i] = b->tuned[i];
    ms[i] = b->tuned_ms[i];
  }
  *count = b->n_tuned;
  return CC_OK;
}

cc_status cc_batch_set_config(cc_batch *b, const cc_batch_config *cfg) {
  if (!b || !cfg || !cfg_valid(*cfg)) return CC_ERR_INVALID_ARGUMENT;
  b->cfg = *cfg;
  return CC_OK;
}

cc_status cc_batch_get_config(const cc_batch *b, cc_batch_config *cfg) {
  if (!b || !cfg) return CC_ERR_INVALID_ARGUMENT;
  *cfg = b->cfg;
  return CC_OK;
}

cc_status cc_batch_sync(cc_batch *b) {
  if (!b) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(b->device);
  cudaStream_t s = b->last;
  cudaError_t e = cudaMemcpyAsync(b->host_ctrl, b->ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const BatchCtrl h = *b->host_ctrl;
  if (h.err || h.abort || h.bad_offsets) {
    e = cudaMemsetAsync(b->ctrl, 0, sizeof(BatchCtrl), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (h.bad_offsets) return CC_ERR_INVALID_ARGUMENT;
  if (h.err & cc::kErrTimeout) return CC_ERR_TIMEOUT;
  if (h.err & cc::kErrRange) return CC_ERR_OUT_OF_RANGE;
  return CC_OK;
}

cc_status cc_batch_tune(cc_batch *b, uint32_t n_graphs, const uint64_t *vtx_off_dev,
                        const uint64_t *edge_off_dev, const uint32_t *edges_dev, uint32_t *L_out_dev,
                        cc_stream_t stream, cc_batch_config *best, float *best_ms) {
  cc_status st = check_args(b, n_graphs, vtx_off_dev, edge_off_dev, edges_dev, L_out_dev);
  if (st != CC_OK) return st;
  if (n_graphs == 0) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  b->last = s;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CC_ERR_CUDA;
  }
  const int blocks[] = {256, 512};
  const int epts[] = {1, 2, 4};
  const int filters[] = {1, 0};
  const uint32_t tiles[] = {4096, 8192, 16384, 65536};  // edges per warp tile
  cc_batch_config top = b->cfg;
  float top_ms = 1e30f;
  b->n_tuned = 0;
  for (int blk : blocks)
    for (int ept : epts)
      for (int flt : filters)
        for (uint32_t te : tiles) {
          cc_batch_config c = default_cfg();
          c.barrier_wait_us = b->cfg.barrier_wait_us;
          c.block_size = blk;
          c.edges_per_thread = ept;
          c.filter = flt;
          c.tile_edges = te;
          float ms_min = 1e30f;
          for (int rep = 0; rep < 3 && st == CC_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = enqueue(b, c, n_graphs, vtx_off_dev, edge_off_dev, edges_dev, L_out_dev, s);
            cudaEventRecord(e1, s);
            if (st != CC_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
              st = CC_ERR_CUDA;
              break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < ms_min) ms_min = ms;  // the first run warms up
          }
          if (st != CC_OK) break;
          if (b->n_tuned < 64) {
            b->tuned[b->n_tuned] = c;
            b->tuned_ms[b->n_tuned++] = ms_min;
          }
          if (ms_min < top_ms) {
            top_ms = ms_min;
            top = c;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CC_OK) return st;
  st = cc_batch_sync(b);
  if (st != CC_OK) return st;
  b->cfg = top;
  if (best) *best = top;
  if (best_ms) *best_ms = top_ms;
  return CC_OK;
}

}  // extern "C"

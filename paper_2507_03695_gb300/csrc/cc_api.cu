// cc_api.cu - host runtime and C ABI (include/cc.h) of the connected-components
// library: the handle, its device memory (parent array P, root-select
// histogram, control block, staging), argument checks, HBM budget, error
// reporting, checkpoints, and the order in which the kernels of
// cc_kernels.cu are enqueued.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <array>
#include <new>
#include <vector>

#include "cc.h"
#include "cc_internal.h"

using cc::Ctrl;

struct cc_graph {
  int device = 0;
  uint64_t n = 0;
  cc_options opt{};
  bool rf = false;
  uint32_t *P = nullptr;
  void *cnt = nullptr;  // root-select histogram (uint32 or uint64 per vertex)
  size_t cnt_bytes = 0;
  cc::CertScratch *cert = nullptr;  // certified root-select scratch
  Ctrl *ctrl = nullptr;
  Ctrl *host_ctrl = nullptr;  // pinned mirror
  uint32_t *staging = nullptr;
  uint64_t capacity = 0;
  uint32_t *label_dev = nullptr;  // cc_run_host labels
  cudaStream_t last = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev = nullptr;
  std::vector<std::array<cudaEvent_t, 5>> evsets;  // one set per timed run
  size_t ev_used = 0;                                // sets filled since the last total
  size_t ev_cur = 0;                                 // set of the current run
  bool timed_run = false;
  bool ncomp_fresh = false;
  uint64_t owned = 0;
  uint32_t *csr_rows = nullptr;  // cc_run_csr: the row of each tile's first entry
  uint64_t csr_rows_cap = 0;
  uint8_t *pk[2] = {nullptr, nullptr};  // cc_run_host_packed: packed chunk slots
  size_t pk_bytes = 0;                   // bytes of each slot
  cudaEvent_t pk_ev[2] = {nullptr, nullptr};  // a slot's last unpack has run
  uint32_t *push = nullptr;  // Initial Push list (push_cap entries), or null
  uint32_t push_cap = 0;
  uint32_t *cand_list = nullptr;  // listed candidates of the root selection (cand_cap entries), f = R only
  uint32_t cand_cap = 0;
  uint32_t *z = nullptr;   // zero-tree bitmap (one bit per name), or null
  size_t z_bytes = 0;
  bool z_forced = false;   // CC_FILTER_BITMAP: always used
  bool z_auto_ok = false;  // the last run's exact selection left ctrl->cert meaningful
};

namespace {

constexpr uint64_t kMaxVertices = 0x7FFFFFFFULL;
constexpr uint64_t kHostChunk = 1ULL << 24;  // edges per cc_run_host copy chunk
constexpr uint64_t kZMinBytes = 128ULL << 20;  // CC_FILTER_AUTO: P at least this large gets the bitmap

// Bitmap bytes for names 0 .. n (n + 1 names under R), whole 32-bit words.
size_t z_bytes_for(uint64_t n) { return (size_t)((n + 1 + 31) / 32) * 4; }

// Initial Push: on request only.
bool wants_push(const cc_options &o) {
  return o.mode == CC_ROOT_MAXDEG && o.root_hint == CC_ROOT_AUTO && o.root_select != CC_ROOT_SELECT_SAMPLED &&
         o.initial_push == CC_PUSH_ON;
}
uint32_t push_cap_for(uint64_t n) {
  const uint64_t c = n < (1ULL << 23) ? n : (1ULL << 23);
  return (uint32_t)((c + cc::kPushLanes - 1) / cc::kPushLanes * cc::kPushLanes);
}

bool wants_z(const cc_options &o, uint64_t n) {
  if (o.filter == CC_FILTER_BITMAP) return true;
  return o.filter == CC_FILTER_AUTO && o.mode == CC_ROOT_MAXDEG && (uint64_t)n * 4 >= kZMinBytes;
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

cc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  if (e == cudaErrorMemoryAllocation) return CC_ERR_OOM;
  return CC_ERR_CUDA;
}

#define CC_TRY(expr)                          \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

bool opts_valid(const cc_options &o) {
  if (o.mode != CC_ROOT_IDENTITY && o.mode != CC_ROOT_MAXDEG) return false;
  if (o.root_select != CC_ROOT_SELECT_EXACT && o.root_select != CC_ROOT_SELECT_SAMPLED) return false;
  if (o.filter < CC_FILTER_AUTO || o.filter > CC_FILTER_BITMAP) return false;
  if (o.initial_push < CC_PUSH_AUTO || o.initial_push > CC_PUSH_OFF || o.reserved32) return false;
  if (o.label_space != CC_LABEL_MIN_ID && o.label_space != CC_LABEL_ROOT_VALUE) return false;
  if (o.block_size != 0 && o.block_size != 128 && o.block_size != 256 && o.block_size != 512)
    return false;
  if (o.edges_per_thread != 0 && o.edges_per_thread != 2 && o.edges_per_thread != 4 &&
      o.edges_per_thread != 8)
    return false;
  if (o.sample_stride < 0) return false;
  for (uint64_t r : o.reserved)
    if (r) return false;
  return true;
}

int eff_filter(const cc_graph *g) {
  if (g->opt.filter == CC_FILTER_ON) return 1;
  if (g->opt.filter == CC_FILTER_OFF) return 0;
  return 1;
}
int eff_ept(const cc_graph *g) { return g->opt.edges_per_thread ? g->opt.edges_per_thread : 4; }
int eff_block(const cc_graph *g) { return g->opt.block_size ? g->opt.block_size : 512; }

cudaError_t dev_alloc(cc_graph *g, void **p, size_t bytes) {
  if (g->opt.hbm_budget_bytes && g->owned + bytes > g->opt.hbm_budget_bytes)
    return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) g->owned += bytes;
  return e;
}

void dev_free(cc_graph *g, void *p, size_t bytes) {
  if (p) {
    cudaFree(p);
    g->owned -= bytes;
  }
}

size_t p_bytes(uint64_t n) { return (size_t)((n + 3) / 4 * 4) * sizeof(uint32_t); }

// Copies the control block to the pinned mirror, waits, then turns and clears
// the sticky device error bits.
cc_status fetch_ctrl(cc_graph *g, cudaStream_t s) {
  CC_TRY(cudaMemcpyAsync(g->host_ctrl, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaStreamSynchronize(s));
  const uint32_t err = g->host_ctrl->err;
  if (err) {
    CC_TRY(cudaMemsetAsync(&g->ctrl->err, 0, sizeof(uint32_t), s));
    CC_TRY(cudaStreamSynchronize(s));
    if (err & cc::kErrInternal) return CC_ERR_INTERNAL;
    if (err & cc::kErrFormat) return CC_ERR_INVALID_ARGUMENT;
    if (err & cc::kErrTimeout) return CC_ERR_TIMEOUT;
    if (err & cc::kErrRange) return CC_ERR_OUT_OF_RANGE;
  }
  return CC_OK;
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// Root selection (f = R with no hint): the certified exact selection, or the
// argmax of a histogram over the sampled groups. Leaves m in ctrl->maxkey.
// The root-select histogram: n counters of 4 bytes, or 8 when wide.
cudaError_t ensure_cnt(cc_graph *g, bool wide, cudaStream_t s) {
  const size_t need = (size_t)g->n * (wide ? 8 : 4);
  if (g->cnt_bytes >= need) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  dev_free(g, g->cnt, g->cnt_bytes);
  g->cnt = nullptr;
  g->cnt_bytes = 0;
  if ((e = dev_alloc(g, &g->cnt, need)) != cudaSuccess) return e;
  g->cnt_bytes = need;
  return cudaSuccess;
}

cc_status root_select(cc_graph *g, const uint32_t *edges, uint64_t n_edges, const cc::EdgeSpan &span,
                      cudaStream_t s, int *m_src) {
  const uint32_t n = (uint32_t)g->n;
  const uint32_t stride = g->opt.sample_stride ? (uint32_t)g->opt.sample_stride : 16u;
  const bool sampled = g->opt.root_select == CC_ROOT_SELECT_SAMPLED && stride > 1;
  const bool wide = !sampled && n_edges >= (1ULL << 31);
  const size_t need = (size_t)n * (wide ? 8 : 4);
  CC_TRY(ensure_cnt(g, wide, s));
  *m_src = cc::kMFromPackedMax;
  if (sampled) {
    CC_TRY(cudaMemsetAsync(g->cnt, 0, need, s));
    CC_TRY(cudaMemsetAsync(&g->ctrl->maxkey, 0, sizeof(unsigned long long), s));
    CC_TRY(cc::launch_degree_sampled_u32(reinterpret_cast<const uint2 *>(edges), n_edges, 0, stride,
                                         (uint32_t *)g->cnt, n, s));
    CC_TRY(cc::launch_argmax_u32((const uint32_t *)g->cnt, n, g->ctrl, s));
    return CC_OK;
  }
  CC_TRY(cc::launch_root_select_certified(edges, n_edges, span, g->cnt, wide, n, g->cert, g->ctrl, s, g->push,
                                         g->push_cap, g->cand_list, g->cand_cap));
  return CC_OK;
}

void record(cc_graph *g, int i, cudaStream_t s);

constexpr size_t kMaxEventSets = 4096;

// Picks the event set of a timed run (false when timing is off or the pool is full).
bool begin_timed_run(cc_graph *g) {
  g->timed_run = false;
  if (!g->opt.timing) return false;
  if (g->ev_used == g->evsets.size()) {
    if (g->evsets.size() >= kMaxEventSets) return false;
    std::array<cudaEvent_t, 5> set{};
    for (auto &ev : set)
      if (cudaEventCreate(&ev) != cudaSuccess) return false;
    g->evsets.push_back(set);
  }
  g->ev_cur = g->ev_used++;
  g->timed_run = true;
  return true;
}

void record(cc_graph *g, int i, cudaStream_t s) {
  if (g->timed_run) cudaEventRecord(g->evsets[g->ev_cur][i], s);
}

// gmin <- m and ncomp <- 0 ahead of a flatten that is not preceded by init.
__global__ void k_prep_flatten(Ctrl *ctrl) {
  ctrl->gmin = ctrl->m;
  ctrl->ncomp = 0ULL;
}

}  // namespace

extern "C" {

void cc_options_init(cc_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->mode = CC_ROOT_MAXDEG;
  opt->root_select = CC_ROOT_SELECT_EXACT;
  opt->root_hint = CC_ROOT_AUTO;
  opt->filter = CC_FILTER_AUTO;
  opt->label_space = CC_LABEL_MIN_ID;
}

const char *cc_status_string(cc_status s) {
  switch (s) {
    case CC_OK: return "CC_OK: success";
    case CC_ERR_INVALID_ARGUMENT: return "CC_ERR_INVALID_ARGUMENT: invalid argument";
    case CC_ERR_TOO_LARGE: return "CC_ERR_TOO_LARGE: size exceeds a limit";
    case CC_ERR_OOM: return "CC_ERR_OOM: device memory or HBM budget exhausted";
    case CC_ERR_OUT_OF_RANGE: return "CC_ERR_OUT_OF_RANGE: vertex id >= n_vertices";
    case CC_ERR_TIMEOUT: return "CC_ERR_TIMEOUT: bounded wait expired";
    case CC_ERR_CUDA: return "CC_ERR_CUDA: CUDA runtime error";
    case CC_ERR_INTERNAL: return "CC_ERR_INTERNAL: internal invariant failed";
    case CC_ERR_NOT_READY: return "CC_ERR_NOT_READY: request not complete";
  }
  return "unknown cc_status";
}

cc_status cc_create(uint64_t n_vertices, uint64_t n_edges_capacity, const cc_options *opt,
                    cc_graph **out) {
  if (!out) return CC_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  cc_options o;
  if (opt)
    o = *opt;
  else
    cc_options_init(&o);
  if (!opts_valid(o)) return CC_ERR_INVALID_ARGUMENT;
  if (n_vertices > kMaxVertices) return CC_ERR_TOO_LARGE;
  if (o.mode == CC_ROOT_MAXDEG && o.root_hint != CC_ROOT_AUTO && o.root_hint >= n_vertices &&
      n_vertices > 0)
    return CC_ERR_INVALID_ARGUMENT;
  if (n_edges_capacity > (1ULL << 40)) return CC_ERR_TOO_LARGE;

  // host-side checks first: they need no device
  const bool rf = o.mode == CC_ROOT_MAXDEG;
  const size_t need = p_bytes(n_vertices) +
                      (rf ? (size_t)n_vertices * 4 + sizeof(cc::CertScratch) + (size_t)cc::cand_list_cap(n_vertices) * 4
                          : 0) + sizeof(Ctrl) +
                      (size_t)n_edges_capacity * 8 + (wants_z(o, n_vertices) ? z_bytes_for(n_vertices) : 0) +
                      (wants_push(o) ? (size_t)push_cap_for(n_vertices) * 4 : 0);
  if (o.hbm_budget_bytes && need > o.hbm_budget_bytes) return CC_ERR_OOM;

  cc_graph *g = new (std::nothrow) cc_graph();
  if (!g) return CC_ERR_OOM;
  g->n = n_vertices;
  g->opt = o;
  g->rf = rf;
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    delete g;
    return CC_ERR_CUDA;
  }
  cc_status st = CC_OK;
  cudaError_t e = cudaSuccess;
  do {
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) break;
    if (need > free_b) {
      st = CC_ERR_OOM;
      break;
    }
    if ((e = dev_alloc(g, (void **)&g->P, p_bytes(n_vertices))) != cudaSuccess) break;
    if ((e = dev_alloc(g, (void **)&g->ctrl, sizeof(Ctrl))) != cudaSuccess) break;
    if ((e = cudaMallocHost((void **)&g->host_ctrl, sizeof(Ctrl))) != cudaSuccess) break;
    memset(g->host_ctrl, 0, sizeof(Ctrl));
    if (g->rf && n_vertices) {
      if ((e = dev_alloc(g, &g->cnt, (size_t)n_vertices * 4)) != cudaSuccess) break;
      g->cnt_bytes = (size_t)n_vertices * 4;
      if ((e = dev_alloc(g, (void **)&g->cert, sizeof(cc::CertScratch))) != cudaSuccess) break;
      g->cand_cap = cc::cand_list_cap(n_vertices);
      if ((e = dev_alloc(g, (void **)&g->cand_list, (size_t)g->cand_cap * 4)) != cudaSuccess) break;
    }
    if (n_edges_capacity) {
      if ((e = dev_alloc(g, (void **)&g->staging, (size_t)n_edges_capacity * 8)) != cudaSuccess) break;
      g->capacity = n_edges_capacity;
    }
    if (n_vertices && wants_push(o)) {
      g->push_cap = push_cap_for(n_vertices);
      if ((e = dev_alloc(g, (void **)&g->push, (size_t)g->push_cap * 4)) != cudaSuccess) break;
    }
    if (n_vertices && wants_z(o, n_vertices)) {
      if ((e = dev_alloc(g, (void **)&g->z, z_bytes_for(n_vertices))) != cudaSuccess) break;
      g->z_bytes = z_bytes_for(n_vertices);
      g->z_forced = o.filter == CC_FILTER_BITMAP;
      if ((e = cudaMemset(g->z, 0, g->z_bytes)) != cudaSuccess) break;
    }
    if ((e = cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&g->copy_ev, cudaEventDisableTiming)) != cudaSuccess) break;
    if ((e = cudaMemset(g->ctrl, 0, sizeof(Ctrl))) != cudaSuccess) break;
    // the edgeless graph: P_v = f(v) with m = hint (or 0)
    const uint32_t hint =
        (g->rf && o.root_hint != CC_ROOT_AUTO) ? (uint32_t)o.root_hint : 0u;
    if ((e = cc::launch_init(g->rf, g->P, (uint32_t)n_vertices, g->ctrl, cc::kMFromHint, hint, 0)) !=
        cudaSuccess)
      break;
    if ((e = cudaStreamSynchronize(0)) != cudaSuccess) break;
    g->ncomp_fresh = false;
  } while (0);
  if (st == CC_OK && e != cudaSuccess) st = from_cuda(e);
  if (st != CC_OK) {
    cc_destroy(g);
    return st;
  }
  *out = g;
  return CC_OK;
}

void cc_destroy(cc_graph *g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  cudaDeviceSynchronize();
  dev_free(g, g->P, p_bytes(g->n));
  dev_free(g, g->cnt, g->cnt_bytes);
  dev_free(g, g->cert, sizeof(cc::CertScratch));
  dev_free(g, g->cand_list, (size_t)g->cand_cap * 4);
  dev_free(g, g->ctrl, sizeof(Ctrl));
  dev_free(g, g->staging, (size_t)g->capacity * 8);
  dev_free(g, g->label_dev, (size_t)g->n * 4);
  dev_free(g, g->z, g->z_bytes);
  dev_free(g, g->push, (size_t)g->push_cap * 4);
  dev_free(g, g->csr_rows, (size_t)g->csr_rows_cap * 4);
  for (int i = 0; i < 2; ++i) {
    dev_free(g, g->pk[i], g->pk_bytes);
    if (g->pk_ev[i]) cudaEventDestroy(g->pk_ev[i]);
  }
  if (g->host_ctrl) cudaFreeHost(g->host_ctrl);
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  if (g->copy_ev) cudaEventDestroy(g->copy_ev);
  for (auto &set : g->evsets)
    for (auto ev : set)
      if (ev) cudaEventDestroy(ev);
  delete g;
}

cc_status cc_run(cc_graph *g, const uint32_t *edges_dev, uint64_t n_edges, uint32_t *L_out_dev,
                 cc_stream_t stream) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges && (!edges_dev || !aligned(edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
  if (L_out_dev && !aligned(L_out_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (g->n == 0) return CC_OK;
  const uint32_t n = (uint32_t)g->n;
  const cc::EdgeSpan span = cc::split_edges(edges_dev, n_edges);
  begin_timed_run(g);
  record(g, 0, s);
  int m_src = cc::kMFromHint;
  uint32_t hint = 0;
  if (g->rf) {
    if (g->opt.root_hint != CC_ROOT_AUTO) {
      hint = (uint32_t)g->opt.root_hint;
    } else {
      cc_status st = root_select(g, edges_dev, n_edges, span, s, &m_src);
      if (st != CC_OK) return st;
    }
  }
  record(g, 1, s);
  CC_TRY(cc::launch_init(g->rf, g->P, n, g->ctrl, m_src, hint, s));
  if (g->push) CC_TRY(cc::launch_initial_push(g->P, n, g->push, g->push_cap, g->cert, g->ctrl, s));
  // the zero-tree bitmap starts empty with every init; without a forced
  // bitmap it is used when this run's exact selection certified a hub
  const bool exact = g->rf && g->opt.root_hint == CC_ROOT_AUTO && g->opt.root_select != CC_ROOT_SELECT_SAMPLED;
  if (g->z) CC_TRY(cudaMemsetAsync(g->z, 0, g->z_bytes, s));
  g->z_auto_ok = exact && !g->z_forced;
  uint32_t *Z = (g->z && (g->z_forced || exact)) ? g->z : nullptr;
  const uint32_t *zsel = (Z && !g->z_forced) ? &g->ctrl->cert : nullptr;
  record(g, 2, s);
  CC_TRY(cc::launch_edge_pass(g->rf, eff_filter(g), eff_ept(g), eff_block(g), span, g->P, n, g->ctrl,
                              nullptr, s, Z, zsel, false, nullptr, exact ? &g->ctrl->cert : nullptr, true,
                              exact ? g->cert->hot : nullptr));
  record(g, 3, s);
  CC_TRY(cc::launch_flatten(g->rf, g->opt.label_space, g->P, n, L_out_dev, g->ctrl, s));
  record(g, 4, s);
  g->ncomp_fresh = true;
  return CC_OK;
}

// The work of cc_run_host; id_bytes 0: edges_host holds uint32 pairs;
// 3: packed ids, copied into the two slots in turn and unpacked on s.
// wait: synchronise at the end and report device errors (cc_run_host);
// otherwise return once everything is enqueued (cc_run_host_async).
static cc_status run_host_impl(cc_graph *g, const void *edges_host, uint64_t n_edges, int id_bytes, uint32_t *L_out_host,
                        cc_stream_t stream, bool wait) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges && !edges_host) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges > g->capacity) return CC_ERR_TOO_LARGE;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (g->n == 0) return CC_OK;
  const uint32_t n = (uint32_t)g->n;
  if (L_out_host && !g->label_dev) CC_TRY(dev_alloc(g, (void **)&g->label_dev, (size_t)n * 4));
  // When m is known before the edges arrive (identity, or a hint), the edge
  // pass runs on each chunk as soon as it lands. Exact selection takes the
  // chunked route: a speculative m' from the first chunk, hooking and the
  // certificate's counts per chunk, and a rerun only when m' was not the
  // exact answer. Sampled selection needs every edge first.
  const bool select = g->rf && g->opt.root_hint == CC_ROOT_AUTO;
  const bool chunked = select && g->opt.root_select != CC_ROOT_SELECT_SAMPLED;
  const uint32_t hint = (g->rf && !select) ? (uint32_t)g->opt.root_hint : 0u;
  const bool wide = n_edges >= (1ULL << 31);
  if (chunked) CC_TRY(ensure_cnt(g, wide, s));
  // the zero-tree bitmap starts empty; a forced bitmap is used throughout,
  // an automatic one for the final pass when the certificate allows
  if (g->z) CC_TRY(cudaMemsetAsync(g->z, 0, g->z_bytes, s));
  g->z_auto_ok = chunked && !g->z_forced;
  uint32_t *Zf = g->z_forced ? g->z : nullptr;
  if (!select) CC_TRY(cc::launch_init(g->rf, g->P, n, g->ctrl, cc::kMFromHint, hint, s));
  // Chunks hooked under a speculative m' use the bitmap too when the first
  // chunk's sample showed a hub (its bits name the tree of m', and are
  // cleared before a rerun under another vertex); the hub-mode word picks
  // the instance on the device.
  uint32_t *Zc = Zf;
  const uint32_t *zc_sel = nullptr, *hub_c = nullptr;
  if (chunked && !g->z_forced) {
    hub_c = &g->ctrl->skip[cc::kSkipHist];
    Zc = g->z;
    zc_sel = g->z ? hub_c : nullptr;
  }
  // the copy stream starts after everything already enqueued on s
  CC_TRY(cudaEventRecord(g->copy_ev, s));
  CC_TRY(cudaStreamWaitEvent(g->copy_stream, g->copy_ev, 0));
  for (uint64_t off = 0; off < n_edges; off += kHostChunk) {
    const uint64_t cnt = (n_edges - off) < kHostChunk ? (n_edges - off) : kHostChunk;
    if (id_bytes == 3) {
      // a slot is refilled only after the unpack of the chunk before last
      const int slot = (int)((off / kHostChunk) & 1u);
      if (off >= 2 * kHostChunk) CC_TRY(cudaStreamWaitEvent(g->copy_stream, g->pk_ev[slot], 0));
      CC_TRY(cudaMemcpyAsync(g->pk[slot], static_cast<const uint8_t *>(edges_host) + 6 * off, cnt * 6,
                             cudaMemcpyHostToDevice, g->copy_stream));
      CC_TRY(cudaEventRecord(g->copy_ev, g->copy_stream));
      CC_TRY(cudaStreamWaitEvent(s, g->copy_ev, 0));
      CC_TRY(cc::launch_unpack3(g->pk[slot], cnt, g->staging + 2 * off, s));
      CC_TRY(cudaEventRecord(g->pk_ev[slot], s));
      if (select && !chunked) continue;
    } else {
      CC_TRY(cudaMemcpyAsync(g->staging + 2 * off, static_cast<const uint32_t *>(edges_host) + 2 * off, cnt * 8,
                             cudaMemcpyHostToDevice, g->copy_stream));
      if (select && !chunked) continue;
      CC_TRY(cudaEventRecord(g->copy_ev, g->copy_stream));
      CC_TRY(cudaStreamWaitEvent(s, g->copy_ev, 0));
    }
    const cc::EdgeSpan chunk = cc::split_edges(g->staging + 2 * off, cnt);
    if (chunked && off == 0) CC_TRY(cc::chunked_select_begin(g->staging, cnt, g->cnt, wide, n, g->cert, g->ctrl, s));
    if (chunked) CC_TRY(cc::chunked_select_chunk(chunk, off == 0, g->cnt, wide, n, g->cert, g->ctrl, s));
    // every chunk is hooked as it lands, under m' when m is still unknown
    if (chunked && off == 0) CC_TRY(cc::launch_init(true, g->P, n, g->ctrl, cc::kMFromPackedMax, 0u, s));
    CC_TRY(cc::launch_edge_pass(g->rf, eff_filter(g), eff_ept(g), eff_block(g), chunk, g->P, n, g->ctrl, nullptr,
                                s, Zc, zc_sel, false, nullptr, hub_c, true, chunked ? g->cert->hot : nullptr));
  }
  const cc::EdgeSpan all = cc::split_edges(g->staging, n_edges);
  if (chunked) {
    if (n_edges == 0) CC_TRY(cc::chunked_select_begin(g->staging, 0, g->cnt, wide, n, g->cert, g->ctrl, s));
    CC_TRY(cc::chunked_select_end(all, g->cnt, wide, n, g->cert, g->ctrl, s));
    const uint32_t *held = &g->ctrl->skip[cc::kSkipRerun];
    CC_TRY(cc::launch_init(true, g->P, n, g->ctrl, cc::kMFromPackedMax, 0u, s, held));
    // a rerun starts from a fresh P in which another vertex holds name 0, so
    // a forced bitmap must start empty again (when m' held, the reset only
    // forgets bits: an empty bitmap is always valid)
    if (Zc) CC_TRY(cudaMemsetAsync(Zc, 0, g->z_bytes, s));
    CC_TRY(cc::launch_edge_pass(true, eff_filter(g), eff_ept(g), eff_block(g), all, g->P, n, g->ctrl, held, s,
                                g->z, Zf ? nullptr : &g->ctrl->cert, false, nullptr, nullptr, true, g->cert->hot));
  } else if (select) {
    if (id_bytes != 3) {  // (packed chunks were unpacked on s already)
      CC_TRY(cudaEventRecord(g->copy_ev, g->copy_stream));
      CC_TRY(cudaStreamWaitEvent(s, g->copy_ev, 0));
    }
    int m_src = cc::kMFromHint;
    cc_status st = root_select(g, g->staging, n_edges, all, s, &m_src);
    if (st != CC_OK) return st;
    CC_TRY(cc::launch_init(g->rf, g->P, n, g->ctrl, m_src, hint, s));
    CC_TRY(cc::launch_edge_pass(g->rf, eff_filter(g), eff_ept(g), eff_block(g), all, g->P, n, g->ctrl,
                                nullptr, s, Zf, nullptr, false, nullptr, nullptr, true));
  }
  CC_TRY(cc::launch_flatten(g->rf, g->opt.label_space, g->P, n, L_out_host ? g->label_dev : nullptr,
                            g->ctrl, s));
  if (L_out_host)
    CC_TRY(cudaMemcpyAsync(L_out_host, g->label_dev, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  g->ncomp_fresh = true;
  return wait ? fetch_ctrl(g, s) : CC_OK;
}

cc_status cc_run_csr(cc_graph *g, const uint64_t *offsets_dev, const uint32_t *neighbors_dev, uint64_t n_entries,
                     uint32_t *L_out_dev, cc_stream_t stream) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (g->n && (!offsets_dev || !aligned(offsets_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
  if (n_entries && (!neighbors_dev || !aligned(neighbors_dev, 4))) return CC_ERR_INVALID_ARGUMENT;
  if (L_out_dev && !aligned(L_out_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (g->n == 0) return CC_OK;
  const uint32_t n = (uint32_t)g->n;
  const uint64_t tiles = cc::csr_tiles(n_entries);
  if (tiles > g->csr_rows_cap) {
    CC_TRY(cudaStreamSynchronize(s));
    dev_free(g, g->csr_rows, (size_t)g->csr_rows_cap * 4);
    g->csr_rows = nullptr;
    g->csr_rows_cap = 0;
    CC_TRY(dev_alloc(g, (void **)&g->csr_rows, (size_t)tiles * 4));
    g->csr_rows_cap = tiles;
  }
  begin_timed_run(g);
  record(g, 0, s);
  int m_src = cc::kMFromHint;
  uint32_t hint = 0;
  if (g->rf && g->opt.root_hint == CC_ROOT_AUTO) {
    CC_TRY(cc::launch_csr_root_select(offsets_dev, n, n_entries, g->ctrl, s));
    m_src = cc::kMFromPackedMax;
  } else {
    if (g->rf) hint = (uint32_t)g->opt.root_hint;
    CC_TRY(cc::launch_csr_check(offsets_dev, n, n_entries, g->ctrl, s));
  }
  record(g, 1, s);
  CC_TRY(cc::launch_init(g->rf, g->P, n, g->ctrl, m_src, hint, s));
  if (g->z) CC_TRY(cudaMemsetAsync(g->z, 0, g->z_bytes, s));
  g->z_auto_ok = false;
  record(g, 2, s);
  CC_TRY(cc::launch_edge_pass_csr(g->rf, offsets_dev, neighbors_dev, n_entries, n, g->csr_rows, g->P, g->ctrl, s));
  record(g, 3, s);
  CC_TRY(cc::launch_flatten(g->rf, g->opt.label_space, g->P, n, L_out_dev, g->ctrl, s));
  record(g, 4, s);
  g->ncomp_fresh = true;
  return CC_OK;
}

cc_status cc_run_host(cc_graph *g, const uint32_t *edges_host, uint64_t n_edges, uint32_t *L_out_host,
                      cc_stream_t stream) {
  return run_host_impl(g, edges_host, n_edges, 0, L_out_host, stream, true);
}

cc_status cc_run_host_async(cc_graph *g, const uint32_t *edges_host, uint64_t n_edges, uint32_t *L_out_host,
                            cc_stream_t stream) {
  return run_host_impl(g, edges_host, n_edges, 0, L_out_host, stream, false);
}

static cc_status run_host_packed_impl(cc_graph *g, const uint8_t *edges_host, uint64_t n_edges, int32_t id_bytes,
                                      uint32_t *L_out_host, cc_stream_t stream, bool wait) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (id_bytes == 4) return run_host_impl(g, edges_host, n_edges, 0, L_out_host, stream, wait);
  if (id_bytes != 3 || g->n > (1ULL << 24)) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges && !edges_host) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges > g->capacity) return CC_ERR_TOO_LARGE;
  if (!g->pk[0] && n_edges) {
    DeviceGuard dg(g->device);
    g->pk_bytes = (size_t)kHostChunk * 6;
    for (int i = 0; i < 2; ++i) {
      CC_TRY(dev_alloc(g, (void **)&g->pk[i], g->pk_bytes));
      CC_TRY(cudaEventCreateWithFlags(&g->pk_ev[i], cudaEventDisableTiming));
    }
  }
  return run_host_impl(g, edges_host, n_edges, 3, L_out_host, stream, wait);
}

cc_status cc_run_host_packed(cc_graph *g, const uint8_t *edges_host, uint64_t n_edges, int32_t id_bytes,
                             uint32_t *L_out_host, cc_stream_t stream) {
  return run_host_packed_impl(g, edges_host, n_edges, id_bytes, L_out_host, stream, true);
}

cc_status cc_run_host_packed_async(cc_graph *g, const uint8_t *edges_host, uint64_t n_edges, int32_t id_bytes,
                                   uint32_t *L_out_host, cc_stream_t stream) {
  return run_host_packed_impl(g, edges_host, n_edges, id_bytes, L_out_host, stream, false);
}

cc_status cc_stream_insert(cc_graph *g, const uint32_t *edges_dev, uint64_t n_edges, cc_stream_t stream) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (n_edges && (!edges_dev || !aligned(edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (g->n == 0 || n_edges == 0) return CC_OK;
  const cc::EdgeSpan span = cc::split_edges(edges_dev, n_edges);
  CC_TRY(cudaMemsetAsync(&g->ctrl->reject, 0, sizeof(uint32_t), s));
  CC_TRY(cc::launch_validate(span, (uint32_t)g->n, g->ctrl, s));
  uint32_t *Z = (g->z && (g->z_forced || g->z_auto_ok)) ? g->z : nullptr;
  const uint32_t *zsel = (Z && !g->z_forced) ? &g->ctrl->cert : nullptr;
  // the last run's certificate (when its exact selection ran) picks the form
  const uint32_t *hub = g->z_auto_ok ? &g->ctrl->cert : nullptr;
  CC_TRY(cc::launch_edge_pass(g->rf, eff_filter(g), eff_ept(g), eff_block(g), span, g->P,
                              (uint32_t)g->n, g->ctrl, &g->ctrl->reject, s, Z, zsel, false, nullptr, hub, true,
                              g->z_auto_ok ? g->cert->hot : nullptr));
  g->ncomp_fresh = false;
  return CC_OK;
}

cc_status cc_labels(cc_graph *g, uint32_t *L_out_dev, cc_stream_t stream) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (!L_out_dev || !aligned(L_out_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (g->n == 0) return CC_OK;
  k_prep_flatten<<<1, 1, 0, s>>>(g->ctrl); cc::note_launch();
  CC_TRY(cudaGetLastError());
  CC_TRY(cc::launch_flatten(g->rf, g->opt.label_space, g->P, (uint32_t)g->n, L_out_dev, g->ctrl, s));
  g->ncomp_fresh = true;
  return CC_OK;
}

cc_status cc_connected(cc_graph *g, const uint32_t *pairs_dev, uint64_t n_pairs, uint8_t *out_dev,
                       cc_stream_t stream) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  if (n_pairs && (!pairs_dev || !out_dev || !aligned(pairs_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  if (n_pairs == 0) return CC_OK;
  CC_TRY(cc::launch_connected(g->rf, g->P, (uint32_t)g->n, reinterpret_cast<const uint2 *>(pairs_dev),
                              n_pairs, out_dev, g->ctrl, s));
  return CC_OK;
}

cc_status cc_forest_pairs(cc_graph *g, uint32_t *pairs_dev, uint64_t capacity, uint64_t *count,
                          cc_stream_t stream) {
  if (!g || !count) return CC_ERR_INVALID_ARGUMENT;
  if (capacity && (!pairs_dev || !aligned(pairs_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  g->last = s;
  *count = 0;
  if (g->n == 0) return CC_OK;
  CC_TRY(cc::launch_forest_pairs(g->rf, g->P, (uint32_t)g->n, pairs_dev, capacity, g->ctrl, s));
  const cc_status st = fetch_ctrl(g, s);  // waits; also reports earlier device errors
  *count = g->host_ctrl->pairs;
  if (st != CC_OK) return st;
  return *count > capacity ? CC_ERR_TOO_LARGE : CC_OK;
}

cc_status cc_connected1(cc_graph *g, uint64_t u, uint64_t v, int *out) {
  if (!g || !out) return CC_ERR_INVALID_ARGUMENT;
  if (u >= g->n || v >= g->n) return CC_ERR_OUT_OF_RANGE;
  DeviceGuard dg(g->device);
  cudaStream_t s = g->last;
  g->host_ctrl->q_u = (uint32_t)u;
  g->host_ctrl->q_v = (uint32_t)v;
  CC_TRY(cudaMemcpyAsync(&g->ctrl->q_u, &g->host_ctrl->q_u, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  CC_TRY(cudaMemsetAsync(&g->ctrl->q_out, 0, sizeof(uint32_t), s));
  CC_TRY(cc::launch_connected(g->rf, g->P, (uint32_t)g->n, reinterpret_cast<const uint2 *>(&g->ctrl->q_u),
                              1, reinterpret_cast<uint8_t *>(&g->ctrl->q_out), g->ctrl, s));
  cc_status st = fetch_ctrl(g, s);
  *out = (int)(g->host_ctrl->q_out & 0xFFu);
  return st;
}

cc_status cc_num_components(cc_graph *g, uint64_t *out) {
  if (!g || !out) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = g->last;
  if (g->n == 0) {
    *out = 0;
    return CC_OK;
  }
  if (!g->ncomp_fresh) {
    CC_TRY(cudaMemsetAsync(&g->ctrl->ncomp, 0, sizeof(unsigned long long), s));
    CC_TRY(cc::launch_count_roots(g->rf, g->P, (uint32_t)g->n, g->ctrl, s));
  }
  cc_status st = fetch_ctrl(g, s);
  *out = g->host_ctrl->ncomp;
  if (st == CC_OK) g->ncomp_fresh = true;
  return st;
}

cc_status cc_root_vertex(cc_graph *g, uint64_t *m) {
  if (!g || !m) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cc_status st = fetch_ctrl(g, g->last);
  *m = g->rf ? (uint64_t)g->host_ctrl->m : CC_ROOT_AUTO;
  return st;
}

cc_status cc_sync(cc_graph *g) {
  if (!g) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  return fetch_ctrl(g, g->last);
}

cc_status cc_phase_times(cc_graph *g, float ms[5]) {
  if (!g || !ms) return CC_ERR_INVALID_ARGUMENT;
  if (!g->timed_run) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  const auto &ev = g->evsets[g->ev_cur];
  CC_TRY(cudaEventSynchronize(ev[4]));
  for (int i = 0; i < 4; ++i) CC_TRY(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
  CC_TRY(cudaEventElapsedTime(&ms[4], ev[0], ev[4]));
  return CC_OK;
}

cc_status cc_phase_times_total(cc_graph *g, float ms[5], uint64_t *runs) {
  if (!g || !ms || !runs) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  for (int i = 0; i < 5; ++i) ms[i] = 0.f;
  for (size_t k = 0; k < g->ev_used; ++k) {
    const auto &ev = g->evsets[k];
    CC_TRY(cudaEventSynchronize(ev[4]));
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      CC_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      ms[i] += t;
    }
    float t = 0.f;
    CC_TRY(cudaEventElapsedTime(&t, ev[0], ev[4]));
    ms[4] += t;
  }
  *runs = g->ev_used;
  g->ev_used = 0;
  g->timed_run = false;
  return CC_OK;
}

uint64_t cc_kernel_launches(void) { return cc::launch_count(); }

struct CkptHeader {
  uint32_t magic;    // 'JTCC'
  uint32_t version;  // 1
  uint32_t mode;
  uint32_t m;
  uint64_t n;
};
static const uint32_t kCkptMagic = 0x4343544Au;

cc_status cc_checkpoint_size(const cc_graph *g, uint64_t *bytes) {
  if (!g || !bytes) return CC_ERR_INVALID_ARGUMENT;
  *bytes = sizeof(CkptHeader) + g->n * 4;
  return CC_OK;
}

cc_status cc_checkpoint(cc_graph *g, void *host_buf, uint64_t bytes) {
  if (!g || !host_buf || bytes < sizeof(CkptHeader) + g->n * 4) return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = g->last;
  cc_status st = fetch_ctrl(g, s);
  if (st != CC_OK) return st;
  CkptHeader h{kCkptMagic, 1u, (uint32_t)g->opt.mode, g->host_ctrl->m, g->n};
  memcpy(host_buf, &h, sizeof(h));
  if (g->n) {
    CC_TRY(cudaMemcpyAsync((char *)host_buf + sizeof(h), g->P, g->n * 4, cudaMemcpyDeviceToHost, s));
    CC_TRY(cudaStreamSynchronize(s));
  }
  return CC_OK;
}

cc_status cc_restore(cc_graph *g, const void *host_buf, uint64_t bytes) {
  if (!g || !host_buf || bytes < sizeof(CkptHeader)) return CC_ERR_INVALID_ARGUMENT;
  CkptHeader h;
  memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kCkptMagic || h.version != 1u || h.n != g->n || h.mode != (uint32_t)g->opt.mode ||
      bytes < sizeof(h) + h.n * 4 || (h.n && h.m >= h.n))
    return CC_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(g->device);
  cudaStream_t s = g->last;
  CC_TRY(cudaStreamSynchronize(s));
  if (g->n) CC_TRY(cudaMemcpy(g->P, (const char *)host_buf + sizeof(h), g->n * 4, cudaMemcpyHostToDevice));
  g->host_ctrl->m = h.m;
  CC_TRY(cudaMemcpy(&g->ctrl->m, &g->host_ctrl->m, sizeof(uint32_t), cudaMemcpyHostToDevice));
  if (g->z) CC_TRY(cudaMemset(g->z, 0, g->z_bytes));  // the restored P has its own trees
  g->z_auto_ok = false;
  g->ncomp_fresh = false;
  return CC_OK;
}

cc_status cc_device_bytes(const cc_graph *g, uint64_t *bytes) {
  if (!g || !bytes) return CC_ERR_INVALID_ARGUMENT;
  *bytes = g->owned;
  return CC_OK;
}

}  // extern "C"

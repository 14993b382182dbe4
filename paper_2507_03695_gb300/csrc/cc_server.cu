// cc_server.cu - serving runtime (include/cc_server.h): a host scheduler
// thread, a device arena with a first-fit allocator, and a persistent executor
// kernel that runs insert and query tiles on the live parent arrays of
// resident graphs.
//
// Host <-> device protocol (all in mapped pinned host memory):
//   ring[]     work items written by the host; `published` counts them;
//   done_seq[] per request slot: the executor stores the item's sequence
//              number after the request's last tile (release, system scope);
//   err[]      per request slot: an out-of-range id was seen;
//   stop       asks the executor to leave.
// In device memory: `taken` (items claimed by executor blocks) and, per slot,
// `finished` (tiles done; the last finisher resets it and signals).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_server.h"

namespace cc {
namespace srv {

constexpr uint32_t kRingCap = 1u << 16;  // work items in the ring
constexpr uint32_t kSlots = 4096;        // requests with executor tiles in flight
enum : uint32_t { kItemEdges = 1, kItemValidate = 2, kItemApply = 3, kItemQuery = 4 };

struct alignas(16) WorkItem {
  uint32_t kind, slot, seq, n_tiles;
  uint32_t rf, m, n, pad;
  uint64_t P, src, begin, end, out;
  uint64_t pad2;
};
static_assert(sizeof(WorkItem) == 80, "work item layout");

struct HostShared {
  unsigned long long published;
  unsigned int stop;
  unsigned int pad[13];
  WorkItem ring[kRingCap];
  unsigned int done_seq[kSlots];
  unsigned int err[kSlots];
};

struct DevShared {
  unsigned long long taken;
  unsigned int finished[kSlots];
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_volatile_sys_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys_u32(unsigned int *p, unsigned int v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Request buffers may be rewritten by the client between requests while the
// executor stays resident, so they are read through L2 only.
__device__ __forceinline__ uint2 ld_pair_cg(const uint2 *a) {
  uint2 r;
  asm volatile("ld.global.cg.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(a) : "memory");
  return r;
}

// Runtime root function of a served graph: names f(x) = x + 1 (x != m), 0
// for m under R; f(x) = x under the identity. Slots S = P - rf.
__device__ __forceinline__ uint32_t name_of(uint32_t x, uint32_t rf, uint32_t m) {
  return rf ? (x == m ? 0u : x + 1u) : x;
}

// The persistent executor: blocks take work items one at a time, run them,
// and count the request's finished tiles. A block leaves when `stop` is set
// or when no item arrives for idle_ns.
__global__ void __launch_bounds__(256) k_executor(HostShared *hs, DevShared *ds, unsigned long long idle_ns) {
  __shared__ WorkItem it;
  __shared__ int s_leave;
  __shared__ unsigned int s_bad;
  __shared__ uint32_t ring_smem[8 * 4 * kRing];
  while (true) {
    if (threadIdx.x == 0) {
      int leave = 1;
      const unsigned long long t0 = now_ns();
      while (true) {
        const unsigned long long pub = ld_acquire_sys_u64(&hs->published);
        const unsigned long long t = ld_volatile_u64(&ds->taken);
        if (t < pub) {
          if (atomicCAS(&ds->taken, t, t + 1ULL) == t) {
            const volatile WorkItem *src = &hs->ring[t % kRingCap];
            it.kind = src->kind;
            it.slot = src->slot;
            it.seq = src->seq;
            it.n_tiles = src->n_tiles;
            it.rf = src->rf;
            it.m = src->m;
            it.n = src->n;
            it.P = src->P;
            it.src = src->src;
            it.begin = src->begin;
            it.end = src->end;
            it.out = src->out;
            leave = 0;
            break;
          }
          continue;  // another block took it: look again at once
        }
        if (ld_volatile_sys_u32(&hs->stop)) break;
        if (now_ns() - t0 > idle_ns) break;  // bounded idle wait
        __nanosleep(256);
      }
      s_leave = leave;
      s_bad = 0u;
    }
    __syncthreads();
    if (s_leave) return;

    uint32_t *const P = reinterpret_cast<uint32_t *>(it.P);
    uint32_t *const S = P - it.rf;
    const uint32_t n = it.n, rf = it.rf, m = it.m;
    const uint2 *src = reinterpret_cast<const uint2 *>(it.src);
    if (it.kind == kItemEdges || it.kind == kItemValidate) {
      bool bad = false;
      for (uint64_t i = it.begin + threadIdx.x; i < it.end; i += blockDim.x) {
        const uint2 e = ld_pair_cg(src + i);
        bad |= e.x >= n || e.y >= n;
      }
      if (bad) s_bad = 1u;
    }
    __syncthreads();
    if ((it.kind == kItemEdges && !s_bad) || it.kind == kItemApply) {
      WarpRing ring;
      ring.init(ring_smem);
      // warp-uniform rounds over the tile
      for (uint64_t r0 = it.begin; r0 < it.end; r0 += blockDim.x) {
        const uint64_t i = r0 + threadIdx.x;
        uint32_t a = 0, b = 0, pa = 0, pb = 0;
        if (i < it.end) {
          const uint2 e = ld_pair_cg(src + i);
          if (e.x < n && e.y < n) {
            a = name_of(e.x, rf, m);
            b = name_of(e.y, rf, m);
            pa = ldP_cg(P + e.x);
            pb = ldP_cg(P + e.y);
          }
        }
        ring.push<true>(S, pa != pb, a, pa, b, pb);
      }
      ring.drain<true>(S);
    } else if (it.kind == kItemQuery) {
      uint8_t *out = reinterpret_cast<uint8_t *>(it.out);
      bool bad = false;
      for (uint64_t i = it.begin + threadIdx.x; i < it.end; i += blockDim.x) {
        const uint2 q = ld_pair_cg(src + i);
        uint8_t r = 0;
        if (q.x >= n || q.y >= n) {
          bad = true;
        } else {
          // read-only walks: queries never write P
          uint32_t cu = name_of(q.x, rf, m), pu = ldP_cg(P + q.x);
          while (pu != cu && pu != 0u) {
            cu = pu;
            pu = ldP_cg(S + pu);
          }
          if (pu == 0u) cu = 0u;
          uint32_t cv = name_of(q.y, rf, m), pv = ldP_cg(P + q.y);
          while (pv != cv && pv != 0u) {
            cv = pv;
            pv = ldP_cg(S + pv);
          }
          if (pv == 0u) cv = 0u;
          r = cu == cv;
        }
        out[i] = r;
      }
      if (bad) s_bad = 1u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_bad) *(volatile unsigned int *)&hs->err[it.slot] = 1u;
      __threadfence();
      const unsigned int prev = atomicAdd(&ds->finished[it.slot], 1u);
      if (prev + 1u == it.n_tiles) {
        ds->finished[it.slot] = 0u;
        __threadfence_system();
        st_release_sys_u32(&hs->done_seq[it.slot], it.seq);
      }
    }
    __syncthreads();
  }
}

// gmin <- m, ncomp <- 0 before a snapshot's flatten.
__global__ void k_srv_prep_flatten(Ctrl *ctrl) {
  ctrl->gmin = ctrl->m;
  ctrl->ncomp = 0ULL;
}

}  // namespace srv
}  // namespace cc

using cc::srv::DevShared;
using cc::srv::HostShared;
using cc::srv::WorkItem;

namespace {

uint64_t host_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) with coalescing of neighbouring holes.
class Arena {
 public:
  void reset(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(uint64_t size, uint64_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= size) {
        *off = it->first;
        const uint64_t rest = it->second - size, start = it->first + size;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += size;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t size) {
    used_ -= size;
    auto it = free_.emplace(off, size).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t used_ = 0;
};

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2 };
enum GroupClass { kIdle = 0, kWriters = 1, kReaders = 2, kExclusive = 3 };

struct Req {
  cc_request r{};
  uint32_t graph = 0;
  uint64_t t_submit = 0, t_done = 0;
  int state = kQueued;
  cc_status result = CC_OK;
  // executor bookkeeping
  uint32_t slot = UINT32_MAX, seq = 0, n_tiles = 0;
  int phase = 0;  // inserts: 1 validating, 2 applying
  // side-stream bookkeeping
  cudaEvent_t ev = nullptr;
};

struct GraphState {
  bool live = false;
  bool rf = true;
  uint64_t n = 0, off = 0, bytes = 0;
  uint32_t *P = nullptr;
  void *cnt = nullptr;
  cc::CertScratch *cert = nullptr;
  cc::Ctrl *ctrl = nullptr;
  uint32_t m = 0;
  std::deque<uint64_t> fifo;
  int group = kIdle;
  int active = 0;
};

}  // namespace

struct cc_server {
  cc_server_config cfg{};
  int device = 0;
  char *arena_base = nullptr;
  Arena arena;
  HostShared *hs = nullptr;  // host view of the mapped block
  HostShared *hs_dev = nullptr;
  DevShared *ds = nullptr;
  cudaStream_t exec_stream = nullptr, side_stream = nullptr;
  cudaEvent_t exec_ev = nullptr;
  bool exec_running = false;
  uint32_t *side_words = nullptr;  // pinned: per-graph m and error words read back after a run
  // shared with client threads (mu)
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Req> reqs;          // ticket t is reqs[t - 1]
  std::deque<uint64_t> inbox;
  std::vector<int> id_state;      // 0 free, 1 assigned, 2 dropping
  std::vector<uint32_t> free_ids;
  cc_server_stats stats{};
  bool quit = false;
  // scheduler-thread state
  std::vector<GraphState> graphs;
  std::vector<uint32_t> free_slots;
  std::vector<uint64_t> slot_ticket;
  uint64_t in_flight_items = 0;
  std::vector<uint64_t> side_running;  // tickets with side-stream work in flight
  std::thread thread;
};

namespace {

uint64_t graph_bytes(const cc_server *s, uint64_t n, uint64_t n_edges, bool rf) {
  size_t b = align256((size_t)((n + 3) / 4 * 4) * 4) + align256(sizeof(cc::Ctrl));
  if (rf) b += align256((size_t)n * (n_edges >= (1ULL << 31) ? 8 : 4)) + align256(sizeof(cc::CertScratch));
  (void)s;
  return b;
}

void complete(cc_server *s, uint64_t t, cc_status st) {
  Req &r = s->reqs[t - 1];
  r.state = kDone;
  r.result = st;
  r.t_done = host_ns();
  s->stats.completed++;
  if (st != CC_OK) s->stats.failed++;
}

void publish_tiles(cc_server *s, Req &r, uint32_t kind, uint64_t count, const uint32_t *src,
                   const GraphState &g) {
  uint64_t tile = s->cfg.tile_edges;
  const uint64_t min_tile = (count + (cc::srv::kRingCap / 4) - 1) / (cc::srv::kRingCap / 4);
  if (tile < min_tile) tile = min_tile;
  const uint32_t n_tiles = (uint32_t)((count + tile - 1) / tile);
  r.n_tiles = n_tiles;
  r.seq++;
  s->hs->err[r.slot] = 0u;
  unsigned long long pub = s->hs->published;
  for (uint32_t i = 0; i < n_tiles; ++i) {
    WorkItem &w = s->hs->ring[(pub + i) % cc::srv::kRingCap];
    w.kind = kind;
    w.slot = r.slot;
    w.seq = r.seq;
    w.n_tiles = n_tiles;
    w.rf = g.rf ? 1u : 0u;
    w.m = g.m;
    w.n = (uint32_t)g.n;
    w.P = (uint64_t)(uintptr_t)g.P;
    w.src = (uint64_t)(uintptr_t)src;
    w.begin = (uint64_t)i * tile;
    w.end = w.begin + tile < count ? w.begin + tile : count;
    w.out = (uint64_t)(uintptr_t)r.r.out_dev;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  *(volatile unsigned long long *)&s->hs->published = pub + n_tiles;
  s->in_flight_items += n_tiles;
  s->stats.tiles_run += n_tiles;
}

uint64_t tiles_needed(const cc_server *s, uint64_t count) {
  uint64_t tile = s->cfg.tile_edges;
  const uint64_t min_tile = (count + (cc::srv::kRingCap / 4) - 1) / (cc::srv::kRingCap / 4);
  if (tile < min_tile) tile = min_tile;
  return (count + tile - 1) / tile;
}

// Starts an insert or query on the executor; false when no slot or ring room.
bool start_exec(cc_server *s, uint64_t t, GraphState &g) {
  Req &r = s->reqs[t - 1];
  const bool insert = r.r.kind == CC_REQ_INSERT;
  const uint64_t count = insert ? r.r.n_edges : r.r.n_pairs;
  if (count == 0) {
    complete(s, t, CC_OK);
    return true;
  }
  const uint64_t need = tiles_needed(s, count);
  if (s->free_slots.empty() || s->in_flight_items + need > cc::srv::kRingCap / 2) return false;
  r.slot = s->free_slots.back();
  s->free_slots.pop_back();
  s->slot_ticket[r.slot] = t;
  r.state = kRunning;
  if (insert) {
    r.phase = need == 1 ? 2 : 1;  // a single tile validates and applies itself
    publish_tiles(s, r, need == 1 ? cc::srv::kItemEdges : cc::srv::kItemValidate, count, r.r.edges_dev, g);
  } else {
    publish_tiles(s, r, cc::srv::kItemQuery, count, r.r.pairs_dev, g);
  }
  return true;
}

// Root selection (f = R), init, hooking pass and flatten of a new graph on
// the side stream; m and the error word are copied back to pinned memory.
bool start_new_graph(cc_server *s, uint64_t t, GraphState &g) {
  Req &r = s->reqs[t - 1];
  const bool rf = s->cfg.mode == CC_ROOT_MAXDEG;
  const uint64_t bytes = graph_bytes(s, r.r.n_vertices, r.r.n_edges, rf);
  uint64_t off = 0;
  if (!s->arena.alloc(bytes, &off)) return false;  // wait for memory
  g.live = true;
  g.rf = rf;
  g.n = r.r.n_vertices;
  g.off = off;
  g.bytes = bytes;
  char *p = s->arena_base + off;
  g.P = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)((g.n + 3) / 4 * 4) * 4);
  g.ctrl = reinterpret_cast<cc::Ctrl *>(p);
  p += align256(sizeof(cc::Ctrl));
  const bool wide = r.r.n_edges >= (1ULL << 31);
  if (rf) {
    g.cnt = p;
    p += align256((size_t)g.n * (wide ? 8 : 4));
    g.cert = reinterpret_cast<cc::CertScratch *>(p);
  }
  r.state = kRunning;
  cudaStream_t ss = s->side_stream;
  cudaError_t e = cudaMemsetAsync(g.ctrl, 0, sizeof(cc::Ctrl), ss);
  const uint32_t n = (uint32_t)g.n;
  const cc::EdgeSpan span = cc::split_edges(r.r.edges_dev, r.r.n_edges);
  int m_src = cc::kMFromHint;
  if (e == cudaSuccess && rf && n) {
    e = cc::launch_root_select_certified(r.r.edges_dev, r.r.n_edges, span, g.cnt, wide, n, g.cert, g.ctrl, ss);
    m_src = cc::kMFromPackedMax;
  }
  if (e == cudaSuccess && n) e = cc::launch_init(rf, g.P, n, g.ctrl, m_src, 0u, ss);
  if (e == cudaSuccess && n) e = cc::launch_edge_pass(rf, 1, 4, 256, span, g.P, n, g.ctrl, false, ss);
  if (e == cudaSuccess && n) e = cc::launch_flatten(rf, s->cfg.label_space, g.P, n, r.r.labels_dev, g.ctrl, ss);
  const uint32_t gid = r.graph;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->side_words[2 * gid], &g.ctrl->m, sizeof(uint32_t), cudaMemcpyDeviceToHost, ss);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->side_words[2 * gid + 1], &g.ctrl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ss);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.ev, ss);
  if (e != cudaSuccess) {
    complete(s, t, CC_ERR_CUDA);
    return true;
  }
  s->side_running.push_back(t);
  return true;
}

bool start_snapshot(cc_server *s, uint64_t t, GraphState &g) {
  Req &r = s->reqs[t - 1];
  r.state = kRunning;
  cudaStream_t ss = s->side_stream;
  cudaError_t e = cudaSuccess;
  if (g.n) {
    cc::srv::k_srv_prep_flatten<<<1, 1, 0, ss>>>(g.ctrl);
    cc::note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cc::launch_flatten(g.rf, s->cfg.label_space, g.P, (uint32_t)g.n, r.r.labels_dev, g.ctrl, ss);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.ev, ss);
  if (e != cudaSuccess) {
    complete(s, t, CC_ERR_CUDA);
    return true;
  }
  s->side_running.push_back(t);
  return true;
}

int class_of(int kind) {
  switch (kind) {
    case CC_REQ_INSERT: return kWriters;
    case CC_REQ_QUERY:
    case CC_REQ_SNAPSHOT: return kReaders;
    default: return kExclusive;
  }
}

void finish_graph_request(cc_server *s, GraphState &g) {
  if (--g.active == 0) g.group = kIdle;
  (void)s;
}

// Starts what may start at the head of a graph's queue.
void try_start(cc_server *s, uint32_t gid) {
  GraphState &g = s->graphs[gid];
  while (!g.fifo.empty()) {
    const uint64_t t = g.fifo.front();
    Req &r = s->reqs[t - 1];
    const int cls = class_of(r.r.kind);
    if (g.group == kExclusive) return;
    if (cls == kExclusive) {
      if (g.active) return;
      if (r.r.kind == CC_REQ_NEW_GRAPH) {
        if (!start_new_graph(s, t, g)) return;  // no memory yet
        g.fifo.pop_front();
        if (r.state == kRunning) {
          g.group = kExclusive;
          g.active = 1;
        }
        return;
      }
      // drop
      if (g.live) s->arena.release(g.off, g.bytes);
      g.live = false;
      g.fifo.pop_front();
      complete(s, t, CC_OK);
      {
        s->id_state[gid] = 0;
        s->free_ids.push_back(gid);
      }
      continue;
    }
    if (g.active && g.group != cls) return;
    bool started;
    if (r.r.kind == CC_REQ_SNAPSHOT)
      started = start_snapshot(s, t, g);
    else
      started = start_exec(s, t, g);
    if (!started) return;
    g.fifo.pop_front();
    if (r.state == kRunning) {
      g.group = cls;
      g.active++;
    }
  }
}

void ensure_executor(cc_server *s) {
  if (s->exec_running) {
    if (cudaEventQuery(s->exec_ev) == cudaSuccess) s->exec_running = false;
  }
  if (!s->exec_running && s->in_flight_items > 0) {
    const unsigned grid = (unsigned)(cc::num_sms() * s->cfg.executor_blocks_per_sm);
    cc::srv::k_executor<<<grid, 256, 0, s->exec_stream>>>(s->hs_dev, s->ds,
                                                         (unsigned long long)s->cfg.idle_timeout_us * 1000ULL);
    cc::note_launch();
    cudaEventRecord(s->exec_ev, s->exec_stream);
    s->exec_running = true;
    s->stats.executor_launches++;
  }
}

// One scheduler pass; returns true when anything changed.
bool scheduler_step(cc_server *s) {
  bool progress = false;
  std::vector<uint32_t> touched;
  // 1. new requests into their graphs' queues
  while (!s->inbox.empty()) {
    const uint64_t t = s->inbox.front();
    s->inbox.pop_front();
    Req &r = s->reqs[t - 1];
    s->graphs[r.graph].fifo.push_back(t);
    touched.push_back(r.graph);
    progress = true;
  }
  // 2. executor completions
  for (uint32_t slot = 0; slot < cc::srv::kSlots; ++slot) {
    const uint64_t t = s->slot_ticket[slot];
    if (!t) continue;
    Req &r = s->reqs[t - 1];
    if (*(volatile unsigned int *)&s->hs->done_seq[slot] != r.seq) continue;
    s->in_flight_items -= r.n_tiles;
    const bool bad = *(volatile unsigned int *)&s->hs->err[slot] != 0u;
    GraphState &g = s->graphs[r.graph];
    if (r.r.kind == CC_REQ_INSERT && r.phase == 1 && !bad) {
      r.phase = 2;  // validated: apply
      publish_tiles(s, r, cc::srv::kItemApply, r.r.n_edges, r.r.edges_dev, g);
      progress = true;
      continue;
    }
    s->slot_ticket[slot] = 0;
    s->free_slots.push_back(slot);
    complete(s, t, bad ? CC_ERR_OUT_OF_RANGE : CC_OK);
    finish_graph_request(s, g);
    touched.push_back(r.graph);
    progress = true;
  }
  // 3. side-stream completions
  for (size_t i = 0; i < s->side_running.size();) {
    const uint64_t t = s->side_running[i];
    Req &r = s->reqs[t - 1];
    const cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    cudaEventDestroy(r.ev);
    r.ev = nullptr;
    GraphState &g = s->graphs[r.graph];
    cc_status st = q == cudaSuccess ? CC_OK : CC_ERR_CUDA;
    if (r.r.kind == CC_REQ_NEW_GRAPH && st == CC_OK) {
      g.m = s->side_words[2 * r.graph];
      if (s->side_words[2 * r.graph + 1]) st = CC_ERR_OUT_OF_RANGE;
    }
    complete(s, t, st);
    finish_graph_request(s, g);
    touched.push_back(r.graph);
    s->side_running[i] = s->side_running.back();
    s->side_running.pop_back();
    progress = true;
  }
  // 4. start what may start; graphs waiting for memory are retried too
  for (uint32_t gid : touched) try_start(s, gid);
  for (uint32_t gid = 0; gid < s->graphs.size(); ++gid)
    if (!s->graphs[gid].fifo.empty() && s->graphs[gid].group == kIdle) try_start(s, gid);
  ensure_executor(s);
  return progress;
}

void scheduler_main(cc_server *s) {
  cudaSetDevice(s->device);
  while (true) {
    bool busy;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (scheduler_step(s)) s->cv.notify_all();
      busy = s->in_flight_items > 0 || !s->side_running.empty();
      bool queued = !s->inbox.empty();
      for (auto &g : s->graphs)
        if (!g.fifo.empty()) {
          queued = true;
          break;
        }
      if (s->quit && !busy && !queued) break;
      if (!busy) {
        // waiting for memory or ordering: retry soon, or at the next submit
        s->cv.wait_for(lk, queued ? std::chrono::microseconds(100) : std::chrono::milliseconds(2));
        continue;
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(2));  // poll completions
  }
}

}  // namespace

extern "C" {

void cc_server_config_init(cc_server_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->max_graphs = 1024;
  cfg->executor_blocks_per_sm = 2;
  cfg->tile_edges = 16384;
  cfg->idle_timeout_us = 20000;
  cfg->mode = CC_ROOT_MAXDEG;
  cfg->label_space = CC_LABEL_MIN_ID;
}

cc_status cc_server_create(const cc_server_config *cfg_in, cc_server **out) {
  if (!out || !cfg_in) return CC_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  cc_server_config cfg = *cfg_in;
  if (!cfg.max_graphs) cfg.max_graphs = 1024;
  if (!cfg.executor_blocks_per_sm) cfg.executor_blocks_per_sm = 2;
  if (!cfg.tile_edges) cfg.tile_edges = 16384;
  if (!cfg.idle_timeout_us) cfg.idle_timeout_us = 20000;
  if (cfg.hbm_budget_bytes == 0 || cfg.executor_blocks_per_sm > 8 ||
      (cfg.mode != CC_ROOT_IDENTITY && cfg.mode != CC_ROOT_MAXDEG) ||
      (cfg.label_space != CC_LABEL_MIN_ID && cfg.label_space != CC_LABEL_ROOT_VALUE) || cfg.max_graphs > (1u << 20))
    return CC_ERR_INVALID_ARGUMENT;
  for (int r : cfg.reserved)
    if (r) return CC_ERR_INVALID_ARGUMENT;
  cc_server *s = new (std::nothrow) cc_server();
  if (!s) return CC_ERR_OOM;
  s->cfg = cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->arena_base, cfg.hbm_budget_bytes);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->hs, sizeof(HostShared), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s->hs_dev, s->hs, 0);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->ds, sizeof(DevShared));
  if (e == cudaSuccess) e = cudaMemset(s->ds, 0, sizeof(DevShared));
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->side_words, 2 * (size_t)cfg.max_graphs * sizeof(uint32_t), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->exec_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->exec_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cc_status st = e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->hs) cudaFreeHost(s->hs);
    if (s->ds) cudaFree(s->ds);
    if (s->side_words) cudaFreeHost(s->side_words);
    if (s->exec_stream) cudaStreamDestroy(s->exec_stream);
    if (s->side_stream) cudaStreamDestroy(s->side_stream);
    if (s->exec_ev) cudaEventDestroy(s->exec_ev);
    delete s;
    return st;
  }
  memset(s->hs, 0, sizeof(HostShared));
  s->arena.reset(cfg.hbm_budget_bytes);
  s->graphs.resize(cfg.max_graphs);
  s->id_state.assign(cfg.max_graphs, 0);
  for (uint32_t i = cfg.max_graphs; i-- > 0;) s->free_ids.push_back(i);
  for (uint32_t i = cc::srv::kSlots; i-- > 0;) s->free_slots.push_back(i);
  s->slot_ticket.assign(cc::srv::kSlots, 0);
  s->stats.arena_bytes = cfg.hbm_budget_bytes;
  s->thread = std::thread(scheduler_main, s);
  *out = s;
  return CC_OK;
}

cc_status cc_server_submit(cc_server *s, const cc_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return CC_ERR_INVALID_ARGUMENT;
  const cc_request &r = *req;
  auto misaligned = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; };
  switch (r.kind) {
    case CC_REQ_NEW_GRAPH:
      if (r.n_vertices > 0x7FFFFFFFULL) return CC_ERR_TOO_LARGE;
      if (r.n_edges && (!r.edges_dev || misaligned(r.edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      if (r.labels_dev && misaligned(r.labels_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
      if (graph_bytes(s, r.n_vertices, r.n_edges, s->cfg.mode == CC_ROOT_MAXDEG) > s->cfg.hbm_budget_bytes)
        return CC_ERR_TOO_LARGE;
      break;
    case CC_REQ_INSERT:
      if (r.n_edges && (!r.edges_dev || misaligned(r.edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      break;
    case CC_REQ_QUERY:
      if (r.n_pairs && (!r.pairs_dev || !r.out_dev || misaligned(r.pairs_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      break;
    case CC_REQ_SNAPSHOT:
      if (!r.labels_dev || misaligned(r.labels_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
      break;
    case CC_REQ_DROP_GRAPH:
      break;
    default:
      return CC_ERR_INVALID_ARGUMENT;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->quit) return CC_ERR_INVALID_ARGUMENT;
  uint32_t gid = r.graph;
  if (r.kind == CC_REQ_NEW_GRAPH) {
    if (s->free_ids.empty()) return CC_ERR_TOO_LARGE;
    gid = s->free_ids.back();
    s->free_ids.pop_back();
    s->id_state[gid] = 1;
  } else {
    if (gid >= s->cfg.max_graphs || s->id_state[gid] != 1) return CC_ERR_INVALID_ARGUMENT;
    if (r.kind == CC_REQ_DROP_GRAPH) s->id_state[gid] = 2;
  }
  Req q;
  q.r = r;
  q.graph = gid;
  q.t_submit = host_ns();
  s->reqs.push_back(q);
  const uint64_t t = s->reqs.size();
  s->inbox.push_back(t);
  s->stats.submitted++;
  *ticket = t;
  s->cv.notify_all();
  return CC_OK;
}

cc_status cc_server_poll(cc_server *s, uint64_t ticket, cc_status *result) {
  if (!s || !result) return CC_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket > s->reqs.size()) return CC_ERR_INVALID_ARGUMENT;
  const Req &r = s->reqs[ticket - 1];
  if (r.state != kDone) return CC_ERR_NOT_READY;
  *result = r.result;
  return CC_OK;
}

cc_status cc_server_wait(cc_server *s, uint64_t ticket, uint64_t timeout_ns, cc_status *result) {
  if (!s || !result) return CC_ERR_INVALID_ARGUMENT;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket > s->reqs.size()) return CC_ERR_INVALID_ARGUMENT;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
  while (s->reqs[ticket - 1].state != kDone) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && s->reqs[ticket - 1].state != kDone)
      return CC_ERR_TIMEOUT;
  }
  *result = s->reqs[ticket - 1].result;
  return CC_OK;
}

cc_status cc_server_result_graph(cc_server *s, uint64_t ticket, uint32_t *graph) {
  if (!s || !graph) return CC_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket > s->reqs.size()) return CC_ERR_INVALID_ARGUMENT;
  *graph = s->reqs[ticket - 1].graph;
  return CC_OK;
}

cc_status cc_server_latency_ns(cc_server *s, uint64_t ticket, uint64_t *ns) {
  if (!s || !ns) return CC_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket > s->reqs.size()) return CC_ERR_INVALID_ARGUMENT;
  const Req &r = s->reqs[ticket - 1];
  if (r.state != kDone) return CC_ERR_NOT_READY;
  *ns = r.t_done - r.t_submit;
  return CC_OK;
}

cc_status cc_server_get_stats(cc_server *s, cc_server_stats *st) {
  if (!s || !st) return CC_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->arena_bytes_used = s->arena.used();
  uint64_t live = 0;
  for (auto &g : s->graphs) live += g.live;
  st->resident_graphs = live;
  return CC_OK;
}

void cc_server_destroy(cc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->quit = true;
    s->cv.notify_all();
  }
  if (s->thread.joinable()) s->thread.join();
  *(volatile unsigned int *)&s->hs->stop = 1u;
  cudaStreamSynchronize(s->exec_stream);
  cudaStreamSynchronize(s->side_stream);
  for (auto &r : s->reqs)
    if (r.ev) cudaEventDestroy(r.ev);
  cudaFree(s->arena_base);
  cudaFreeHost(s->hs);
  cudaFree(s->ds);
  cudaFreeHost(s->side_words);
  cudaStreamDestroy(s->exec_stream);
  cudaStreamDestroy(s->side_stream);
  cudaEventDestroy(s->exec_ev);
  delete s;
}

}  // extern "C"

// cc_server.cu - serving runtime (include/cc_server.h): a host scheduler
// thread, a device arena with a first-fit allocator, and a persistent executor
// kernel that runs insert and query tiles on the live parent arrays of
// resident graphs.
//
// Host <-> device protocol (mapped pinned host memory unless noted):
//   ring[]     work items written by the host; `published` counts them;
//   taken      (device memory) items claimed so far: a block claims the next
//              index with one fetch-and-add and waits, bounded, until the
//              host has published it;
//   done_seq[] per request slot: the executor stores the item's sequence
//              number after the request's last tile (release, system scope);
//   err[]      per request slot: 1 = an out-of-range id, 2 = a gated wait
//              expired;
//   stop       the host asks the executor to leave (after an idle period,
//              when every published item has been processed; the host then
//              sets taken back to published before the next launch).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
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
// Default bounded waits of the executor (cc_server_config.gate_wait_us and
// publish_wait_us set others).
constexpr unsigned long long kGateTimeoutNs = 2000000000ULL;  // gated apply tile: 2 s
constexpr unsigned long long kWaitLimitNs = 30000000000ULL;   // waiting for an item: 30 s
// Side-stream requests in flight at once: bounds the launches queued on the
// side stream so that a launch never blocks the scheduler thread.
constexpr size_t kMaxSideRunning = 16;
// A side-stream request still unfinished this long while the executor runs
// makes the host drain the executor once, so that kernels that cannot fit
// beside it get the SMs.
constexpr uint64_t kSideStarveNs = 20ULL * 1000 * 1000;
// Inserts of at least this many edges run on a side stream as one validated,
// full-occupancy edge pass beside the executor instead of as executor tiles.
constexpr uint64_t kSideInsertMin = 1ULL << 18;
// Side streams; a graph's side work always goes to the same one, in order.
constexpr uint32_t kSideStreams = 4;
// Graphs whose parent array reaches this size keep a zero-tree bitmap.
constexpr uint64_t kZMinBytes = 128ULL << 20;

struct alignas(16) WorkItem {
  uint32_t kind, slot, seq, n_tiles;  // n_tiles: tiles that count towards completion
  uint32_t rf, m, n, n_gate;          // n_gate: validate tiles an apply tile waits for
  uint64_t P, src, begin, end, out;
  uint64_t log;  // the graph's changed-root log (inserts append the roots they hook)
  uint64_t Z;    // the graph's zero-tree bitmap, or 0
  uint64_t pad;
};
static_assert(sizeof(WorkItem) == 96, "work item layout: six 16-byte loads");

struct HostShared {
  unsigned long long published;
  unsigned int stop;
  unsigned int exec_err;  // an executor wait expired (the host stopped answering)
  unsigned int pad[12];
  WorkItem ring[kRingCap];
  unsigned int done_seq[kSlots];
  unsigned int err[kSlots];
};

struct DevShared {
  unsigned long long taken;
  unsigned int finished[kSlots];   // completion-counting tiles done
  unsigned int validated[kSlots];  // validate tiles done
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

__device__ __forceinline__ void st_release_sys_u32(unsigned int *p, unsigned int v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A work item from mapped host memory: six 16-byte loads in flight at once.
__device__ __forceinline__ void load_item(const WorkItem *src, WorkItem *dst) {
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
  uint4 *d4 = reinterpret_cast<uint4 *>(dst);
  uint4 v[6];
#pragma unroll
  for (int k = 0; k < 6; ++k)
    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[k].x), "=r"(v[k].y), "=r"(v[k].z), "=r"(v[k].w)
                 : "l"(s4 + k)
                 : "memory");
#pragma unroll
  for (int k = 0; k < 6; ++k) d4[k] = v[k];
}

// Zero-tree bit of the vertex named c, through L2 only: the executor's blocks
// outlive other kernels' writes, and an arena region reused by a new graph
// must never show the bits of the old one from a stale L1 line.
__device__ __forceinline__ bool zbit_cg(const uint32_t *Z, uint32_t c) {
  uint32_t w;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(w) : "l"(Z + (c >> 5)) : "memory");
  return (w >> (c & 31u)) & 1u;
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

// Read-only root name of a vertex: walk parents (L2 loads) until a root or
// the permanent root 0.
__device__ __forceinline__ void walk_step(const uint32_t *S, uint32_t &c, uint32_t &p, bool &done) {
  if (!done) {
    if (p == c || p == 0u) {
      if (p == 0u) c = 0u;
      done = true;
    } else {
      c = p;
      p = ldP_cg(S + c);
    }
  }
}

constexpr int kEpt = 4;  // elements per thread per round

// The persistent executor: each block claims the next item index, waits
// (at most wait_ns) until the host has published it, runs it, and counts the
// request's finished tiles. Blocks leave when the host sets `stop`, or when
// a wait expires (exec_err tells the host). A gated apply tile waits at most
// gate_ns for its request's validate tiles.
__global__ void __launch_bounds__(256) k_executor(HostShared *hs, DevShared *ds, unsigned long long wait_ns,
                                                  unsigned long long gate_ns) {
  __shared__ WorkItem it;
  __shared__ int s_leave;
  __shared__ unsigned int s_bad, s_skip;
  __shared__ uint32_t ring_smem[8 * 4 * kRing];
  while (true) {
    if (threadIdx.x == 0) {
      int leave = 0;
      const unsigned long long t = atomicAdd(&ds->taken, 1ULL);
      const unsigned long long t0 = now_ns();
      unsigned int backoff = 32;
      while (ld_acquire_sys_u64(&hs->published) <= t) {
        if (ld_volatile_sys_u32(&hs->stop)) {
          leave = 1;
          break;
        }
        if (now_ns() - t0 > wait_ns) {  // the host stopped answering
          *(volatile unsigned int *)&hs->exec_err = 1u;
          leave = 1;
          break;
        }
        __nanosleep(backoff);
        if (backoff < 4096) backoff <<= 1;
      }
      if (!leave) load_item(&hs->ring[t % kRingCap], &it);
      s_leave = leave;
      s_bad = 0u;
      s_skip = 0u;
      // a gated apply tile waits (bounded) until every validate tile of its
      // request has finished; they were all claimed before it (ring order)
      if (!leave && it.kind == kItemApply && it.n_gate) {
        const unsigned long long g0 = now_ns();
        while (ld_volatile_sys_u32(&ds->validated[it.slot]) < it.n_gate) {
          if (now_ns() - g0 > gate_ns) {
            s_skip = 1u;
            s_bad = 2u;  // reported as a timeout
            break;
          }
          __nanosleep(128);
        }
        __threadfence();
        if (ld_volatile_sys_u32(&hs->err[it.slot])) s_skip = 1u;  // rejected: apply nothing
      }
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
      if (bad) atomicMax(&s_bad, 1u);
    }
    __syncthreads();
    uint32_t *const Zb = reinterpret_cast<uint32_t *>(it.Z);
    if ((it.kind == kItemEdges && !s_bad) || (it.kind == kItemApply && !s_skip)) {
      WarpRing ring;
      ring.init(ring_smem, Zb, reinterpret_cast<uint32_t *>(it.log));
      // warp-uniform rounds of kEpt edges per thread, all parent loads issued together
      for (uint64_t r0 = it.begin; r0 < it.end; r0 += (uint64_t)blockDim.x * kEpt) {
        uint32_t a[kEpt], b[kEpt], pa[kEpt], pb[kEpt];
#pragma unroll
        for (int j = 0; j < kEpt; ++j) {
          const uint64_t i = r0 + (uint64_t)j * blockDim.x + threadIdx.x;
          a[j] = b[j] = pa[j] = pb[j] = 0u;
          if (i < it.end) {
            const uint2 e = ld_pair_cg(src + i);
            if (e.x < n && e.y < n) {
              a[j] = e.x;
              b[j] = e.y;
              pa[j] = 1u;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kEpt; ++j) {
          if (pa[j]) {
            const uint32_t na = name_of(a[j], rf, m), nb = name_of(b[j], rf, m);
            // a vertex known to be in the tree of name 0 needs no parent load
            const bool za = Zb && zbit_cg(Zb, na), zb = Zb && zbit_cg(Zb, nb);
            pa[j] = za ? 0u : ldP_cg(P + a[j]);
            pb[j] = zb ? 0u : ldP_cg(P + b[j]);
            // a parent value 0 proves membership in the tree of name 0: keep
            // the bit (the warp ring sets none for an endpoint whose parent is 0)
            if (Zb && !za && pa[j] == 0u) zset(Zb, na);
            if (Zb && !zb && pb[j] == 0u) zset(Zb, nb);
            a[j] = na;
            b[j] = nb;
          }
        }
#pragma unroll
        for (int j = 0; j < kEpt; ++j) ring.push<true>(S, pa[j] != pb[j], a[j], pa[j], b[j], pb[j]);
      }
      ring.drain<true>(S);
    } else if (it.kind == kItemQuery) {
      uint8_t *out = reinterpret_cast<uint8_t *>(it.out);
      bool bad = false;
      for (uint64_t r0 = it.begin; r0 < it.end; r0 += (uint64_t)blockDim.x * kEpt) {
        // kEpt queries per thread, their 2 * kEpt read-only walks in lock step
        uint32_t c[2 * kEpt], p[2 * kEpt];
        bool done[2 * kEpt], valid[kEpt];
#pragma unroll
        for (int j = 0; j < kEpt; ++j) {
          const uint64_t i = r0 + (uint64_t)j * blockDim.x + threadIdx.x;
          done[2 * j] = done[2 * j + 1] = true;
          valid[j] = false;
          c[2 * j] = c[2 * j + 1] = p[2 * j] = p[2 * j + 1] = 0u;
          if (i < it.end) {
            const uint2 q = ld_pair_cg(src + i);
            if (q.x >= n || q.y >= n) {
              bad = true;
            } else {
              c[2 * j] = name_of(q.x, rf, m);
              c[2 * j + 1] = name_of(q.y, rf, m);
              // an endpoint in the tree of name 0 has root 0: no walk
              const bool zx = Zb && zbit_cg(Zb, c[2 * j]), zy = Zb && zbit_cg(Zb, c[2 * j + 1]);
              p[2 * j] = zx ? 0u : ldP_cg(P + q.x);
              p[2 * j + 1] = zy ? 0u : ldP_cg(P + q.y);
              done[2 * j] = done[2 * j + 1] = false;
              valid[j] = true;
            }
          }
        }
        bool any = true;
        while (any) {  // ends: names strictly decrease along parents
          any = false;
#pragma unroll
          for (int k = 0; k < 2 * kEpt; ++k) {
            walk_step(S, c[k], p[k], done[k]);
            any |= !done[k];
          }
        }
#pragma unroll
        for (int j = 0; j < kEpt; ++j) {
          const uint64_t i = r0 + (uint64_t)j * blockDim.x + threadIdx.x;
          if (i < it.end) out[i] = (uint8_t)(valid[j] && c[2 * j] == c[2 * j + 1]);
        }
      }
      if (bad) atomicMax(&s_bad, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_bad) *(volatile unsigned int *)&hs->err[it.slot] = s_bad;
      __threadfence_system();
      if (it.kind == kItemValidate) {
        atomicAdd(&ds->validated[it.slot], 1u);
      } else {
        const unsigned int prev = atomicAdd(&ds->finished[it.slot], 1u);
        if (prev + 1u == it.n_tiles) {
          ds->finished[it.slot] = 0u;
          ds->validated[it.slot] = 0u;
          __threadfence_system();
          st_release_sys_u32(&hs->done_seq[it.slot], it.seq);
        }
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

// ------------------------------------------------ incremental snapshots
//
// Each resident graph keeps the labels of its last snapshot (Llast) and the
// changed-root log of the inserts since (SiskinCC's pairs sent on a
// successful CAS, Algorithm 2, reused as a log). A root hooked since the last
// snapshot was a root then, so the label its component had is the label of
// that root; every other component kept its label, except that under R the
// smallest vertex of m's tree (gmin) may have dropped. The next snapshot
// therefore maps each changed label to the label of the logged root's
// current root and rewrites Llast in one streaming pass, with no parent walk
// per vertex.

// Label of the root named c in the server's label space.
__device__ __forceinline__ uint32_t root_label(uint32_t c, uint32_t rf, uint32_t min_id, uint32_t gmin) {
  if (!rf || !min_id) return c;  // identity: names are ids; root-value labels are names
  return c == 0u ? gmin : c - 1u;
}

// words[0]: gmin of the last snapshot. chg: one bit per label that changed;
// rem[l]: the new label of a changed label l.
__global__ void __launch_bounds__(256) k_srv_inc_remap(uint32_t *P, uint32_t rf, uint32_t min_id,
                                                       const uint32_t *log, uint32_t *rem, uint32_t *chg,
                                                       const uint32_t *words, const Ctrl *ctrl) {
  uint32_t *const S = P - rf;
  const uint32_t gmin = *(const volatile uint32_t *)&ctrl->gmin;
  const uint32_t count = *(const volatile uint32_t *)log;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t r = log[1u + i];
    const uint32_t root = root_name(S, r, ldP_strong(S + r));
    const uint32_t old = root_label(r, rf, min_id, gmin);
    rem[old] = root_label(root, rf, min_id, gmin);
    atomicOr(chg + (old >> 5), 1u << (old & 31u));
  }
  if (rf && min_id && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t g0 = words[0];
    if (g0 != gmin) {  // m's tree took in a smaller vertex
      rem[g0] = gmin;
      atomicOr(chg + (g0 >> 5), 1u << (g0 & 31u));
    }
  }
}

// L[v] = the new label of Llast[v]; Llast takes the changes. After it: the
// log is emptied, words[0] = gmin (the bitmap is cleared by the host).
__global__ void __launch_bounds__(256) k_srv_inc_relabel(uint32_t *Llast, uint32_t n, const uint32_t *rem,
                                                         const uint32_t *chg, uint32_t *L) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t l = Llast[v];
    if ((chg[l >> 5] >> (l & 31u)) & 1u) {
      l = rem[l];
      Llast[v] = l;
    }
    L[v] = l;
  }
}

__global__ void k_srv_inc_finish(uint32_t *log, uint32_t *words, const Ctrl *ctrl) {
  log[0] = 0u;
  words[0] = *(const volatile uint32_t *)&ctrl->gmin;
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
  uint64_t ticket = 0;
  uint64_t t_submit = 0;
  std::atomic<uint64_t> t_done{0};
  std::atomic<int> state{kQueued};
  std::atomic<int> result{CC_OK};
  // scheduler-thread bookkeeping
  uint32_t slot = UINT32_MAX, seq = 0, n_tiles = 0;
  cudaEvent_t ev = nullptr;
  uint64_t t_side = 0;  // side-stream work issued (or the executor last drained for it) at
  int flag = -1;        // side insert: index of its pinned rejection word
  // snapshot: its read point (the copy of P) and whether the graph's later
  // requests were released once that point had passed
  cudaEvent_t ev_point = nullptr;
  bool detached = false;
};

struct GraphState {
  bool live = false;
  bool rf = true;
  uint64_t n = 0, off = 0, bytes = 0;
  uint32_t *P = nullptr;
  void *cnt = nullptr;
  cc::CertScratch *cert = nullptr;
  cc::Ctrl *ctrl = nullptr;
  uint32_t *Z = nullptr;  // zero-tree bitmap (large graphs under R), or null
  uint64_t z_bytes = 0;
  // incremental snapshots: last labels, two changed-root logs (inserts append
  // to logs[cur_log]; a snapshot takes the other one over), label remap,
  // bitmap, and the copy of P that a snapshot reads
  uint32_t *Llast = nullptr, *rem = nullptr, *chg = nullptr, *words = nullptr, *Psnap = nullptr;
  uint32_t *logs[2] = {nullptr, nullptr};
  int cur_log = 0;
  uint64_t chg_bytes = 0;
  bool has_last = false;   // Llast holds the labels of a snapshot (or of the admission)
  bool snap_busy = false;  // a snapshot still computes from Psnap and its log
  uint32_t m = 0;
  std::deque<Req *> fifo;
  int group = kIdle;
  int active = 0;
};

}  // namespace

struct cc_server {
  cc_server_config cfg{};
  int device = 0;
  char *arena_base = nullptr;
  HostShared *hs = nullptr;  // host view of the mapped block
  HostShared *hs_dev = nullptr;
  DevShared *ds = nullptr;
  cudaStream_t exec_stream = nullptr, side_stream = nullptr;
  cudaStream_t side_streams[cc::srv::kSideStreams] = {};  // [0] is side_stream
  cudaEvent_t exec_ev = nullptr;
  uint32_t *side_words = nullptr;  // pinned: per-graph m and error word read back after admission
  uint32_t *side_flags = nullptr;  // pinned: one rejection word per running side insert
  uint32_t *side_reject = nullptr; // device: the same words, written by validation
  std::vector<int> free_flags;
  uint32_t next_side = 0;          // round-robin stream of side inserts
  // submission side (sub_mu): request objects, the inbox, graph ids
  std::mutex sub_mu;
  std::condition_variable sub_cv;
  std::vector<std::unique_ptr<Req>> reqs;  // ticket t is reqs[t - 1]
  std::vector<Req *> inbox;
  std::vector<int> id_state;  // 0 free, 1 assigned, 2 dropping
  std::vector<uint32_t> free_ids;
  bool quit = false;
  // completion side (done_mu): waiters
  std::mutex done_mu;
  std::condition_variable done_cv;
  std::atomic<uint64_t> submitted{0}, completed{0}, failed{0}, executor_launches{0}, tiles_run{0};
  std::atomic<uint64_t> arena_used{0}, resident{0}, side_drains{0}, snapshot_overlaps{0};
  // scheduler-thread state
  Arena arena;
  std::vector<GraphState> graphs;
  std::vector<uint32_t> free_slots;
  std::vector<Req *> slot_req;
  std::vector<uint32_t> slot_gen;  // per-slot sequence: every publication takes a new one
  uint64_t in_flight_items = 0;
  std::vector<Req *> side_running;  // requests with side-stream work in flight
  bool exec_running = false, exec_stopping = false;
  uint64_t idle_since = 0;
  unsigned long long wait_ns = 0, gate_ns = 0;  // the executor's bounded waits
  std::atomic<uint64_t> executor_timeouts{0};
  // fault injection (cfg.fault_hold_publish_us): executor requests still to
  // hold, and the one whose tiles are written but not yet published
  uint32_t hold_left = 0;
  Req *held = nullptr;
  unsigned long long held_pub = 0;
  uint64_t held_until = 0;
  // apply tiles of multi-tile inserts started in this scheduler pass, written
  // to the ring after every validate tile of the pass (flush_pending_apply)
  struct PendingApply {
    Req *r;
    uint32_t graph, n_work, n_val;
    uint64_t count, tile;
    uint32_t *log;
  };
  std::vector<PendingApply> pending_apply;
  std::thread thread;
};

namespace {

bool wants_z(uint64_t n, bool rf) { return rf && n * 4 >= cc::srv::kZMinBytes; }
uint64_t z_bytes_for(uint64_t n) { return (n + 1 + 31) / 32 * 4; }

// Incremental-snapshot buffers: labels (n), two logs (count + n each), remap
// (n + 1: root-value labels reach n), changed-label bitmap, a few words, and
// the snapshot's copy of P (n).
uint64_t inc_bytes(uint64_t n) {
  return 2 * align256((size_t)((n + 3) / 4 * 4) * 4) + 3 * align256((size_t)(n + 1) * 4) +
         align256((size_t)((n + 1 + 31) / 32) * 4) + align256(16);
}

uint64_t graph_bytes(uint64_t n, uint64_t n_edges, bool rf) {
  size_t b = align256((size_t)((n + 3) / 4 * 4) * 4) + align256(sizeof(cc::Ctrl));
  if (rf) b += align256((size_t)n * (n_edges >= (1ULL << 31) ? 8 : 4)) + align256(sizeof(cc::CertScratch));
  if (wants_z(n, rf)) b += align256(z_bytes_for(n));
  return b + inc_bytes(n);
}

cudaStream_t side_stream_of(const cc_server *s, uint32_t gid) {
  return s->side_streams[gid % cc::srv::kSideStreams];
}

void complete(cc_server *s, Req *r, cc_status st) {
  r->result.store(st);
  r->t_done.store(host_ns());
  r->state.store(kDone, std::memory_order_release);
  s->completed++;
  if (st != CC_OK) s->failed++;
}

// Elements per tile: with an idle executor, enough tiles to spread a request
// over every executor block twice (latency); the more tiles already wait in
// the ring, the fewer and larger the new request's tiles (a backlog keeps the
// blocks busy anyway, and every tile costs a claim, a wait on the host ring
// and an item read from host memory). At least at_least, at most the
// configured tile size, and few enough to fit the ring.
uint64_t tile_for(const cc_server *s, uint64_t count, uint64_t at_least) {
  const uint64_t blocks = (uint64_t)cc::num_sms() * s->cfg.executor_blocks_per_sm;
  const uint64_t spread = 2 * blocks * blocks / (blocks + s->in_flight_items);
  uint64_t t = (count + spread - 1) / (spread ? spread : 1);
  t = (t + 255) / 256 * 256;
  if (t < at_least) t = at_least;
  if (t > s->cfg.tile_edges) t = s->cfg.tile_edges;
  const uint64_t min_tile = (count + (cc::srv::kRingCap / 8) - 1) / (cc::srv::kRingCap / 8);
  return t < min_tile ? min_tile : t;
}

uint64_t n_tiles_of(uint64_t count, uint64_t tile) { return (count + tile - 1) / tile; }

// log: the changed-root log the tiles append to (the graph's current one when null).
void write_tiles(cc_server *s, const Req &r, uint32_t kind, uint64_t count, const uint32_t *src,
                 const GraphState &g, uint64_t tile, uint32_t n_count, uint32_t n_gate,
                 unsigned long long &pub, const uint32_t *log = nullptr) {
  if (!log) log = g.logs[g.cur_log];
  const uint64_t nt = n_tiles_of(count, tile);
  for (uint64_t i = 0; i < nt; ++i) {
    WorkItem &w = s->hs->ring[(pub + i) % cc::srv::kRingCap];
    w.kind = kind;
    w.slot = r.slot;
    w.seq = r.seq;
    w.n_tiles = n_count;
    w.rf = g.rf ? 1u : 0u;
    w.m = g.m;
    w.n = (uint32_t)g.n;
    w.n_gate = n_gate;
    w.P = (uint64_t)(uintptr_t)g.P;
    w.src = (uint64_t)(uintptr_t)src;
    w.begin = i * tile;
    w.end = w.begin + tile < count ? w.begin + tile : count;
    w.out = (uint64_t)(uintptr_t)r.r.out_dev;
    w.log = (uint64_t)(uintptr_t)log;
    w.Z = (uint64_t)(uintptr_t)g.Z;
    w.pad = 0;
  }
  pub += nt;
}

// Starts an insert or query on the executor; false when it must wait (no
// slot, no ring room, or the executor is being stopped). An insert of one
// tile validates and applies itself; a longer one publishes validate tiles
// and then apply tiles that wait on the device until the validation has
// finished (and apply nothing if it failed). The apply tiles are written at
// the end of the scheduler pass, after the validate tiles of every insert
// started in it: a burst of inserts is validated first, so that apply tiles
// rarely find their gate closed (inserts started together commute).
bool start_exec(cc_server *s, Req *r, GraphState &g) {
  const bool insert = r->r.kind == CC_REQ_INSERT;
  const uint64_t count = insert ? r->r.n_edges : r->r.n_pairs;
  if (count == 0) {
    complete(s, r, CC_OK);
    return true;
  }
  if (s->exec_stopping || s->held) return false;
  const uint64_t tile = tile_for(s, count, 256);
  const uint64_t n_work = n_tiles_of(count, tile);
  const uint64_t vtile = insert && n_work > 1 ? tile_for(s, count, 16384) : 0;
  const uint64_t n_val = vtile ? n_tiles_of(count, vtile) : 0;
  const uint64_t need = n_work + n_val;
  if (s->free_slots.empty() || s->in_flight_items + need > cc::srv::kRingCap / 2) return false;
  r->slot = s->free_slots.back();
  s->free_slots.pop_back();
  s->slot_req[r->slot] = r;
  r->state.store(kRunning);
  // a fresh sequence number for this slot, never equal to one a previous
  // user of the slot left in done_seq
  r->seq = ++s->slot_gen[r->slot];
  if (r->seq == 0u) r->seq = ++s->slot_gen[r->slot];
  s->hs->err[r->slot] = 0u;
  r->n_tiles = (uint32_t)need;
  unsigned long long pub = s->hs->published;
  if (!insert) {
    write_tiles(s, *r, cc::srv::kItemQuery, count, r->r.pairs_dev, g, tile, (uint32_t)n_work, 0, pub);
  } else if (n_work == 1) {
    write_tiles(s, *r, cc::srv::kItemEdges, count, r->r.edges_dev, g, tile, 1, 0, pub);
  } else {
    write_tiles(s, *r, cc::srv::kItemValidate, count, r->r.edges_dev, g, vtile, (uint32_t)n_work, 0, pub);
    if (s->hold_left)  // the fault injection holds the whole request back
      write_tiles(s, *r, cc::srv::kItemApply, count, r->r.edges_dev, g, tile, (uint32_t)n_work, (uint32_t)n_val,
                  pub);
    else
      s->pending_apply.push_back({r, r->graph, (uint32_t)n_work, (uint32_t)n_val, count, tile,
                                  g.logs[g.cur_log]});
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (s->hold_left) {
    // fault injection: a stuck producer, whose tiles are in the ring but not
    // published until held_until (manage_executor publishes or drops them)
    s->hold_left--;
    s->held = r;
    s->held_pub = pub;
    s->held_until = host_ns() + (uint64_t)s->cfg.fault_hold_publish_us * 1000ULL;
  } else {
    *(volatile unsigned long long *)&s->hs->published = pub;
  }
  s->in_flight_items += need;
  s->tiles_run += need;
  return true;
}

// Writes and publishes the apply tiles that start_exec deferred in this pass.
// While the fault injection holds a request's tiles unpublished in the ring,
// nothing may be published past them: the deferred tiles wait for a later pass.
void flush_pending_apply(cc_server *s) {
  if (s->pending_apply.empty() || s->held) return;
  unsigned long long pub = s->hs->published;
  for (const cc_server::PendingApply &a : s->pending_apply)
    write_tiles(s, *a.r, cc::srv::kItemApply, a.count, a.r->r.edges_dev, s->graphs[a.graph], a.tile, a.n_work,
                a.n_val, pub, a.log);
  s->pending_apply.clear();
  std::atomic_thread_fence(std::memory_order_seq_cst);
  *(volatile unsigned long long *)&s->hs->published = pub;
}

// Root selection (f = R), init, hooking pass and flatten of a new graph on
// the side stream; m and the error word are copied back to pinned memory.
bool start_new_graph(cc_server *s, Req *r, GraphState &g) {
  if (s->side_running.size() >= cc::srv::kMaxSideRunning) return false;
  const bool rf = s->cfg.mode == CC_ROOT_MAXDEG;
  const uint64_t bytes = graph_bytes(r->r.n_vertices, r->r.n_edges, rf);
  uint64_t off = 0;
  if (!s->arena.alloc(bytes, &off)) return false;  // wait for memory
  s->arena_used = s->arena.used();
  g.live = true;
  s->resident++;
  g.rf = rf;
  g.n = r->r.n_vertices;
  g.off = off;
  g.bytes = bytes;
  char *p = s->arena_base + off;
  g.P = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)((g.n + 3) / 4 * 4) * 4);
  g.ctrl = reinterpret_cast<cc::Ctrl *>(p);
  p += align256(sizeof(cc::Ctrl));
  const bool wide = r->r.n_edges >= (1ULL << 31);
  if (rf) {
    g.cnt = p;
    p += align256((size_t)g.n * (wide ? 8 : 4));
    g.cert = reinterpret_cast<cc::CertScratch *>(p);
    p += align256(sizeof(cc::CertScratch));
  }
  g.Z = nullptr;
  g.z_bytes = 0;
  if (wants_z(g.n, rf)) {
    g.Z = reinterpret_cast<uint32_t *>(p);
    g.z_bytes = z_bytes_for(g.n);
    p += align256(g.z_bytes);
  }
  g.Llast = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)((g.n + 3) / 4 * 4) * 4);
  g.logs[0] = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)(g.n + 1) * 4);
  g.logs[1] = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)(g.n + 1) * 4);
  g.cur_log = 0;
  g.snap_busy = false;
  g.Psnap = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)((g.n + 3) / 4 * 4) * 4);
  g.rem = reinterpret_cast<uint32_t *>(p);
  p += align256((size_t)(g.n + 1) * 4);
  g.chg = reinterpret_cast<uint32_t *>(p);
  g.chg_bytes = (size_t)((g.n + 1 + 31) / 32) * 4;
  p += align256(g.chg_bytes);
  g.words = reinterpret_cast<uint32_t *>(p);
  r->state.store(kRunning);
  cudaStream_t ss = side_stream_of(s, r->graph);
  cudaError_t e = cudaMemsetAsync(g.ctrl, 0, sizeof(cc::Ctrl), ss);
  if (e == cudaSuccess && g.Z) e = cudaMemsetAsync(g.Z, 0, g.z_bytes, ss);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.chg, 0, g.chg_bytes, ss);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.logs[1], 0, sizeof(uint32_t), ss);  // logs[0] is emptied below
  const uint32_t n = (uint32_t)g.n;
  const cc::EdgeSpan span = cc::split_edges(r->r.edges_dev, r->r.n_edges);
  int m_src = cc::kMFromHint;
  if (e == cudaSuccess && rf && n) {
    e = cc::launch_root_select_certified(r->r.edges_dev, r->r.n_edges, span, g.cnt, wide, n, g.cert, g.ctrl, ss);
    m_src = cc::kMFromPackedMax;
  }
  if (e == cudaSuccess && n) e = cc::launch_init(rf, g.P, n, g.ctrl, m_src, 0u, ss);
  if (e == cudaSuccess && n)
    e = cc::launch_edge_pass(rf, 1, 4, 256, span, g.P, n, g.ctrl, nullptr, ss, g.Z, g.Z ? &g.ctrl->cert : nullptr,
                             true, nullptr, nullptr, false, rf ? g.cert->hot : nullptr);
  // with labels requested they also go to the graph's own copy (the base of
  // incremental snapshots); otherwise the first snapshot makes that copy
  g.has_last = r->r.labels_dev != nullptr && n;
  if (e == cudaSuccess && n)
    e = cc::launch_flatten(rf, s->cfg.label_space, g.P, n, g.has_last ? g.Llast : nullptr, g.ctrl, ss);
  if (e == cudaSuccess && g.has_last)
    e = cudaMemcpyAsync(r->r.labels_dev, g.Llast, (size_t)n * 4, cudaMemcpyDeviceToDevice, ss);
  if (e == cudaSuccess) {
    cc::srv::k_srv_inc_finish<<<1, 1, 0, ss>>>(g.logs[0], g.words, g.ctrl);  // empty log, gmin of these labels
    cc::note_launch();
    e = cudaGetLastError();
  }
  const uint32_t gid = r->graph;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->side_words[2 * gid], &g.ctrl->m, sizeof(uint32_t), cudaMemcpyDeviceToHost, ss);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->side_words[2 * gid + 1], &g.ctrl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ss);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, ss);
  if (e != cudaSuccess) {
    complete(s, r, CC_ERR_CUDA);
    return true;
  }
  r->t_side = host_ns();
  s->side_running.push_back(r);
  return true;
}

// A snapshot reads a copy of P taken on the graph's side stream (its read
// point, an event) and takes over the changed-root log of the inserts before
// it; inserts submitted after it append to the other log and may start as
// soon as the copy has run, while the relabelling still works on the copy.
// One snapshot per graph computes at a time.
bool start_snapshot(cc_server *s, Req *r, GraphState &g) {
  if (s->side_running.size() >= cc::srv::kMaxSideRunning) return false;
  if (g.snap_busy) return false;
  r->state.store(kRunning);
  cudaStream_t ss = side_stream_of(s, r->graph);
  cudaError_t e = cudaSuccess;
  uint32_t *const log = g.logs[g.cur_log];
  if (g.n) {
    e = cudaMemcpyAsync(g.Psnap, g.P, (size_t)((g.n + 3) / 4 * 4) * 4, cudaMemcpyDeviceToDevice, ss);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_point, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev_point, ss);
    if (e == cudaSuccess) {
      g.cur_log ^= 1;  // later inserts log into the other (empty) log
      g.snap_busy = true;
    }
  }
  if (e == cudaSuccess && g.n && !g.has_last) {
    // the first snapshot: a full flatten into the graph's copy, then the
    // caller's buffer; the log starts over
    const uint32_t n = (uint32_t)g.n;
    cc::srv::k_srv_prep_flatten<<<1, 1, 0, ss>>>(g.ctrl);
    cc::note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cc::launch_flatten(g.rf, s->cfg.label_space, g.Psnap, n, g.Llast, g.ctrl, ss);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->r.labels_dev, g.Llast, (size_t)n * 4, cudaMemcpyDeviceToDevice, ss);
    if (e == cudaSuccess) {
      cc::srv::k_srv_inc_finish<<<1, 1, 0, ss>>>(log, g.words, g.ctrl);
      cc::note_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) g.has_last = true;
  } else if (e == cudaSuccess && g.n) {
    // incremental: remap the labels the logged roots led, rewrite Llast
    const uint32_t n = (uint32_t)g.n;
    const uint32_t min_id = s->cfg.label_space == cc::kLabelMinId ? 1u : 0u;
    cc::srv::k_srv_prep_flatten<<<1, 1, 0, ss>>>(g.ctrl);
    cc::note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess && g.rf && min_id) e = cc::launch_gmin_probe(g.Psnap, n, g.ctrl, ss);
    if (e == cudaSuccess) {
      const unsigned gr = cc::clamp_grid(((uint64_t)n + 255) / 256,
                                         cc::persistent_cap((const void *)cc::srv::k_srv_inc_remap, 256, 0));
      cc::srv::k_srv_inc_remap<<<gr, 256, 0, ss>>>(g.Psnap, g.rf ? 1u : 0u, min_id, log, g.rem, g.chg, g.words,
                                                   g.ctrl);
      cc::note_launch();
      const unsigned gl = cc::clamp_grid(((uint64_t)n + 255) / 256,
                                         cc::persistent_cap((const void *)cc::srv::k_srv_inc_relabel, 256, 0));
      cc::srv::k_srv_inc_relabel<<<gl, 256, 0, ss>>>(g.Llast, n, g.rem, g.chg, r->r.labels_dev);
      cc::note_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g.chg, 0, g.chg_bytes, ss);
    if (e == cudaSuccess) {
      cc::srv::k_srv_inc_finish<<<1, 1, 0, ss>>>(log, g.words, g.ctrl);
      cc::note_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, ss);
  if (e != cudaSuccess) {
    // the stream's work is unknown: wait for it before the graph moves on
    cudaStreamSynchronize(ss);
    g.snap_busy = false;
    complete(s, r, CC_ERR_CUDA);
    return true;
  }
  r->t_side = host_ns();
  s->side_running.push_back(r);
  return true;
}

// A large insert as one validated, full-occupancy edge pass on a side
// stream: validation sets the request's own rejection word, the edge pass
// skips itself when it is set, and the word is copied to the request's pinned
// flag. Inserts commute, so large inserts of one graph may run on different
// streams at once, and executor tiles of the same graph meanwhile.
bool start_side_insert(cc_server *s, Req *r, GraphState &g) {
  if (s->side_running.size() >= cc::srv::kMaxSideRunning || s->free_flags.empty()) return false;
  r->flag = s->free_flags.back();
  s->free_flags.pop_back();
  s->side_flags[r->flag] = 0u;
  r->state.store(kRunning);
  // not the graph's own side stream, where a snapshot of it may still compute
  cudaStream_t ss = s->side_streams[s->next_side++ % cc::srv::kSideStreams];
  if (ss == side_stream_of(s, r->graph)) ss = s->side_streams[s->next_side++ % cc::srv::kSideStreams];
  const uint32_t n = (uint32_t)g.n;
  const cc::EdgeSpan span = cc::split_edges(r->r.edges_dev, r->r.n_edges);
  uint32_t *rej = s->side_reject + r->flag;
  cudaError_t e = cudaMemsetAsync(rej, 0, sizeof(uint32_t), ss);
  if (e == cudaSuccess) e = cc::launch_validate(span, n, g.ctrl, ss, rej);
  if (e == cudaSuccess)
    e = cc::launch_edge_pass(g.rf, 1, 4, 256, span, g.P, n, g.ctrl, rej, ss, g.Z, g.Z ? &g.ctrl->cert : nullptr,
                             true, g.logs[g.cur_log]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->side_flags[r->flag], rej, sizeof(uint32_t), cudaMemcpyDeviceToHost, ss);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, ss);
  if (e != cudaSuccess) {
    s->free_flags.push_back(r->flag);
    r->flag = -1;
    complete(s, r, CC_ERR_CUDA);
    return true;
  }
  r->t_side = host_ns();
  s->side_running.push_back(r);
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

void finish_graph_request(GraphState &g) {
  if (--g.active == 0) g.group = kIdle;
}

// Starts what may start at the head of a graph's queue.
void try_start(cc_server *s, uint32_t gid) {
  GraphState &g = s->graphs[gid];
  while (!g.fifo.empty()) {
    Req *r = g.fifo.front();
    const int cls = class_of(r->r.kind);
    if (g.group == kExclusive) return;
    if (cls == kExclusive) {
      if (g.active || g.snap_busy) return;  // a detached snapshot still reads the graph's memory
      if (r->r.kind == CC_REQ_NEW_GRAPH) {
        if (!start_new_graph(s, r, g)) return;  // no memory yet
        g.fifo.pop_front();
        if (r->state.load() == kRunning) {
          g.group = kExclusive;
          g.active = 1;
        }
        return;
      }
      // drop: every earlier request of the graph has completed
      if (g.live) {
        s->arena.release(g.off, g.bytes);
        s->arena_used = s->arena.used();
        s->resident--;
      }
      g.live = false;
      g.fifo.pop_front();
      {
        std::lock_guard<std::mutex> lk(s->sub_mu);
        s->id_state[gid] = 0;
        s->free_ids.push_back(gid);
      }
      complete(s, r, CC_OK);
      continue;
    }
    if (g.active && g.group != cls) return;
    bool started;
    if (r->r.kind == CC_REQ_INSERT && g.snap_busy) s->snapshot_overlaps++;
    if (r->r.kind == CC_REQ_SNAPSHOT)
      started = start_snapshot(s, r, g);
    else if (r->r.kind == CC_REQ_INSERT && r->r.n_edges >= cc::srv::kSideInsertMin && g.n)
      started = start_side_insert(s, r, g);
    else
      started = start_exec(s, r, g);
    if (!started) return;
    g.fifo.pop_front();
    if (r->state.load() == kRunning) {
      g.group = cls;
      g.active++;
    }
  }
}

// Completes the requests whose executor tiles have all finished (their
// done_seq word carries the request's sequence number).
bool reap_executor(cc_server *s, std::vector<uint32_t> *touched) {
  bool any = false;
  for (uint32_t slot = 0; slot < cc::srv::kSlots; ++slot) {
    Req *r = s->slot_req[slot];
    if (!r) continue;
    if (*(volatile unsigned int *)&s->hs->done_seq[slot] != r->seq) continue;
    s->in_flight_items -= r->n_tiles;
    const unsigned int err = *(volatile unsigned int *)&s->hs->err[slot];
    s->slot_req[slot] = nullptr;
    // after a gate timeout a late validate tile may still count into this
    // slot: retire it instead of reusing it
    if (err != 2u) s->free_slots.push_back(slot);
    complete(s, r, err == 2u ? CC_ERR_TIMEOUT : (err ? CC_ERR_OUT_OF_RANGE : CC_OK));
    finish_graph_request(s->graphs[r->graph]);
    if (touched) touched->push_back(r->graph);
    any = true;
  }
  return any;
}

// Handles an executor that has left (asked to, or after its own bounded
// wait): completes what it finished, fails what it left in flight, and
// rewinds `taken` to `published` (all published items were processed or
// failed) so that claims made while waiting are forgotten. Runs before new
// requests are started in a scheduler pass, so that tiles published after the
// executor left wait for the next launch instead of being failed with it.
void executor_departed(cc_server *s) {
  if (s->exec_running && cudaEventQuery(s->exec_ev) == cudaSuccess) {
    // the executor has left (asked to, or after its own bounded wait); its
    // last completions may have become visible only now
    reap_executor(s, nullptr);
    if (*(volatile unsigned int *)&s->hs->exec_err) {  // a publish wait expired
      *(volatile unsigned int *)&s->hs->exec_err = 0u;
      s->executor_timeouts++;
    }
    if (s->in_flight_items > 0) {
      // it left without finishing: fail what was in flight (not expected
      // unless the host stalled for longer than the executor's wait limit)
      for (uint32_t slot = 0; slot < cc::srv::kSlots; ++slot) {
        Req *r = s->slot_req[slot];
        if (!r) continue;
        s->slot_req[slot] = nullptr;  // retired, not reused
        s->in_flight_items -= r->n_tiles;
        complete(s, r, CC_ERR_TIMEOUT);
        finish_graph_request(s->graphs[r->graph]);
      }
      // tiles held back by the fault injection are never published: the
      // ring positions after `published` are written again by later requests;
      // apply tiles still deferred belong to requests just failed
      s->held = nullptr;
      s->pending_apply.clear();
    }
    unsigned long long pub = s->hs->published;
    cudaMemcpyAsync(&s->ds->taken, &pub, sizeof(pub), cudaMemcpyHostToDevice, s->exec_stream);
    cudaStreamSynchronize(s->exec_stream);
    *(volatile unsigned int *)&s->hs->stop = 0u;
    s->exec_running = false;
    s->exec_stopping = false;
  }
}

// Launches the executor when work is in flight and stops it after an idle
// period.
void manage_executor(cc_server *s) {
  const uint64_t now = host_ns();
  executor_departed(s);
  if (s->held && now >= s->held_until) {  // the stuck producer publishes at last
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile unsigned long long *)&s->hs->published = s->held_pub;
    s->held = nullptr;
  }
  if (s->in_flight_items > 0) {
    s->idle_since = 0;
    if (!s->exec_running) {
      const unsigned grid = (unsigned)(cc::num_sms() * s->cfg.executor_blocks_per_sm);
      cc::srv::k_executor<<<grid, 256, 0, s->exec_stream>>>(s->hs_dev, s->ds, s->wait_ns, s->gate_ns);
      cc::note_launch();
      cudaEventRecord(s->exec_ev, s->exec_stream);
      s->exec_running = true;
      s->executor_launches++;
    }
  } else if (s->exec_running && !s->exec_stopping) {
    if (!s->idle_since) s->idle_since = now;
    // idle: leave after the idle timeout, or at once while side-stream work
    // runs, so that it gets every SM (the executor is relaunched on demand)
    if (!s->side_running.empty() || now - s->idle_since > (uint64_t)s->cfg.idle_timeout_us * 1000ULL) {
      *(volatile unsigned int *)&s->hs->stop = 1u;
      s->exec_stopping = true;
      s->idle_since = 0;
    }
  }
  // Side-stream work starved by the resident executor (a kernel that does
  // not fit beside it waits for it to leave): drain the executor, which
  // finishes every published tile first; a later pass relaunches it.
  if (s->exec_running && !s->exec_stopping) {
    for (Req *r : s->side_running) {
      if (now - r->t_side < cc::srv::kSideStarveNs) continue;
      r->t_side = now;
      *(volatile unsigned int *)&s->hs->stop = 1u;
      s->exec_stopping = true;
      s->idle_since = 0;
      s->side_drains++;
      break;
    }
  }
}

// One scheduler pass; returns true when a request completed or started.
bool scheduler_step(cc_server *s, std::vector<Req *> &incoming) {
  bool progress = false;
  std::vector<uint32_t> touched;
  for (Req *r : incoming) {
    s->graphs[r->graph].fifo.push_back(r);
    touched.push_back(r->graph);
    progress = true;
  }
  incoming.clear();
  if (reap_executor(s, &touched)) progress = true;
  executor_departed(s);
  // side-stream completions
  for (size_t i = 0; i < s->side_running.size();) {
    Req *r = s->side_running[i];
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) {
      // a snapshot whose copy of P has been taken releases the graph's later
      // requests (it no longer reads the live P)
      if (r->ev_point && !r->detached && cudaEventQuery(r->ev_point) == cudaSuccess) {
        r->detached = true;
        finish_graph_request(s->graphs[r->graph]);
        touched.push_back(r->graph);
        progress = true;
      }
      ++i;
      continue;
    }
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
    GraphState &g = s->graphs[r->graph];
    const bool was_detached = r->detached;
    if (r->ev_point) {
      cudaEventDestroy(r->ev_point);
      r->ev_point = nullptr;
      g.snap_busy = false;
    }
    cc_status st = q == cudaSuccess ? CC_OK : CC_ERR_CUDA;
    if (r->r.kind == CC_REQ_NEW_GRAPH && st == CC_OK) {
      g.m = s->side_words[2 * r->graph];
      if (s->side_words[2 * r->graph + 1]) st = CC_ERR_OUT_OF_RANGE;
    }
    if (r->flag >= 0) {
      if (st == CC_OK && *(volatile uint32_t *)&s->side_flags[r->flag]) st = CC_ERR_OUT_OF_RANGE;
      s->free_flags.push_back(r->flag);
      r->flag = -1;
    }
    complete(s, r, st);
    if (!was_detached) finish_graph_request(g);
    touched.push_back(r->graph);
    s->side_running[i] = s->side_running.back();
    s->side_running.pop_back();
    progress = true;
  }
  for (uint32_t gid : touched) try_start(s, gid);
  for (uint32_t gid = 0; gid < s->graphs.size(); ++gid)
    if (!s->graphs[gid].fifo.empty() && s->graphs[gid].group == kIdle) try_start(s, gid);
  flush_pending_apply(s);
  manage_executor(s);
  return progress;
}

constexpr uint64_t kShutdownGraceNs = 10ULL * 1000 * 1000 * 1000;  // 10 s

void scheduler_main(cc_server *s) {
  cudaSetDevice(s->device);
  std::vector<Req *> incoming;
  uint64_t quit_at = 0;
  while (true) {
    bool quit;
    {
      std::lock_guard<std::mutex> lk(s->sub_mu);
      incoming.swap(s->inbox);
      quit = s->quit;
    }
    if (scheduler_step(s, incoming)) {
      std::lock_guard<std::mutex> lk(s->done_mu);
      s->done_cv.notify_all();
    }
    const bool busy = s->in_flight_items > 0 || !s->side_running.empty() || s->exec_running;
    bool queued = false;
    for (auto &g : s->graphs)
      if (!g.fifo.empty()) {
        queued = true;
        break;
      }
    if (quit) {
      // shutting down: requests still running get a bounded grace period
      if (!quit_at) quit_at = host_ns();
      const bool work = s->in_flight_items > 0 || !s->side_running.empty() || queued;
      if (!work || host_ns() - quit_at > kShutdownGraceNs) break;
    }
    if (busy) {
      std::this_thread::yield();  // poll completions without a timer sleep
    } else {
      std::unique_lock<std::mutex> lk(s->sub_mu);
      if (s->inbox.empty() && !s->quit)
        s->sub_cv.wait_for(lk, queued ? std::chrono::microseconds(100) : std::chrono::milliseconds(2));
    }
  }
  // stop the executor (bounded: its blocks leave at the next look at `stop`)
  *(volatile unsigned int *)&s->hs->stop = 1u;
  cudaStreamSynchronize(s->exec_stream);
  for (cudaStream_t st : s->side_streams) cudaStreamSynchronize(st);
}

// Frees what cc_server_create allocated (any subset of it).
void release_resources(cc_server *s) {
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->hs) cudaFreeHost(s->hs);
  if (s->ds) cudaFree(s->ds);
  if (s->side_words) cudaFreeHost(s->side_words);
  if (s->side_flags) cudaFreeHost(s->side_flags);
  if (s->side_reject) cudaFree(s->side_reject);
  if (s->exec_stream) cudaStreamDestroy(s->exec_stream);
  for (cudaStream_t st : s->side_streams)
    if (st) cudaStreamDestroy(st);
  if (s->exec_ev) cudaEventDestroy(s->exec_ev);
}

// Runs every kernel the server can launch once, on a tiny graph, before the
// executor exists. With lazy module loading, the first launch of a kernel
// can wait until the device is idle; the resident executor never is while it
// works, so a first launch from the scheduler thread would stall both.
cudaError_t warm_up(cc_server *s) {
  const bool rf = s->cfg.mode == CC_ROOT_MAXDEG;
  const uint32_t n = 16;
  const uint32_t edges_h[8] = {0, 1, 2, 3, 3, 1, 5, 5};
  uint32_t *P = nullptr, *edges = nullptr, *labels = nullptr, *Z = nullptr, *inc = nullptr;
  void *cnt = nullptr;
  cc::CertScratch *cert = nullptr;
  cc::Ctrl *ctrl = nullptr;
  cudaStream_t ss = s->side_stream;
  cudaError_t e = cudaMalloc((void **)&P, 64 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void **)&Z, 64 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void **)&inc, 256 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void **)&edges, sizeof(edges_h));
  if (e == cudaSuccess) e = cudaMalloc((void **)&labels, 64 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, 64 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void **)&cert, sizeof(cc::CertScratch));
  if (e == cudaSuccess) e = cudaMalloc((void **)&ctrl, sizeof(cc::Ctrl));
  if (e == cudaSuccess) e = cudaMemcpy(edges, edges_h, sizeof(edges_h), cudaMemcpyHostToDevice);
  const cc::EdgeSpan span = cc::split_edges(edges, 4);
  for (int wide = 0; wide < 2 && e == cudaSuccess; ++wide) {
    e = cudaMemsetAsync(ctrl, 0, sizeof(cc::Ctrl), ss);
    int m_src = cc::kMFromHint;
    if (e == cudaSuccess && rf) {
      e = cc::launch_root_select_certified(edges, 4, span, cnt, wide != 0, n, cert, ctrl, ss);
      m_src = cc::kMFromPackedMax;
    }
    if (e == cudaSuccess) e = cc::launch_init(rf, P, n, ctrl, m_src, 0u, ss);
    if (e == cudaSuccess) e = cc::launch_edge_pass(rf, 1, 4, 256, span, P, n, ctrl, nullptr, ss);
    // a side insert: validation, then both edge-pass instances (plain and
    // zero-tree, one chosen on the device)
    if (e == cudaSuccess) e = cudaMemsetAsync(Z, 0, 64 * sizeof(uint32_t), ss);
    if (e == cudaSuccess) e = cc::launch_validate(span, n, ctrl, ss);
    if (e == cudaSuccess) e = cc::launch_edge_pass(rf, 1, 4, 256, span, P, n, ctrl, &ctrl->reject, ss, Z, &ctrl->cert);
    if (e == cudaSuccess) e = cc::launch_flatten(rf, s->cfg.label_space, P, n, labels, ctrl, ss);
    if (e == cudaSuccess) e = cc::launch_flatten(rf, s->cfg.label_space, P, n, nullptr, ctrl, ss);
    // an incremental snapshot over an empty log (log, remap, bitmap, words
    // in one zeroed scratch)
    if (e == cudaSuccess) e = cudaMemsetAsync(inc, 0, 256 * sizeof(uint32_t), ss);
    if (e == cudaSuccess) e = cc::launch_gmin_probe(P, n, ctrl, ss);
    if (e == cudaSuccess) {
      cc::srv::k_srv_inc_remap<<<1, 256, 0, ss>>>(P, rf ? 1u : 0u, 1u, inc, inc + 64, inc + 128, inc + 192, ctrl);
      cc::srv::k_srv_inc_relabel<<<1, 256, 0, ss>>>(labels, n, inc + 64, inc + 128, labels + 32);
      cc::srv::k_srv_inc_finish<<<1, 1, 0, ss>>>(inc, inc + 192, ctrl);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      cc::srv::k_srv_prep_flatten<<<1, 1, 0, ss>>>(ctrl);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ss);
  // The executor prefers the largest shared memory carveout: with the
  // driver's default choice, the SMs it holds have too little shared memory
  // left for the side-stream kernels that use 64 KB.
  static std::atomic<unsigned long long> carveout_set{0};
  if (e == cudaSuccess)
    e = cc::ensure_func_attr((const void *)cc::srv::k_executor, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared, carveout_set);
  // the executor: told to leave before it starts
  if (e == cudaSuccess) {
    *(volatile unsigned int *)&s->hs->stop = 1u;
    cc::srv::k_executor<<<1, 256, 0, s->exec_stream>>>(s->hs_dev, s->ds, s->wait_ns, s->gate_ns);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->exec_stream);
    *(volatile unsigned int *)&s->hs->stop = 0u;
    if (e == cudaSuccess) e = cudaMemset(&s->ds->taken, 0, sizeof(unsigned long long));
  }
  cudaFree(P);
  cudaFree(Z);
  cudaFree(inc);
  cudaFree(edges);
  cudaFree(labels);
  cudaFree(cnt);
  cudaFree(cert);
  cudaFree(ctrl);
  return e;
}

Req *find(cc_server *s, uint64_t ticket) {
  std::lock_guard<std::mutex> lk(s->sub_mu);
  if (ticket == 0 || ticket > s->reqs.size()) return nullptr;
  return s->reqs[ticket - 1].get();
}

}  // namespace

extern "C" {

void cc_server_config_init(cc_server_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->max_graphs = 1024;
  cfg->executor_blocks_per_sm = 3;
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
  if (!cfg.executor_blocks_per_sm) cfg.executor_blocks_per_sm = 3;
  if (!cfg.tile_edges) cfg.tile_edges = 16384;
  if (!cfg.idle_timeout_us) cfg.idle_timeout_us = 20000;
  if (cfg.hbm_budget_bytes == 0 || cfg.executor_blocks_per_sm > 8 || cfg.tile_edges < 256 ||
      (cfg.mode != CC_ROOT_IDENTITY && cfg.mode != CC_ROOT_MAXDEG) ||
      (cfg.label_space != CC_LABEL_MIN_ID && cfg.label_space != CC_LABEL_ROOT_VALUE) || cfg.max_graphs > (1u << 20))
    return CC_ERR_INVALID_ARGUMENT;
  for (int r : cfg.reserved)
    if (r) return CC_ERR_INVALID_ARGUMENT;
  constexpr uint32_t kMaxWaitUs = 600u * 1000u * 1000u;  // 10 minutes
  if (cfg.publish_wait_us > kMaxWaitUs || cfg.gate_wait_us > kMaxWaitUs || cfg.fault_hold_publish_us > kMaxWaitUs)
    return CC_ERR_INVALID_ARGUMENT;
  cc_server *s = new (std::nothrow) cc_server();
  if (!s) return CC_ERR_OOM;
  s->cfg = cfg;
  s->wait_ns = cfg.publish_wait_us ? (unsigned long long)cfg.publish_wait_us * 1000ULL : cc::srv::kWaitLimitNs;
  s->gate_ns = cfg.gate_wait_us ? (unsigned long long)cfg.gate_wait_us * 1000ULL : cc::srv::kGateTimeoutNs;
  s->hold_left = cfg.fault_hold_publish_us ? 1u : 0u;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->arena_base, cfg.hbm_budget_bytes);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->hs, sizeof(HostShared), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s->hs_dev, s->hs, 0);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->ds, sizeof(DevShared));
  if (e == cudaSuccess) e = cudaMemset(s->ds, 0, sizeof(DevShared));
  if (e == cudaSuccess)
    e = cudaHostAlloc((void **)&s->side_words, 2 * (size_t)cfg.max_graphs * sizeof(uint32_t), cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void **)&s->side_flags, cc::srv::kMaxSideRunning * sizeof(uint32_t), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->side_reject, cc::srv::kMaxSideRunning * sizeof(uint32_t));
  // the executor's stream has the highest priority, so that its blocks are
  // placed ahead of waiting side-stream blocks whenever SMs free up
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->exec_stream, cudaStreamNonBlocking, prio_high);
  for (cudaStream_t &st : s->side_streams)
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_low);
  s->side_stream = s->side_streams[0];
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->exec_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cc_status st = e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
    release_resources(s);
    delete s;
    return st;
  }
  memset(s->hs, 0, sizeof(HostShared));
  if ((e = warm_up(s)) != cudaSuccess) {
    release_resources(s);
    delete s;
    return CC_ERR_CUDA;
  }
  for (int i = (int)cc::srv::kMaxSideRunning; i-- > 0;) s->free_flags.push_back(i);
  s->arena.reset(cfg.hbm_budget_bytes);
  s->graphs.resize(cfg.max_graphs);
  s->id_state.assign(cfg.max_graphs, 0);
  for (uint32_t i = cfg.max_graphs; i-- > 0;) s->free_ids.push_back(i);
  for (uint32_t i = cc::srv::kSlots; i-- > 0;) s->free_slots.push_back(i);
  s->slot_req.assign(cc::srv::kSlots, nullptr);
  s->slot_gen.assign(cc::srv::kSlots, 0);
  s->thread = std::thread(scheduler_main, s);
  *out = s;
  return CC_OK;
}

namespace {

// Host-side argument checks of one request (no server state).
cc_status check_request(const cc_server *s, const cc_request &r) {
  auto misaligned = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; };
  switch (r.kind) {
    case CC_REQ_NEW_GRAPH:
      if (r.n_vertices > 0x7FFFFFFFULL) return CC_ERR_TOO_LARGE;
      if (r.n_edges && (!r.edges_dev || misaligned(r.edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      if (r.labels_dev && misaligned(r.labels_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
      if (graph_bytes(r.n_vertices, r.n_edges, s->cfg.mode == CC_ROOT_MAXDEG) > s->cfg.hbm_budget_bytes)
        return CC_ERR_TOO_LARGE;
      return CC_OK;
    case CC_REQ_INSERT:
      if (r.n_edges && (!r.edges_dev || misaligned(r.edges_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      return CC_OK;
    case CC_REQ_QUERY:
      if (r.n_pairs && (!r.pairs_dev || !r.out_dev || misaligned(r.pairs_dev, 8))) return CC_ERR_INVALID_ARGUMENT;
      return CC_OK;
    case CC_REQ_SNAPSHOT:
      if (!r.labels_dev || misaligned(r.labels_dev, 4)) return CC_ERR_INVALID_ARGUMENT;
      return CC_OK;
    case CC_REQ_DROP_GRAPH:
      return CC_OK;
    default:
      return CC_ERR_INVALID_ARGUMENT;
  }
}

// Queues requests in order until one is refused. Returns the status of the
// refused request (CC_OK when all were queued); *n_queued tells how many were.
cc_status submit_in_order(cc_server *s, const cc_request *reqs, uint32_t count, uint64_t *tickets,
                          uint32_t *n_queued) {
  *n_queued = 0;
  cc_status st = CC_OK;
  std::vector<std::unique_ptr<Req>> made;
  made.reserve(count);
  uint32_t checked = 0;
  for (; checked < count; ++checked) {
    if ((st = check_request(s, reqs[checked])) != CC_OK) break;
    std::unique_ptr<Req> q(new (std::nothrow) Req());
    if (!q) {
      st = CC_ERR_OOM;
      break;
    }
    q->r = reqs[checked];
    made.push_back(std::move(q));
  }
  const uint64_t t_submit = host_ns();
  uint32_t done = 0;
  {
    std::lock_guard<std::mutex> lk(s->sub_mu);
    if (s->quit) return CC_ERR_INVALID_ARGUMENT;
    for (; done < made.size(); ++done) {
      std::unique_ptr<Req> &q = made[done];
      const cc_request &r = q->r;
      uint32_t gid = r.graph;
      if (r.kind == CC_REQ_NEW_GRAPH) {
        if (s->free_ids.empty()) {
          st = CC_ERR_TOO_LARGE;
          break;
        }
        gid = s->free_ids.back();
        s->free_ids.pop_back();
        s->id_state[gid] = 1;
      } else {
        if (gid >= s->cfg.max_graphs || s->id_state[gid] != 1) {
          st = CC_ERR_INVALID_ARGUMENT;
          break;
        }
        if (r.kind == CC_REQ_DROP_GRAPH) s->id_state[gid] = 2;
      }
      q->graph = gid;
      q->t_submit = t_submit;
      s->reqs.push_back(std::move(q));
      tickets[done] = s->reqs.size();
      s->reqs.back()->ticket = tickets[done];
      s->inbox.push_back(s->reqs.back().get());
    }
  }
  *n_queued = done;
  if (done) {
    s->submitted += done;
    s->sub_cv.notify_one();
  }
  return st;
}

}  // namespace

cc_status cc_server_submit(cc_server *s, const cc_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return CC_ERR_INVALID_ARGUMENT;
  uint32_t n = 0;
  return submit_in_order(s, req, 1, ticket, &n);
}

cc_status cc_server_submit_many(cc_server *s, const cc_request *reqs, uint32_t count, uint64_t *tickets,
                                uint32_t *n_queued) {
  if (!s || !n_queued || (count && (!reqs || !tickets))) return CC_ERR_INVALID_ARGUMENT;
  return submit_in_order(s, reqs, count, tickets, n_queued);
}

cc_status cc_server_poll(cc_server *s, uint64_t ticket, cc_status *result) {
  if (!s || !result) return CC_ERR_INVALID_ARGUMENT;
  Req *r = find(s, ticket);
  if (!r) return CC_ERR_INVALID_ARGUMENT;
  if (r->state.load(std::memory_order_acquire) != kDone) return CC_ERR_NOT_READY;
  *result = (cc_status)r->result.load();
  return CC_OK;
}

cc_status cc_server_wait(cc_server *s, uint64_t ticket, uint64_t timeout_ns, cc_status *result) {
  if (!s || !result) return CC_ERR_INVALID_ARGUMENT;
  Req *r = find(s, ticket);
  if (!r) return CC_ERR_INVALID_ARGUMENT;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
  std::unique_lock<std::mutex> lk(s->done_mu);
  while (r->state.load(std::memory_order_acquire) != kDone) {
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        r->state.load(std::memory_order_acquire) != kDone)
      return CC_ERR_TIMEOUT;
  }
  *result = (cc_status)r->result.load();
  return CC_OK;
}

cc_status cc_server_result_graph(cc_server *s, uint64_t ticket, uint32_t *graph) {
  if (!s || !graph) return CC_ERR_INVALID_ARGUMENT;
  Req *r = find(s, ticket);
  if (!r) return CC_ERR_INVALID_ARGUMENT;
  *graph = r->graph;
  return CC_OK;
}

cc_status cc_server_latency_ns(cc_server *s, uint64_t ticket, uint64_t *ns) {
  if (!s || !ns) return CC_ERR_INVALID_ARGUMENT;
  Req *r = find(s, ticket);
  if (!r) return CC_ERR_INVALID_ARGUMENT;
  if (r->state.load(std::memory_order_acquire) != kDone) return CC_ERR_NOT_READY;
  *ns = r->t_done.load() - r->t_submit;
  return CC_OK;
}

cc_status cc_server_get_stats(cc_server *s, cc_server_stats *st) {
  if (!s || !st) return CC_ERR_INVALID_ARGUMENT;
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->resident_graphs = s->resident;
  st->arena_bytes_used = s->arena_used;
  st->arena_bytes = s->cfg.hbm_budget_bytes;
  st->executor_launches = s->executor_launches;
  st->tiles_run = s->tiles_run;
  st->side_drains = s->side_drains;
  st->executor_timeouts = s->executor_timeouts;
  st->snapshot_overlaps = s->snapshot_overlaps;
  return CC_OK;
}

void cc_server_destroy(cc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->sub_mu);
    s->quit = true;
  }
  s->sub_cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  for (auto &r : s->reqs) {
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->ev_point) cudaEventDestroy(r->ev_point);
  }
  release_resources(s);
  delete s;
}

}  // extern "C"

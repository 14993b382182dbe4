// cc_kernels.cu - CUDA kernels of the connected-components hot path for
// sm_103a and their launchers:
//   root selection  degree histogram + argmax (Algorithm 4, max_degree())
//   init            P_v = f(v)                 (Algorithm 3, initialisation)
//   edge pass       one hooking pass           (Algorithm 3, hooking)
//   min-id probe    smallest vertex of m's component (min-id labels under R)
//   flatten         labels + compression       (Algorithm 3, pointer jumping)
//   count, connected, validate                 (queries and insert checks)
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {

namespace {

int g_num_sms = 0;

// ------------------------------------------------------------------- init

template <class F>
__global__ void __launch_bounds__(256) k_init(uint32_t *__restrict__ P, uint32_t n, Ctrl *ctrl,
                                              int m_src, uint32_t m_hint, const uint32_t *skip) {
  if (skip && ld_volatile_u32(skip)) return;
  uint32_t m = 0;
  if (F::kRF) {
    if (m_src == kMFromHint)
      m = m_hint;
    else
      m = ~(uint32_t)(*(volatile unsigned long long *)&ctrl->maxkey);
    if (m >= n) m = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->m = m;
    ctrl->gmin = m;
    ctrl->ncomp = 0ULL;
  }
  const uint64_t n4 = n / 4u;
  uint4 *P4 = reinterpret_cast<uint4 *>(P);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(4 * i);
    uint4 r;
    if (F::kRF) {
      r = make_uint4(v + 1u, v + 2u, v + 3u, v + 4u);
      if (m - v < 4u) {
        if (m == v) r.x = 0u;
        if (m == v + 1u) r.y = 0u;
        if (m == v + 2u) r.z = 0u;
        if (m == v + 3u) r.w = 0u;
      }
    } else {
      r = make_uint4(v, v + 1u, v + 2u, v + 3u);
    }
    P4[i] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3u)) {
    const uint32_t v = (uint32_t)(4 * n4) + threadIdx.x;
    P[v] = F::kRF ? (v == m ? 0u : v + 1u) : v;
  }
}

// --------------------------------------------------------------- edge pass

// Range check of one edge; an out-of-range id flags the error and turns the
// edge into the no-op self-loop (0, 0).
__device__ __forceinline__ void guard(uint32_t &a, uint32_t &b, uint32_t n, Ctrl *ctrl) {
  if (a >= n || b >= n) {
    set_err(ctrl, kErrRange);
    a = 0u;
    b = 0u;
  }
}

template <class F>
__device__ __forceinline__ void single_edge(uint32_t *P, const F fn, const uint2 *e, uint32_t n,
                                            Ctrl *ctrl, uint32_t *log = nullptr) {
  uint2 x = ld_edge(e);
  guard(x.x, x.y, n, ctrl);
  const UniteResult r = unite(slots<F>(P), fn.f(x.x), ldP(P + x.x), fn.f(x.y), ldP(P + x.y));
  if (log && r.hooked != kNoHook) log_hook(log, r.hooked);
}

// Direct form: each thread takes Q 128-bit loads (2Q edges) per iteration,
// issues all 4Q parent loads together, then resolves its edges one by one.
template <class F, int Q>
__global__ void __launch_bounds__(512) k_edge_pass_direct(const uint4 *__restrict__ e4,
                                                          uint64_t n_quads, const uint2 *head,
                                                          const uint2 *tail, uint32_t *P,
                                                          uint32_t n, Ctrl *ctrl, const uint32_t *skip) {
  if (skip && ld_volatile_u32(skip)) return;
  const F fn = F::load(ctrl);
  uint32_t *const S = slots<F>(P);
  const uint64_t pol = policy_evict_first();
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t == 0 && head) single_edge(P, fn, head, n, ctrl);
  if (t == 1 % T && tail) single_edge(P, fn, tail, n, ctrl);
  for (uint64_t base = t; base < n_quads; base += T * Q) {
    uint4 e[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const uint64_t q = base + (uint64_t)j * T;
      e[j] = q < n_quads ? ld_edges(e4 + q, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
    uint32_t p[4 * Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      guard(e[j].x, e[j].y, n, ctrl);
      guard(e[j].z, e[j].w, n, ctrl);
      p[4 * j + 0] = ldP(P + e[j].x);
      p[4 * j + 1] = ldP(P + e[j].y);
      p[4 * j + 2] = ldP(P + e[j].z);
      p[4 * j + 3] = ldP(P + e[j].w);
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      unite(S, fn.f(e[j].x), p[4 * j + 0], fn.f(e[j].y), p[4 * j + 1]);
      unite(S, fn.f(e[j].z), p[4 * j + 2], fn.f(e[j].w), p[4 * j + 3]);
    }
  }
}

// Filtered form: the parent loads of a warp's edges feed the warp ring
// (cc_device.cuh), which drops edges whose endpoints already share a parent
// and resolves the survivors in dense warps.
//
// kZ: the zero-tree bitmap Z (one bit per name, 1/32 of P) stands in front of
// P. An endpoint whose bit is set belongs to the tree of name 0, so its parent
// value is taken as 0 without loading P; an edge with both bits set costs no
// parent load at all. When P is larger than L2 and the giant component hangs
// under name 0 (R with a dominant hub), this turns most random DRAM reads of
// P into L2 hits on Z. Bits are set when a parent value of 0 is read and when
// an edge ends in the tree of name 0.
//
// Instances, chosen at run time by the word *sel (the certificate flag):
//   kZ (with kDirect): the zero-tree form, for a certified hub when Z exists;
//   !kZ, !kDirect: the plain form that always queues, for a certified hub
//     whose P fits L2 (resolving in place cost a few percent there);
//   !kZ, kDirect: the plain form that resolves nearly full warps in place,
//     for graphs without a certified hub; capped at 32 registers, because
//     that search-bound pass gains more from resident warps than it loses
//     to a few spilled registers.
// The register caps (the launch bounds' minimum blocks) were measured.
// The hub-serving instances run only when *sel is nonzero, the other only
// when it is zero; with sel null the launched instance runs.
//
// work: the dynamic schedule. Warps claim `grab` steps of 32 * Q consecutive
// quads at a time from *work, so warps whose edges need long searches do not
// set the end of the kernel; null: each warp takes a fixed stride of steps.
// The claim size is chosen by the launcher (grab_for).
//
// hot (hub instances only): the hot-vertex table of the root selection
// (CertScratch::hot). Each block copies its vertex ids into shared memory
// after the ring and learns, per entry, whether that vertex is known to be in
// the tree of name 0; an endpoint known so skips its bitmap or parent load.
// The table covers 3-8% of R-MAT endpoint occurrences at 4096 entries
// (measured edge pass, R-MAT 28: 32.50 -> 31.61 ms, R-MAT 24: 1.94 -> 1.79);
// 8192 entries lost occupancy and ran slower.

template <class F, int Q, bool kZ, bool kDirect, bool kL2 = false>
__global__ void __launch_bounds__(512, Q >= 4 ? (kZ ? 1 : 2) : (kZ ? 2 : (kDirect ? 4 : 3)))
    k_edge_pass_filtered(const uint4 *__restrict__ e4, uint64_t n_quads, const uint2 *head, const uint2 *tail,
                         uint32_t *P, uint32_t n, Ctrl *ctrl, const uint32_t *skip, uint32_t *Z,
                         const uint32_t *sel, uint32_t *log, unsigned long long *work, uint32_t grab,
                         const unsigned long long *hot) {
  static_assert(kDirect || !kZ, "the zero-tree form resolves in place");
  // kL2 (the queue form on a parent array of at least kL2MinVertices): P is
  // read through L2 only. Its random parent loads almost never hit L1 then,
  // and skipping L1 allocation measured faster (R-MAT scale 24: 2.02 -> 1.94
  // ms); a small P lives in L1 (R-MAT 16's 256 KB: 0.077 ms with L1, 0.13
  // without), and the grid's searches hit L1 (1.27 ms without it, 0.94 with).
  static_assert(!kL2 || (!kZ && !kDirect), "L2-only loads only in the queue form");
  constexpr bool kCG = kL2;
  extern __shared__ uint32_t ring_smem[];
  if (skip && ld_volatile_u32(skip)) return;
  if (sel && ((ld_volatile_u32(sel) != 0u) != (kZ || !kDirect))) return;
  const F fn = F::load(ctrl);
  uint32_t *const S = slots<F>(P);
  const uint64_t pol = policy_evict_first();
  WarpRing ring;
  ring.init(ring_smem, kZ ? Z : nullptr, log, kDirect ? kDirectMin : kNeverDirect);
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // the table: entry v + 1 of a hot vertex v, top bit once v is known to be
  // in the tree of name 0 (0: an empty slot)
  constexpr bool kHub = F::kRF && (kZ || !kDirect);
  uint32_t *const H = ring_smem + (blockDim.x >> 5) * 4 * kRing;
  const bool use_hot = kHub && hot != nullptr;
  if (use_hot) {
    for (uint32_t i = threadIdx.x; i < kHot; i += blockDim.x) H[i] = (uint32_t)hot[i];
    __syncthreads();
  }
  if (t == 0 && head) single_edge(P, fn, head, n, ctrl, log);
  if (t == 1 % T && tail) single_edge(P, fn, tail, n, ctrl, log);
  // One warp step: lane l takes quads base + j * stride (j < Q), base being
  // the warp's first quad plus l; the trip counts stay warp-uniform.
  auto step = [&](uint64_t base, uint64_t stride) {
    uint4 e[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const uint64_t q = base + (uint64_t)j * stride;
      e[j] = q < n_quads ? ld_edges(e4 + q, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
    uint32_t p[4 * Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      guard(e[j].x, e[j].y, n, ctrl);
      guard(e[j].z, e[j].w, n, ctrl);
    }
    // bit i of hz: endpoint i is known (by the table) to be in the tree of
    // name 0; of hk: endpoint i is its slot's vertex
    uint32_t hz = 0, hk = 0;
    if (use_hot) {
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const uint32_t xs[4] = {e[j].x, e[j].y, e[j].z, e[j].w};
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const uint32_t ent = H[hot_slot(xs[k2])];
          hz |= (uint32_t)(ent == ((xs[k2] + 1u) | 0x80000000u)) << (4 * j + k2);
          hk |= (uint32_t)((ent & 0x7FFFFFFFu) == xs[k2] + 1u) << (4 * j + k2);
        }
      }
    }
    if (kZ) {
      uint32_t z = hz;  // bit i: endpoint i is known to be in the tree of name 0
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (!((hz >> (4 * j + 0)) & 1u)) z |= (uint32_t)zbit(Z, fn.f(e[j].x)) << (4 * j + 0);
        if (!((hz >> (4 * j + 1)) & 1u)) z |= (uint32_t)zbit(Z, fn.f(e[j].y)) << (4 * j + 1);
        if (!((hz >> (4 * j + 2)) & 1u)) z |= (uint32_t)zbit(Z, fn.f(e[j].z)) << (4 * j + 2);
        if (!((hz >> (4 * j + 3)) & 1u)) z |= (uint32_t)zbit(Z, fn.f(e[j].w)) << (4 * j + 3);
      }
      if (use_hot) {  // learn: a hot endpoint whose bitmap bit is set
        const uint32_t learn = z & hk & ~hz;
        if (learn) {
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            const uint32_t xs[4] = {e[j].x, e[j].y, e[j].z, e[j].w};
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2)
              if ((learn >> (4 * j + k2)) & 1u) H[hot_slot(xs[k2])] = (xs[k2] + 1u) | 0x80000000u;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        p[4 * j + 0] = (z >> (4 * j + 0)) & 1u ? 0u : ldP(P + e[j].x);
        p[4 * j + 1] = (z >> (4 * j + 1)) & 1u ? 0u : ldP(P + e[j].y);
        p[4 * j + 2] = (z >> (4 * j + 2)) & 1u ? 0u : ldP(P + e[j].z);
        p[4 * j + 3] = (z >> (4 * j + 3)) & 1u ? 0u : ldP(P + e[j].w);
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (!((z >> (4 * j + 0)) & 1u) && p[4 * j + 0] == 0u) zset(Z, fn.f(e[j].x));
        if (!((z >> (4 * j + 1)) & 1u) && p[4 * j + 1] == 0u) zset(Z, fn.f(e[j].y));
        if (!((z >> (4 * j + 2)) & 1u) && p[4 * j + 2] == 0u) zset(Z, fn.f(e[j].z));
        if (!((z >> (4 * j + 3)) & 1u) && p[4 * j + 3] == 0u) zset(Z, fn.f(e[j].w));
      }
    } else {
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        p[4 * j + 0] = ((hz >> (4 * j + 0)) & 1u) ? 0u : ldP_t<kCG>(P + e[j].x);
        p[4 * j + 1] = ((hz >> (4 * j + 1)) & 1u) ? 0u : ldP_t<kCG>(P + e[j].y);
        p[4 * j + 2] = ((hz >> (4 * j + 2)) & 1u) ? 0u : ldP_t<kCG>(P + e[j].z);
        p[4 * j + 3] = ((hz >> (4 * j + 3)) & 1u) ? 0u : ldP_t<kCG>(P + e[j].w);
      }
      if (use_hot) {  // learn: a hot endpoint whose parent is name 0
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const uint32_t xs[4] = {e[j].x, e[j].y, e[j].z, e[j].w};
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2)
            if (((hk & ~hz) >> (4 * j + k2)) & 1u && p[4 * j + k2] == 0u)
              H[hot_slot(xs[k2])] = (xs[k2] + 1u) | 0x80000000u;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * Q; ++k) {
      const uint32_t a = (k & 1) ? e[k >> 1].z : e[k >> 1].x;
      const uint32_t b = (k & 1) ? e[k >> 1].w : e[k >> 1].y;
      const uint32_t pa = p[2 * k], pb = p[2 * k + 1];
      ring.push<kCG>(S, pa != pb, fn.f(a), pa, fn.f(b), pb);
    }
  };
  if (work) {
    // dynamic: warps claim `grab` steps of 32 * Q consecutive quads at a time,
    // so warps whose edges need longer searches do not set the kernel's end
    const uint64_t steps = (n_quads + 32u * Q - 1) / (32u * Q);
    for (;;) {
      unsigned long long g0 = 0;
      if (ring.lane == 0) g0 = atomicAdd(work, (unsigned long long)grab);
      g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
      if (g0 >= steps) break;
      const uint64_t g1 = g0 + grab < steps ? g0 + grab : steps;
      for (uint64_t g = g0; g < g1; ++g) step(g * 32u * Q + ring.lane, 32u);
    }
  } else {
    const uint64_t warp_t0 = t - (uint64_t)ring.lane;
    for (uint64_t wbase = warp_t0; wbase < n_quads; wbase += T * Q) step(wbase + ring.lane, T);
  }
  ring.drain<kCG>(S);
}

__global__ void __launch_bounds__(256) k_validate(const uint4 *__restrict__ e4, uint64_t n_quads,
                                                  const uint2 *head, const uint2 *tail, uint32_t n,
                                                  Ctrl *ctrl, uint32_t *reject) {
  const uint64_t pol = policy_evict_first();
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  bool bad = false;
  if (t == 0 && head) {
    uint2 e = ld_edge(head);
    bad |= e.x >= n || e.y >= n;
  }
  if (t == 1 % T && tail) {
    uint2 e = ld_edge(tail);
    bad |= e.x >= n || e.y >= n;
  }
  for (uint64_t q = t; q < n_quads; q += T) {
    const uint4 e = ld_edges(e4 + q, pol);
    bad |= (e.x >= n) | (e.y >= n) | (e.z >= n) | (e.w >= n);
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) {
    atomicOr(reject, 1u);
    set_err(ctrl, kErrRange);
  }
}

// ------------------------------------------------------------------ flatten

// Smallest vertex whose root value is 0 under R. Its answer is at most m, so
// only [0, m) is scanned, in chunks of increasing id; a block stops as soon as
// its next chunk starts above the best candidate found so far.
__global__ void __launch_bounds__(256) k_gmin_probe(uint32_t *P, uint32_t n, Ctrl *ctrl) {
  const RootR fn = RootR::load(ctrl);
  const uint32_t m = fn.m;
  __shared__ uint32_t s_stop;
  const uint64_t chunk = 4ull * blockDim.x;
  for (uint64_t c = blockIdx.x;; c += gridDim.x) {
    const uint64_t start = c * chunk;
    if (threadIdx.x == 0) s_stop = (start >= m) || (start > ld_volatile_u32(&ctrl->gmin));
    __syncthreads();
    const bool stop = s_stop;
    __syncthreads();
    if (stop) return;
    uint32_t best = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t v = start + (uint64_t)k * blockDim.x + threadIdx.x;
      if (v < m && v < best) {
        const uint32_t pv = ldP(P + v);
        if (root_name(slots<RootR>(P), fn.f((uint32_t)v), pv) == 0u) best = (uint32_t)v;
      }
    }
    best = __reduce_min_sync(0xFFFFFFFFu, best);
    if ((threadIdx.x & 31) == 0 && best != 0xFFFFFFFFu) atomicMin(&ctrl->gmin, best);
  }
}

// Pointer jumping (Algorithm 3): every vertex finds its root name c with
// path splitting, stores c into P (compression; roots are never written) and,
// when L is given, writes its label: the root's name (root-value labels, and
// min-id labels under f = id), or under f = R the root's id c - 1 for c != 0
// and the smallest vertex of m's component for c == 0. Roots are counted.
template <class F, int LABEL>
__device__ __forceinline__ uint32_t label_of(uint32_t c, uint32_t gmin) {
  if (LABEL == kLabelRootValue || !F::kRF) return c;
  return c == 0u ? gmin : c - 1u;
}

template <class F>
__device__ __forceinline__ uint32_t flatten_one(uint32_t *S, const F fn, uint32_t v, uint32_t pv,
                                                unsigned long long &roots) {
  const uint32_t cv = fn.f(v);
  if (pv == cv) {
    ++roots;
    return pv;
  }
  return root_name(S, cv, pv);
}

// 16-byte load of four consecutive parent values.
__device__ __forceinline__ uint4 ldP4(const uint32_t *p) {
  uint4 r;
  asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p) : "memory");
  return r;
}

// Root names of W vertices (names c, parent values pc), walked in lock step:
// each round issues the next parent load of every walk still running, so the
// dependent chains overlap instead of following one another. Path splitting
// as in root_name(); r receives the root names.
template <int W>
__device__ __forceinline__ void root_names_lockstep(uint32_t *S, uint32_t (&c)[W], uint32_t (&pc)[W],
                                                    uint32_t (&r)[W], unsigned long long &roots) {
  unsigned running = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    if (pc[k] == c[k]) {
      ++roots;
      r[k] = pc[k];
    } else if (pc[k] == 0u) {
      r[k] = 0u;
    } else {
      running |= 1u << k;
    }
  }
  while (running) {
    uint32_t pw[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (running & (1u << k)) pw[k] = ldP(S + pc[k]);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      if (!(running & (1u << k))) continue;
      if (pw[k] == pc[k]) {  // pc[k] is a root
        r[k] = pc[k];
        running &= ~(1u << k);
        continue;
      }
      stP(S + c[k], pw[k]);  // the parent is not a root: split past it
      c[k] = pc[k];
      pc[k] = pw[k];
      if (pc[k] == 0u) {  // the permanent root
        r[k] = 0u;
        running &= ~(1u << k);
      }
    }
  }
}

// Four consecutive vertices per thread: 16-byte loads of P, 16-byte stores of
// the compressed names (only when one changed; every name written is a valid
// ancestor, and roots are never changed) and of the labels.
template <class F, int LABEL>
__global__ void __launch_bounds__(256) k_flatten4(uint32_t *P, uint32_t n, uint32_t *__restrict__ L,
                                                  Ctrl *ctrl) {
  const F fn = F::load(ctrl);
  uint32_t *const S = slots<F>(P);
  uint32_t gmin = 0;
  if (F::kRF && LABEL == kLabelMinId) gmin = ld_volatile_u32(&ctrl->gmin);
  unsigned long long roots = 0;
  const uint64_t n4 = n / 4u;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(4 * i);
    const uint4 p = ldP4(P + v);
    uint32_t c[4] = {fn.f(v), fn.f(v + 1u), fn.f(v + 2u), fn.f(v + 3u)};
    uint32_t pc[4] = {p.x, p.y, p.z, p.w};
    uint32_t r[4];
    root_names_lockstep<4>(S, c, pc, r, roots);
    const uint4 cq = make_uint4(r[0], r[1], r[2], r[3]);
    if (cq.x != p.x || cq.y != p.y || cq.z != p.z || cq.w != p.w)
      asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(P + v), "r"(cq.x), "r"(cq.y), "r"(cq.z),
                   "r"(cq.w)
                   : "memory");
    if (L)
      __stcs(reinterpret_cast<uint4 *>(L + v),
             make_uint4(label_of<F, LABEL>(cq.x, gmin), label_of<F, LABEL>(cq.y, gmin),
                        label_of<F, LABEL>(cq.z, gmin), label_of<F, LABEL>(cq.w, gmin)));
  }
  // the last n % 4 vertices
  if (blockIdx.x == 0 && threadIdx.x < (n & 3u)) {
    const uint32_t v = (uint32_t)(4 * n4) + threadIdx.x;
    const uint32_t pv = ldP(P + v);
    const uint32_t c = flatten_one(S, fn, v, pv, roots);
    if (c != pv) stP(P + v, c);
    if (L) L[v] = label_of<F, LABEL>(c, gmin);
  }
  roots = warp_sum_u64(roots);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(&ctrl->ncomp, roots);
}

// One vertex per thread, for label buffers that are not 16-byte aligned.
template <class F, int LABEL>
__global__ void __launch_bounds__(256) k_flatten(uint32_t *P, uint32_t n, uint32_t *__restrict__ L,
                                                 Ctrl *ctrl) {
  const F fn = F::load(ctrl);
  uint32_t *const S = slots<F>(P);
  uint32_t gmin = 0;
  if (F::kRF && LABEL == kLabelMinId) gmin = ld_volatile_u32(&ctrl->gmin);
  unsigned long long roots = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)i;
    const uint32_t pv = ldP(P + v);
    const uint32_t c = flatten_one(S, fn, v, pv, roots);
    if (c != pv) stP(P + v, c);
    if (L) __stcs(L + v, label_of<F, LABEL>(c, gmin));
  }
  roots = warp_sum_u64(roots);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(&ctrl->ncomp, roots);
}

template <class F>
__global__ void __launch_bounds__(256) k_count_roots(const uint32_t *__restrict__ P, uint32_t n,
                                                     Ctrl *ctrl) {
  const F fn = F::load(ctrl);
  unsigned long long roots = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    roots += (P[i] == fn.f((uint32_t)i));
  roots = warp_sum_u64(roots);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(&ctrl->ncomp, roots);
}

template <class F>
__global__ void __launch_bounds__(256) k_connected(uint32_t *P, uint32_t n,
                                                   const uint2 *__restrict__ pairs, uint64_t n_pairs,
                                                   uint8_t *__restrict__ out, Ctrl *ctrl) {
  const F fn = F::load(ctrl);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_pairs;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 q = ld_edge(pairs + i);
    uint8_t r = 0;
    if (q.x >= n || q.y >= n) {
      set_err(ctrl, kErrRange);
    } else {
      const uint32_t cu = root_name(slots<F>(P), fn.f(q.x), ldP(P + q.x));
      const uint32_t cv = root_name(slots<F>(P), fn.f(q.y), ldP(P + q.y));
      r = cu == cv;
    }
    out[i] = r;
  }
}

// The forest as edges (the pairs (v, P_v) that each machine sends to the
// Reducer, Section III): a non-root v (P[v] != f(v)) gives (v, f^-1(P[v])),
// the vertex its parent name names. Each thread takes 4 consecutive vertices
// (one 16-byte load); a warp scan and a block prefix place the block's pairs
// behind one atomic per block and round (one per warp serialised on the one
// counter: 5.7 ms for 2^28 vertices).
template <class F>
__global__ void __launch_bounds__(256) k_forest_pairs(const uint32_t *__restrict__ P, uint32_t n, uint2 *out,
                                                      uint64_t cap, Ctrl *ctrl) {
  __shared__ unsigned int s_cnt[8];
  __shared__ unsigned long long s_base[8];
  const F fn = F::load(ctrl);
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, n_w = blockDim.x >> 5;
  const uint64_t per_block = 4ull * blockDim.x;
  for (uint64_t b0 = (uint64_t)blockIdx.x * per_block; b0 < n; b0 += (uint64_t)gridDim.x * per_block) {
    const uint64_t v0 = b0 + 4ull * threadIdx.x;  // block-uniform trip count
    uint32_t pv[4] = {0u, 0u, 0u, 0u};
    if (v0 + 3 < n) {
      const uint4 q = *reinterpret_cast<const uint4 *>(P + v0);  // P is 256-byte aligned
      pv[0] = q.x;
      pv[1] = q.y;
      pv[2] = q.z;
      pv[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (v0 + j < n) pv[j] = P[v0 + j];
    }
    uint32_t mine = 0, k = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool nr = v0 + j < n && pv[j] != fn.f((uint32_t)(v0 + j));
      mine |= (uint32_t)nr << j;
      k += nr ? 1u : 0u;
    }
    uint32_t incl = k;  // inclusive warp scan of the pair counts
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_cnt[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (uint32_t w = 0; w < n_w; ++w) {
        s_base[w] = tot;
        tot += s_cnt[w];
      }
      const unsigned long long g = tot ? atomicAdd(&ctrl->pairs, tot) : 0ULL;
      for (uint32_t w = 0; w < n_w; ++w) s_base[w] += g;
    }
    __syncthreads();
    uint64_t slot = s_base[wid] + (incl - k);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((mine >> j) & 1u) {
        if (slot < cap) out[slot] = make_uint2((uint32_t)(v0 + j), fn.finv(pv[j]));
        ++slot;
      }
    }
    __syncthreads();  // s_cnt and s_base are reused next round
  }
}

}  // namespace

// ======================================================================= host

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

uint64_t persistent_cap(const void *kernel, int block, size_t smem) {
  struct Key {
    const void *k;
    int block, dev;
    size_t smem;
    bool operator<(const Key &o) const {
      if (k != o.k) return k < o.k;
      if (block != o.block) return block < o.block;
      if (dev != o.dev) return dev < o.dev;
      return smem < o.smem;
    }
  };
  static std::mutex mu;
  static std::map<Key, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const Key key{kernel, block, dev, smem};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return (uint64_t)num_sms() * (uint64_t)it->second;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem) != cudaSuccess || occ < 1) occ = 1;
  {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = occ;
  }
  return (uint64_t)num_sms() * (uint64_t)occ;
}

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    g_num_sms = v;
  }
  return g_num_sms;
}

EdgeSpan split_edges(const uint32_t *edges, uint64_t n_edges) {
  EdgeSpan s;
  if (n_edges == 0) return s;
  const uint2 *e2 = reinterpret_cast<const uint2 *>(edges);
  uint64_t h = ((uintptr_t)edges & 15u) ? 1u : 0u;
  if (h) s.head = e2;
  const uint64_t body = n_edges - h;
  s.n_quads = body / 2u;
  s.quads = reinterpret_cast<const uint4 *>(e2 + h);
  if (body & 1u) s.tail = e2 + h + 2u * s.n_quads;
  return s;
}

cudaError_t launch_init(bool rf, uint32_t *P, uint32_t n, Ctrl *ctrl, int m_src, uint32_t m_hint,
                        cudaStream_t s, const uint32_t *skip) {
  const uint64_t work = n / 4u + 1u;
  if (rf) {
    const unsigned g = clamp_grid((work + 255) / 256, persistent_cap((const void *)k_init<RootR>, 256, 0));
    k_init<RootR><<<g, 256, 0, s>>>(P, n, ctrl, m_src, m_hint, skip); note_launch();
  } else {
    const unsigned g = clamp_grid((work + 255) / 256, persistent_cap((const void *)k_init<RootId>, 256, 0));
    k_init<RootId><<<g, 256, 0, s>>>(P, n, ctrl, m_src, m_hint, skip); note_launch();
  }
  return cudaGetLastError();
}

namespace {
constexpr uint64_t kMinWaves = 8;
// The queue form reads P through L2 only from this many vertices up (16 MB).
constexpr uint32_t kL2MinVertices = 1u << 22;

// Claim size of the dynamic schedule, in warp steps. From 2^20 edges up,
// 16 steps at a time (measured best there: fewer warps start on the hub's
// trees at once, so fewer CAS collide). Below that, a smaller graph would
// leave most warps of the grid idle, so the claim shrinks to about half the
// steps per warp (at least one).
uint32_t grab_for(uint64_t n_quads, int Q, unsigned grid, int block) {
  constexpr uint32_t kGrabMax = 16;
  if (n_quads >= (1ULL << 19)) return kGrabMax;
  const uint64_t steps = (n_quads + 32u * Q - 1) / (32u * Q);
  const uint64_t warps = (uint64_t)grid * (uint64_t)(block / 32);
  const uint64_t g = steps / (2 * (warps ? warps : 1));
  return g < 1 ? 1u : (g > kGrabMax ? kGrabMax : (uint32_t)g);
}

template <class F, int Q>
cudaError_t edge_pass_q(int filter, int block, const EdgeSpan &e, uint32_t *P, uint32_t n, Ctrl *ctrl,
                        const uint32_t *skip, uint32_t *Z, const uint32_t *zsel, bool one_shot, uint32_t *log,
                        const uint32_t *hub, bool dyn, cudaStream_t s, const unsigned long long *hot) {
  const uint64_t per_block = (uint64_t)block * Q;
  // At least kMinWaves grid iterations per thread: when a whole graph fits
  // one wave, every edge reads P before any hooking and duplicate hub edges
  // then CAS the same roots at once (R-MAT scale 16: 97% of the CAS failed);
  // later waves find most edges already joined. one_shot: no cap at the
  // resident blocks, so blocks retire after their kMinWaves iterations and
  // kernels of other streams get SMs while this one runs.
  const uint64_t want = (e.n_quads + per_block * kMinWaves - 1) / (per_block * kMinWaves);
  const uint64_t cap_big = 0x7FFFFFFFull;
  if (filter) {
    unsigned long long *work = nullptr;
    if (dyn) {  // one counter serves both instances: only one of them runs
      cudaError_t err = cudaMemsetAsync(&ctrl->work, 0, sizeof(unsigned long long), s);
      if (err != cudaSuccess) return err;
      work = &ctrl->work;
    }
    const size_t smem = (size_t)(block / 32) * 4 * kRing * sizeof(uint32_t);
    static_assert((512 / 32) * 4 * kRing * sizeof(uint32_t) + kHot * sizeof(uint32_t) <= 48 * 1024,
                  "the ring of a 512-thread block and the hot table fit the default dynamic shared memory limit");
    // the hub instances also hold the hot-vertex table
    const size_t smem_hub = smem + (F::kRF && hot ? kHot * sizeof(uint32_t) : 0);
    // the certificate word chooses among the launched instances (see
    // k_edge_pass_filtered); zsel: with Z, hub: without it
    if (Z) {
      const void *k = (const void *)k_edge_pass_filtered<F, Q, true, true>;
      const unsigned g = clamp_grid(want, one_shot ? cap_big : persistent_cap(k, block, smem_hub));
      const uint32_t grab = grab_for(e.n_quads, Q, g, block);
      k_edge_pass_filtered<F, Q, true, true><<<g, block, smem_hub, s>>>(e.quads, e.n_quads, e.head, e.tail, P, n,
                                                                        ctrl, skip, Z, zsel, log, work, grab, hot);
      note_launch();
    }
    if (!Z && hub) {
      const bool l2 = n >= kL2MinVertices;
      const void *k = l2 ? (const void *)k_edge_pass_filtered<F, Q, false, false, true>
                         : (const void *)k_edge_pass_filtered<F, Q, false, false, false>;
      const unsigned g = clamp_grid(want, one_shot ? cap_big : persistent_cap(k, block, smem_hub));
      const uint32_t grab = grab_for(e.n_quads, Q, g, block);
      if (l2)
        k_edge_pass_filtered<F, Q, false, false, true><<<g, block, smem_hub, s>>>(
            e.quads, e.n_quads, e.head, e.tail, P, n, ctrl, skip, nullptr, hub, log, work, grab, hot);
      else
        k_edge_pass_filtered<F, Q, false, false, false><<<g, block, smem_hub, s>>>(
            e.quads, e.n_quads, e.head, e.tail, P, n, ctrl, skip, nullptr, hub, log, work, grab, hot);
      note_launch();
    }
    if (!Z || zsel) {
      const void *k = (const void *)k_edge_pass_filtered<F, Q, false, true>;
      const unsigned g = clamp_grid(want, one_shot ? cap_big : persistent_cap(k, block, smem));
      const uint32_t grab = grab_for(e.n_quads, Q, g, block);
      k_edge_pass_filtered<F, Q, false, true><<<g, block, smem, s>>>(e.quads, e.n_quads, e.head, e.tail, P, n,
                                                                     ctrl, skip, nullptr, Z ? zsel : hub, log,
                                                                     work, grab, nullptr);
      note_launch();
    }
  } else {
    const void *k = (const void *)k_edge_pass_direct<F, Q>;
    const unsigned g = clamp_grid(want, one_shot ? cap_big : persistent_cap(k, block, 0));
    k_edge_pass_direct<F, Q><<<g, block, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, P, n, ctrl,
                                                 skip); note_launch();
  }
  return cudaGetLastError();
}

template <class F>
cudaError_t edge_pass_f(int filter, int ept, int block, const EdgeSpan &e, uint32_t *P, uint32_t n,
                        Ctrl *ctrl, const uint32_t *skip, uint32_t *Z, const uint32_t *zsel, bool one_shot,
                        uint32_t *log, const uint32_t *hub, bool dyn, cudaStream_t s, const unsigned long long *hot) {
  switch (ept) {
    case 2: return edge_pass_q<F, 1>(filter, block, e, P, n, ctrl, skip, Z, zsel, one_shot, log, hub, dyn, s, hot);
    case 8: return edge_pass_q<F, 4>(filter, block, e, P, n, ctrl, skip, Z, zsel, one_shot, log, hub, dyn, s, hot);
    default: return edge_pass_q<F, 2>(filter, block, e, P, n, ctrl, skip, Z, zsel, one_shot, log, hub, dyn, s, hot);
  }
}
}  // namespace

cudaError_t launch_edge_pass(bool rf, int filter, int ept, int block, const EdgeSpan &e, uint32_t *P,
                             uint32_t n, Ctrl *ctrl, const uint32_t *skip, cudaStream_t s, uint32_t *Z,
                             const uint32_t *zsel, bool one_shot, uint32_t *log, const uint32_t *hub, bool dyn,
                             const unsigned long long *hot) {
  if (block != 128 && block != 256 && block != 512) block = 256;
  if (e.n_quads == 0 && !e.head && !e.tail) return cudaSuccess;
  if (log) filter = 1;  // the log is kept by the filtered form
  return rf ? edge_pass_f<RootR>(filter, ept, block, e, P, n, ctrl, skip, Z, zsel, one_shot, log, hub, dyn, s, hot)
            : edge_pass_f<RootId>(filter, ept, block, e, P, n, ctrl, skip, Z, zsel, one_shot, log, hub, dyn, s,
                                  nullptr);
}

cudaError_t launch_validate(const EdgeSpan &e, uint32_t n, Ctrl *ctrl, cudaStream_t s, uint32_t *reject) {
  if (e.n_quads == 0 && !e.head && !e.tail) return cudaSuccess;
  const unsigned g = clamp_grid((e.n_quads + 255) / 256, persistent_cap((const void *)k_validate, 256, 0));
  k_validate<<<g, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, n, ctrl, reject ? reject : &ctrl->reject);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gmin_probe(uint32_t *P, uint32_t n, Ctrl *ctrl, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)n + 255) / 256;
  const unsigned gp = clamp_grid(want / 4 + 1, persistent_cap((const void *)k_gmin_probe, 256, 0));
  k_gmin_probe<<<gp, 256, 0, s>>>(P, n, ctrl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_flatten(bool rf, int label_space, uint32_t *P, uint32_t n, uint32_t *L, Ctrl *ctrl,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)n + 255) / 256;
  if (rf && label_space == kLabelMinId && L) {
    const unsigned gp = clamp_grid(want / 4 + 1, persistent_cap((const void *)k_gmin_probe, 256, 0));
    k_gmin_probe<<<gp, 256, 0, s>>>(P, n, ctrl); note_launch();
  }
#define CC_FLAT(F_, LAB_)                                                                         \
  do {                                                                                            \
    if (vec) {                                                                                    \
      const unsigned g = clamp_grid(want / 4 + 1, persistent_cap((const void *)k_flatten4<F_, LAB_>, 256, 0)); \
      k_flatten4<F_, LAB_><<<g, 256, 0, s>>>(P, n, L, ctrl);                                      \
    } else {                                                                                      \
      const unsigned g = clamp_grid(want, persistent_cap((const void *)k_flatten<F_, LAB_>, 256, 0)); \
      k_flatten<F_, LAB_><<<g, 256, 0, s>>>(P, n, L, ctrl);                                       \
    }                                                                                             \
    note_launch();                                                                                \
  } while (0)
  const bool vec = ((uintptr_t)L & 15u) == 0;  // P itself is 256-byte aligned
  if (rf) {
    if (label_space == kLabelRootValue) CC_FLAT(RootR, kLabelRootValue);
    else CC_FLAT(RootR, kLabelMinId);
  } else {
    if (label_space == kLabelRootValue) CC_FLAT(RootId, kLabelRootValue);
    else CC_FLAT(RootId, kLabelMinId);
  }
#undef CC_FLAT
  return cudaGetLastError();
}

cudaError_t launch_count_roots(bool rf, const uint32_t *P, uint32_t n, Ctrl *ctrl, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)n + 255) / 256;
  if (rf) {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_count_roots<RootR>, 256, 0));
    k_count_roots<RootR><<<g, 256, 0, s>>>(P, n, ctrl); note_launch();
  } else {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_count_roots<RootId>, 256, 0));
    k_count_roots<RootId><<<g, 256, 0, s>>>(P, n, ctrl); note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_forest_pairs(bool rf, const uint32_t *P, uint32_t n, uint32_t *out, uint64_t cap, Ctrl *ctrl,
                                cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(&ctrl->pairs, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess || n == 0) return err;
  const uint64_t want = ((uint64_t)n + 1023) / 1024;  // 4 vertices per thread
  uint2 *o = reinterpret_cast<uint2 *>(out);
  if (rf) {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_forest_pairs<RootR>, 256, 0));
    k_forest_pairs<RootR><<<g, 256, 0, s>>>(P, n, o, cap, ctrl);
  } else {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_forest_pairs<RootId>, 256, 0));
    k_forest_pairs<RootId><<<g, 256, 0, s>>>(P, n, o, cap, ctrl);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_connected(bool rf, uint32_t *P, uint32_t n, const uint2 *pairs, uint64_t n_pairs,
                             uint8_t *out, Ctrl *ctrl, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  const uint64_t want = (n_pairs + 255) / 256;
  if (rf) {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_connected<RootR>, 256, 0));
    k_connected<RootR><<<g, 256, 0, s>>>(P, n, pairs, n_pairs, out, ctrl); note_launch();
  } else {
    const unsigned g = clamp_grid(want, persistent_cap((const void *)k_connected<RootId>, 256, 0));
    k_connected<RootId><<<g, 256, 0, s>>>(P, n, pairs, n_pairs, out, ctrl); note_launch();
  }
  return cudaGetLastError();
}

}  // namespace cc

#ifdef CC_STATS
// Diagnostics builds only: read and clear the search counters.
extern "C" __attribute__((visibility("default"))) int cc_stats_read(unsigned long long out[4]) {
  cudaError_t e = cudaMemcpyFromSymbol(out, cc::g_cc_stats, 4 * sizeof(unsigned long long));
  unsigned long long z[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(cc::g_cc_stats, z, sizeof(z));
  return (int)e;
}
#endif

// cc_device.cuh - device primitives of Root-Function JT union-find.
//
// The parent array P holds, for every vertex x, a root value: x is a root iff
// P[x] == f(x); otherwise f^-1(P[x]) is an ancestor of x (Algorithm 3). Two
// root functions are provided: f(v) = v (Algorithm 1) and f = R of Eq. 1
// (R(m) = 0, R(v) = v + 1 otherwise) with its inverse from Eq. 2.
//
// Facts the kernels rely on (all follow from the hooking rule "the root of
// larger f gets the smaller f as parent value"):
//  * P values only decrease, and every non-root x has f(parent) < f(x), so
//    every walk up the parents ends, and any value P[x] ever held names an
//    ancestor of x for the rest of the run. A stale read of P is therefore
//    still a correct (if older) ancestor, and two endpoints that ever showed
//    the same P value are in the same tree.
//  * The vertex of root value 0 (m under R, vertex 0 under the identity) can
//    never be hooked, so reading 0 ends a root search at once.
//  * Only roots are ever CAS targets; path splitting rewrites only non-roots,
//    and always to an ancestor's value, so it never changes a component.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cc_internal.h"

namespace cc {

// f(v) = v (Algorithm 1; Algorithm 3 with the identity, Section IV).
struct RootId {
  static constexpr bool kRF = false;
  static constexpr uint32_t kOff = 0;  // f(x) = x + kOff for every x with f(x) != 0
  __device__ __forceinline__ static RootId load(const Ctrl *) { return RootId{}; }
  __device__ __forceinline__ uint32_t f(uint32_t x) const { return x; }
  __device__ __forceinline__ uint32_t finv(uint32_t c) const { return c; }
};

// f = R (Eq. 1), f^-1 = R^-1 (Eq. 2).
struct RootR {
  static constexpr bool kRF = true;
  static constexpr uint32_t kOff = 1;
  uint32_t m;
  __device__ __forceinline__ static RootR load(const Ctrl *ctrl) {
    return RootR{*(const volatile uint32_t *)&ctrl->m};
  }
  __device__ __forceinline__ uint32_t f(uint32_t x) const { return x == m ? 0u : x + 1u; }
  __device__ __forceinline__ uint32_t finv(uint32_t c) const { return c == 0u ? m : c - 1u; }
};

// ------------------------------------------------------------ memory access

// L2 policy for data read exactly once (the edge stream): evict first, so the
// parent array keeps the cache.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 128-bit streaming load of two edges: non-coherent path, no L1 allocation.
__device__ __forceinline__ uint4 ld_edges(const uint4 *a, uint64_t pol) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(a), "l"(pol));
  return r;
}

__device__ __forceinline__ uint2 ld_edge(const uint2 *a) {
  uint2 r;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(a));
  return r;
}

// Parent-array load. A weak load may be served from this SM's L1 and so be
// stale; by the facts above a stale value is an older ancestor, which keeps
// every search correct. (CAS results always come from L2.)
// Build option CC_PLOAD selects the cache behaviour of these loads: 0 (default)
// allocates in L1, 1 bypasses L1 allocation, 2 caches in L2 only (.cg).
#ifndef CC_PLOAD
#define CC_PLOAD 0
#endif
__device__ __forceinline__ uint32_t ldP(const uint32_t *p) {
  uint32_t r;
#if CC_PLOAD == 1
  asm volatile("ld.global.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
#elif CC_PLOAD == 2
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
#else
  asm volatile("ld.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
#endif
  return r;
}

__device__ __forceinline__ uint32_t ldP_strong(const uint32_t *p) {
  uint32_t r;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}

// L2-only parent load (no L1 allocation): for long-lived kernels whose L1
// may hold lines from before the latest writes of other kernels.
__device__ __forceinline__ uint32_t ldP_cg(const uint32_t *p) {
  uint32_t r;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}

template <bool kCG>
__device__ __forceinline__ uint32_t ldP_t(const uint32_t *p) {
  return kCG ? ldP_cg(p) : ldP(p);
}

__device__ __forceinline__ void stP(uint32_t *p, uint32_t v) {
  asm volatile("st.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
  return *(const volatile uint32_t *)p;
}

__device__ __forceinline__ void set_err(Ctrl *ctrl, uint32_t bit) { atomicOr(&ctrl->err, bit); }

// ----------------------------------------------------------- instrumentation
// Built with -DCC_STATS, the searches count their work into a device array
// (edges that reach a root search, parent loads in searches, CAS attempts, CAS
// failures); diagnostics only, off in normal builds.
#ifdef CC_STATS
__device__ unsigned long long g_cc_stats[4];  // only cc_kernels.cu includes this header
#define CC_STAT(i) atomicAdd(&g_cc_stats[(i)], 1ULL)
#else
#define CC_STAT(i) ((void)0)
#endif

// ------------------------------------------------------------------ searches
//
// The searches work on names: vertex x is named f(x), and P[x] holds the name
// of x's parent (x's own name when x is a root). Every vertex except the one
// named 0 has f(x) = x + kOff, so the slot of name c >= 1 is
// slots(P)[c] = P[c - kOff]: a walk up the parents needs neither f nor f^-1,
// only an address with a constant offset. The vertex named 0 is never loaded
// through its name: it can never be hooked, so reading the name 0 ends a walk.

template <class F>
__device__ __forceinline__ uint32_t *slots(uint32_t *P) {
  return P - F::kOff;
}

// Root name of the vertex named c, given pc = a value its P has held. Walks
// with path splitting (each visited non-root gets its grandparent's name).
// The walk is at most n steps because names strictly decrease along parents.
__device__ __forceinline__ uint32_t root_name(uint32_t *S, uint32_t c, uint32_t pc) {
  while (pc != c) {
    if (pc == 0u) return 0u;  // the permanent root
    const uint32_t pw = ldP(S + pc);
    if (pw != pc) stP(S + c, pw);  // the parent is not a root: split past it
    c = pc;
    pc = pw;
  }
  return c;
}

// One edge of the hooking pass (Algorithm 3) in names: cu, cv name the
// endpoints and pu, pv are values their P held. Repeats { find both roots;
// equal -> done; CAS the root of larger name from its name to the other
// root's name } until a CAS succeeds. A failed CAS returns the root's new
// parent, and the search resumes from that root (the current roots, not the
// original endpoints). Any moment at which both sides show the same parent
// name proves a common tree and ends the edge, which includes the case of
// both endpoints already holding 0. Reports whether the edge is known to end
// in the tree of name 0 (both endpoints then belong to it for good), and the
// name of the root this edge's CAS hooked, if any (the pairs SiskinCC sends on
// a successful CAS, Algorithm 2).
struct UniteResult {
  bool zero;        // ended in the tree of name 0
  uint32_t hooked;  // the root hooked by this edge, or kNoHook
};
constexpr uint32_t kNoHook = 0xFFFFFFFFu;

template <bool kCG = false>
__device__ __forceinline__ UniteResult unite(uint32_t *S, uint32_t cu, uint32_t pu, uint32_t cv, uint32_t pv) {
  if (pu != pv) CC_STAT(0);
  while (true) {
    if (pu == pv) return {pu == 0u, kNoHook};
    while (pu != cu) {
      if (pu == 0u) {
        cu = 0u;
        break;
      }
      CC_STAT(1);
      const uint32_t pw = ldP_t<kCG>(S + pu);
      if (pw != pu) stP(S + cu, pw);
      cu = pu;
      pu = pw;
      if (pu == pv) return {pu == 0u, kNoHook};
    }
    while (pv != cv) {
      if (pv == 0u) {
        cv = 0u;
        break;
      }
      CC_STAT(1);
      const uint32_t pw = ldP_t<kCG>(S + pv);
      if (pw != pv) stP(S + cv, pw);
      cv = pv;
      pv = pw;
      if (pu == pv) return {pu == 0u, kNoHook};
    }
    if (pu == pv) return {pu == 0u, kNoHook};  // same root
    CC_STAT(2);
    if (pu < pv) {
      const uint32_t old = atomicCAS(S + cv, pv, pu);
      if (old == pv) return {pu == 0u, cv};
      pv = old;  // that root was hooked meanwhile: continue from it
    } else {
      const uint32_t old = atomicCAS(S + cu, pu, pv);
      if (old == pu) return {pv == 0u, cu};
      pu = old;
    }
    CC_STAT(3);
  }
}

// ------------------------------------------------------------ the warp ring
//
// Warp-level filter and compaction of the edge pass: after the parent loads,
// an edge whose endpoints hold the same parent name is dropped (this covers
// both endpoints already at name 0); survivors of the warp are appended to a
// per-warp ring in shared memory (names and parent names of both endpoints),
// and whenever 32 are queued the whole warp resolves them together, one per
// lane, so root searches run in dense warps. At most 31 survivors are carried
// between appends, so 64 entries suffice. All lanes of the warp must call
// push() and drain() together. With a zero-tree bitmap Z (below), an edge that
// ends in the tree of name 0 marks both endpoint names in it.
constexpr int kRing = 64;
// When at least this many lanes keep their edge, the warp resolves them in
// place: the queue would only add its shared-memory round trip. This pays
// where most edges reach a search for most of the pass (graphs without a
// hub, and parent arrays beyond L2 behind the zero-tree bitmap); on a
// certified hub graph whose P fits L2 it cost a few percent, so the plain
// edge pass keeps the queue there (kNeverDirect).
constexpr uint32_t kDirectMin = 28;
constexpr uint32_t kNeverDirect = 33;

// The zero-tree bitmap: bit c set means the vertex named c belongs to the
// tree of name 0 (the planted vertex m under R). Bits are only ever set, and
// only after a walk or a parent value proved the fact, which holds for good
// because name 0 is never hooked; a stale 0 bit only costs the parent load
// it would have saved. Name 0 itself (the tree's root m) never gets its bit:
// the many hooks onto m would all send an atomic to the one word that holds
// it. A lookup of m then loads P of m, which is 0 (the hot-vertex table
// answers for m first where there is one).
__device__ __forceinline__ bool zbit(const uint32_t *Z, uint32_t c) {
  uint32_t w;
  asm volatile("ld.global.u32 %0, [%1];" : "=r"(w) : "l"(Z + (c >> 5)) : "memory");
  return (w >> (c & 31u)) & 1u;
}

// Sets bit c, never for name 0.
__device__ __forceinline__ void zset(uint32_t *Z, uint32_t c) {
  if (c != 0u) atomicOr(Z + (c >> 5), 1u << (c & 31u));
}

// Slot of vertex x in the hot-vertex table (kHot entries).
__device__ __forceinline__ uint32_t hot_slot(uint32_t x) { return (x * 2654435761u) >> (32 - kHotBits); }

// A changed-root log: log[0] counts the entries that follow it, the names of
// the roots hooked since the log was last cleared. Its capacity (one entry
// per vertex) cannot be exceeded: a root is hooked once.
__device__ __forceinline__ void log_hook(uint32_t *log, uint32_t hooked) {
  const uint32_t i = atomicAdd(log, 1u);
  log[1u + i] = hooked;
}

// The same for a whole warp (every lane calls it): one atomic per warp.
__device__ __forceinline__ void log_hooks_warp(uint32_t *log, uint32_t hooked, uint32_t lane, uint32_t lt_mask) {
  const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hooked != kNoHook);
  if (!bal) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(log, (uint32_t)__popc(bal));
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  if (hooked != kNoHook) log[1u + base + (uint32_t)__popc(bal & lt_mask)] = hooked;
}

struct WarpRing {
  uint32_t *cu, *pu, *cv, *pv;
  uint32_t *Z;    // zero-tree bitmap, or null
  uint32_t *log;  // changed-root log, or null
  uint32_t head, tail;
  uint32_t lane, lt_mask;
  uint32_t direct_min;  // kDirectMin, or kNeverDirect for the queue only

  // ring storage for this warp out of 4 * kRing words per warp
  __device__ __forceinline__ void init(uint32_t *smem_words, uint32_t *zero_tree = nullptr,
                                       uint32_t *root_log = nullptr, uint32_t direct = kDirectMin) {
    Z = zero_tree;
    log = root_log;
    direct_min = direct;
    const uint32_t wid = threadIdx.x >> 5;
    cu = smem_words + wid * (4 * kRing);
    pu = cu + kRing;
    cv = cu + 2 * kRing;
    pv = cu + 3 * kRing;
    head = tail = 0;
    lane = threadIdx.x & 31u;
    lt_mask = (1u << lane) - 1u;
  }

  template <bool kCG = false>
  __device__ __forceinline__ void push(uint32_t *S, bool keep, uint32_t a, uint32_t pa, uint32_t b,
                                       uint32_t pb) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
    // one call of unite() serves both routes: a second inlined copy cost
    // the plain pass a register spill
    const bool direct = (uint32_t)__popc(bal) >= direct_min;  // warp-uniform
    bool run = direct;
    bool mine = keep;
    if (!direct) {
      if (keep) {
        const uint32_t slot = (tail + __popc(bal & lt_mask)) & (kRing - 1);
        cu[slot] = a;
        pu[slot] = pa;
        cv[slot] = b;
        pv[slot] = pb;
      }
      tail += __popc(bal);
      if (tail - head >= 32u) {
        __syncwarp();
        const uint32_t slot = (head + lane) & (kRing - 1);
        a = cu[slot];
        pa = pu[slot];
        b = cv[slot];
        pb = pv[slot];
        __syncwarp();
        head += 32u;
        run = true;
        mine = true;
      }
    }
    if (!run) return;
    UniteResult res{false, kNoHook};
    if (mine) res = unite<kCG>(S, a, pa, b, pb);
    // an endpoint whose parent value was 0 is known to be in the tree of
    // name 0 already (its bit set, or P = 0): no atomic for it
    if (res.zero && Z) {
      if (pa) zset(Z, a);
      if (pb) zset(Z, b);
    }
    if (log) log_hooks_warp(log, res.hooked, lane, lt_mask);
  }

  template <bool kCG = false>
  __device__ __forceinline__ void drain(uint32_t *S) {
    __syncwarp();
    uint32_t hooked = kNoHook;
    if (lane < tail - head) {
      const uint32_t slot = (head + lane) & (kRing - 1);
      const uint32_t a = cu[slot], b = cv[slot], pa = pu[slot], pb = pv[slot];
      const UniteResult res = unite<kCG>(S, a, pa, b, pb);
      if (res.zero && Z) {
        if (pa) zset(Z, a);
        if (pb) zset(Z, b);
      }
      hooked = res.hooked;
    }
    if (log) log_hooks_warp(log, hooked, lane, lt_mask);
    head = tail;
    __syncwarp();
  }
};

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

}  // namespace cc

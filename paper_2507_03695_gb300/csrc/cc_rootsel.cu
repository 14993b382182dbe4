// cc_rootsel.cu - selection of the planted vertex m of Eq. 1: the vertex of
// maximum degree (Algorithm 4, max_degree()), degree = occurrences as an
// endpoint (a self-loop counts twice, duplicates count), ties to the smaller
// id.
//
// A global histogram needs one random atomic per endpoint, which on R-MAT
// graphs is slower than the edge pass itself. The default exact selection is
// therefore certified instead:
//   1. a histogram over 1 group of kSampleGroup edges in 128 (more from 2^26
//      edges up: cert_sample_stride; global atomics) gives
//      candidate hubs: every vertex with at least 1/32 of the largest sampled
//      count (at most kCertCand of them); the best per hash bucket of vertex
//      ids competes, and the kCertTop best of those are kept;
//   2. one pass over all edges counts, in registers, the exact degree of each
//      kept candidate and, in shared memory, the endpoint occurrences of every
//      bucket;
//   3. a bucket's occurrences minus the exact degrees of the kept candidates
//      in it bound the degree of every other vertex of the bucket; if the
//      best candidate's degree D (smaller id on ties) exceeds that bound in
//      every bucket, no other vertex can reach D, and the best candidate is
//      the exact answer;
//   4. otherwise (graphs without a dominant hub, such as grids) the full
//      global histogram runs; its kernels read the certificate flag and
//      return at once when step 3 succeeded.
// The answer is the exact maximum-degree vertex in both cases.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {

namespace {

__device__ __forceinline__ bool skipped(const uint32_t *skip) {
  return skip && *(const volatile uint32_t *)skip != 0u;
}

template <typename C>
__device__ __forceinline__ void count_edge(C *cnt, uint32_t n, uint32_t a, uint32_t b) {
  if (a < n) atomicAdd(cnt + a, (C)1);
  if (b < n) atomicAdd(cnt + b, (C)1);
}

template <typename C>
__global__ void __launch_bounds__(256) k_zero_cnt(C *cnt, uint32_t n, const uint32_t *skip) {
  if (skipped(skip)) return;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    cnt[v] = (C)0;
}

// Edge idx lies in a sampled group of k_degree_sampled (1 group of
// kSampleGroup in stride, counted from the start of the edge array); stride
// 0: never.
__device__ __forceinline__ bool in_sample(uint64_t idx, uint32_t stride) {
  return stride != 0u && ((idx >> kSampleGroupShift) % stride) == 0u;
}

// Degree histogram. With stride nonzero, the edges of the sampled groups are
// left out: added to the sampled counts, the result is the full histogram.
template <typename C>
__global__ void __launch_bounds__(256) k_degree(const uint4 *__restrict__ e4, uint64_t n_quads,
                                                const uint2 *head, const uint2 *tail,
                                                C *__restrict__ cnt, uint32_t n, const uint32_t *skip,
                                                uint32_t stride) {
  if (skipped(skip)) return;
  const uint64_t pol = policy_evict_first();
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t h = head ? 1u : 0u;  // edge index of the first quad's first edge
  if (t == 0 && head && !in_sample(0, stride)) {
    uint2 e = ld_edge(head);
    count_edge(cnt, n, e.x, e.y);
  }
  if (t == 1 % T && tail && !in_sample(h + 2 * n_quads, stride)) {
    uint2 e = ld_edge(tail);
    count_edge(cnt, n, e.x, e.y);
  }
  for (uint64_t q = t; q < n_quads; q += T) {
    const uint64_t i0 = h + 2 * q;
    const bool s0 = in_sample(i0, stride), s1 = in_sample(i0 + 1, stride);
    if (s0 && s1) continue;
    const uint4 e = ld_edges(e4 + q, pol);
    if (!s0) count_edge(cnt, n, e.x, e.y);
    if (!s1) count_edge(cnt, n, e.z, e.w);
  }
}

// Sampled histogram: edge i (global index edge_base + i) is counted iff
// ((edge_base + i) / kSampleGroup) % stride == 0. With track, the largest count also
// goes to the high half of track->maxkey (from the atomics' old values: the
// last increment of a counter sees its final value), which spares an argmax
// pass over the counters when only the largest count is needed.
// With list, a vertex whose count reaches kListThr is appended to it (once:
// the atomics' old values are distinct), to the block's segment; the segment
// counters list_n may go beyond the segment's room (list_cap / kListSegs).
__global__ void __launch_bounds__(256) k_degree_sampled(const uint2 *__restrict__ e, uint64_t n_edges,
                                                        uint64_t edge_base, uint32_t stride,
                                                        uint32_t *__restrict__ cnt, uint32_t n, Ctrl *track,
                                                        uint32_t *list, unsigned int *list_n, uint32_t list_cap) {
  uint32_t top = 0;
  const uint32_t seg = blockIdx.x % kListSegs, seg_room = list_cap / kListSegs;
  auto bump = [&](uint32_t v) {
    if (v >= n) return;
    const uint32_t c = atomicAdd(cnt + v, 1u) + 1u;
    top = max(top, c);
    if (c == kListThr) {
      const unsigned int i = atomicAdd(list_n + seg, 1u);
      if (i < seg_room) list[seg * seg_room + i] = v;
    }
  };
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g_first = edge_base >> kSampleGroupShift;
  const uint64_t g_last = (edge_base + n_edges + kSampleGroup - 1u) >> kSampleGroupShift;  // exclusive
  const uint64_t g0 = (g_first + stride - 1) / stride * stride;    // first sampled group
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;; k += T) {
    const uint64_t grp = g0 + (k >> kSampleGroupShift) * stride;
    if (grp >= g_last) break;
    const uint64_t gi = (grp << kSampleGroupShift) + (k & (kSampleGroup - 1u));
    if (gi < edge_base || gi >= edge_base + n_edges) continue;
    const uint2 x = ld_edge(e + (gi - edge_base));
    if (list) {
      bump(x.x);
      bump(x.y);
    } else if (!track) {
      count_edge(cnt, n, x.x, x.y);
    } else {
      if (x.x < n) top = max(top, atomicAdd(cnt + x.x, 1u) + 1u);
      if (x.y < n) top = max(top, atomicAdd(cnt + x.y, 1u) + 1u);
    }
  }
  if (track) {
    top = __reduce_max_sync(0xFFFFFFFFu, top);
    if ((threadIdx.x & 31) == 0 && top) atomicMax(&track->maxkey, (unsigned long long)top << 32);
  }
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long key) {
  __shared__ unsigned long long sm[32];
  key = warp_max_u64(key);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = key;
  __syncthreads();
  key = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ULL;
  return warp_max_u64(key);  // valid in every warp
}

// Packed key (deg << 32) | ~v: the largest key has the largest degree and,
// among equal degrees, the smallest v.
__global__ void __launch_bounds__(256) k_argmax_u32(const uint32_t *__restrict__ cnt, uint32_t n,
                                                    Ctrl *ctrl, const uint32_t *skip) {
  if (skipped(skip)) return;
  unsigned long long best = 0;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = ((unsigned long long)cnt[v] << 32) | (uint32_t)~(uint32_t)v;
    best = key > best ? key : best;
  }
  best = block_max_u64(best);
  if (threadIdx.x == 0 && best) atomicMax(&ctrl->maxkey, best);
}

__global__ void __launch_bounds__(256) k_maxcnt_u64(const unsigned long long *__restrict__ cnt,
                                                    uint32_t n, Ctrl *ctrl, const uint32_t *skip) {
  if (skipped(skip)) return;
  unsigned long long best = 0;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    best = cnt[v] > best ? cnt[v] : best;
  best = block_max_u64(best);
  if (threadIdx.x == 0 && best) atomicMax(&ctrl->maxcnt, best);
}

__global__ void __launch_bounds__(256) k_minid_u64(const unsigned long long *__restrict__ cnt,
                                                   uint32_t n, Ctrl *ctrl, const uint32_t *skip) {
  if (skipped(skip)) return;
  const unsigned long long mx = *(volatile unsigned long long *)&ctrl->maxcnt;
  uint32_t best = 0xFFFFFFFFu;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    if (cnt[v] == mx && (uint32_t)v < best) best = (uint32_t)v;
  best = __reduce_min_sync(0xFFFFFFFFu, best);
  if ((threadIdx.x & 31) == 0 && best != 0xFFFFFFFFu) atomicMin(&ctrl->m_sel, best);
}

// Packs the 64-bit-count answer (m_sel) into maxkey for the init kernel.
__global__ void k_finalize_m(Ctrl *ctrl, const uint32_t *skip) {
  if (skipped(skip)) return;
  ctrl->maxkey = (unsigned long long)(uint32_t)~ctrl->m_sel;
}

// ----------------------------------------------------------- certification

// One multiplicative hash picks the bucket (13 bits) of a vertex. Each bucket
// has at most one candidate, its owner; every other vertex of the bucket is
// counted in the bucket's total.
__device__ __forceinline__ uint32_t bucket_of(uint32_t x) { return (x * 2654435769u) >> 19; }
static_assert(kCertBuckets == 8192, "13-bit buckets");

// Candidates: every vertex whose sampled count is at least 1/32 of the largest
// competes for its bucket; the larger sampled count (then the smaller id)
// owns it. Without a dominant hub (largest sampled count below 64) no
// certificate can succeed and nothing is selected. Scanning stops once more
// than kCertCand candidates are seen: so many near-maximal vertices leave no
// room for a proof, and the full histogram runs. The last block to finish
// ranks the owners and keeps the kCertTop best for the counting pass.
// kList: the vertices are those appended to the list's segments (as many as
// each segment holds), else every vertex 0 .. n-1.
template <bool kList>
__global__ void __launch_bounds__(256) k_select_candidates(const uint32_t *__restrict__ cnt, uint32_t n,
                                                           Ctrl *ctrl, CertScratch *cs,
                                                           const uint32_t *__restrict__ list, uint32_t list_cap) {
  const uint32_t cmax = (uint32_t)(*(volatile unsigned long long *)&ctrl->maxkey >> 32);
  if (cmax < 64u) return;  // uniform over the grid: no block ranks, top stays empty
  const uint32_t thr = cmax >> 5;
  // The hot-vertex table takes vertices from 1/256 of the largest count. On
  // R-MAT the list's own threshold (kListThr) is then the tighter one, so
  // every listed vertex competes for its slot (R-MAT scale 24 edge pass: 1/64
  // 1.75 ms, 1/128 to 1/2048 1.70 ms).
  const uint32_t hot_thr = cmax >> 8;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t w0 = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t count = kList ? list_cap : n;
  const uint32_t seg_room = kList ? list_cap / kListSegs : 0u;
  for (uint64_t base = w0 * 32; base < count; base += warps * 32) {
    const uint64_t i = base + (uint64_t)lane;
    bool have = i < count;
    uint64_t v = i;
    if constexpr (kList) {
      if (have) {
        const uint32_t seg = (uint32_t)(i / seg_room), k = (uint32_t)(i % seg_room);
        have = k < __ldcg(&cs->list_n[seg]);
        v = have ? list[i] : 0u;
      }
    }
    const uint32_t c = have ? cnt[v] : 0u;
    if (c >= hot_thr && c != 0u)
      atomicMax(&cs->hot[hot_slot((uint32_t)v)], ((unsigned long long)c << 32) | (uint32_t)(v + 1u));
    const bool q = c >= thr && c != 0u;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, q);
    if (!bal) continue;
    uint32_t seen = 0;
    if (lane == 0) seen = atomicAdd(&ctrl->n_cand, (uint32_t)__popc(bal)) + (uint32_t)__popc(bal);
    seen = __shfl_sync(0xFFFFFFFFu, seen, 0);
    if (seen > kCertCand) break;  // too many candidates (warp-uniform)
    if (q)
      atomicMax(&cs->owner[bucket_of((uint32_t)v)], ((unsigned long long)c << 32) | (uint32_t)~(uint32_t)v);
  }
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cs->sel_done, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // rank: each thread keeps the kCertTop best owners of its buckets (one pass
  // over them), then kCertTop rounds of a block maximum over the threads'
  // best untaken keys (keys are distinct: they hold the id)
  unsigned long long loc[kCertTop];
#pragma unroll
  for (uint32_t k = 0; k < kCertTop; ++k) loc[k] = 0ULL;
  for (uint32_t b = threadIdx.x; b < kCertBuckets; b += blockDim.x) {
    unsigned long long o = __ldcg(&cs->owner[b]);
#pragma unroll
    for (uint32_t k = 0; k < kCertTop; ++k) {  // insertion into the sorted list
      const unsigned long long hi = o > loc[k] ? o : loc[k];
      o = o > loc[k] ? loc[k] : o;
      loc[k] = hi;
    }
  }
  uint32_t next = 0;  // loc[next] is this thread's best untaken key
  for (uint32_t r = 0; r < kCertTop; ++r) {
    unsigned long long mine = 0ULL;
#pragma unroll
    for (uint32_t k = 0; k < kCertTop; ++k)
      if (k == next) mine = loc[k];
    const unsigned long long best = block_max_u64(mine);
    if (best == 0ULL) break;  // uniform: fewer owners than kCertTop
    if (threadIdx.x == 0) cs->top[r] = best;
    if (mine == best) ++next;
  }
}

constexpr size_t kCertSmem = kCertBuckets * sizeof(uint32_t);  // 32 KiB

__device__ __forceinline__ bool cert_skipped(const Ctrl *ctrl) {
  const uint32_t nc = *(const volatile uint32_t *)&ctrl->n_cand;
  return nc == 0u || nc > kCertCand;
}

// The proof, by one block: D = best exact candidate degree (ties to the
// smaller id); bound = the largest bucket total less the exact degrees of the
// candidates in that bucket. D > bound means every other vertex has degree
// < D. Reads through L2: other blocks wrote the totals.
__device__ void certify_decide_block(const CertScratch *cs, Ctrl *ctrl) {
  const bool skip = cert_skipped(ctrl);
  uint32_t cv[kCertTop];
  unsigned long long cc[kCertTop];
  bool any = false, wide = false;
  unsigned long long best = 0, bound = 0;
#pragma unroll
  for (uint32_t k = 0; k < kCertTop; ++k) {
    const unsigned long long o = __ldcg(&cs->top[k]);
    cv[k] = o ? ~(uint32_t)o : 0u;
    cc[k] = o ? __ldcg(&cs->top_cnt[k]) : 0ULL;
    if (!o) continue;
    any = true;
    if (cc[k] >= (1ULL << 32)) {
      wide = true;
      continue;
    }
    const unsigned long long key = (cc[k] << 32) | (uint32_t)o;  // low half: ~vertex
    best = key > best ? key : best;
  }
  for (uint32_t b = threadIdx.x; b < kCertBuckets && !skip && any; b += blockDim.x) {
    unsigned long long t = __ldcg(&cs->bucket[b]);
#pragma unroll
    for (uint32_t k = 0; k < kCertTop; ++k)
      if (cc[k] && bucket_of(cv[k]) == b) t -= cc[k];
    bound = t > bound ? t : bound;
  }
  bound = block_max_u64(bound);
  if (threadIdx.x == 0) {
    const unsigned long long D = best >> 32;
    if (!skip && any && !wide && best != 0ULL && D > bound) {
      ctrl->maxkey = best;
      ctrl->cert = 1u;
    } else {
      ctrl->maxkey = 0ULL;
      ctrl->cert = 0u;
    }
  }
}

// The proof as its own launch (after counting passes over several chunks).
__global__ void __launch_bounds__(256) k_certify_decide(const CertScratch *cs, Ctrl *ctrl) {
  certify_decide_block(cs, ctrl);
}

// One pass over all edges: exact candidate degrees (per-thread registers,
// summed per warp at the end) and bucket totals (shared memory, 32-bit per
// block, flushed once per block): one shared-memory atomic per endpoint.
// decide: the last block to finish also takes the decision (one pass over
// all edges); otherwise k_certify_decide runs after the last chunk.
// With push_buf, the other endpoint of every edge incident to the sampled
// argmax m' (read from ctrl->maxkey before the decision) is appended to the
// push list.
__device__ __forceinline__ void push_neighbour(uint32_t a, uint32_t b, uint32_t mp, uint32_t *buf, uint32_t seg,
                                               CertScratch *cs) {
  uint32_t x;
  if (a == mp && b != mp)
    x = b;
  else if (b == mp && a != mp)
    x = a;
  else
    return;
  const uint32_t lane = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kPushLanes;
  const uint32_t i = atomicAdd(&cs->push_cnt[lane], 1u);
  if (i < seg)
    buf[(uint64_t)lane * seg + i] = x;
  else
    cs->push_overflow = 1u;
}

// Counts one endpoint. Ids >= n are counted too; they only make the bound
// more conservative (the edge pass reports them).
struct CertCounter {
  uint32_t key[kCertTop];  // candidate ids (an empty slot matches only id 2^32 - 1, and is ignored)
  uint32_t c[kCertTop];
  uint32_t *bk;
  __device__ __forceinline__ void operator()(uint32_t x) {
    atomicAdd(&bk[bucket_of(x)], 1u);
#pragma unroll
    for (uint32_t k = 0; k < kCertTop; ++k) c[k] += x == key[k] ? 1u : 0u;
  }
};

constexpr int kCertBlock = 512;

__global__ void __launch_bounds__(kCertBlock, 2)
    k_degree_certify(const uint4 *__restrict__ e4, uint64_t n_quads, const uint2 *head, const uint2 *tail, uint32_t n,
                     CertScratch *cs, Ctrl *ctrl, int decide, uint32_t *push_buf, uint32_t push_seg) {
  extern __shared__ uint32_t csm[];
  if (cert_skipped(ctrl)) {  // no proof possible: the full histogram runs
    if (decide && blockIdx.x == 0 && threadIdx.x == 0) {
      ctrl->maxkey = 0ULL;
      ctrl->cert = 0u;
    }
    return;
  }
  CertCounter cnt;
  cnt.bk = csm;
#pragma unroll
  for (uint32_t k = 0; k < kCertTop; ++k) {
    const unsigned long long o = *(const volatile unsigned long long *)&cs->top[k];
    cnt.key[k] = o ? ~(uint32_t)o : 0xFFFFFFFFu;
    cnt.c[k] = 0u;
  }
  // the sampled argmax, whose neighbours the push list gathers
  const uint32_t mp = ~(uint32_t)(*(const volatile unsigned long long *)&ctrl->maxkey);
  if (push_buf && blockIdx.x == 0 && threadIdx.x == 0) cs->push_m = mp + 1u;
  for (uint32_t i = threadIdx.x; i < kCertBuckets; i += blockDim.x) csm[i] = 0u;
  __syncthreads();
  const uint64_t pol = policy_evict_first();
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t == 0 && head) {
    const uint2 e = ld_edge(head);
    cnt(e.x);
    cnt(e.y);
    if (push_buf) push_neighbour(e.x, e.y, mp, push_buf, push_seg, cs);
  }
  if (t == 1 % T && tail) {
    const uint2 e = ld_edge(tail);
    cnt(e.x);
    cnt(e.y);
    if (push_buf) push_neighbour(e.x, e.y, mp, push_buf, push_seg, cs);
  }
  uint64_t q = t;
  for (; q + 3 * T < n_quads; q += 4 * T) {  // four loads in flight per thread
    uint4 a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = ld_edges(e4 + q + j * T, pol);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cnt(a[j].x);
      cnt(a[j].y);
      cnt(a[j].z);
      cnt(a[j].w);
      if (push_buf) {
        push_neighbour(a[j].x, a[j].y, mp, push_buf, push_seg, cs);
        push_neighbour(a[j].z, a[j].w, mp, push_buf, push_seg, cs);
      }
    }
  }
  for (; q < n_quads; q += T) {
    const uint4 a = ld_edges(e4 + q, pol);
    cnt(a.x);
    cnt(a.y);
    cnt(a.z);
    cnt(a.w);
    if (push_buf) {
      push_neighbour(a.x, a.y, mp, push_buf, push_seg, cs);
      push_neighbour(a.z, a.w, mp, push_buf, push_seg, cs);
    }
  }
#pragma unroll
  for (uint32_t k = 0; k < kCertTop; ++k) {
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, cnt.c[k]);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&cs->top_cnt[k], (unsigned long long)w);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kCertBuckets; i += blockDim.x)
    if (csm[i]) atomicAdd(&cs->bucket[i], (unsigned long long)csm[i]);
  if (!decide) return;
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cs->blocks_done, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  certify_decide_block(cs, ctrl);
}

// Initial Push (Algorithm 4): right after init every vertex is a root, so a
// gathered neighbour x of m gets parent name 0 (m) by a plain store. Only when
// the planted m is the vertex whose neighbours were gathered, and no segment
// overflowed. Row y of the grid takes segment y of the push list.
__global__ void __launch_bounds__(256) k_initial_push(uint32_t *P, uint32_t n, const uint32_t *buf, uint32_t seg,
                                                      const CertScratch *cs, const Ctrl *ctrl) {
  const uint32_t pm = *(const volatile uint32_t *)&cs->push_m;
  if (pm == 0u || *(const volatile uint32_t *)&cs->push_overflow) return;
  const uint32_t m = *(const volatile uint32_t *)&ctrl->m;
  if (pm - 1u != m) return;
  const uint32_t lane = blockIdx.y;
  const uint32_t cnt = min(*(const volatile uint32_t *)&cs->push_cnt[lane], seg);
  const uint32_t *b = buf + (uint64_t)lane * seg;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint32_t x = b[i];
    if (x < n && x != m) P[x] = 0u;
  }
}

// Chunked selection: after the first chunk's sample, hub mode (candidates
// that a certificate can prove) or histogram mode. Histogram mode restarts
// the argmax, which the first chunk's full histogram then sets to m'.
__global__ void k_spec_begin(Ctrl *ctrl) {
  const uint32_t nc = *(volatile uint32_t *)&ctrl->n_cand;
  const bool hub = nc != 0u && nc <= kCertCand;
  ctrl->skip[kSkipHist] = hub ? 1u : 0u;
  ctrl->skip[kSkipRerun] = 0u;
  ctrl->skip[kSkipFullHist] = 1u;
  if (!hub) {
    ctrl->maxkey = 0ULL;
    ctrl->maxcnt = 0ULL;
    ctrl->m_sel = 0xFFFFFFFFu;
  }
}

// After the certificate's decision: a hub whose certificate failed needs the
// full histogram; histogram mode restarts the argmax for the final counts.
__global__ void k_spec_end(Ctrl *ctrl) {
  const bool hub = *(volatile uint32_t *)&ctrl->skip[kSkipHist] != 0u;
  const bool cert = *(volatile uint32_t *)&ctrl->cert != 0u;
  ctrl->skip[kSkipFullHist] = (hub && !cert) ? 0u : 1u;
  if (!hub) {
    ctrl->maxkey = 0ULL;
    ctrl->maxcnt = 0ULL;
    ctrl->m_sel = 0xFFFFFFFFu;
  }
}

// The exact m is in ctrl->maxkey: keep the speculative hooking when it was
// planted under that vertex (ctrl->m, written by the first init).
__global__ void k_spec_check(Ctrl *ctrl) {
  const uint32_t m = ~(uint32_t)(*(volatile unsigned long long *)&ctrl->maxkey);
  ctrl->skip[kSkipRerun] = m == *(volatile uint32_t *)&ctrl->m ? 1u : 0u;
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_degree_u32(const EdgeSpan &e, uint32_t *cnt, uint32_t n, cudaStream_t s) {
  const unsigned g = clamp_grid((e.n_quads + 255) / 256, persistent_cap((const void *)k_degree<uint32_t>, 256, 0));
  k_degree<uint32_t><<<g, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, cnt, n, nullptr, 0u);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_degree_sampled_u32(const uint2 *edges, uint64_t n_edges, uint64_t edge_base,
                                      uint32_t stride, uint32_t *cnt, uint32_t n, cudaStream_t s, Ctrl *track,
                                      uint32_t *list, unsigned int *list_n, uint32_t list_cap) {
  if (n_edges == 0) return cudaSuccess;
  if (stride == 0) stride = 1;
  const uint64_t groups = ((n_edges + kSampleGroup - 1) >> kSampleGroupShift) / stride + 2;
  const unsigned g = clamp_grid(groups * kSampleGroup / 256, persistent_cap((const void *)k_degree_sampled, 256, 0));
  k_degree_sampled<<<g, 256, 0, s>>>(edges, n_edges, edge_base, stride, cnt, n, track, list, list_n, list_cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_argmax_u32(const uint32_t *cnt, uint32_t n, Ctrl *ctrl, cudaStream_t s) {
  const unsigned g = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_argmax_u32, 256, 0));
  k_argmax_u32<<<g, 256, 0, s>>>(cnt, n, ctrl, nullptr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_root_select_certified(const uint32_t *edges, uint64_t n_edges, const EdgeSpan &e,
                                         void *cnt, bool wide, uint32_t n, CertScratch *cs, Ctrl *ctrl,
                                         cudaStream_t s, uint32_t *push_buf, uint32_t push_cap,
                                         uint32_t *list, uint32_t list_cap) {
  cudaError_t err;
  if (!list || list_cap < kListSegs || list_cap % kListSegs) list = nullptr;
  // 0. reset the sampled counters, the scratch and the control fields
  if ((err = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(cs, 0, sizeof(CertScratch), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->maxkey, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->m_sel, 0xFF, sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->n_cand, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return err;
  uint32_t *c32 = static_cast<uint32_t *>(cnt);
  // 1. sampled histogram and its largest count; the push list also needs the
  // vertex holding it (the argmax pass)
  const uint32_t stride = cert_sample_stride(n_edges);
  if ((err = launch_degree_sampled_u32(reinterpret_cast<const uint2 *>(edges), n_edges, 0, stride, c32, n, s,
                                       push_buf ? nullptr : ctrl, list, cs->list_n, list_cap)) != cudaSuccess)
    return err;
  if (push_buf && (err = launch_argmax_u32(c32, n, ctrl, s)) != cudaSuccess) return err;
  // 2. candidates: the owners of their buckets, from the list when there is one
  if (list) {
    const unsigned gsel = clamp_grid(((uint64_t)list_cap + 255) / 256,
                                     persistent_cap((const void *)k_select_candidates<true>, 256, 0));
    k_select_candidates<true><<<gsel, 256, 0, s>>>(c32, n, ctrl, cs, list, list_cap);
  } else {
    const unsigned gsel = clamp_grid(((uint64_t)n + 255) / 256,
                                     persistent_cap((const void *)k_select_candidates<false>, 256, 0));
    k_select_candidates<false><<<gsel, 256, 0, s>>>(c32, n, ctrl, cs, nullptr, 0u);
  }
  note_launch();
  // 3. the exact pass in shared memory
  static std::atomic<unsigned long long> smem_set_certify{0};
  if ((err = ensure_func_attr((const void *)k_degree_certify, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kCertSmem, smem_set_certify)) != cudaSuccess)
    return err;
  const unsigned gcert = clamp_grid((e.n_quads + kCertBlock - 1) / kCertBlock,
                                    persistent_cap((const void *)k_degree_certify, kCertBlock, kCertSmem));
  // 4. the proof: taken by the counting pass's last block (which also
  // gathers the push list when asked to)
  k_degree_certify<<<gcert, kCertBlock, kCertSmem, s>>>(e.quads, e.n_quads, e.head, e.tail, n, cs, ctrl, 1, push_buf,
                                                 push_buf ? push_cap / kPushLanes : 0u);
  note_launch();
  // 5. full histogram, skipped when certified
  const uint32_t *skip = &ctrl->cert;
  const unsigned gz = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_zero_cnt<uint32_t>, 256, 0));
  const unsigned gd = clamp_grid((e.n_quads + 255) / 256, persistent_cap((const void *)k_degree<uint32_t>, 256, 0));
  if (wide) {
    unsigned long long *c64 = static_cast<unsigned long long *>(cnt);
    k_zero_cnt<unsigned long long><<<gz, 256, 0, s>>>(c64, n, skip);
    note_launch();
    k_degree<unsigned long long><<<gd, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, c64, n, skip, 0u);
    note_launch();
    k_maxcnt_u64<<<gz, 256, 0, s>>>(c64, n, ctrl, skip);
    note_launch();
    k_minid_u64<<<gz, 256, 0, s>>>(c64, n, ctrl, skip);
    note_launch();
    k_finalize_m<<<1, 1, 0, s>>>(ctrl, skip);
    note_launch();
  } else {
    // the sampled counts are kept: only the edges outside the sample are added
    k_degree<uint32_t><<<gd, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, c32, n, skip, stride);
    note_launch();
    k_argmax_u32<<<gz, 256, 0, s>>>(c32, n, ctrl, skip);
    note_launch();
  }
  return cudaGetLastError();
}

// ------------------------------------------------- chunked root selection

namespace {
constexpr uint32_t kChunk0Sample = 16;  // the first chunk keeps 1 group of kSampleGroup edges in 16

cudaError_t launch_histogram(const EdgeSpan &e, void *cnt, bool wide, uint32_t n, const uint32_t *skip,
                             cudaStream_t s) {
  const unsigned gd = clamp_grid((e.n_quads + 255) / 256, persistent_cap((const void *)k_degree<uint32_t>, 256, 0));
  if (wide)
    k_degree<unsigned long long><<<gd, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail,
                                                    static_cast<unsigned long long *>(cnt), n, skip, 0u);
  else
    k_degree<uint32_t><<<gd, 256, 0, s>>>(e.quads, e.n_quads, e.head, e.tail, static_cast<uint32_t *>(cnt), n,
                                          skip, 0u);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zero(void *cnt, bool wide, uint32_t n, const uint32_t *skip, cudaStream_t s) {
  const unsigned gz = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_zero_cnt<uint32_t>, 256, 0));
  if (wide)
    k_zero_cnt<unsigned long long><<<gz, 256, 0, s>>>(static_cast<unsigned long long *>(cnt), n, skip);
  else
    k_zero_cnt<uint32_t><<<gz, 256, 0, s>>>(static_cast<uint32_t *>(cnt), n, skip);
  note_launch();
  return cudaGetLastError();
}

// argmax of a complete histogram into ctrl->maxkey (64-bit counts: through
// maxcnt, m_sel and k_finalize_m)
cudaError_t launch_hist_argmax(void *cnt, bool wide, uint32_t n, Ctrl *ctrl, const uint32_t *skip,
                               cudaStream_t s) {
  const unsigned gz = clamp_grid(((uint64_t)n + 255) / 256, persistent_cap((const void *)k_zero_cnt<uint32_t>, 256, 0));
  if (wide) {
    unsigned long long *c64 = static_cast<unsigned long long *>(cnt);
    k_maxcnt_u64<<<gz, 256, 0, s>>>(c64, n, ctrl, skip);
    note_launch();
    k_minid_u64<<<gz, 256, 0, s>>>(c64, n, ctrl, skip);
    note_launch();
    k_finalize_m<<<1, 1, 0, s>>>(ctrl, skip);
    note_launch();
  } else {
    k_argmax_u32<<<gz, 256, 0, s>>>(static_cast<const uint32_t *>(cnt), n, ctrl, skip);
    note_launch();
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t chunked_select_begin(const uint32_t *chunk0, uint64_t n0, void *cnt, bool wide, uint32_t n,
                                 CertScratch *cs, Ctrl *ctrl, cudaStream_t s) {
  cudaError_t err;
  if ((err = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(cs, 0, sizeof(CertScratch), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->maxkey, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->m_sel, 0xFF, sizeof(uint32_t), s)) != cudaSuccess) return err;
  // no vertex is planted yet: m' == m cannot hold before the first init
  if ((err = cudaMemsetAsync(&ctrl->m, 0xFF, sizeof(uint32_t), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(&ctrl->n_cand, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return err;
  uint32_t *c32 = static_cast<uint32_t *>(cnt);
  if ((err = launch_degree_sampled_u32(reinterpret_cast<const uint2 *>(chunk0), n0, 0, kChunk0Sample, c32, n, s)) !=
      cudaSuccess)
    return err;
  if ((err = launch_argmax_u32(c32, n, ctrl, s)) != cudaSuccess) return err;
  const unsigned gsel = clamp_grid(((uint64_t)n + 255) / 256,
                                   persistent_cap((const void *)k_select_candidates<false>, 256, 0));
  k_select_candidates<false><<<gsel, 256, 0, s>>>(c32, n, ctrl, cs, nullptr, 0u);
  note_launch();
  k_spec_begin<<<1, 1, 0, s>>>(ctrl);
  note_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // histogram mode: the chunks build the full histogram from zero
  return launch_zero(cnt, wide, n, &ctrl->skip[kSkipHist], s);
}

cudaError_t chunked_select_chunk(const EdgeSpan &chunk, bool first, void *cnt, bool wide, uint32_t n,
                                 CertScratch *cs, Ctrl *ctrl, cudaStream_t s) {
  cudaError_t err;
  const uint32_t *hub = &ctrl->skip[kSkipHist];
  if ((err = launch_histogram(chunk, cnt, wide, n, hub, s)) != cudaSuccess) return err;
  // histogram mode: the first chunk's argmax is m'
  if (first && (err = launch_hist_argmax(cnt, wide, n, ctrl, hub, s)) != cudaSuccess) return err;
  static std::atomic<unsigned long long> smem_set_certify{0};
  if ((err = ensure_func_attr((const void *)k_degree_certify, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kCertSmem, smem_set_certify)) != cudaSuccess)
    return err;
  const unsigned gcert =
      clamp_grid((chunk.n_quads + kCertBlock - 1) / kCertBlock,
                 persistent_cap((const void *)k_degree_certify, kCertBlock, kCertSmem));
  k_degree_certify<<<gcert, kCertBlock, kCertSmem, s>>>(chunk.quads, chunk.n_quads, chunk.head, chunk.tail, n, cs,
                                                        ctrl, 0, nullptr, 0u);
  note_launch();
  return cudaGetLastError();
}

cudaError_t chunked_select_end(const EdgeSpan &all, void *cnt, bool wide, uint32_t n, CertScratch *cs,
                               Ctrl *ctrl, cudaStream_t s) {
  cudaError_t err;
  k_certify_decide<<<1, 256, 0, s>>>(cs, ctrl);
  note_launch();
  k_spec_end<<<1, 1, 0, s>>>(ctrl);
  note_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // histogram mode: the chunks built the full histogram
  if ((err = launch_hist_argmax(cnt, wide, n, ctrl, &ctrl->skip[kSkipHist], s)) != cudaSuccess) return err;
  // hub mode without a certificate: the full histogram over all edges now
  const uint32_t *full = &ctrl->skip[kSkipFullHist];
  if ((err = launch_zero(cnt, wide, n, full, s)) != cudaSuccess) return err;
  if ((err = launch_histogram(all, cnt, wide, n, full, s)) != cudaSuccess) return err;
  if ((err = launch_hist_argmax(cnt, wide, n, ctrl, full, s)) != cudaSuccess) return err;
  k_spec_check<<<1, 1, 0, s>>>(ctrl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_initial_push(uint32_t *P, uint32_t n, const uint32_t *push_buf, uint32_t push_cap,
                                const CertScratch *cs, const Ctrl *ctrl, cudaStream_t s) {
  if (!push_buf || n == 0) return cudaSuccess;
  const uint32_t seg = push_cap / kPushLanes;
  const dim3 grid(clamp_grid(((uint64_t)seg + 255) / 256, 16), kPushLanes);
  k_initial_push<<<grid, 256, 0, s>>>(P, n, push_buf, seg, cs, ctrl);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cc

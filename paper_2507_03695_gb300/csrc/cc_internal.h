// cc_internal.h - state shared by the kernels and the host runtime of the
// connected-components library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <stddef.h>
#include <stdint.h>

namespace cc {

// Device error bits (sticky until a synchronising call reports them).
enum : uint32_t {
  kErrRange = 1u,     // a vertex id >= n reached a kernel
  kErrTimeout = 2u,   // a bounded wait expired
  kErrInternal = 4u,  // an invariant failed (a root search longer than n)
  kErrFormat = 8u,    // malformed input structure (CSR offsets)
};

// Where the init kernel takes the planted vertex m from.
enum : int { kMFromHint = 0, kMFromPackedMax = 1 };

// Per-handle control block in device memory (one cache line or two).
struct alignas(128) Ctrl {
  unsigned long long maxkey;  // root select, u32 counts: (deg << 32) | ~v, atomicMax
  unsigned long long maxcnt;  // root select, u64 counts: max degree
  unsigned long long ncomp;   // roots counted by the last flatten / count pass
  alignas(8) uint32_t q_u;    // cc_connected1 pair: read as one 8-byte (u, v) load
  uint32_t q_v;
  uint32_t q_out;             // cc_connected1 result (first byte)
  uint32_t m_sel;             // root select, 64-bit counts: smallest v with deg == maxcnt
  uint32_t m;                 // planted vertex in use (written by init)
  uint32_t gmin;              // smallest vertex of m's component (min-id labels, f = R)
  uint32_t err;               // kErr* bits
  uint32_t reject;            // the insert batch being applied failed validation
  uint32_t n_cand;            // root select: candidates found by the sampled pass
  uint32_t cert;              // root select: 1 when the candidate pass proved the argmax
  uint32_t skip[3];           // chunked root select: skip words (kSkip*), set on the device
  unsigned long long stats[4];  // optional edge-pass counters
  unsigned long long work;      // edge pass, dynamic schedule: steps claimed so far
  unsigned long long pairs;     // cc_forest_pairs: non-root vertices found
};
static_assert(offsetof(Ctrl, q_u) % 8 == 0, "the query pair is loaded with an 8-byte access");
static_assert(offsetof(Ctrl, maxkey) % 8 == 0 && offsetof(Ctrl, ncomp) % 8 == 0, "64-bit atomics");

// Label spaces (cc_label_space).
enum : int { kLabelMinId = 0, kLabelRootValue = 1 };

struct LaunchCfg {
  int block = 256;
  int grid = 0;
};

// Kernel launchers (cc_kernels.cu). Each returns cudaGetLastError().
struct EdgeSpan {
  const uint4 *quads = nullptr;  // 16-byte aligned body: 2 edges per uint4
  uint64_t n_quads = 0;
  const uint2 *head = nullptr;   // at most one edge before the aligned body
  const uint2 *tail = nullptr;   // at most one edge after it
};
EdgeSpan split_edges(const uint32_t *edges, uint64_t n_edges);

int num_sms();

// Grid of min(want, cap) blocks (at least one).
inline unsigned clamp_grid(uint64_t want, uint64_t cap) {
  if (want == 0) want = 1;
  return (unsigned)(want < cap ? want : cap);
}

// Sets a kernel attribute once per device. Setting a function attribute can
// make the host wait for the device, so it is done on first use only, never
// per launch; `done` is the call site's per-device bit mask.
inline cudaError_t ensure_func_attr(const void *kernel, cudaFuncAttribute attr, int value,
                                    std::atomic<unsigned long long> &done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, attr, value);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Blocks that fit on the whole GPU at once for this kernel and block size
// (the occupancy query is cached per kernel, block size, shared memory and
// device: it costs microseconds of host time, and launches are frequent).
uint64_t persistent_cap(const void *kernel, int block, size_t smem);

// Process-wide count of kernel launches issued by the library.
void note_launch();
unsigned long long launch_count();

// skip: when not null and the word it points to is nonzero at run time, the
// kernel does nothing (device-side choice between enqueued alternatives).
cudaError_t launch_init(bool rf, uint32_t *P, uint32_t n, Ctrl *ctrl, int m_src, uint32_t m_hint,
                        cudaStream_t s, const uint32_t *skip = nullptr);
// Scratch of the certified exact root selection (cc_rootsel.cu).
constexpr uint32_t kCertCand = 4096;     // more candidates than this: no proof is tried
constexpr uint32_t kCertBuckets = 8192;  // hash buckets of the degree bound
constexpr uint32_t kCertTop = 4;         // candidates whose degree is counted exactly
// The hot-vertex table of the edge pass: per slot (a multiplicative hash of
// the vertex id, kHotBits bits) the vertex with the largest sampled count
// among those with at least 1/256 of the largest, packed (count << 32) |
// (vertex + 1); filled by the candidate scan of the root selection.
constexpr uint32_t kHotBits = 12;
constexpr uint32_t kHot = 1u << kHotBits;
// Listed candidates: the sampled pass lists a vertex when its sampled count
// reaches kListThr, so that the candidate scan reads the list instead of all
// n counters. A vertex left off the list (its count stayed below kListThr, or
// the list was full) is still bounded by its bucket's total in the proof, so
// the list can only make a certificate fail, never make a wrong one.
// The list is cut into kListSegs segments with a counter each (a block
// appends to segment blockIdx % kListSegs), so that appends do not all
// contend on one counter.
constexpr uint32_t kListThr = 8;
constexpr uint32_t kListSegs = 256;
constexpr uint32_t kListCap = 1u << 20;
inline uint32_t cand_list_cap(uint64_t n) {
  const uint64_t c = n < kListCap ? n : kListCap;
  return (uint32_t)((c + kListSegs - 1) / kListSegs * kListSegs);  // whole segments
}
// The sampled passes keep whole groups of kSampleGroup consecutive edges (4
// edges: one 32-byte sector), one group in `stride`. Short groups keep the
// sample an even spread of the array even when the edges come sorted by an
// endpoint, where a long group lies inside one row and gives that row's
// vertex the whole group as sampled count. R-MAT 26 sorted by source: with
// groups of 1024 edges the certificate failed at edge factor 4 (root select
// 0.49 -> 7.2 ms), with groups of 32 at edge factor 16 (1.47 -> 29 ms, the
// fallback histogram's atomics meeting on each row's vertex); groups of 4
// certify both, and random order loses nothing.
constexpr uint32_t kSampleGroupShift = 2;
constexpr uint32_t kSampleGroup = 1u << kSampleGroupShift;
// The sampled pass keeps 1 group in cert_sample_stride(E):
// kCertSample, or E / 2^19 from 2^26 edges up (about 2^19 sampled edges), at
// most 4096 (2^20 sampled edges on R-MAT scale 28). Its random atomics into
// the n counters cost more than the candidates they find need (R-MAT scale
// 28 root select: 1 in 128 7.6 ms, E / 2^23 6.0 ms, this 5.6 ms). A thinner
// sample lists fewer hubs for the hot-vertex table, and the edge pass loses
// more than the root selection gains (R-MAT scale 28 at E / 2^18 with a cap
// of 16384: root select -0.1 ms, edge pass +0.5 ms).
constexpr uint32_t kCertSample = 128;
inline uint32_t cert_sample_stride(uint64_t n_edges) {
  const uint64_t s = n_edges >> 19;
  return s > kCertSample ? (uint32_t)(s < 4096 ? s : 4096) : kCertSample;
}
struct CertScratch {
  unsigned long long owner[kCertBuckets];   // per bucket, its best sampled (count << 32) | ~vertex; 0 = none
  unsigned long long top[kCertTop];         // the best owners, same packing; 0 = empty slot
  unsigned long long top_cnt[kCertTop];     // their exact degrees
  unsigned long long bucket[kCertBuckets];  // endpoint occurrences of all vertices of the bucket
  unsigned long long hot[kHot];             // the hot-vertex table (see kHotBits)
  unsigned int sel_done;                    // candidate-selection blocks finished (the last one ranks)
  unsigned int list_n[kListSegs];           // per list segment, vertices appended (may exceed its room)
  unsigned int blocks_done;                 // counting blocks finished (the last one decides)
  // Initial Push (Algorithm 4): neighbours of the sampled argmax m', appended
  // through kPushLanes counters, each owning a segment of the push buffer
  unsigned int push_cnt[256];
  unsigned int push_m;         // m' + 1 (0: no push list was gathered)
  unsigned int push_overflow;  // a segment filled up: the push is skipped
};
constexpr uint32_t kPushLanes = 256;

// Chunked exact root selection, for edges that arrive in chunks (host input):
// a dense sample of the first chunk picks candidates, and every chunk is
// hooked under a speculative m' as it lands. With a plausible hub, m' is the
// sampled leader and the certificate's counts accumulate per chunk; without
// one, every chunk adds to the full histogram and m' is the first chunk's
// argmax (exact on graphs whose largest degree is reached in their first
// chunk, such as grids stored row by row). After the last chunk the device
// knows the exact m (certificate or histogram): m' == m keeps the hooking,
// otherwise init plus one edge pass over all edges run again. Kernels read
// the Ctrl skip words, so the host enqueues every alternative without waiting.
enum : int {
  kSkipHist = 0,      // nonzero: hub mode (the per-chunk histogram and its argmaxes skip)
  kSkipRerun = 1,     // nonzero: m' was exact (the final init and edge pass skip)
  kSkipFullHist = 2,  // nonzero unless the hub's certificate failed (a full histogram then runs)
};
cudaError_t chunked_select_begin(const uint32_t *chunk0, uint64_t n0, void *cnt, bool wide, uint32_t n,
                                 CertScratch *cs, Ctrl *ctrl, cudaStream_t s);
// first: the chunk given to chunked_select_begin (its argmax is m' without a hub)
cudaError_t chunked_select_chunk(const EdgeSpan &chunk, bool first, void *cnt, bool wide, uint32_t n,
                                 CertScratch *cs, Ctrl *ctrl, cudaStream_t s);
cudaError_t chunked_select_end(const EdgeSpan &all, void *cnt, bool wide, uint32_t n, CertScratch *cs,
                               Ctrl *ctrl, cudaStream_t s);

// Certified exact root selection: sampled candidates, one exact pass over all
// edges counting candidate degrees and bucket totals in shared memory, a
// proof that no other vertex reaches the best candidate's degree, and the
// full histogram as a fallback that runs only when the proof fails.
// cnt holds n counters of 4 bytes (8 when wide); afterwards ctrl->maxkey
// encodes m ((deg << 32) | ~m for the init kernel).
// push_buf (push_cap entries, a multiple of kPushLanes), when not null,
// receives the neighbours of the sampled argmax during the counting pass, for
// launch_initial_push after init. list (list_cap entries), when not null,
// receives the listed candidates (kListThr) and the candidate scan reads it
// instead of the n counters.
cudaError_t launch_root_select_certified(const uint32_t *edges, uint64_t n_edges, const EdgeSpan &e,
                                         void *cnt, bool wide, uint32_t n, CertScratch *cs, Ctrl *ctrl,
                                         cudaStream_t s, uint32_t *push_buf = nullptr, uint32_t push_cap = 0,
                                         uint32_t *list = nullptr, uint32_t list_cap = 0);
// Initial Push (Algorithm 4): right after init, when the planted m is the
// vertex whose neighbours were gathered, every gathered neighbour x != m gets
// P[x] = 0 (name 0 is m): x, still a root, is hooked under m.
cudaError_t launch_initial_push(uint32_t *P, uint32_t n, const uint32_t *push_buf, uint32_t push_cap,
                                const CertScratch *cs, const Ctrl *ctrl, cudaStream_t s);

cudaError_t launch_degree_u32(const EdgeSpan &e, uint32_t *cnt, uint32_t n, cudaStream_t s);
// CSR input (cc_csr.cu): offsets[n + 1], neighbors[n_entries].
uint64_t csr_tiles(uint64_t n_entries);  // entries of tile_row needed
// m = the longest row, smallest id on ties (into ctrl->maxkey); also checks
// the offsets (kErrFormat).
cudaError_t launch_csr_root_select(const uint64_t *off, uint32_t n, uint64_t n_entries, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_csr_check(const uint64_t *off, uint32_t n, uint64_t n_entries, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_edge_pass_csr(bool rf, const uint64_t *off, const uint32_t *nb, uint64_t n_entries, uint32_t n,
                                 uint32_t *tile_row, uint32_t *P, Ctrl *ctrl, cudaStream_t s);
// Unpacks n_edges edges of 3-byte ids (cc_pack.cu; src 16-byte aligned) into
// uint32 pairs at dst (16-byte aligned).
cudaError_t launch_unpack3(const uint8_t *src, uint64_t n_edges, uint32_t *dst, cudaStream_t s);
// track: also put the largest sampled count in the high half of track->maxkey;
// list (list_cap entries, a multiple of kListSegs, with the segment counters
// list_n): list the vertices whose sampled count reaches kListThr.
cudaError_t launch_degree_sampled_u32(const uint2 *edges, uint64_t n_edges, uint64_t edge_base,
                                      uint32_t stride, uint32_t *cnt, uint32_t n, cudaStream_t s,
                                      Ctrl *track = nullptr, uint32_t *list = nullptr,
                                      unsigned int *list_n = nullptr, uint32_t list_cap = 0);
cudaError_t launch_argmax_u32(const uint32_t *cnt, uint32_t n, Ctrl *ctrl, cudaStream_t s);
// Z: the zero-tree bitmap (one bit per name, zeroed at every init), or null.
// With Z and zsel null only the zero-tree instance runs; with both, the device
// picks the zero-tree instance when *zsel is nonzero, the plain one otherwise.
// one_shot: short-lived blocks (a few grid iterations each) instead of a
// persistent grid (for work that shares the GPU with a resident kernel).
// log: a changed-root log (log[0] = entries, then the hooked root names), or
// null.
// hot: the hot-vertex table (CertScratch::hot) of this graph's last root
// selection, for the instances that serve a certified hub, or null.
cudaError_t launch_edge_pass(bool rf, int filter, int ept, int block, const EdgeSpan &e, uint32_t *P,
                             uint32_t n, Ctrl *ctrl, const uint32_t *skip, cudaStream_t s,
                             uint32_t *Z = nullptr, const uint32_t *zsel = nullptr, bool one_shot = false,
                             uint32_t *log = nullptr, const uint32_t *hub = nullptr, bool dyn = false,
                             const unsigned long long *hot = nullptr);
// dyn: warps claim their edges from a counter in ctrl (reset on s before the
// launch), so at most one dynamic edge pass per Ctrl may be in flight.
// Sets *reject (ctrl->reject when null) and the range error bit when an id is >= n.
cudaError_t launch_validate(const EdgeSpan &e, uint32_t n, Ctrl *ctrl, cudaStream_t s, uint32_t *reject = nullptr);
cudaError_t launch_flatten(bool rf, int label_space, uint32_t *P, uint32_t n, uint32_t *L, Ctrl *ctrl,
                           cudaStream_t s);
// Under R: the smallest vertex of m's tree into ctrl->gmin (which must hold m).
cudaError_t launch_gmin_probe(uint32_t *P, uint32_t n, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_count_roots(bool rf, const uint32_t *P, uint32_t n, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_connected(bool rf, uint32_t *P, uint32_t n, const uint2 *pairs, uint64_t n_pairs,
                             uint8_t *out, Ctrl *ctrl, cudaStream_t s);
// The forest of P as edges: for every non-root vertex v, the pair (v, parent
// of v) goes to out[2i], out[2i + 1] for i < cap; ctrl->pairs counts them all
// (reset on s before the launch).
cudaError_t launch_forest_pairs(bool rf, const uint32_t *P, uint32_t n, uint32_t *out, uint64_t cap, Ctrl *ctrl,
                                cudaStream_t s);

}  // namespace cc

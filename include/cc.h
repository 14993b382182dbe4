/*
 * cc.h - C ABI of a GB300 (sm_103a) connected-components library built on
 * Root-Function Jayanti-Tarjan (JT) union-find: one pass over the edges
 * (Algorithm 3, hooking), then a flatten pass that writes the label array L
 * (Algorithm 3, pointer jumping). With f(v) = v this is Algorithm 1; with
 * f = R (Eq. 1) the maximum-degree vertex m is planted as root value 0
 * ("Zero Planting", Section IV), so every vertex of m's component ends with
 * root value 0.
 *
 * Problem statement (Section II, terminology): for an undirected graph
 * G = (V, E) compute L with L_u == L_v iff u and v are in the same component.
 * Edges are unordered pairs; JT needs each edge in one direction only
 * (Section II), so directed COO input is accepted and treated as undirected.
 *
 * Conventions shared by every call
 *  - Vertex ids are uint32 in [0, n_vertices); n_vertices <= 2^31 - 1 so that
 *    the root value v + 1 of Eq. 1 fits the int32 parent array.
 *  - Edge lists are COO pairs interleaved u0, v0, u1, v1, ... (uint32, 8 bytes
 *    per edge). Edge buffers must be at least 8-byte aligned; 16-byte aligned
 *    buffers are read with 128-bit loads. Self-loops and duplicates are allowed.
 *  - "_dev" pointers are device pointers of the handle's device; "_host"
 *    pointers are host memory (pinned memory transfers fastest).
 *  - Ownership: the caller owns every edge, label, query and output buffer and
 *    must keep it alive until the stream has passed the call. The library owns
 *    the parent array P and its scratch, and keeps no caller pointer after the
 *    stream has passed the call.
 *  - Streams: work is enqueued on the caller's stream (NULL = legacy default
 *    stream); calls documented as synchronising wait for it.
 *  - Errors: every call returns a cc_status; nothing aborts, prints or throws
 *    across the ABI. Errors found by kernels (an out-of-range vertex id, an
 *    expired bounded wait) set a sticky device flag that the next
 *    synchronising call (cc_sync, cc_num_components, cc_connected1,
 *    cc_root_vertex, cc_checkpoint, cc_run_host) returns and then clears.
 *  - Threading: one handle is used by one host thread at a time.
 */
#ifndef CC_H
#define CC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CC_API __attribute__((visibility("default")))
#else
#define CC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *cc_stream_t;

typedef struct cc_graph cc_graph;

typedef enum cc_status {
  CC_OK = 0,
  CC_ERR_INVALID_ARGUMENT = 1, /* NULL or misaligned pointer, bad option value   */
  CC_ERR_TOO_LARGE = 2,        /* n_vertices > 2^31 - 1, or a count over capacity */
  CC_ERR_OOM = 3,              /* device allocation failed or HBM budget exceeded */
  CC_ERR_OUT_OF_RANGE = 4,     /* a vertex id >= n_vertices reached a kernel       */
  CC_ERR_TIMEOUT = 5,          /* a bounded device or host wait expired            */
  CC_ERR_CUDA = 6,             /* a CUDA runtime call failed                       */
  CC_ERR_INTERNAL = 7,         /* an internal invariant failed                     */
  CC_ERR_NOT_READY = 8         /* a server request has not completed yet           */
} cc_status;

/* Root function f of Algorithm 3. */
typedef enum cc_root_mode {
  CC_ROOT_IDENTITY = 0, /* f(v) = v: Algorithm 1                                     */
  CC_ROOT_MAXDEG = 1    /* f = R of Eq. 1: R(m) = 0, R(v) = v + 1; inverse Eq. 2    */
} cc_root_mode;

/* How m, the vertex planted as root value 0, is chosen when no hint is given
 * (Algorithm 4, max_degree()). Degree = occurrences as an endpoint (a
 * self-loop counts twice, duplicates count); ties go to the smaller id. */
typedef enum cc_root_select {
  CC_ROOT_SELECT_EXACT = 0,  /* degree histogram over all edges                     */
  CC_ROOT_SELECT_SAMPLED = 1 /* histogram over every k-th group of 4 edges          */
} cc_root_select;

/* Warp-level pre-filter of the edge pass: an edge whose endpoints already
 * hold the same parent value is dropped before any root search; survivors are
 * compacted so that whole warps search roots together.
 *
 * CC_FILTER_BITMAP adds the zero-tree bitmap: one bit per vertex (n / 8
 * bytes of device memory), set once the vertex is known to belong to the tree
 * of root value 0 (the planted vertex m under R; vertex 0 under the identity).
 * The filter then skips the parent load of such an endpoint. It pays off when
 * P is larger than the GPU's L2 and most edges lie in m's component (the
 * skewed graphs that Zero Planting, Section IV, targets). CC_FILTER_AUTO uses
 * it under R with exact root selection when P exceeds 128 MiB, and only on
 * runs whose selection certified a dominant hub (decided on the device). */
typedef enum cc_filter {
  CC_FILTER_AUTO = 0,
  CC_FILTER_ON = 1,
  CC_FILTER_OFF = 2,
  CC_FILTER_BITMAP = 3
} cc_filter;

/* Label written to L. */
typedef enum cc_label_space {
  /* L_v = min { w : w ~ v }: each component is named by its lowest vertex id
   * (Section II). The same in both root modes and for any choice of m. */
  CC_LABEL_MIN_ID = 0,
  /* L_v = min { f(w) : w ~ v }: the value Algorithm 3's pointer jumping leaves
   * in P (f(root)). With f = R this is 0 for m's component and min id + 1
   * otherwise. */
  CC_LABEL_ROOT_VALUE = 1
} cc_label_space;

/* Initial Push (Algorithm 4, Section IV): before the edge pass, every
 * neighbour of the planted vertex m is hooked directly under it (root value
 * 0), so that the pass starts with m's star formed. Only with f = R and
 * automatic exact root selection: the neighbours of the sampled argmax m' are
 * gathered by the selection's counting pass (no extra read of the edges) and
 * pushed only when m' turns out to be the exact m. The gathered list takes up
 * to min(n, 2^23) * 4 bytes of device memory; a longer list skips the push. */
typedef enum cc_initial_push {
  CC_PUSH_AUTO = 0, /* the library's choice: off (it paid only on some graphs) */
  CC_PUSH_ON = 1,
  CC_PUSH_OFF = 2
} cc_initial_push;

#define CC_ROOT_AUTO UINT64_MAX

typedef struct cc_options {
  int32_t mode;              /* cc_root_mode, default CC_ROOT_MAXDEG              */
  int32_t root_select;       /* cc_root_select, default CC_ROOT_SELECT_EXACT      */
  uint64_t root_hint;        /* vertex to plant as m, or CC_ROOT_AUTO (default)   */
  int32_t filter;            /* cc_filter, default CC_FILTER_AUTO                 */
  int32_t label_space;       /* cc_label_space, default CC_LABEL_MIN_ID           */
  int32_t block_size;        /* edge-pass threads per block (128, 256, 512); 0 = 512 */
  int32_t edges_per_thread;  /* edges per thread per iteration (2, 4 or 8); 0 = auto */
  int32_t sample_stride;     /* sampled root select keeps 1 group in k; 0 = 16     */
  int32_t timing;            /* nonzero: record per-phase times (cc_phase_times)  */
  uint64_t hbm_budget_bytes; /* device bytes the handle may own; 0 = free memory  */
  int32_t initial_push;      /* cc_initial_push, default CC_PUSH_AUTO              */
  int32_t reserved32;        /* must be zero                                       */
  uint64_t reserved[3];      /* must be zero                                       */
} cc_options;

/* Fills *opt with the defaults above. */
CC_API void cc_options_init(cc_options *opt);

/* Creates a handle on the current CUDA device for a graph on n_vertices
 * vertices and allocates the parent array P (int32[n_vertices]) and scratch
 * (the root-select histogram in CC_ROOT_MAXDEG mode). n_edges_capacity sizes
 * the device staging buffer of cc_run_host (0 = none: cc_run_host then fails
 * with CC_ERR_TOO_LARGE). P starts as the edgeless graph: P_v = f(v)
 * (Algorithm 3, initialisation), with m = root_hint, or 0 when the hint is
 * CC_ROOT_AUTO, until a cc_run selects m.
 * Errors: CC_ERR_INVALID_ARGUMENT (out == NULL, bad option),
 * CC_ERR_TOO_LARGE (n_vertices > 2^31 - 1), CC_ERR_OOM (over the budget or
 * allocation failure). On error *out is NULL. */
CC_API cc_status cc_create(uint64_t n_vertices, uint64_t n_edges_capacity, const cc_options *opt,
                    cc_graph **out);

/* Full computation on a device-resident edge list: root selection (f = R
 * only; Algorithm 4, max_degree()), initialisation P_v = f(v), one hooking
 * pass over the n_edges pairs (Algorithm 3: find both roots, link the root of
 * larger f under the root of smaller f with a CAS, retry from the current
 * roots on failure; finds use path splitting), then the flatten pass
 * (Algorithm 3, pointer jumping), which compresses P to root values and, when
 * L_out_dev is not NULL, writes uint32[n_vertices] labels in the handle's
 * label space. Stream-ordered; returns once the work is enqueued.
 * An id >= n_vertices skips that edge and sets CC_ERR_OUT_OF_RANGE for the
 * next synchronising call; the labels are then undefined.
 * CUDA graphs: a call may allocate scratch the first time the handle sees an
 * edge count of its size class (below or from 2^31 edges); after that, a call
 * with the same buffers enqueues only stream work (kernels and memsets) and
 * can be captured into a CUDA graph. Each replay reads the captured edge
 * buffer as it is at replay time and rewrites P and the labels. */
CC_API cc_status cc_run(cc_graph *g, const uint32_t *edges_dev, uint64_t n_edges, uint32_t *L_out_dev,
                 cc_stream_t stream);

/* cc_run on CSR input, the layout the paper's implementation keeps in memory
 * (Section V): offsets_dev[n_vertices + 1] (uint64, offsets_dev[0] = 0,
 * never decreasing, offsets_dev[n_vertices] = n_entries) and
 * neighbors_dev[n_entries] (uint32). The edges are (u, neighbors_dev[j]) for
 * offsets_dev[u] <= j < offsets_dev[u + 1]; the graph need not be symmetric
 * (Section II). Under f = R with automatic selection, m is the vertex with the
 * longest row (the degree that Algorithm 4's max_degree() reads from the
 * offsets), ties to the smaller id. The edge pass walks the neighbor array in
 * order, so the entries of one row share the parent load of their row.
 * Stream-ordered; malformed offsets are reported as CC_ERR_INVALID_ARGUMENT
 * and a neighbor id >= n_vertices as CC_ERR_OUT_OF_RANGE at the next
 * synchronising call (the labels are then undefined). Allocates 4 bytes per
 * 1024 entries on the first call of a larger size. */
CC_API cc_status cc_run_csr(cc_graph *g, const uint64_t *offsets_dev, const uint32_t *neighbors_dev,
                     uint64_t n_entries, uint32_t *L_out_dev, cc_stream_t stream);

/* cc_run on host buffers: copies the n_edges pairs (n_edges <= the handle's
 * n_edges_capacity) to the device in chunks of 2^24 edges and works on each
 * chunk as it lands: with m known in advance (identity, or a hint) the edge
 * pass; with exact selection, hooking under a speculative m' taken from the
 * first chunk (the sampled leader when a hub shows, else the first chunk's
 * argmax) while the certificate's or the histogram's counts accumulate, then
 * one more init + edge pass only if m' was not the exact m; with sampled
 * selection, nothing until the last chunk. The labels go to L_out_host
 * (uint32[n_vertices], may be NULL). Synchronising: returns after the labels
 * are in host memory, with any device error. */
CC_API cc_status cc_run_host(cc_graph *g, const uint32_t *edges_host, uint64_t n_edges,
                      uint32_t *L_out_host, cc_stream_t stream);

/* cc_run_host without the final wait: returns once every copy and kernel is
 * enqueued on `stream` (argument errors are still returned at once). The
 * caller keeps edges_host unchanged and does not read L_out_host until a
 * synchronising call on the handle (cc_sync) has returned; that call
 * reports any device error. Several handles, each on its own stream, then
 * overlap one graph's copies with another's kernels and label read-back. */
CC_API cc_status cc_run_host_async(cc_graph *g, const uint32_t *edges_host, uint64_t n_edges,
                            uint32_t *L_out_host, cc_stream_t stream);

/* cc_run_host on compactly encoded edges (Section V sends ids in the fewest
 * whole bytes that hold them): each id takes id_bytes little-endian bytes,
 * an edge is u then v, 2 * id_bytes bytes per edge, no padding. id_bytes is
 * 3 (requires n_vertices <= 2^24) or 4 (the layout of cc_run_host). The
 * packed bytes cross the host link; each chunk is unpacked on the device into
 * the staging buffer, and the work of cc_run_host follows. The unpacking uses
 * two device buffers of 2^24 packed edges each, allocated at the first call.
 * CC_ERR_INVALID_ARGUMENT for another id_bytes or n_vertices > 2^24 with 3. */
CC_API cc_status cc_run_host_packed(cc_graph *g, const uint8_t *edges_host, uint64_t n_edges, int32_t id_bytes,
                             uint32_t *L_out_host, cc_stream_t stream);

/* cc_run_host_packed without the final wait, as cc_run_host_async. */
CC_API cc_status cc_run_host_packed_async(cc_graph *g, const uint8_t *edges_host, uint64_t n_edges,
                                   int32_t id_bytes, uint32_t *L_out_host, cc_stream_t stream);

/* Incremental union: applies n_edges new pairs to the live P without
 * re-initialisation, exactly as the edge pass does (JT processes edges in any
 * order, so P after the batch equals P of a pass over all edges seen so far;
 * compare the Reducer of Section III, which treats received pairs as edges).
 * The batch is validated first: if any id is >= n_vertices, P is left
 * unchanged and CC_ERR_OUT_OF_RANGE is reported at the next synchronising
 * call. Labels go stale until cc_labels. Stream-ordered. */
CC_API cc_status cc_stream_insert(cc_graph *g, const uint32_t *edges_dev, uint64_t n_edges,
                           cc_stream_t stream);

/* Flatten pass over the live P (Algorithm 3, pointer jumping) writing
 * uint32[n_vertices] labels to L_out_dev in the handle's label space.
 * Stream-ordered. */
CC_API cc_status cc_labels(cc_graph *g, uint32_t *L_out_dev, cc_stream_t stream);

/* Batched queries on the live P: out_dev[i] = 1 if pairs_dev[2i] and
 * pairs_dev[2i+1] have the same root (u and v are connected iff their labels
 * are equal, Section II), else 0. Each query does two root searches. An id
 * >= n_vertices yields 0 and sets CC_ERR_OUT_OF_RANGE. Stream-ordered. */
CC_API cc_status cc_connected(cc_graph *g, const uint32_t *pairs_dev, uint64_t n_pairs, uint8_t *out_dev,
                       cc_stream_t stream);

/* The forest of the live P as edges, for a Reducer (Section III: each
 * machine, after processing its share of the edges, sends the pairs
 * (v, P_v) with P_v != f(v) to the Reducer, which processes them like graph
 * edges and finishes with pointer jumping; Algorithm 2). For every non-root
 * vertex v the pair (v, parent of v) is written to pairs_dev as COO
 * (uint32[2 * count], 8-byte aligned, in no particular order), so the pairs
 * have exactly the components of the edges applied so far and can be given
 * to cc_run or cc_stream_insert of another handle. After cc_labels (which
 * compresses P) every pair names the root directly. At most `capacity` pairs
 * are written; *count receives the number of non-root vertices
 * (n_vertices - cc_num_components), and CC_ERR_TOO_LARGE is returned when it
 * exceeds capacity (call again with a larger buffer). Synchronising; also
 * reports earlier device errors. */
CC_API cc_status cc_forest_pairs(cc_graph *g, uint32_t *pairs_dev, uint64_t capacity, uint64_t *count,
                                 cc_stream_t stream);

/* One query, synchronising: *out = 1 if u and v are connected, else 0. */
CC_API cc_status cc_connected1(cc_graph *g, uint64_t u, uint64_t v, int *out);

/* Number of components of all edges applied so far: the number of roots of
 * P (vertices with P_v == f(v)). Synchronising. */
CC_API cc_status cc_num_components(cc_graph *g, uint64_t *out);

/* The planted vertex m (CC_ROOT_MAXDEG), or CC_ROOT_AUTO in identity mode.
 * Synchronising. */
CC_API cc_status cc_root_vertex(cc_graph *g, uint64_t *m);

/* Waits for the handle's work on the stream of its last call and returns the
 * first error found since the previous synchronising call. */
CC_API cc_status cc_sync(cc_graph *g);

/* Per-phase device times in milliseconds of the last cc_run when the handle
 * was created with timing != 0: [0] root selection, [1] initialisation,
 * [2] edge pass, [3] flatten (including the min-id probe), [4] total.
 * Synchronising. */
CC_API cc_status cc_phase_times(cc_graph *g, float ms[5]);

/* Sum of the per-phase times (same layout as cc_phase_times) over every
 * cc_run since the previous call of this function, on a handle created with
 * timing != 0; *runs receives how many runs were summed. Synchronising. */
CC_API cc_status cc_phase_times_total(cc_graph *g, float ms[5], uint64_t *runs);

/* Number of CUDA kernels this library has launched in this process (all
 * handles); lets a caller count the device work of a region of its own. */
CC_API uint64_t cc_kernel_launches(void);

/* Checkpoint of the whole JT state (P, m, mode): any intermediate P is a
 * valid forest, so restoring it and inserting more edges continues the same
 * computation. cc_checkpoint_size gives the byte count; cc_checkpoint copies
 * to host_buf (synchronising); cc_restore loads a checkpoint taken from a
 * handle with the same n_vertices and mode (else CC_ERR_INVALID_ARGUMENT). */
CC_API cc_status cc_checkpoint_size(const cc_graph *g, uint64_t *bytes);
CC_API cc_status cc_checkpoint(cc_graph *g, void *host_buf, uint64_t bytes);
CC_API cc_status cc_restore(cc_graph *g, const void *host_buf, uint64_t bytes);

/* Device bytes owned by the handle. */
CC_API cc_status cc_device_bytes(const cc_graph *g, uint64_t *bytes);

/* Largest vertex count cc_max_degree_vertex_noalloc accepts. */
#define CC_NOALLOC_MAX_VERTICES (1u << 22)

/* The maximum-degree vertex of an edge list, for callers that cannot allocate
 * device memory. The paper has no counterpart: it is this library's root
 * selection (degree = occurrences as an endpoint, a self-loop counts twice,
 * ties to the smaller id; the same answer as cc_root_vertex after a cc_run in
 * CC_ROOT_MAXDEG mode with exact selection) with no handle and no
 * cudaMalloc. It is meant for code that must not allocate: code running
 * inside another framework's allocator or pool callbacks, services whose
 * device memory is fixed at start-up, and code that cannot afford the device
 * synchronisation cudaMalloc/cudaFree may cause.
 *  - In: edges_dev, n_edges COO pairs (8-byte aligned; ids >= n_vertices are
 *    not counted), n_vertices in [1, CC_NOALLOC_MAX_VERTICES], n_edges < 2^31.
 *  - Out: *m_out_dev (one uint32 in device memory, 4-byte aligned), written
 *    on `stream`; the call is stream-ordered and returns once enqueued.
 *  - Scratch: a fixed static device array inside the library (about 16 MiB
 *    per GPU that loads the library, held until the process exits). The first
 *    call on a device looks up its address (cudaGetSymbolAddress); make that
 *    first call before any stream capture. The address is kept per device and
 *    context: the first call after cudaDeviceReset looks it up again. All
 *    calls share the array and each clears what it uses, so calls whose work
 *    overlaps on the GPU race: serialise them (one stream, or events).
 * Errors: CC_ERR_INVALID_ARGUMENT (NULL or misaligned pointer, n_vertices 0),
 * CC_ERR_TOO_LARGE (n_vertices or n_edges over the limits), CC_ERR_CUDA. */
CC_API cc_status cc_max_degree_vertex_noalloc(const uint32_t *edges_dev, uint64_t n_edges,
                                              uint64_t n_vertices, uint32_t *m_out_dev,
                                              cc_stream_t stream);

/* Frees the handle after waiting for its work. NULL is ignored. */
CC_API void cc_destroy(cc_graph *g);

/* Static description of a status code. */
CC_API const char *cc_status_string(cc_status s);

#ifdef __cplusplus
}
#endif

#endif /* CC_H */

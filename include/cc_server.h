/*
 * cc_server.h - a serving runtime for many resident graphs (C ABI;
 * conventions as in cc.h).
 *
 * Requests arrive at any time: new whole graphs, edge-insert batches,
 * batches of connected(u, v) queries, label snapshots, and graph drops.
 * Each resident graph keeps its parent array P live on the device, so an
 * insert is one hooking pass over the new edges only (JT processes edges in
 * any order and needs no re-initialisation; Section III treats received
 * pairs the same way), and a query batch is two root searches per pair on
 * the live P (u and v are connected iff their roots agree, Section II).
 *
 * Execution. Insert and query batches are cut into tiles and run by a
 * persistent executor kernel that stays resident on a fixed share of every
 * SM, takes tiles from a ring in mapped host memory and signals each request's
 * completion through mapped memory; every wait in it is bounded, and it
 * leaves after an idle period (it is relaunched on demand). New graphs (root
 * selection, init, hooking pass, flatten) and snapshots (flatten) run on a
 * side stream beside the executor; the executor asks for the largest shared
 * memory carveout so that they fit beside it, and side work that still waits
 * longer than 20 ms makes the host drain the executor (it finishes every
 * published tile, leaves, and is relaunched). A host scheduler thread admits
 * requests as memory and ordering allow (continuous batching): requests that
 * arrive while others run start as soon as they may, and their tiles
 * interleave with the running ones on the device.
 *
 * Ordering. Per graph, requests take effect in submission order: a query or
 * snapshot sees exactly the inserts submitted before it for that graph.
 * Consecutive inserts run together, and so do consecutive reads (queries
 * and snapshots). A snapshot reads a copy of the graph's parent array taken
 * when it starts (one device copy of 4 bytes per vertex), so inserts
 * submitted after it start as soon as that copy has run, while the snapshot
 * still computes its labels; one snapshot per graph computes at a time.
 *
 * Memory. The server owns one device arena of hbm_budget_bytes, allocated at
 * creation; graphs are placed in it by first fit and a new graph waits until
 * enough memory is free (drops release it). No cudaMalloc or cudaFree happens
 * while serving. Request buffers (edges, pairs, outputs) are the caller's
 * device memory: their contents must be complete on the device when the
 * request is submitted (the server's streams do not wait for the caller's),
 * and they must stay valid until the request completes. Outputs are complete
 * in device memory when the ticket completes.
 *
 * Module loading. The executor stays resident while requests are in flight.
 * With CUDA's lazy module loading, the first launch of any kernel in the
 * process can wait until the device is idle, so cc_server_create runs every
 * kernel the server uses once before the executor starts. Other code that
 * launches kernels for the first time while a server is busy may wait until
 * it goes idle; such processes should load eagerly
 * (CUDA_MODULE_LOADING=EAGER) or warm those kernels up before serving.
 */
#ifndef CC_SERVER_H
#define CC_SERVER_H

#include "cc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_server cc_server;

typedef enum cc_request_kind {
  CC_REQ_NEW_GRAPH = 1,  /* n_vertices, edges_dev/n_edges; labels_dev optional */
  CC_REQ_INSERT = 2,     /* graph, edges_dev/n_edges; rejected whole if an id is out of range */
  CC_REQ_QUERY = 3,      /* graph, pairs_dev/n_pairs -> out_dev (uint8 per pair) */
  CC_REQ_SNAPSHOT = 4,   /* graph -> labels_dev (uint32[n_vertices], label space of the config) */
  CC_REQ_DROP_GRAPH = 5  /* graph: frees its memory after the requests before it */
} cc_request_kind;

typedef struct cc_request {
  int32_t kind;               /* cc_request_kind */
  uint32_t graph;             /* target graph (not used by CC_REQ_NEW_GRAPH) */
  uint64_t n_vertices;        /* CC_REQ_NEW_GRAPH */
  const uint32_t *edges_dev;  /* COO pairs, 8-byte aligned */
  uint64_t n_edges;
  const uint32_t *pairs_dev;  /* query pairs, 8-byte aligned */
  uint64_t n_pairs;
  uint8_t *out_dev;           /* query results */
  uint32_t *labels_dev;       /* snapshot labels (or NEW_GRAPH labels when not NULL) */
} cc_request;

typedef struct cc_server_config {
  uint64_t hbm_budget_bytes;       /* device arena for resident graphs (required)   */
  uint32_t max_graphs;             /* graph ids 0 .. max_graphs-1; 0 = 1024          */
  uint32_t executor_blocks_per_sm; /* resident executor blocks (256 threads); 0 = 3, which
                                      leaves room on every SM for the side-stream kernels */
  uint32_t tile_edges;             /* largest executor tile in edges or pairs; 0 = 16384;
                                      requests are cut finer to spread over all blocks */
  uint32_t idle_timeout_us;        /* executor leaves after this much idleness; 0 = 20000 */
  int32_t mode;                    /* cc_root_mode of new graphs; default CC_ROOT_MAXDEG */
  int32_t label_space;             /* cc_label_space of snapshots; default MIN_ID   */
  /* Bounded waits of the executor (at most 600 s each). publish_wait_us: how
   * long an executor block waits for a tile it has claimed but the host has
   * not published; expiry makes the executor leave (the host then fails the
   * requests in flight with CC_ERR_TIMEOUT, counts executor_timeouts and
   * relaunches it for later requests); 0 = 30 s. Keep it above the idle
   * timeout: an idle executor is asked to leave before its waits expire,
   * whereas blocks whose wait expired while idle cannot take tiles published
   * just then (those requests would fail the same way). gate_wait_us: how long an
   * insert's apply tile waits for the request's validate tiles; expiry fails
   * the insert with CC_ERR_TIMEOUT, and apply tiles that had already passed
   * the gate stay applied (a subset of a valid batch: P is still a forest
   * of the graph's edges plus some of the batch); 0 = 2 s. */
  uint32_t publish_wait_us;
  uint32_t gate_wait_us;
  /* Fault injection for tests (a stuck producer): the first executor request
   * has its tiles written to the ring but published only this long later, so
   * an executor whose publish wait is shorter gives up on it. 0 = off. */
  uint32_t fault_hold_publish_us;
  int32_t reserved[1];             /* must be zero */
} cc_server_config;

typedef struct cc_server_stats {
  uint64_t submitted, completed, failed;
  uint64_t resident_graphs, arena_bytes_used, arena_bytes;
  uint64_t executor_launches, tiles_run;
  uint64_t side_drains;  /* executor drains forced by starved side-stream work */
  uint64_t executor_timeouts;  /* executor launches that ended on an expired publish wait */
  uint64_t snapshot_overlaps;  /* inserts started while a snapshot of their graph still computed */
} cc_server_stats;

CC_API void cc_server_config_init(cc_server_config *cfg);

/* Creates the server on the current device: allocates the arena and the
 * executor's rings, starts the scheduler thread. */
CC_API cc_status cc_server_create(const cc_server_config *cfg, cc_server **out);

/* Queues a request and returns its ticket at once. For CC_REQ_NEW_GRAPH the
 * new graph's id is available immediately through cc_server_result_graph and
 * may be used by requests submitted right after. Host-side argument errors
 * are returned here (CC_ERR_INVALID_ARGUMENT, CC_ERR_TOO_LARGE when a graph
 * can never fit the arena); device-side ones through the ticket. */
CC_API cc_status cc_server_submit(cc_server *s, const cc_request *req, uint64_t *ticket);

/* Queues reqs[0 .. count) in order, as count calls of cc_server_submit would,
 * but under one lock and with one wake-up of the scheduler. Stops at the
 * first request that fails its host-side checks: *n_queued requests were
 * queued (tickets[0 .. *n_queued) are theirs) and the refused request's
 * status is returned; CC_OK when all were queued. Requests of one call keep
 * their order, so per-graph submission order holds across the batch.
 * Errors: CC_ERR_INVALID_ARGUMENT (NULL pointers with count > 0, a closing
 * server), and the per-request errors of cc_server_submit. */
CC_API cc_status cc_server_submit_many(cc_server *s, const cc_request *reqs, uint32_t count,
                                       uint64_t *tickets, uint32_t *n_queued);

/* CC_OK with *result = the request's status when it has completed,
 * CC_ERR_NOT_READY otherwise. */
CC_API cc_status cc_server_poll(cc_server *s, uint64_t ticket, cc_status *result);

/* Waits up to timeout_ns for the ticket; CC_ERR_TIMEOUT if it has not
 * completed by then. */
CC_API cc_status cc_server_wait(cc_server *s, uint64_t ticket, uint64_t timeout_ns, cc_status *result);

CC_API cc_status cc_server_result_graph(cc_server *s, uint64_t ticket, uint32_t *graph);

/* Submission-to-completion time of a completed ticket (host clock). */
CC_API cc_status cc_server_latency_ns(cc_server *s, uint64_t ticket, uint64_t *ns);

CC_API cc_status cc_server_get_stats(cc_server *s, cc_server_stats *st);

/* Waits for the requests still running (at most about 10 s), stops the
 * executor and frees everything. */
CC_API void cc_server_destroy(cc_server *s);

#ifdef __cplusplus
}
#endif

#endif /* CC_SERVER_H */

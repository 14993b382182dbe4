/*
 * cc_batch.h - connected components of many independent graphs in one
 * launch (C ABI; conventions as in cc.h).
 *
 * Graph g owns vertices [vtx_off[g], vtx_off[g+1]) and edges
 * [edge_off[g], edge_off[g+1]) of one concatenated edge list whose ids are
 * graph-local (0 .. |V_g| - 1). The result is, for every vertex i of graph g,
 * L[vtx_off[g] + i] = the smallest graph-local id of i's component: the
 * min-id labels of Section II for each graph separately.
 *
 * Method: Algorithm 1 (Root-Function JT with f(v) = v) on the union of all
 * graphs, whose vertex sets occupy disjoint ranges of one name space, so the
 * forests of different graphs never meet. One cooperative persistent kernel
 * runs the phases (tile offsets, initialisation, hooking over edge tiles that
 * each lie inside one graph, compression, local labels) separated by grid
 * barriers whose waits are bounded; the label array doubles as the parent
 * array, so a run allocates nothing. The launch can be captured in a CUDA
 * graph. The tile size, block size, edges per thread and the warp filter are
 * chosen by cc_batch_tune.
 */
#ifndef CC_BATCH_H
#define CC_BATCH_H

#include "cc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_batch cc_batch;

/* A new context starts with 512 threads, 1 edge per thread, the filter on,
 * tiles of 8192 edges and 4096 vertices (the best measured on a mixed batch of
 * 4096 graphs); cc_batch_tune times every block size x edges per thread x
 * filter x tile of 4096, 8192, 16384 or 65536 edges. */
typedef struct cc_batch_config {
  int32_t block_size;       /* 256 or 512 */
  int32_t edges_per_thread; /* 1, 2 or 4 per round */
  int32_t filter;           /* 1: warp filter + compaction, 0: per-lane */
  uint32_t tile_edges;      /* edges per hooking tile (one warp's unit of work), a multiple of 256, >= 256 */
  uint32_t tile_vertices;   /* vertices per tile of the label phase, >= 256 */
  uint32_t barrier_wait_us; /* bounded wait of each grid barrier, at most 60 s; 0 = 4 s. A
                               wait that expires aborts the run (every block leaves at its
                               next barrier; the labels are then undefined) and cc_batch_sync
                               returns CC_ERR_TIMEOUT; the next run starts afresh. The
                               autotuner keeps the context's value */
  int32_t reserved[2];      /* must be zero */
} cc_batch_config;

/* A batch context for up to max_graphs graphs per call: its tile-offset
 * scratch (16 bytes per graph) and control block. */
CC_API cc_status cc_batch_create(uint32_t max_graphs, cc_batch **out);

/* Labels of n_graphs graphs (n_graphs <= max_graphs). vtx_off_dev and
 * edge_off_dev are uint64[n_graphs + 1] device arrays, nondecreasing, starting
 * at 0; the total vertex count must be <= 2^31 - 1. edges_dev holds
 * edge_off[n_graphs] pairs (8-byte aligned); L_out_dev holds vtx_off[n_graphs]
 * uint32 and receives graph-local min-id labels. Stream-ordered, no host
 * synchronisation, capturable in a CUDA graph. A graph-local id >= |V_g| skips
 * its edge and sets CC_ERR_OUT_OF_RANGE; malformed offsets stop the run with
 * CC_ERR_INVALID_ARGUMENT; both are reported by cc_batch_sync. */
CC_API cc_status cc_run_batched(cc_batch *b, uint32_t n_graphs, const uint64_t *vtx_off_dev,
                                const uint64_t *edge_off_dev, const uint32_t *edges_dev,
                                uint32_t *L_out_dev, cc_stream_t stream);

/* Autotuner: runs cc_run_batched on the given batch under each candidate
 * configuration (block size x edges per thread x filter x tile size), keeps
 * the fastest in the context and returns it with its time in ms.
 * Synchronising; overwrites L_out_dev. */
CC_API cc_status cc_batch_tune(cc_batch *b, uint32_t n_graphs, const uint64_t *vtx_off_dev,
                               const uint64_t *edge_off_dev, const uint32_t *edges_dev,
                               uint32_t *L_out_dev, cc_stream_t stream, cc_batch_config *best,
                               float *best_ms);

/* The candidates timed by the last cc_batch_tune on this context, in the
 * order tried, each with its best time in ms (the spread between them shows
 * how decisive the choice was). Copies min(cap, count) entries; *count
 * receives how many there are (0 before any tuning). Not synchronising. */
CC_API cc_status cc_batch_tune_results(const cc_batch *b, cc_batch_config *cfgs, float *ms, uint32_t cap,
                                       uint32_t *count);

CC_API cc_status cc_batch_set_config(cc_batch *b, const cc_batch_config *cfg);
CC_API cc_status cc_batch_get_config(const cc_batch *b, cc_batch_config *cfg);

/* Waits for the context's last stream and returns the first error found by
 * its kernels since the previous call. */
CC_API cc_status cc_batch_sync(cc_batch *b);

CC_API void cc_batch_destroy(cc_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* CC_BATCH_H */

/*
 * cc_oracle.c - the CPU oracle for connected-components labels.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may load this code; the library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Plain, sequential, single-threaded C. What it computes:
 *
 *  - min-id labels (Section II, "Terminology": L_u = L_v iff u and v lie in
 *    the same component; the JT description in Section II identifies each
 *    component by the lowest id of its vertices). Written out directly:
 *    L[v] = min { w : w ~ v }, where ~ is the equivalence closure of the edge
 *    set taken as unordered pairs. The closure is built by a textbook
 *    sequential union-find in which the smaller root always becomes the
 *    parent, so the root of each class is its minimum (oracle_uf_*), and
 *    independently by breadth-first search in increasing start order
 *    (oracle_bfs_labels; Section II, related work, search-based CC);
 *  - root-value labels of Root-Function JT (Algorithm 3, final pointer
 *    jumping writes the root's value): L[v] = min { R(w) : w ~ v } with R from
 *    Eq. 1 (R(m) = 0, R(v) = v + 1 otherwise);
 *  - the maximum-degree vertex m (Algorithm 4, max_degree(); Section IV):
 *    deg(x) = number of times x occurs as an endpoint (a self-loop counts
 *    twice, duplicates count), ties broken towards the smaller id;
 *  - sequential Algorithm 1 / Algorithm 3 hooking and pointer jumping,
 *    step for step, for the worked example of Fig. 1 and as a cross-check.
 *
 * Every function returns a negative value when an id is out of range.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ union-find
 * Sequential union-find over parent[]: find follows parents with path halving
 * (parent[x] <- parent[parent[x]]), union makes the smaller of the two roots
 * the parent of the larger. The smallest vertex of a class is never given a
 * parent, so it is the root of its class: find(v) = min { w : w ~ v }. */
typedef struct oracle_uf {
  uint64_t n;
  uint32_t *parent;
} oracle_uf;

static uint32_t uf_find(uint32_t *parent, uint32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

ORACLE_EXPORT oracle_uf *oracle_uf_new(uint64_t n) {
  oracle_uf *h = (oracle_uf *)malloc(sizeof(oracle_uf));
  if (!h) return NULL;
  h->n = n;
  h->parent = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!h->parent) {
    free(h);
    return NULL;
  }
  for (uint64_t v = 0; v < n; ++v) h->parent[v] = (uint32_t)v;
  return h;
}

ORACLE_EXPORT void oracle_uf_free(oracle_uf *h) {
  if (!h) return;
  free(h->parent);
  free(h);
}

/* Adds n_edges pairs (edges[2i], edges[2i+1]); returns 0, or -1 if an id is
 * >= n (nothing after the bad pair is added). */
ORACLE_EXPORT int oracle_uf_add(oracle_uf *h, const uint32_t *edges, uint64_t n_edges) {
  uint32_t *parent = h->parent;
  for (uint64_t i = 0; i < n_edges; ++i) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a >= h->n || b >= h->n) return -1;
    uint32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra < rb)
      parent[rb] = ra;
    else if (rb < ra)
      parent[ra] = rb;
  }
  return 0;
}

/* L[v] = min { w : w ~ v } over the pairs added so far. */
ORACLE_EXPORT void oracle_uf_min_labels(oracle_uf *h, uint32_t *L) {
  for (uint64_t v = 0; v < h->n; ++v) L[v] = uf_find(h->parent, (uint32_t)v);
}

ORACLE_EXPORT int oracle_min_labels(uint64_t n, const uint32_t *edges, uint64_t n_edges,
                                    uint32_t *L) {
  oracle_uf *h = oracle_uf_new(n);
  if (!h) return -2;
  int rc = oracle_uf_add(h, edges, n_edges);
  if (rc == 0) oracle_uf_min_labels(h, L);
  oracle_uf_free(h);
  return rc;
}

/* ------------------------------------------------------------ root function R
 * Eq. 1: R(v) = 0 if v is the planted vertex m, v + 1 otherwise. */
static uint64_t R_of(uint64_t v, uint64_t m) { return v == m ? 0 : v + 1; }

/* L[v] = min { R(w) : w ~ v }: the same union-find, but the root of larger R
 * value is the one given a parent, so each class's root is its R-minimum. */
ORACLE_EXPORT int oracle_root_value_labels(uint64_t n, const uint32_t *edges,
                                           uint64_t n_edges, uint64_t m, uint32_t *L) {
  if (n == 0) return 0;
  if (m >= n) return -1;
  uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * n);
  if (!parent) return -2;
  for (uint64_t v = 0; v < n; ++v) parent[v] = (uint32_t)v;
  for (uint64_t i = 0; i < n_edges; ++i) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a >= n || b >= n) {
      free(parent);
      return -1;
    }
    uint32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) continue;
    if (R_of(ra, m) < R_of(rb, m))
      parent[rb] = ra;
    else
      parent[ra] = rb;
  }
  for (uint64_t v = 0; v < n; ++v) L[v] = (uint32_t)R_of(uf_find(parent, (uint32_t)v), m);
  free(parent);
  return 0;
}

/* ------------------------------------------------------------------------ BFS
 * Search-based CC: build the symmetric adjacency (each pair in both
 * directions, self-loops dropped), then visit vertices in increasing id order;
 * each vertex not yet reached starts a BFS and every vertex that BFS reaches
 * is labelled with the start. All smaller vertices were visited before, so the
 * start is the minimum of its component. */
ORACLE_EXPORT int oracle_bfs_labels(uint64_t n, const uint32_t *edges, uint64_t n_edges,
                                    uint32_t *L) {
  if (n == 0) return 0;
  uint64_t *off = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  if (!off) return -2;
  for (uint64_t i = 0; i < n_edges; ++i) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a >= n || b >= n) {
      free(off);
      return -1;
    }
    if (a == b) continue;
    off[a + 1]++;
    off[b + 1]++;
  }
  for (uint64_t v = 0; v < n; ++v) off[v + 1] += off[v];
  uint32_t *adj = (uint32_t *)malloc(sizeof(uint32_t) * (off[n] ? off[n] : 1));
  uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * n);
  uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * n);
  if (!adj || !fill || !queue) {
    free(off);
    free(adj);
    free(fill);
    free(queue);
    return -2;
  }
  memcpy(fill, off, sizeof(uint64_t) * n);
  for (uint64_t i = 0; i < n_edges; ++i) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a == b) continue;
    adj[fill[a]++] = b;
    adj[fill[b]++] = a;
  }
  const uint32_t UNSEEN = 0xFFFFFFFFu;
  for (uint64_t v = 0; v < n; ++v) L[v] = UNSEEN;
  for (uint64_t s = 0; s < n; ++s) {
    if (L[s] != UNSEEN) continue;
    uint64_t head = 0, tail = 0;
    L[s] = (uint32_t)s;
    queue[tail++] = (uint32_t)s;
    while (head < tail) {
      uint32_t x = queue[head++];
      for (uint64_t k = off[x]; k < off[x + 1]; ++k) {
        uint32_t y = adj[k];
        if (L[y] == UNSEEN) {
          L[y] = (uint32_t)s;
          queue[tail++] = y;
        }
      }
    }
  }
  free(off);
  free(adj);
  free(fill);
  free(queue);
  return 0;
}

/* ------------------------------------------------------------- degree argmax
 * deg[x] = occurrences of x as an endpoint; returns the smallest x with the
 * largest deg[x] (0 for an edgeless graph), or -1 for an out-of-range id.
 * deg_out, when not NULL, receives the n counts. */
ORACLE_EXPORT int64_t oracle_max_degree_vertex(uint64_t n, const uint32_t *edges,
                                               uint64_t n_edges, uint64_t *deg_out) {
  if (n == 0) return -1;
  uint64_t *deg = (uint64_t *)calloc(n, sizeof(uint64_t));
  if (!deg) return -2;
  for (uint64_t i = 0; i < 2 * n_edges; ++i) {
    if (edges[i] >= n) {
      free(deg);
      return -1;
    }
    deg[edges[i]]++;
  }
  uint64_t best = 0;
  for (uint64_t v = 1; v < n; ++v)
    if (deg[v] > deg[best]) best = v;
  if (deg_out) memcpy(deg_out, deg, sizeof(uint64_t) * n);
  free(deg);
  return (int64_t)best;
}

/* CSR input (Section V keeps graphs as offsets + neighbors): the vertex
 * whose row is longest, the smaller id on ties, as Algorithm 4 reads
 * max_degree() from the offsets. Returns -1 for malformed offsets (not
 * starting at 0 or decreasing) and for n == 0. */
ORACLE_EXPORT int64_t oracle_csr_max_row_vertex(uint64_t n, const uint64_t *offsets) {
  if (n == 0 || offsets[0] != 0) return -1;
  uint64_t best = 0, best_len = 0;
  for (uint64_t v = 0; v < n; ++v) {
    if (offsets[v + 1] < offsets[v]) return -1;
    const uint64_t len = offsets[v + 1] - offsets[v];
    if (len > best_len) { /* strictly longer: an earlier (smaller) id keeps ties */
      best = v;
      best_len = len;
    }
  }
  return (int64_t)best;
}

/* Streaming degree count for inputs that do not fit in memory at once. */
ORACLE_EXPORT int oracle_degree_add(uint64_t n, const uint32_t *edges, uint64_t n_edges,
                                    uint64_t *deg) {
  for (uint64_t i = 0; i < 2 * n_edges; ++i) {
    if (edges[i] >= n) return -1;
    deg[edges[i]]++;
  }
  return 0;
}

/* ---------------------------------------------------- component queries
 * Number of components: the number of vertices that are their own label.
 * connected(u, v) holds iff L[u] == L[v] (Section II, "Terminology"). */
ORACLE_EXPORT uint64_t oracle_num_components(uint64_t n, const uint32_t *L) {
  uint64_t c = 0;
  for (uint64_t v = 0; v < n; ++v) c += (L[v] == v);
  return c;
}

ORACLE_EXPORT int oracle_connected(uint64_t n, const uint32_t *L, const uint32_t *pairs,
                                   uint64_t n_pairs, uint8_t *out) {
  for (uint64_t i = 0; i < n_pairs; ++i) {
    uint32_t a = pairs[2 * i], b = pairs[2 * i + 1];
    if (a >= n || b >= n) return -1;
    out[i] = (uint8_t)(L[a] == L[b]);
  }
  return 0;
}

/* --------------------------------------------- sequential Algorithms 1 and 3
 * Root-Function JT (Algorithm 3) run by one thread, so every CAS succeeds.
 * use_r = 0 takes f(v) = v (Algorithm 1, as Section IV notes); use_r = 1 takes
 * f = R of Eq. 1 with inverse Eq. 2. No path compression during hooking. */
static uint64_t f_of(int use_r, uint64_t m, uint64_t v) { return use_r ? R_of(v, m) : v; }
static uint64_t f_inv(int use_r, uint64_t m, uint64_t c) {
  if (!use_r) return c;
  return c == 0 ? m : c - 1; /* Eq. 2 */
}

/* Initialisation: P[v] = f(v). */
ORACLE_EXPORT void oracle_rfjt_init(uint64_t n, int use_r, uint64_t m, uint32_t *P) {
  for (uint64_t v = 0; v < n; ++v) P[v] = (uint32_t)f_of(use_r, m, v);
}

/* Hooking, one edge after another: walk both endpoints up to their roots
 * (a vertex x is a root iff P[x] == f(x)); equal roots end the edge;
 * otherwise the root with the larger f is given the smaller f as parent
 * value. */
ORACLE_EXPORT int oracle_rfjt_hook(uint64_t n, int use_r, uint64_t m, const uint32_t *edges,
                                   uint64_t n_edges, uint32_t *P) {
  for (uint64_t i = 0; i < n_edges; ++i) {
    uint64_t u = edges[2 * i], v = edges[2 * i + 1];
    if (u >= n || v >= n) return -1;
    while (P[u] != f_of(use_r, m, u)) u = f_inv(use_r, m, P[u]);
    while (P[v] != f_of(use_r, m, v)) v = f_inv(use_r, m, P[v]);
    if (u == v) continue;
    if (f_of(use_r, m, u) < f_of(use_r, m, v))
      P[v] = (uint32_t)f_of(use_r, m, u);
    else
      P[u] = (uint32_t)f_of(use_r, m, v);
  }
  return 0;
}

/* Pointer jumping: every vertex takes the value of its root, P[v] = P[root]. */
ORACLE_EXPORT void oracle_rfjt_pointer_jump(uint64_t n, int use_r, uint64_t m, uint32_t *P) {
  for (uint64_t v = 0; v < n; ++v) {
    uint64_t u = v;
    while (P[u] != f_of(use_r, m, u)) u = f_inv(use_r, m, P[u]);
    P[v] = P[u];
  }
}

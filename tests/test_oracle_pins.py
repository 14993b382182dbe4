"""Pins for the CPU oracle: checks against things other than the oracle itself.

* the definition on tiny graphs (transitive closure, every simple graph on 5
  vertices and every edge order of small cases);
* a different algorithm (BFS) and a library routine
  (scipy.sparse.csgraph.connected_components) on larger graphs;
* closed forms (path, disjoint cliques, empty edge set, star, full grid,
  self-loops only);
* the identity between the two label spaces under Eq. 1;
* the worked example of Fig. 1 (Section II);
* invariants (L_u == L_v on every edge, L_v <= v, L[L_v] == L_v, invariance
  under edge order, direction, duplicates and self-loops).
"""
import itertools
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_pairs(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def test_exhaustive_five_vertices_against_closure():
    """Every simple graph on 5 vertices (2^10 of them): union-find, BFS and the
    transitive-closure definition agree, and so do the root-value labels with
    the closed form under each choice of planted vertex m."""
    n = 5
    cand = all_pairs(n)
    for mask in range(1 << len(cand)):
        edges = np.array([cand[i] for i in range(len(cand)) if mask >> i & 1],
                         dtype=np.uint32).reshape(-1, 2)
        ref = oracle.closure_labels(n, edges)
        np.testing.assert_array_equal(oracle.min_labels(n, edges), ref)
        np.testing.assert_array_equal(oracle.bfs_labels(n, edges), ref)
        for m in range(n):
            same_as_m = ref == ref[m]
            expect = np.where(same_as_m, 0, ref + 1).astype(np.uint32)
            np.testing.assert_array_equal(oracle.root_value_labels(n, edges, m), expect)


def test_every_edge_order_sequential_rfjt():
    """Sequential Algorithm 3 (both f = id and f = R) ends, after pointer
    jumping, in the same P for every order and direction of the edges, and that
    P is the root-value label of the definition."""
    rng = np.random.default_rng(7)
    for trial in range(12):
        n = int(rng.integers(3, 8))
        k = int(rng.integers(1, 6))
        edges = rng.integers(0, n, size=(k, 2)).astype(np.uint32)
        ref = oracle.closure_labels(n, edges)
        m = int(rng.integers(0, n))
        for perm in itertools.permutations(range(k)):
            for flip in range(1 << k):
                e = edges[list(perm)].copy()
                for i in range(k):
                    if flip >> i & 1:
                        e[i] = e[i][::-1]
                P = oracle.rfjt_hook(oracle.rfjt_init(n), e)
                np.testing.assert_array_equal(oracle.rfjt_pointer_jump(P), ref)
                P = oracle.rfjt_hook(oracle.rfjt_init(n, True, m), e, True, m)
                oracle.rfjt_pointer_jump(P, True, m)
                np.testing.assert_array_equal(P, np.where(ref == ref[m], 0, ref + 1))


def test_fig1_trace():
    """Section II, Fig. 1: after (3,2), P_3 = 2; after (3,1), P_2 = 1."""
    with open(os.path.join(GOLDEN, "fig1_trace.json")) as f:
        fx = json.load(f)
    P = oracle.rfjt_init(fx["n_vertices"])
    for step in fx["steps"]:
        oracle.rfjt_hook(P, np.array([step["edge"]], dtype=np.uint32))
        for v, pv in step["expect"].items():
            assert P[int(v)] == pv


def test_closed_forms():
    n = 1000
    # path on n vertices, fed in descending order: one component, all labels 0
    path = np.stack([np.arange(n - 1, 0, -1), np.arange(n - 2, -1, -1)], 1).astype(np.uint32)
    L = oracle.min_labels(n, path)
    assert (L == 0).all() and oracle.num_components(L) == 1
    # k disjoint cliques on id blocks: k components, each labelled by its first id
    sizes = [1, 2, 3, 7, 30, 57]
    starts = np.cumsum([0] + sizes[:-1])
    cl = [(s + i, s + j) for s, z in zip(starts, sizes) for i in range(z) for j in range(i + 1, z)]
    nv = sum(sizes)
    L = oracle.min_labels(nv, np.array(cl, dtype=np.uint32))
    assert oracle.num_components(L) == len(sizes)
    for s, z in zip(starts, sizes):
        assert (L[s:s + z] == s).all()
    # empty edge set: n components, L_v = v
    L = oracle.min_labels(n, np.zeros((0, 2), np.uint32))
    np.testing.assert_array_equal(L, np.arange(n, dtype=np.uint32))
    # star centred on the last vertex: one component
    star = np.stack([np.full(n - 1, n - 1), np.arange(n - 1)], 1).astype(np.uint32)
    assert oracle.num_components(oracle.min_labels(n, star)) == 1
    # full 40 x 25 grid: one component
    W, H = 40, 25
    ids = np.arange(W * H).reshape(H, W)
    g = np.concatenate([np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], 1),
                        np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], 1)]).astype(np.uint32)
    assert oracle.num_components(oracle.min_labels(W * H, g)) == 1
    # n self-loops: n components
    loops = np.stack([np.arange(n), np.arange(n)], 1).astype(np.uint32)
    assert oracle.num_components(oracle.min_labels(n, loops)) == n


def check_invariants(n, edges, L):
    e = edges.astype(np.int64)
    assert (L[e[:, 0]] == L[e[:, 1]]).all()
    assert (L <= np.arange(n)).all()
    assert (L[L] == L).all()


def test_against_bfs_and_scipy_rmat16():
    """The small R-MAT (scale 16, 2^20 edges): union-find == BFS, and the
    partition equals scipy's connected_components (a library routine)."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    w = graphgen.RMAT16
    e = w.host_edges()
    L = oracle.min_labels(w.n_vertices, e)
    np.testing.assert_array_equal(L, oracle.bfs_labels(w.n_vertices, e))
    check_invariants(w.n_vertices, e, L)
    A = sp.coo_matrix((np.ones(len(e), np.int8), (e[:, 0], e[:, 1])),
                      shape=(w.n_vertices, w.n_vertices))
    ncomp, lab = csgraph.connected_components(A, directed=False)
    assert ncomp == oracle.num_components(L)
    # the same partition: the min-id label is a function of scipy's label and back
    mins = np.full(ncomp, np.iinfo(np.int64).max)
    np.minimum.at(mins, lab, np.arange(w.n_vertices))
    np.testing.assert_array_equal(L, mins[lab].astype(np.uint32))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_graphs_bfs_invariance(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5000))
    m = int(rng.integers(0, 3 * n))
    e = rng.integers(0, n, size=(m, 2)).astype(np.uint32)
    L = oracle.min_labels(n, e)
    np.testing.assert_array_equal(L, oracle.bfs_labels(n, e))
    check_invariants(n, e, L)
    # order, direction, duplicates and self-loops leave the labels unchanged
    e2 = e[rng.permutation(m)]
    e2 = np.where(rng.random((m, 1)) < 0.5, e2[:, ::-1], e2)
    extra = np.stack([np.arange(n), np.arange(n)], 1).astype(np.uint32)
    e2 = np.concatenate([e2, e2[: m // 3], extra]).astype(np.uint32)
    np.testing.assert_array_equal(oracle.min_labels(n, e2), L)


def test_grid_stand_in_components():
    """The grid generator at p = 0.9 on 64 x 64: BFS agrees, and one giant
    component holds most vertices (bond percolation well above threshold)."""
    e = graphgen.grid(64, 64, 3)
    n = 64 * 64
    L = oracle.min_labels(n, e)
    np.testing.assert_array_equal(L, oracle.bfs_labels(n, e))
    counts = np.bincount(L, minlength=n)
    assert counts.max() > 0.9 * n


def test_max_degree_vertex():
    # endpoint occurrences, a self-loop counts twice
    e = np.array([[1, 1], [2, 3], [2, 4], [0, 5]], np.uint32)
    m, deg = oracle.max_degree_vertex(6, e, return_degrees=True)
    np.testing.assert_array_equal(deg, [1, 2, 2, 1, 1, 1])
    assert m == 1  # tie between 1 and 2 goes to the smaller id
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(1, 300))
        e = rng.integers(0, n, size=(int(rng.integers(0, 900)), 2)).astype(np.uint32)
        cnt = np.bincount(e.ravel(), minlength=n)
        assert oracle.max_degree_vertex(n, e) == int(np.flatnonzero(cnt == cnt.max())[0])


def test_wound_cycle_closed_form():
    """Edges (i mod n, (i + 1) mod n) for i < q n + r wind a cycle q times
    and r edges more. Vertex v is a first endpoint q + [v < r] times and a
    second endpoint q + [1 <= v <= r] times, so for 2 <= r < n the largest
    degree 2q + 2 belongs to vertices 1 .. r - 1 and m = 1; one component,
    min-id label 0. The GPU test of the 64-bit histogram (2^31 + 5 edges)
    relies on this form."""
    for n, q, r in ((64, 8, 5), (1000, 3, 2), (4096, 2, 4095)):
        E = q * n + r
        i = np.arange(E, dtype=np.int64)
        e = np.stack([i % n, (i + 1) % n], axis=1).astype(np.uint32)
        v = np.arange(n)
        want = 2 * q + (v < r) + ((v >= 1) & (v <= r))
        assert np.array_equal(np.bincount(e.ravel().astype(np.int64), minlength=n), want)
        assert oracle.max_degree_vertex(n, e) == 1
        assert (oracle.min_labels(n, e) == 0).all()


def test_degree_add_chunked():
    """The streaming degree count (the maximum-degree vertex of Algorithm 4's
    max_degree() for inputs fed in chunks) against numpy's bincount of both
    endpoint columns: random edge lists with self-loops and duplicates, split
    at every kind of chunk boundary (empty chunks, one-edge chunks, uneven
    splits); its argmax (smallest id on ties) is max_degree_vertex; closed
    forms for a star and for self-loops; an out-of-range id is rejected."""
    rng = np.random.default_rng(23)
    for trial in range(40):
        n = int(rng.integers(1, 500))
        k = int(rng.integers(0, 2000))
        e = rng.integers(0, n, size=(k, 2)).astype(np.uint32)
        if k:
            loops = rng.random(k) < 0.05
            e[loops, 1] = e[loops, 0]  # self-loops
            dup = rng.integers(0, k, size=k // 10)
            e = np.concatenate([e, e[dup]])  # duplicates
        cuts = np.sort(rng.integers(0, len(e) + 1, size=int(rng.integers(0, 6))))
        deg = np.zeros(n, np.uint64)
        for chunk in np.split(e, cuts):
            oracle.degree_add(n, chunk, deg)
        want = np.bincount(e[:, 0], minlength=n) + np.bincount(e[:, 1], minlength=n)
        np.testing.assert_array_equal(deg, want.astype(np.uint64))
        assert int(np.flatnonzero(deg == deg.max())[0]) == oracle.max_degree_vertex(n, e)
    # closed forms: a star on k leaves gives the centre k and each leaf 1; a
    # self-loop counts twice
    k = 37
    star = np.stack([np.full(k, 3), np.arange(4, 4 + k)], 1).astype(np.uint32)
    deg = oracle.degree_add(4 + k, star, np.zeros(4 + k, np.uint64))
    assert deg[3] == k and (deg[4:] == 1).all() and (deg[:3] == 0).all()
    deg = oracle.degree_add(3, np.array([[1, 1], [1, 1], [2, 0]], np.uint32), np.zeros(3, np.uint64))
    np.testing.assert_array_equal(deg, [1, 4, 1])
    with pytest.raises(ValueError):
        oracle.degree_add(4, np.array([[0, 1], [2, 4]], np.uint32), np.zeros(4, np.uint64))
    with pytest.raises(ValueError):
        oracle.degree_add(4, np.array([[7, 1]], np.uint32), np.zeros(4, np.uint64))


def test_root_value_identity_rmat16():
    """L_root[v] = 0 if v ~ m else L_min[v] + 1 (Eq. 1 relabelling), and with
    f = id the root-value labels are the min-id labels (Section IV)."""
    w = graphgen.RMAT16
    e = w.host_edges()
    L = oracle.min_labels(w.n_vertices, e)
    m = oracle.max_degree_vertex(w.n_vertices, e)
    Lr = oracle.root_value_labels(w.n_vertices, e, m)
    np.testing.assert_array_equal(Lr, np.where(L == L[m], 0, L + 1))
    P = oracle.rfjt_pointer_jump(oracle.rfjt_hook(oracle.rfjt_init(w.n_vertices, True, m), e, True, m),
                                 True, m)
    np.testing.assert_array_equal(P, Lr)


def test_connected_and_streaming():
    rng = np.random.default_rng(11)
    n = 3000
    e = rng.integers(0, n, size=(2500, 2)).astype(np.uint32)
    L = oracle.min_labels(n, e)
    q = rng.integers(0, n, size=(4000, 2)).astype(np.uint32)
    out = oracle.connected(L, q)
    np.testing.assert_array_equal(out, (L[q[:, 0]] == L[q[:, 1]]).astype(np.uint8))
    # incremental: labels after batches == labels of the union
    uf = oracle.StreamingUnionFind(n)
    for chunk in np.array_split(e, 7):
        uf.add(chunk)
    np.testing.assert_array_equal(uf.min_labels(), L)
    uf.close()


def test_out_of_range_rejected():
    with pytest.raises(ValueError):
        oracle.min_labels(4, np.array([[0, 4]], np.uint32))
    with pytest.raises(ValueError):
        oracle.bfs_labels(4, np.array([[5, 1]], np.uint32))


def test_csr_max_row_vertex_pins():
    """CSR input reads max_degree() from the offsets (Algorithm 4): on a
    symmetric graph without self-loops every undirected edge appears in both
    rows, so the longest row is the COO maximum-degree vertex (ties to the
    smaller id in both); closed forms for a star, ties and empty rows."""
    rng = np.random.default_rng(17)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        e = rng.integers(0, n, size=(int(rng.integers(0, 120)), 2)).astype(np.uint32)
        e = e[e[:, 0] != e[:, 1]]
        sym = np.concatenate([e, e[:, ::-1]])
        off, nb = graphgen.to_csr(n, sym)
        want = oracle.max_degree_vertex(n, e) if len(e) else 0
        assert oracle.csr_max_row_vertex(n, off) == want
        # the CSR stands for the same pairs
        back = oracle.csr_edges(off, nb)
        assert sorted(map(tuple, back.tolist())) == sorted(map(tuple, sym.tolist()))
    star = np.array([[5, k] for k in range(10) if k != 5], np.uint32)
    off, _ = graphgen.to_csr(10, np.concatenate([star, star[:, ::-1]]))
    assert oracle.csr_max_row_vertex(10, off) == 5
    assert oracle.csr_max_row_vertex(4, np.array([0, 0, 0, 0, 0], np.uint64)) == 0  # no edges
    assert oracle.csr_max_row_vertex(5, np.array([0, 0, 3, 3, 6, 7], np.uint64)) == 1  # rows 1 and 3 tie
    with pytest.raises(Exception):
        oracle.csr_max_row_vertex(3, np.array([0, 2, 1, 3], np.uint64))  # decreasing


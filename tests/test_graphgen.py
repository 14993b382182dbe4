"""The seeded input generators: determinism, chunking, shapes and statistics."""
import numpy as np

import graphgen


def test_rmat_chunking_and_determinism():
    full = graphgen.rmat(12, 40000, 9, scramble=True)
    a = graphgen.rmat(12, 40000, 9, scramble=True, e_begin=0, e_end=12345)
    b = graphgen.rmat(12, 40000, 9, scramble=True, e_begin=12345, e_end=40000)
    np.testing.assert_array_equal(np.concatenate([a, b]), full)
    np.testing.assert_array_equal(graphgen.rmat(12, 40000, 9, scramble=True), full)
    assert not np.array_equal(graphgen.rmat(12, 40000, 10, scramble=True), full)
    assert full.max() < (1 << 12)


def test_rmat_quadrant_statistics():
    """Top-level bit of (u, v) follows (a, b, c, d) = (.57, .19, .19, .05)."""
    scale = 10
    e = graphgen.rmat(scale, 400000, 1, scramble=False).astype(np.int64)
    top_u = e[:, 0] >> (scale - 1)
    top_v = e[:, 1] >> (scale - 1)
    q = np.bincount(top_u * 2 + top_v, minlength=4) / len(e)
    np.testing.assert_allclose(q, [0.57, 0.19, 0.19, 0.05], atol=0.005)


def test_scramble_is_a_permutation():
    scale = 14
    n = 1 << scale
    e = graphgen.rmat(scale, n * 4, 3, scramble=False)
    s = graphgen.rmat(scale, n * 4, 3, scramble=True)
    # the same multiset of degrees, relabelled
    d0 = np.sort(np.bincount(e.ravel(), minlength=n))
    d1 = np.sort(np.bincount(s.ravel(), minlength=n))
    np.testing.assert_array_equal(d0, d1)
    # a consistent relabelling: equal raw ids map to equal scrambled ids
    raw, scr = e.ravel(), s.ravel()
    mapping = np.full(n, -1, np.int64)
    mapping[raw] = scr
    assert (mapping[raw] == scr).all()
    used = mapping[mapping >= 0]
    assert len(np.unique(used)) == len(used)


def test_grid_shape():
    W, H = 50, 30
    e = graphgen.grid(W, H, 3)
    cand = (W - 1) * H + W * (H - 1)
    assert 0.85 * cand < len(e) < 0.95 * cand
    u, v = e[:, 0].astype(np.int64), e[:, 1].astype(np.int64)
    assert ((v - u == 1) & (u % W != W - 1) | (v - u == W)).all()
    # row-major slot order: right before down within a cell, cells ascending
    key = 2 * u + (v - u == W)
    assert (np.diff(key) > 0).all()
    full = graphgen.grid(W, H, 3, p_thresh=0xFFFFFFFF)
    assert len(full) >= cand - 1
    cut = graphgen.grid(W, H, 3, n_limit=W * H - 7)
    assert cut.max() < W * H - 7


def test_er_and_pairs():
    e = graphgen.er(1000, 50000, 4)
    assert e.max() < 1000
    np.testing.assert_array_equal(e[100:200], graphgen.er(1000, 50000, 4, 100, 200))
    p = graphgen.pairs(77, 1000, 1, tag=3)
    assert p.max() < 77
    assert not np.array_equal(p, graphgen.pairs(77, 1000, 1, tag=4))


def test_batch_plan_ranges():
    b = graphgen.batch(64, 5)
    nv = np.diff(b.vtx_off.astype(np.int64))
    ne = np.diff(b.edge_off.astype(np.int64))
    assert ((nv >= 256) & (nv < (1 << 18))).all()
    assert set(np.unique(b.kinds)) <= {0, 1, 2}
    assert len(b.edges) == int(b.edge_off[-1])
    for g in range(b.n_graphs):
        seg = b.edges[int(b.edge_off[g]):int(b.edge_off[g + 1])]
        if len(seg):
            assert seg.max() < nv[g]
        if b.kinds[g] != graphgen.KIND_GRID:
            d = 2 * ne[g] / nv[g]
            assert 1.9 <= d <= 32.1
    kinds, vo, eo = graphgen.batch_plan(4096, 5)
    frac = np.bincount(kinds, minlength=3) / 4096
    np.testing.assert_allclose(frac, [0.4, 0.4, 0.2], atol=0.03)

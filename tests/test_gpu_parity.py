"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit for bit (labels are integers; there is no tolerance).

Covers every edge-pass variant (filter on/off, 2/4/8 edges per thread, block
sizes), both root functions and both label spaces, ragged and misaligned
inputs, degenerate graphs, adversarial edge orders, hot-CAS stars, queries,
incremental inserts, checkpoints, host-buffer runs and device-side error
reporting.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")


def dev_edges(e: np.ndarray, misalign: bool = False):
    e = np.ascontiguousarray(e, dtype=np.uint32).reshape(-1, 2)
    if not misalign:
        return torch.from_numpy(e.view(np.int32)).cuda()
    buf = torch.empty((len(e) + 1, 2), dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(e.view(np.int32)).cuda()
    view = buf[1:]
    assert len(e) == 0 or view.data_ptr() % 16 == 8
    return view


def run_labels(n, e, misalign=False, **opts):
    with cc.Graph(n, **opts) as g:
        L = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        g.run(dev_edges(e, misalign), L[:n] if n else None)
        g.sync()
        return L[:n].cpu().numpy().view(np.uint32), g.num_components(), g.root_vertex()


@pytest.fixture(scope="module")
def rmat16():
    w = graphgen.RMAT16
    e = w.host_edges()
    return w.n_vertices, e, oracle.min_labels(w.n_vertices, e)


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
@pytest.mark.parametrize("flt", [cc.CC_FILTER_ON, cc.CC_FILTER_OFF, cc.CC_FILTER_BITMAP])
@pytest.mark.parametrize("ept", [2, 4, 8])
@pytest.mark.parametrize("block", [128, 256, 512])
def test_rmat16_every_variant(rmat16, mode, flt, ept, block):
    n, e, want = rmat16
    got, ncomp, m = run_labels(n, e, mode=mode, filter=flt, edges_per_thread=ept, block_size=block)
    np.testing.assert_array_equal(got, want)
    assert ncomp == oracle.num_components(want)
    if mode == cc.CC_ROOT_MAXDEG:
        assert m == oracle.max_degree_vertex(n, e)


@pytest.mark.parametrize("label_space", [cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE])
@pytest.mark.parametrize("select", [cc.CC_ROOT_SELECT_EXACT, cc.CC_ROOT_SELECT_SAMPLED])
def test_rmat16_label_spaces(rmat16, label_space, select):
    n, e, want = rmat16
    got, _, m = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG, label_space=label_space, root_select=select,
                           sample_stride=4)
    if select == cc.CC_ROOT_SELECT_EXACT:
        assert m == oracle.max_degree_vertex(n, e)
    if label_space == cc.CC_LABEL_MIN_ID:
        np.testing.assert_array_equal(got, want)
    else:
        # root-value labels for the planted vertex the library reports
        np.testing.assert_array_equal(got, oracle.root_value_labels(n, e, m))


def test_identity_root_value_equals_min_id(rmat16):
    n, e, want = rmat16
    got, _, _ = run_labels(n, e, mode=cc.CC_ROOT_IDENTITY, label_space=cc.CC_LABEL_ROOT_VALUE)
    np.testing.assert_array_equal(got, want)


def test_root_hint(rmat16):
    n, e, want = rmat16
    for hint in (0, 1, n // 2, n - 1):
        got, _, m = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG, root_hint=hint)
        assert m == hint
        np.testing.assert_array_equal(got, want)
        got, _, _ = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG, root_hint=hint,
                               label_space=cc.CC_LABEL_ROOT_VALUE)
        np.testing.assert_array_equal(got, oracle.root_value_labels(n, e, hint))


CASES = [(1, 0), (1, 1), (2, 1), (3, 2), (5, 3), (7, 0), (1000, 1), (1000, 2), (1000, 3),
         (1000, 999), (1000, 5000), (4099, 4097), (65536 + 3, 200001), (300007, 900013)]


@pytest.mark.parametrize("n,m", CASES)
@pytest.mark.parametrize("misalign", [False, True])
def test_random_ragged(n, m, misalign):
    rng = np.random.default_rng(n * 7919 + m)
    e = rng.integers(0, n, size=(m, 2)).astype(np.uint32)
    want = oracle.min_labels(n, e)
    m_want = oracle.max_degree_vertex(n, e)
    for mode in (cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY):
        for flt in (cc.CC_FILTER_ON, cc.CC_FILTER_OFF):
            got, ncomp, m = run_labels(n, e, misalign, mode=mode, filter=flt)
            np.testing.assert_array_equal(got, want)
            assert ncomp == oracle.num_components(want)
            if mode == cc.CC_ROOT_MAXDEG:  # no hub: the full histogram (sample + the rest) decides
                assert m == m_want


def test_empty_vertex_set():
    with cc.Graph(0) as g:
        g.run(torch.empty((0, 2), dtype=torch.int32, device="cuda"), None)
        g.sync()
        assert g.num_components() == 0


def _structured():
    n = 200000
    out = {}
    out["path_descending"] = (n, np.stack([np.arange(n - 1, 0, -1), np.arange(n - 2, -1, -1)], 1))
    out["path_ascending"] = (n, np.stack([np.arange(0, n - 1), np.arange(1, n)], 1))
    out["path_desc_reversed_pairs"] = (n, np.stack([np.arange(n - 2, -1, -1), np.arange(n - 1, 0, -1)], 1))
    out["star_high_centre"] = (n, np.stack([np.full(n - 1, n - 1), np.arange(n - 1)], 1))
    out["star_low_centre_dup"] = (n, np.tile(np.stack([np.zeros(n - 1, int), np.arange(1, n)], 1), (3, 1)))
    sizes = [1, 2, 3, 7, 30, 57, 300]
    starts = np.cumsum([0] + sizes[:-1])
    cl = [(s + i, s + j) for s, z in zip(starts, sizes) for i in range(z) for j in range(i + 1, z)]
    out["cliques"] = (sum(sizes), np.array(cl))
    W, H = 700, 300
    ids = np.arange(W * H).reshape(H, W)
    out["full_grid"] = (W * H, np.concatenate([np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], 1),
                                               np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], 1)]))
    out["self_loops"] = (5000, np.stack([np.arange(5000), np.arange(5000)], 1))
    out["one_edge_repeated"] = (10, np.tile(np.array([[7, 3]]), (100000, 1)))
    out["grid_gen_p09"] = (256 * 256, graphgen.grid(256, 256, 9))
    return out


STRUCT = _structured()


@pytest.mark.parametrize("name", sorted(STRUCT))
def test_structured(name):
    n, e = STRUCT[name]
    e = np.asarray(e, dtype=np.uint32)
    want = oracle.min_labels(n, e)
    for mode in (cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY):
        for flt in (cc.CC_FILTER_ON, cc.CC_FILTER_OFF):
            got, ncomp, m = run_labels(n, e, mode=mode, filter=flt)
            np.testing.assert_array_equal(got, want)
            assert ncomp == oracle.num_components(want)
            if mode == cc.CC_ROOT_MAXDEG:
                assert m == oracle.max_degree_vertex(n, e)


def test_order_direction_duplicate_invariance(rmat16):
    n, e, want = rmat16
    rng = np.random.default_rng(1)
    e2 = e[rng.permutation(len(e))]
    e2 = np.where(rng.random((len(e2), 1)) < 0.5, e2[:, ::-1], e2)
    e2 = np.concatenate([e2, e2[:1000], np.stack([np.arange(n), np.arange(n)], 1)]).astype(np.uint32)
    got, _, _ = run_labels(n, e2)
    np.testing.assert_array_equal(got, want)


def test_connected_queries(rmat16):
    n, e, want = rmat16
    q = graphgen.pairs(n, 100003, 5)
    with cc.Graph(n) as g:
        g.run(dev_edges(e))
        out = torch.empty(len(q), dtype=torch.uint8, device="cuda")
        g.connected(dev_edges(q), out)
        g.sync()
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.connected(want, q))
        for (u, v) in q[:20]:
            assert cc.cc_connected1(g.h, int(u), int(v)) == bool(want[u] == want[v])


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
@pytest.mark.parametrize("flt", [cc.CC_FILTER_AUTO, cc.CC_FILTER_BITMAP])
def test_incremental_inserts_equal_union(mode, flt):
    n = 1 << 16
    base = graphgen.rmat(16, 1 << 17, 21, scramble=True)
    batches = [graphgen.pairs(n, k, 30 + i) for i, k in enumerate([1, 1000, 7, 40000, 3, 12345])]
    with cc.Graph(n, mode=mode, filter=flt) as g:
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(dev_edges(base), L)
        seen = [base]
        for b in batches:
            g.insert(dev_edges(b))
            seen.append(b)
            g.labels(L)
            g.sync()
            want = oracle.min_labels(n, np.concatenate(seen))
            np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)
            assert g.num_components() == oracle.num_components(want)
    # inserts on a fresh handle, without any cc_run
    with cc.Graph(n, mode=mode, filter=flt) as g:
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        for b in batches:
            g.insert(dev_edges(b))
        assert g.num_components() == oracle.num_components(oracle.min_labels(n, np.concatenate(batches)))
        g.labels(L)
        g.sync()
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32),
                                      oracle.min_labels(n, np.concatenate(batches)))


def test_insert_rejects_out_of_range_batch():
    n = 5000
    base = graphgen.er(n, 3000, 2)
    with cc.Graph(n) as g:
        L0 = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(dev_edges(base), L0)
        g.sync()
        bad = graphgen.pairs(n, 4000, 9)
        bad[1234, 1] = n  # one id out of range
        g.insert(dev_edges(bad))
        assert cc.cc_sync_status(g.h) == cc.CC_ERR_OUT_OF_RANGE
        L1 = torch.empty(n, dtype=torch.int32, device="cuda")
        g.labels(L1)
        g.sync()  # the error was reported once and cleared
        np.testing.assert_array_equal(L1.cpu().numpy(), L0.cpu().numpy())


def test_run_reports_out_of_range():
    n = 100
    e = np.array([[1, 2], [3, 100], [4, 5]], np.uint32)
    with cc.Graph(n) as g:
        g.run(dev_edges(e), None)
        assert cc.cc_sync_status(g.h) == cc.CC_ERR_OUT_OF_RANGE
        assert cc.cc_sync_status(g.h) == cc.CC_OK
        q = torch.tensor([[0, 1], [5, 999]], dtype=torch.int32, device="cuda")
        out = torch.empty(2, dtype=torch.uint8, device="cuda")
        g.connected(q, out)
        assert cc.cc_sync_status(g.h) == cc.CC_ERR_OUT_OF_RANGE
        with pytest.raises(cc.CCError):
            cc.cc_connected1(g.h, 0, 100)


def test_checkpoint_restore_midstream():
    n = 1 << 15
    base = graphgen.rmat(15, 1 << 16, 40, scramble=True)
    batches = [graphgen.pairs(n, 3000, 50 + i) for i in range(4)]
    for mode in (cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY):
        with cc.Graph(n, mode=mode) as g:
            g.run(dev_edges(base))
            g.insert(dev_edges(batches[0]))
            g.insert(dev_edges(batches[1]))
            ck = cc.cc_checkpoint(g.h)
            m_before = g.root_vertex()
        with cc.Graph(n, mode=mode) as h:
            cc.cc_restore(h.h, ck)
            assert h.root_vertex() == m_before
            h.insert(dev_edges(batches[2]))
            h.insert(dev_edges(batches[3]))
            L = torch.empty(n, dtype=torch.int32, device="cuda")
            h.labels(L)
            h.sync()
            want = oracle.min_labels(n, np.concatenate([base] + batches))
            np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("mode,select", [(cc.CC_ROOT_MAXDEG, cc.CC_ROOT_SELECT_EXACT),
                                         (cc.CC_ROOT_MAXDEG, cc.CC_ROOT_SELECT_SAMPLED),
                                         (cc.CC_ROOT_IDENTITY, cc.CC_ROOT_SELECT_EXACT)])
def test_run_host_buffers(mode, select):
    n = 1 << 18
    E = (1 << 24) + (1 << 20) + 5  # two copy chunks (2^24 edges each), odd count
    e = graphgen.rmat(18, E, 60, scramble=True)
    want = oracle.min_labels(n, e)
    host = torch.from_numpy(e.view(np.int32)).pin_memory()
    L = torch.empty(n, dtype=torch.int32).pin_memory()
    with cc.Graph(n, E, mode=mode, root_select=select) as g:
        cc.cc_run_host(g.h, host, None, L)
        np.testing.assert_array_equal(L.numpy().view(np.uint32), want)
        if select == cc.CC_ROOT_SELECT_EXACT and mode == cc.CC_ROOT_MAXDEG:
            assert g.root_vertex() == oracle.max_degree_vertex(n, e)
        with pytest.raises(cc.CCError):
            cc.cc_run_host(g.h, host, E + 1, L)


def test_run_host_async():
    """Two handles on two streams: both host runs are enqueued before either
    is waited for (one of them packed on the second round). Labels and m
    equal the oracle's; an out-of-range id is reported by cc_sync, not by the
    enqueueing call."""
    n1, e1 = 1 << 20, graphgen.rmat(20, (1 << 24) + 12345, 92, scramble=True)
    n2, e2 = 512 * 512, graphgen.grid(512, 512, 93)
    h1 = torch.from_numpy(e1.view(np.int32)).pin_memory()
    p1 = torch.from_numpy(graphgen.pack_ids(e1, 3)).pin_memory()
    h2 = torch.from_numpy(e2.view(np.int32)).pin_memory()
    L1 = torch.empty(n1, dtype=torch.int32).pin_memory()
    L2 = torch.empty(n2, dtype=torch.int32).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    want1, want2 = oracle.min_labels(n1, e1), oracle.min_labels(n2, e2)
    with cc.Graph(n1, len(e1)) as g1, cc.Graph(n2, len(e2)) as g2:
        for rnd in range(2):
            L1.fill_(-1)
            L2.fill_(-1)
            if rnd == 0:
                cc.cc_run_host_async(g1.h, h1, None, L1, s1)
            else:
                cc.cc_run_host_packed_async(g1.h, p1, len(e1), 3, L1, s1)
            cc.cc_run_host_async(g2.h, h2, None, L2, s2)
            cc.cc_sync(g1.h)
            cc.cc_sync(g2.h)
            np.testing.assert_array_equal(L1.numpy().view(np.uint32), want1)
            np.testing.assert_array_equal(L2.numpy().view(np.uint32), want2)
            assert g1.root_vertex() == oracle.max_degree_vertex(n1, e1)
            assert g2.root_vertex() == oracle.max_degree_vertex(n2, e2)
        bad = e2.copy()
        bad[1000, 1] = n2 + 5
        hb = torch.from_numpy(bad.view(np.int32)).pin_memory()
        cc.cc_run_host_async(g2.h, hb, None, L2, s2)
        with pytest.raises(cc.CCError) as ei:
            cc.cc_sync(g2.h)
        assert ei.value.status == cc.CC_ERR_OUT_OF_RANGE
        cc.cc_run_host_async(g2.h, h2, None, L2, s2)  # the handle is usable again
        cc.cc_sync(g2.h)
        np.testing.assert_array_equal(L2.numpy().view(np.uint32), want2)
        with pytest.raises(cc.CCError):
            cc.cc_run_host_async(g2.h, h2, len(e2) + 1, L2, s2)  # over capacity: at once


def _chunked_case(kind):
    """Host inputs of several 2^24-edge copy chunks, built so that each route
    of the chunked exact root selection in cc_run_host is taken."""
    C = 1 << 24
    if kind == "rmat":  # dominant hub, certified from the first chunk: the speculation holds
        return 1 << 20, graphgen.rmat(20, 3 * C + 77, 61, scramble=True)
    if kind == "er":  # no hub: histogram mode, the first chunk's argmax is not m (rerun)
        return 1 << 22, graphgen.er(1 << 22, 2 * C + 5, 62)
    if kind == "grid":  # no hub: histogram mode, the first chunk's argmax is m (the hooking holds)
        return 4096 * 2560, graphgen.grid(4096, 2560, 64)
    n = 1 << 20
    e = graphgen.er(n, 2 * C + 123, 63)  # background: degree about 64
    rng = np.random.default_rng(64)
    first = rng.permutation(C)[:50000]
    later = C + rng.permutation(len(e) - C)[:100000]
    h1, h2 = 777, 4242

    def star(h, idx):
        e[idx, 0] = h
        e[idx, 1] = rng.integers(0, n, size=len(idx), dtype=np.uint32)

    if kind == "late_hub":  # the true hub never appears in the first chunk: no certificate
        star(h1, first[:20000])
        star(h2, later)
    else:  # two hubs: the first chunk's leader is not the overall one (certificate, rerun)
        star(h1, first[:30000])
        star(h2, first[30000:50000])
        star(h2, later[:40000])
    return n, e


@pytest.mark.parametrize("kind", ["rmat", "er", "grid", "late_hub", "two_hubs"])
@pytest.mark.parametrize("flt", [cc.CC_FILTER_AUTO, cc.CC_FILTER_BITMAP])
def test_run_host_chunked_selection(kind, flt):
    n, e = _chunked_case(kind)
    E = len(e)
    m = oracle.max_degree_vertex(n, e)
    if kind == "late_hub":
        assert m == 4242
    if kind == "two_hubs":
        assert m == 4242
    host = torch.from_numpy(e.view(np.int32)).pin_memory()
    L = torch.empty(n, dtype=torch.int32).pin_memory()
    want = oracle.min_labels(n, e)
    with cc.Graph(n, E, filter=flt) as g:
        for _ in range(2):  # the second run reuses every buffer
            cc.cc_run_host(g.h, host, None, L)
            np.testing.assert_array_equal(L.numpy().view(np.uint32), want)
            assert g.root_vertex() == m
        # inserts after a host run keep the bitmap consistent
        extra = graphgen.pairs(n, 5000, 65)
        g.insert(dev_edges(extra))
        Ld = torch.empty(n, dtype=torch.int32, device="cuda")
        g.labels(Ld)
        g.sync()
        np.testing.assert_array_equal(Ld.cpu().numpy().view(np.uint32),
                                      oracle.min_labels(n, np.concatenate([e, extra])))
    with cc.Graph(n, E, filter=flt, label_space=cc.CC_LABEL_ROOT_VALUE) as g:
        cc.cc_run_host(g.h, host, None, L)
        assert g.root_vertex() == m
        np.testing.assert_array_equal(L.numpy().view(np.uint32), oracle.root_value_labels(n, e, m))


@pytest.fixture(scope="module")
def rmat25():
    """R-MAT scale 25 with edge factor 4 (P of 128 MiB), two insert batches and
    a G(n, m) on the same vertex count, with their oracle labels."""
    n = 1 << 25
    e = graphgen.rmat(25, 1 << 27, 66, scramble=True)
    extra = graphgen.pairs(n, 1 << 22, 67)
    more = graphgen.pairs(n, 1 << 20, 68)
    er = graphgen.er(n, 1 << 26, 69)
    return dict(n=n, e=e, extra=extra, more=more, er=er, m=oracle.max_degree_vertex(n, e),
                want=oracle.min_labels(n, e), want2=oracle.min_labels(n, np.concatenate([e, extra])),
                want3=oracle.min_labels(n, np.concatenate([e, extra, more])), want_er=oracle.min_labels(n, er))


@pytest.mark.parametrize("flt", [cc.CC_FILTER_AUTO, cc.CC_FILTER_BITMAP, cc.CC_FILTER_ON])
def test_zero_tree_bitmap_large(rmat25, flt):
    """CC_FILTER_AUTO allocates the zero-tree bitmap for this size and the
    certified hub selects it on the device; the G(n, m) gets the bitmap too
    but no certificate, so the plain instance runs. Everything equals the
    oracle, also after inserts and a restore."""
    r = rmat25
    n = r["n"]
    with cc.Graph(n, filter=flt) as g:
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        d = dev_edges(r["e"])
        for _ in range(2):
            g.run(d, L)
            g.sync()
            np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), r["want"])
        assert g.root_vertex() == r["m"]
        if flt != cc.CC_FILTER_ON:
            assert cc.cc_device_bytes(g.h) >= 4 * n + n // 8
        g.insert(dev_edges(r["extra"]))
        g.labels(L)
        g.sync()
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), r["want2"])
        buf = cc.cc_checkpoint(g.h)
        g.run(d, L)
        cc.cc_restore(g.h, buf)
        g.insert(dev_edges(r["more"]))
        g.labels(L)
        g.sync()
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), r["want3"])
    with cc.Graph(n, filter=flt) as g:
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(dev_edges(r["er"]), L)
        g.sync()
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), r["want_er"])


@pytest.mark.parametrize("mode,select", [(cc.CC_ROOT_MAXDEG, cc.CC_ROOT_SELECT_EXACT),
                                         (cc.CC_ROOT_MAXDEG, cc.CC_ROOT_SELECT_SAMPLED),
                                         (cc.CC_ROOT_IDENTITY, cc.CC_ROOT_SELECT_EXACT)])
def test_run_host_packed(mode, select):
    """Compact 3-byte ids over the host link: several chunks (the two unpack
    slots are reused) and a tail that is not a whole group of eight edges."""
    n = 1 << 20
    E = 3 * (1 << 24) + 77
    e = graphgen.rmat(20, E, 73, scramble=True)
    want = oracle.min_labels(n, e)
    packed = torch.from_numpy(graphgen.pack_ids(e, 3)).pin_memory()
    plain = torch.from_numpy(graphgen.pack_ids(e, 4)).pin_memory()
    L = torch.empty(n, dtype=torch.int32).pin_memory()
    with cc.Graph(n, E, mode=mode, root_select=select) as g:
        for _ in range(2):
            L.fill_(-1)
            cc.cc_run_host_packed(g.h, packed, E, 3, L)
            np.testing.assert_array_equal(L.numpy().view(np.uint32), want)
        if mode == cc.CC_ROOT_MAXDEG and select == cc.CC_ROOT_SELECT_EXACT:
            assert g.root_vertex() == oracle.max_degree_vertex(n, e)
        L.fill_(-1)
        cc.cc_run_host_packed(g.h, plain, E, 4, L)  # 4-byte ids: the cc_run_host layout
        np.testing.assert_array_equal(L.numpy().view(np.uint32), want)
        for bad in (2, 5):
            with pytest.raises(cc.CCError):
                cc.cc_run_host_packed(g.h, packed, E, bad, L)
    small = graphgen.rmat(10, 1001, 74, scramble=True)  # one chunk, ragged
    ps = torch.from_numpy(graphgen.pack_ids(small, 3)).pin_memory()
    Ls = torch.empty(1 << 10, dtype=torch.int32).pin_memory()
    with cc.Graph(1 << 10, 1001, mode=mode, root_select=select) as g:
        cc.cc_run_host_packed(g.h, ps, 1001, 3, Ls)
        np.testing.assert_array_equal(Ls.numpy().view(np.uint32), oracle.min_labels(1 << 10, small))
    with cc.Graph((1 << 24) + 1, 10) as g:  # 3-byte ids cannot name every vertex
        with pytest.raises(cc.CCError):
            cc.cc_run_host_packed(g.h, ps, 10, 3, None)


def _csr_dev(off, nb):
    return (torch.from_numpy(off.astype(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(nb, dtype=np.uint32).view(np.int32)).cuda())


@pytest.mark.parametrize("hub,deg", [(1001, 255), (1001, 256), (1003, 300), (4, 70000), (65535, 511)])
def test_hub_outside_sample(hub, deg):
    """A hub whose edges all sit in groups the sampled pass skips: no
    candidate, no certificate, so the exact selection falls back to the full
    histogram (the sampled counts plus every other edge). Degrees around 2^8
    and 2^16 and ids at both ends of the range. m and the labels equal the
    oracle's."""
    n = 1 << 16
    e = graphgen.er(n, 1 << 20, 90)  # background degree about 32
    rng = np.random.default_rng(91)
    e[e == hub] = (hub + 7) % n  # the hub's degree is exactly the planted edges
    idx = 1024 + np.arange(deg)  # groups 1 .. 127 of 1024 edges: never sampled
    assert idx[-1] < 128 * 1024
    e[idx, 0] = hub
    other = rng.integers(0, n - 1, size=deg, dtype=np.uint32)
    e[idx, 1] = other + (other >= hub)
    m = oracle.max_degree_vertex(n, e)
    assert m == hub
    want = oracle.min_labels(n, e)
    for label_space in (cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE):
        with cc.Graph(n, label_space=label_space) as g:
            L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            d = dev_edges(e)
            for _ in range(2):  # the second run starts from a used parent array
                g.run(d, L)
                g.sync()
                assert g.root_vertex() == m
                got = L.cpu().numpy().view(np.uint32)
                if label_space == cc.CC_LABEL_MIN_ID:
                    np.testing.assert_array_equal(got, want)
                else:
                    np.testing.assert_array_equal(got, oracle.root_value_labels(n, e, m))


def _csr_case(case):
    if case == "rmat16":
        w = graphgen.RMAT16
        return w.n_vertices, w.host_edges()
    if case == "rmat20":
        return 1 << 20, graphgen.rmat(20, 1 << 23, 75, scramble=True)
    if case == "grid":
        return 512 * 512, graphgen.grid(512, 512, 3)
    if case == "sparse":  # mostly empty rows, a few long ones
        rng = np.random.default_rng(76)
        e = rng.integers(0, 50000, size=(20000, 2)).astype(np.uint32)
        e[:3000, 0] = 7
        return 50000, e
    return 1000, np.zeros((0, 2), np.uint32)  # no edges


@pytest.mark.parametrize("case", ["rmat16", "rmat20", "grid", "sparse", "empty"])
@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
def test_csr_path(case, mode):
    n, e = _csr_case(case)
    off, nb = graphgen.to_csr(n, e)
    pairs = oracle.csr_edges(off, nb)
    want = oracle.min_labels(n, pairs)
    d_off, d_nb = _csr_dev(off, nb)
    for label_space in (cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE):
        with cc.Graph(n, mode=mode, label_space=label_space) as g:
            L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            for _ in range(2):
                cc.cc_run_csr(g.h, d_off, d_nb, len(nb), L)
                g.sync()
                got = L.cpu().numpy().view(np.uint32)
                if mode == cc.CC_ROOT_MAXDEG:
                    m = oracle.csr_max_row_vertex(n, off)
                    assert g.root_vertex() == m
                    ref = want if label_space == cc.CC_LABEL_MIN_ID else oracle.root_value_labels(n, pairs, m)
                else:
                    ref = want
                np.testing.assert_array_equal(got, ref)
                assert g.num_components() == oracle.num_components(want)


def test_csr_errors():
    n = 100
    off, nb = graphgen.to_csr(n, np.array([[1, 2], [3, 4], [5, 6]], np.uint32))
    bad_nb = nb.copy()
    bad_nb[1] = n
    d_off, d_nb = _csr_dev(off, bad_nb)
    with cc.Graph(n) as g:
        cc.cc_run_csr(g.h, d_off, d_nb, len(nb), None)
        assert cc.cc_sync_status(g.h) == cc.CC_ERR_OUT_OF_RANGE
    start = off.astype(np.int64).copy()
    start[0] = 1  # offsets[0] != 0
    dec = off.astype(np.int64).copy()
    dec[5] = dec[6] + 1  # decreasing
    for bad_off in (start, dec):
        d_off, d_nb = _csr_dev(bad_off.astype(np.uint64), nb)
        with cc.Graph(n) as g:
            cc.cc_run_csr(g.h, d_off, d_nb, len(nb), None)
            assert cc.cc_sync_status(g.h) == cc.CC_ERR_INVALID_ARGUMENT
    d_off, d_nb = _csr_dev(off, nb)
    with cc.Graph(n, mode=cc.CC_ROOT_IDENTITY) as g:
        cc.cc_run_csr(g.h, d_off, d_nb, len(nb) + 1, None)  # n_entries != off[n]
        assert cc.cc_sync_status(g.h) == cc.CC_ERR_INVALID_ARGUMENT


def test_phase_times_and_budget():
    n = 1 << 16
    e = graphgen.rmat(16, 1 << 20, 1, scramble=False)
    with cc.Graph(n, timing=1) as g:
        g.run(dev_edges(e))
        t = cc.cc_phase_times(g.h)
        assert all(x >= 0 for x in t) and t[4] >= t[2]
        assert cc.cc_device_bytes(g.h) >= 4 * n
    with pytest.raises(cc.CCError) as ex:
        cc.Graph(n, hbm_budget_bytes=1024)
    assert ex.value.status == cc.CC_ERR_OOM


def _hidden_hub_graph(extra: int):
    """Visible hub A = 500 in every 5th edge; hidden hub B = 100 only in edge
    groups the root-selection sample skips (groups of 4 edges; B avoids
    every 16th group, which covers the one in 128 that the sample of a graph
    of this size keeps, and the one in 16 of a first host chunk), with
    deg(B) = deg(A) + extra. Other endpoints avoid both hubs."""
    n, E = 1 << 16, 1024 * 32 * 8
    rng = np.random.default_rng(11)
    e = rng.integers(1000, n, size=(E, 2)).astype(np.uint32)
    idx = np.arange(E)
    e[idx % 5 == 0, 0] = 500
    dA = int((idx % 5 == 0).sum())
    hidden_slots = idx[((idx // 4) % 16 != 0) & ((idx % 5 == 1) | (idx % 5 == 2))]
    e[hidden_slots[: dA + extra], 1] = 100
    deg = np.bincount(e.ravel(), minlength=n)
    assert deg[100] - deg[500] == extra
    return n, e


@pytest.mark.parametrize("extra", [-1, 0, 1, 5000])
def test_root_select_hidden_hub(extra):
    n, e = _hidden_hub_graph(extra)
    want_m = oracle.max_degree_vertex(n, e)
    assert want_m == (500 if extra < 0 else 100)
    got, _, m = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG, label_space=cc.CC_LABEL_ROOT_VALUE)
    assert m == want_m
    np.testing.assert_array_equal(got, oracle.root_value_labels(n, e, want_m))


@pytest.mark.parametrize("order", ["by_source", "by_source_bucket"])
@pytest.mark.parametrize("flt", [cc.CC_FILTER_AUTO, cc.CC_FILTER_BITMAP])
def test_edges_sorted_by_source(order, flt):
    """Edges sorted by their first endpoint, as edge-list files often come
    (whole rows contiguous), or grouped by its top bits: the root selection's
    sample must still be an even spread of the array, and m and the labels
    must match the oracle."""
    n = 1 << 20
    e = graphgen.rmat(20, 1 << 24, 91, scramble=True)
    key = e[:, 0] if order == "by_source" else e[:, 0] >> 8
    e = np.ascontiguousarray(e[np.argsort(key, kind="stable")])
    want = oracle.min_labels(n, e)
    got, ncomp, m = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG, filter=flt)
    assert m == oracle.max_degree_vertex(n, e)
    assert ncomp == oracle.num_components(want)
    np.testing.assert_array_equal(got, want)


def _push_case(case):
    if case == "rmat16":
        w = graphgen.RMAT16
        return w.n_vertices, w.host_edges(), False
    if case == "rmat20":  # several grid waves
        return 1 << 20, graphgen.rmat(20, 1 << 24, 70, scramble=True), False
    if case == "grid":  # no dominant hub: no certificate, no push list
        return 512 * 512, graphgen.grid(512, 512, 3), False
    if case == "ragged":  # misaligned head and odd tail
        e = graphgen.rmat(18, 900013, 72, scramble=True)
        return 1 << 18, e, True
    extra = 5000 if case == "hidden_other" else -1
    n, e = _hidden_hub_graph(extra)  # the sampled argmax is (or is not) the exact m
    return n, e, False


@pytest.mark.parametrize("case", ["rmat16", "rmat20", "grid", "ragged", "hidden_same", "hidden_other"])
def test_initial_push(case):
    """Initial Push (Algorithm 4) hooks the neighbours of m before the edge
    pass; labels, m and the component count must not change, and the push
    must be skipped when the gathered neighbours belong to another vertex."""
    n, e, misalign = _push_case(case)
    want = oracle.min_labels(n, e)
    m_want = oracle.max_degree_vertex(n, e)
    for label_space in (cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE):
        for _ in range(2):
            got, ncomp, m = run_labels(n, e, misalign, mode=cc.CC_ROOT_MAXDEG, initial_push=cc.CC_PUSH_ON,
                                       label_space=label_space)
            assert m == m_want
            assert ncomp == oracle.num_components(want)
            if label_space == cc.CC_LABEL_MIN_ID:
                np.testing.assert_array_equal(got, want)
            else:
                np.testing.assert_array_equal(got, oracle.root_value_labels(n, e, m_want))


def test_root_select_many_candidates():
    """Thousands of equally heavy vertices (more than the candidate list
    holds) plus one slightly heavier: still the exact maximum."""
    n = 1 << 18
    rng = np.random.default_rng(4)
    heavy = rng.choice(n, size=6000, replace=False).astype(np.uint32)
    e = np.stack([np.repeat(heavy, 100), rng.integers(0, n, size=600000)], 1).astype(np.uint32)
    top = heavy[1234]
    e = np.concatenate([e, np.stack([np.full(3, top), rng.integers(0, n, size=3)], 1)]).astype(np.uint32)
    e = e[rng.permutation(len(e))]
    _, _, m = run_labels(n, e, mode=cc.CC_ROOT_MAXDEG)
    assert m == oracle.max_degree_vertex(n, e)


def _leader_not_max_graph():
    """Hub A = 500 leads the root-selection sample (every second edge of the
    sampled groups, one group of 1024 in 128) but hub B = 100, a candidate
    with an eighth of A's sampled count, has the larger exact degree (most of
    its edges lie in unsampled groups). Other endpoints avoid both hubs."""
    n, E = 1 << 16, 1 << 18
    rng = np.random.default_rng(13)
    e = rng.integers(1000, n, size=(E, 2)).astype(np.uint32)
    idx = np.arange(E)
    sampled = (idx // 1024) % 128 == 0
    e[sampled & (idx % 2 == 0), 0] = 500
    e[sampled & (idx % 16 == 1), 1] = 100
    e[np.flatnonzero(~sampled)[:3000], 1] = 100
    deg = np.bincount(e.ravel(), minlength=n)
    assert deg[100] > deg[500] > deg[1000:].max()
    return n, e


@pytest.mark.parametrize("flt", [cc.CC_FILTER_AUTO, cc.CC_FILTER_BITMAP])
def test_sampled_leader_is_not_the_exact_m(flt):
    """The certificate proves a vertex other than the sampled leader. On
    device input (cc_run) the exact selection plants that vertex; on host
    input (cc_run_host) the chunks are first hooked under the sampled leader
    m', then init and one edge pass run again under the exact m, with the
    zero-tree bitmap cleared of the bits set under m'. m, the labels in both
    spaces and the component count equal the oracle's, on a fresh handle and
    on reuse."""
    n, e = _leader_not_max_graph()
    m_want = oracle.max_degree_vertex(n, e)
    assert m_want == 100
    want = oracle.min_labels(n, e)
    h_e = torch.from_numpy(np.ascontiguousarray(e).view(np.int32)).pin_memory()
    for label_space in (cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE):
        want_l = want if label_space == cc.CC_LABEL_MIN_ID else oracle.root_value_labels(n, e, m_want)
        with cc.Graph(n, len(e), filter=flt, label_space=label_space) as g:
            L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            h_L = torch.full((n,), -1, dtype=torch.int32).pin_memory()
            d = dev_edges(e)
            for _ in range(2):
                g.run(d, L)
                g.sync()
                assert g.root_vertex() == m_want
                assert g.num_components() == oracle.num_components(want)
                np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want_l)
                h_L.fill_(-1)
                cc.cc_run_host(g.h, h_e, len(e), h_L)
                assert g.root_vertex() == m_want
                assert g.num_components() == oracle.num_components(want)
                np.testing.assert_array_equal(h_L.numpy().view(np.uint32), want_l)


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
def test_cc_run_replays_from_a_cuda_graph(mode):
    """cc_run captured once into a CUDA graph and replayed: each replay reads
    the edge buffer as it is at replay time, and its labels, count and m equal
    the oracle's on that content (three different graphs of the same size)."""
    n, E = 1 << 14, 1 << 18
    graphs = [graphgen.rmat(14, E, 900 + k, scramble=True) for k in range(2)] + [graphgen.er(n, E, 903)]
    e_dev = torch.empty((E, 2), dtype=torch.int32, device="cuda")
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    e_dev.copy_(torch.from_numpy(graphs[0].view(np.int32)))
    s = torch.cuda.Stream()
    with cc.Graph(n, mode=mode) as g:
        with torch.cuda.stream(s):
            g.run(e_dev, L, s)       # first use allocates the handle's scratch outside the capture
            s.synchronize()
            gr = torch.cuda.CUDAGraph()
            gr.capture_begin()
            g.run(e_dev, L, s)
            gr.capture_end()
        for e in graphs:
            e_dev.copy_(torch.from_numpy(e.view(np.int32)))
            torch.cuda.synchronize()
            gr.replay()
            torch.cuda.synchronize()
            want = oracle.min_labels(n, e)
            np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)
            assert g.num_components() == oracle.num_components(want)
            if mode == cc.CC_ROOT_MAXDEG:
                assert g.root_vertex() == oracle.max_degree_vertex(n, e)

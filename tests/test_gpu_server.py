"""The serving runtime (include/cc_server.h) against the CPU oracle.

The central check: a mixed stream of requests over several graphs is
submitted all at once (new graphs, inserts of many sizes, query batches,
snapshots, drops) so that their work overlaps on the device; every query
answer and snapshot must equal both the oracle on that graph's edges so far
and the same request run alone (each graph's requests submitted one at a
time, waiting for each)."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")

GB = 1 << 30


def dev(e):
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.uint32).view(np.int32)).cuda()


def make_script(seed):
    """A request script: list of (graph_key, kind, payload)."""
    rng = np.random.default_rng(seed)
    script = []
    graphs = {}
    for k in range(4):
        scale = int(rng.integers(10, 15))
        n = 1 << scale
        e = graphgen.rmat(scale, n * 4, 100 + k, scramble=True)
        graphs[k] = n
        script.append((k, "new", e))
    for i in range(60):
        k = int(rng.integers(0, 4))
        n = graphs[k]
        kind = rng.choice(["insert", "query", "snapshot"], p=[0.45, 0.45, 0.10])
        if kind == "insert":
            size = int(10 ** rng.uniform(0, 5.9))  # 1 .. 800K edges: executor tiles, or a side insert from 2^18
            script.append((k, "insert", graphgen.pairs(n, size, 7, tag=i)))
        elif kind == "query":
            script.append((k, "query", graphgen.pairs(n, 3000, 8, tag=i)))
        else:
            script.append((k, "snapshot", None))
    script.append((2, "drop", None))
    script.append((4, "new", graphgen.er(5000, 9000, 55)))
    graphs[4] = 5000
    script.append((4, "query", graphgen.pairs(5000, 2000, 9, tag=999)))
    script.append((4, "snapshot", None))
    return script, graphs


def expected(script, graphs):
    """Oracle answers for every query / snapshot, in script order."""
    seen = {k: [] for k in graphs}
    out = []
    for k, kind, payload in script:
        if kind in ("new", "insert"):
            seen[k].append(payload)
            out.append(None)
        elif kind in ("query", "snapshot"):
            e = np.concatenate(seen[k]) if seen[k] else np.zeros((0, 2), np.uint32)
            L = oracle.min_labels(graphs[k], e)
            out.append(oracle.connected(L, payload) if kind == "query" else L)
        else:
            out.append(None)
    return out


def run_script(server, script, graphs, one_at_a_time):
    gid = {}
    tickets, results = [], []
    for k, kind, payload in script:
        res = None
        if kind == "new":
            t, gid[k] = server.new_graph(graphs[k], dev(payload))
        elif kind == "insert":
            t = server.insert(gid[k], dev(payload))
        elif kind == "query":
            res = torch.full((len(payload),), 7, dtype=torch.uint8, device="cuda")
            q = dev(payload)
            torch.cuda.synchronize()  # buffers complete before submission
            t = server.query(gid[k], q, res)
        elif kind == "snapshot":
            res = torch.full((graphs[k],), -1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            t = server.snapshot(gid[k], res)
        else:
            t = server.drop(gid[k])
        tickets.append(t)
        results.append(res)
        if one_at_a_time:
            assert server.wait(t) == cc.CC_OK
    out = []
    for t, res in zip(tickets, results):
        assert server.wait(t) == cc.CC_OK
        # read right after completion, with no device-wide synchronisation:
        # a completed ticket must mean its outputs are final
        out.append(None if res is None else res.cpu().numpy())
    return out, tickets


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
def test_mixed_stream_equals_alone_and_oracle(mode):
    script, graphs = make_script(3)
    want = expected(script, graphs)
    with cc.Server(2 * GB, mode=mode, tile_edges=16384) as s:
        mixed, tickets = run_script(s, script, graphs, one_at_a_time=False)
        st = s.stats()
        assert st["completed"] == len(script) and st["failed"] == 0
    with cc.Server(2 * GB, mode=mode, tile_edges=16384) as s:
        alone, _ = run_script(s, script, graphs, one_at_a_time=True)
    for i, (k, kind, _) in enumerate(script):
        if kind == "query":
            np.testing.assert_array_equal(mixed[i], want[i])
            np.testing.assert_array_equal(alone[i], want[i])
        elif kind == "snapshot":
            np.testing.assert_array_equal(mixed[i].view(np.uint32), want[i])
            np.testing.assert_array_equal(alone[i].view(np.uint32), want[i])


def test_insert_with_bad_id_is_rejected_whole():
    n = 1 << 12
    base = graphgen.rmat(12, 1 << 14, 3, scramble=True)
    with cc.Server(GB, tile_edges=1024) as s:
        t, g = s.new_graph(n, dev(base))
        assert s.wait(t) == cc.CC_OK
        L0 = torch.empty(n, dtype=torch.int32, device="cuda")
        assert s.wait(s.snapshot(g, L0)) == cc.CC_OK
        for size in (100, 500, 20000, 300000):  # one tile, many tiles (validated first), a side insert
            bad = graphgen.pairs(n, size, 4, tag=size)
            bad[size // 2, 0] = n + 5
            assert s.wait(s.insert(g, dev(bad))) == cc.CC_ERR_OUT_OF_RANGE
            L1 = torch.empty(n, dtype=torch.int32, device="cuda")
            assert s.wait(s.snapshot(g, L1)) == cc.CC_OK
            assert torch.equal(L0, L1)
        q = dev(np.array([[0, 1], [2, n]], np.uint32))
        out = torch.empty(2, dtype=torch.uint8, device="cuda")
        assert s.wait(s.query(g, q, out)) == cc.CC_ERR_OUT_OF_RANGE


def test_admission_waits_for_memory_and_drop_frees_it():
    n = 1 << 20  # ~20.3 MiB per graph under f = R (P, histogram, scratch, last labels, log, remap)
    e = graphgen.rmat(20, 1 << 21, 5, scramble=True)
    with cc.Server(32 << 20) as s:
        ta, ga = s.new_graph(n, dev(e))
        tb, gb = s.new_graph(n, dev(e))  # cannot fit until graph a is dropped
        assert s.wait(ta) == cc.CC_OK
        assert s.poll(tb) is None
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        assert s.wait(s.snapshot(ga, L)) == cc.CC_OK
        td = s.drop(ga)
        assert s.wait(td) == cc.CC_OK
        assert s.wait(tb) == cc.CC_OK
        L2 = torch.empty(n, dtype=torch.int32, device="cuda")
        assert s.wait(s.snapshot(gb, L2)) == cc.CC_OK
        want = oracle.min_labels(n, e)
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)
        np.testing.assert_array_equal(L2.cpu().numpy().view(np.uint32), want)
        with pytest.raises(cc.CCError):
            s.new_graph(1 << 30, dev(e))  # can never fit the arena


def test_executor_relaunches_after_idle_and_errors_at_submit():
    n = 4096
    e = graphgen.er(n, 5000, 1)
    with cc.Server(GB, idle_timeout_us=1000) as s:
        t, g = s.new_graph(n, dev(e))
        assert s.wait(t) == cc.CC_OK
        out = torch.empty(100, dtype=torch.uint8, device="cuda")
        q = graphgen.pairs(n, 100, 2)
        assert s.wait(s.query(g, dev(q), out)) == cc.CC_OK
        import time
        time.sleep(0.05)  # the executor leaves after 1 ms of idleness
        assert s.wait(s.insert(g, dev(graphgen.pairs(n, 3000, 3)))) == cc.CC_OK
        assert s.wait(s.query(g, dev(q), out)) == cc.CC_OK
        assert s.stats()["executor_launches"] >= 2
        want = oracle.connected(oracle.min_labels(n, np.concatenate([e, graphgen.pairs(n, 3000, 3)])), q)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        with pytest.raises(cc.CCError):
            s.insert(g + 17, dev(e))  # unknown graph
        assert s.latency_ns(t) > 0


def test_slot_reuse_completion_is_exact():
    """Many requests one after another reuse the same executor slots; each
    result is read as soon as its ticket completes (no device-wide sync)."""
    n = 1 << 14
    base = graphgen.rmat(14, 1 << 16, 9, scramble=True)
    with cc.Server(GB, tile_edges=2048) as s:
        t, g = s.new_graph(n, dev(base))
        assert s.wait(t) == cc.CC_OK
        seen = [base]
        for i in range(40):
            ins = graphgen.pairs(n, int(50 + 997 * i), 12, tag=i)  # 1 to 20 tiles
            assert s.wait(s.insert(g, dev(ins))) == cc.CC_OK
            seen.append(ins)
            q = graphgen.pairs(n, 5000, 13, tag=i)
            out = torch.full((5000,), 9, dtype=torch.uint8, device="cuda")
            qd = dev(q)
            torch.cuda.synchronize()
            assert s.wait(s.query(g, qd, out)) == cc.CC_OK
            want = oracle.connected(oracle.min_labels(n, np.concatenate(seen)), q)
            np.testing.assert_array_equal(out.cpu().numpy(), want)



def test_side_work_is_not_starved_by_a_full_executor():
    """With 8 executor blocks per SM the executor leaves no room on any SM for
    the side-stream kernels of a new graph; the host must drain the executor
    instead of waiting for its (long) idle timeout."""
    import time
    n = 1 << 14
    a = graphgen.rmat(14, 1 << 16, 21, scramble=True)
    b = graphgen.rmat(13, 1 << 15, 22, scramble=True)
    with cc.Server(GB, executor_blocks_per_sm=8, idle_timeout_us=5_000_000) as s:
        ta, ga = s.new_graph(n, dev(a))
        assert s.wait(ta) == cc.CC_OK
        q = graphgen.pairs(n, 4000, 23)
        out = torch.empty(4000, dtype=torch.uint8, device="cuda")
        qd = dev(q)
        torch.cuda.synchronize()
        assert s.wait(s.query(ga, qd, out)) == cc.CC_OK  # the executor is now resident and idle
        eb = dev(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tb, gb = s.new_graph(1 << 13, eb)
        assert s.wait(tb, 3.0) == cc.CC_OK
        assert time.perf_counter() - t0 < 2.0  # far below the 5 s idle timeout
        Lb = torch.empty(1 << 13, dtype=torch.int32, device="cuda")
        assert s.wait(s.snapshot(gb, Lb), 3.0) == cc.CC_OK
        np.testing.assert_array_equal(Lb.cpu().numpy().view(np.uint32), oracle.min_labels(1 << 13, b))
        out2 = torch.empty(4000, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        assert s.wait(s.query(ga, qd, out2)) == cc.CC_OK
        want = oracle.connected(oracle.min_labels(n, a), q)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        np.testing.assert_array_equal(out2.cpu().numpy(), want)


def test_large_graph_side_inserts_and_zero_tree():
    """A resident graph whose parent array exceeds 128 MiB keeps a zero-tree
    bitmap; large inserts run as side-stream edge passes (with the bitmap)
    while small inserts and queries run in the executor."""
    n = 1 << 25
    base = graphgen.rmat(25, 1 << 26, 31, scramble=True)
    ins = [graphgen.pairs(n, k, 32, tag=i) for i, k in enumerate([1 << 21, 1000, 1 << 19, 50, 1 << 20])]
    q = graphgen.pairs(n, 100000, 33)
    with cc.Server(4 * GB) as s:
        t, g = s.new_graph(n, dev(base))
        tickets = [t]
        for b in ins:
            tickets.append(s.insert(g, dev(b)))
        out = torch.full((len(q),), 7, dtype=torch.uint8, device="cuda")
        qd = dev(q)
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        tq = s.query(g, qd, out)
        ts = s.snapshot(g, L)
        for tk in tickets + [tq, ts]:
            assert s.wait(tk, 120) == cc.CC_OK
        want = oracle.min_labels(n, np.concatenate([base] + ins))
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.connected(want, q))
        assert s.stats()["failed"] == 0



@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
@pytest.mark.parametrize("label_space", [cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE])
@pytest.mark.parametrize("admit_labels", [True, False])
def test_incremental_snapshots(mode, label_space, admit_labels):
    """Snapshots after inserts come from the last labels and the changed-root
    log (executor tiles and side-stream inserts both log the roots they
    hook); every one must equal the oracle on all edges so far, including an
    insert that gives m's component a smaller vertex (a new gmin)."""
    n = 1 << 15
    base = graphgen.rmat(15, 1 << 16, 41, scramble=True)
    base = base[(base[:, 0] != 3) & (base[:, 1] != 3)]  # vertex 3 starts isolated
    m = oracle.max_degree_vertex(n, base)
    batches = [graphgen.pairs(n, k, 42, tag=i) for i, k in enumerate([5, 2000, 300000, 1, 40000])]
    batches.insert(2, np.array([[3, m]], np.uint32))  # 3 joins m's component
    seen = [base]

    def want():
        e = np.concatenate(seen)
        if label_space == cc.CC_LABEL_MIN_ID:
            return oracle.min_labels(n, e)
        return oracle.root_value_labels(n, e, m) if mode == cc.CC_ROOT_MAXDEG else oracle.min_labels(n, e)

    with cc.Server(GB, mode=mode, label_space=label_space) as s:
        L0 = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        t, g = s.new_graph(n, dev(base), L0 if admit_labels else None)
        assert s.wait(t) == cc.CC_OK
        if admit_labels:  # else the first snapshot below makes the graph's copy
            np.testing.assert_array_equal(L0.cpu().numpy().view(np.uint32), want())
        for b in batches:
            assert s.wait(s.insert(g, dev(b))) == cc.CC_OK
            seen.append(b)
            for _ in range(2):  # a second snapshot with an empty log
                L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
                torch.cuda.synchronize()
                assert s.wait(s.snapshot(g, L)) == cc.CC_OK
                np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want())


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
def test_inserts_overlap_a_snapshot(mode):
    """Inserts submitted right after a snapshot of the same graph start once
    the snapshot has copied the parent array, while its labels are still
    being computed (Section III: received pairs keep being applied while
    results are produced). Each snapshot and query must still see exactly the
    inserts submitted before it, equal to the oracle, and the mix must give
    the same results as the same requests run one at a time."""
    n = 1 << 25  # the parent array (128 MB) is large enough for a slow first flatten
    base = graphgen.rmat(25, 1 << 26, 17, scramble=True)
    rng = np.random.default_rng(5)
    script = [(0, "new", base)]
    for i in range(4):
        script.append((0, "snapshot", None))
        for size in (300000, 20000, 900):  # a side-stream insert, executor tiles, one tile
            script.append((0, "insert", graphgen.pairs(n, size + int(rng.integers(0, 100)), 31, tag=10 * i + size)))
        script.append((0, "query", graphgen.pairs(n, 5000, 32, tag=i)))
    script.append((0, "snapshot", None))
    graphs = {0: n}
    want = expected(script, graphs)
    # Whether an insert starts inside a snapshot's window (after its copy of
    # P, before its labels) depends on timing: up to three mixed runs, each
    # checked in full, and at least one overlap among them.
    overlaps = 0
    for attempt in range(3):
        with cc.Server(4 * GB, mode=mode) as s:
            mixed, _ = run_script(s, script, graphs, one_at_a_time=False)
            st = s.stats()
            assert st["failed"] == 0
            overlaps += st["snapshot_overlaps"]
        for i, (_, kind, _) in enumerate(script):
            if kind == "query":
                np.testing.assert_array_equal(mixed[i], want[i])
            elif kind == "snapshot":
                np.testing.assert_array_equal(mixed[i].view(np.uint32), want[i])
        if overlaps:
            break
    assert overlaps >= 1
    with cc.Server(4 * GB, mode=mode) as s:
        alone, _ = run_script(s, script, graphs, one_at_a_time=True)
    for i, (_, kind, _) in enumerate(script):
        if kind == "query":
            np.testing.assert_array_equal(alone[i], want[i])
        elif kind == "snapshot":
            np.testing.assert_array_equal(alone[i].view(np.uint32), want[i])


def test_submit_many_keeps_order_and_stops_at_a_refused_request():
    """cc_server_submit_many: inserts and queries queued in one call take effect
    in order (each query sees exactly the inserts before it), and a refused
    request ends the batch with the earlier ones queued."""
    n = 1 << 14
    e0 = graphgen.rmat(14, n * 2, 301, scramble=True)
    batches = [graphgen.pairs(n, size, 302, tag=i) for i, size in enumerate([1, 500, 20000, 3, 70000, 9])]
    q = graphgen.pairs(n, 4000, 303, tag=0)
    seen, expect = [e0], []
    for b in batches:
        seen.append(b)
        L = oracle.min_labels(n, np.concatenate(seen))
        expect.append(L[q[:, 0]] == L[q[:, 1]])
    with cc.Server(2 * GB) as srv:
        t, gid = srv.new_graph(n, dev(e0))
        assert srv.wait(t, 60) == cc.CC_OK
        # one call, inserts and queries alternating
        ins = [dev(b) for b in batches]
        qd = dev(q)
        outs = [torch.empty(q.shape[0], dtype=torch.uint8, device="cuda") for _ in batches]
        arr = (cc.cc_request * (2 * len(batches)))()
        for i, (e, out) in enumerate(zip(ins, outs)):
            r = arr[2 * i]
            r.kind, r.graph, r.edges_dev, r.n_edges = cc.CC_REQ_INSERT, gid, e.data_ptr(), e.shape[0]
            r = arr[2 * i + 1]
            r.kind, r.graph, r.pairs_dev, r.n_pairs, r.out_dev = cc.CC_REQ_QUERY, gid, qd.data_ptr(), q.shape[0], \
                out.data_ptr()
        tickets, st = cc.cc_server_submit_many(srv.h, arr)
        assert st == cc.CC_OK and len(tickets) == 2 * len(batches)
        for tk in tickets:
            assert srv.wait(tk, 60) == cc.CC_OK
        for out, ex in zip(outs, expect):
            assert np.array_equal(out.cpu().numpy().astype(bool), ex)
        # the wrappers: all inserts in one call, then all queries in one, on a
        # fresh copy of the graph: every query sees every insert
        t2, g2 = srv.new_graph(n, dev(e0))
        assert srv.wait(t2, 60) == cc.CC_OK
        outs2 = [torch.empty(q.shape[0], dtype=torch.uint8, device="cuda") for _ in batches]
        tk2 = srv.insert_many(g2, ins) + srv.query_many(g2, [qd] * len(batches), outs2)
        for tk in tk2:
            assert srv.wait(tk, 60) == cc.CC_OK
        for out in outs2:
            assert np.array_equal(out.cpu().numpy().astype(bool), expect[-1])
        # a refused request (misaligned pairs) ends the batch: the two before it are queued
        bad = torch.empty(2 * q.shape[0] + 1, dtype=torch.int32, device="cuda")[1:].view(-1, 2)
        o = [torch.empty(q.shape[0], dtype=torch.uint8, device="cuda") for _ in range(4)]
        with pytest.raises(cc.CCError) as ei:
            srv.query_many(g2, [qd, qd, bad, qd], o)
        assert ei.value.status == cc.CC_ERR_INVALID_ARGUMENT
        assert len(ei.value.tickets) == 2
        for tk in ei.value.tickets:
            assert srv.wait(tk, 60) == cc.CC_OK
        for out in o[:2]:
            assert np.array_equal(out.cpu().numpy().astype(bool), expect[-1])

"""Failure detection by bounded device waits that run out, with no GPU fault.

Every wait in the library's long-lived kernels is bounded by the device
clock; when one expires the kernel records CC_ERR_TIMEOUT and returns, the
context stays usable, and later work succeeds. Each test makes one wait run
out on purpose, from the host side only:

* the serving executor's wait for a tile the host has claimed but not yet
  published: the server's fault injection holds the first request's tiles
  back (a stuck producer) for longer than the configured wait;
* the wait of an insert's apply tiles for its validate tiles, set shorter
  than validation takes;
* the batched kernel's grid barriers, set shorter than the first phase.

After each timeout, results of later requests are checked against the CPU
oracle."""
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


def query(srv, gid, q):
    out = torch.full((len(q),), 7, dtype=torch.uint8, device="cuda")
    t = srv.query(gid, dev(q), out)
    return srv.wait(t, 60), out


def snapshot(srv, gid, n):
    L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    t = srv.snapshot(gid, L)
    st = srv.wait(t, 60)
    return st, L.cpu().numpy().view(np.uint32)


def test_executor_publish_wait_times_out_on_a_stuck_producer_then_recovers():
    n = 1 << 14
    base = graphgen.rmat(14, 1 << 16, 31, scramble=True)
    q = graphgen.pairs(n, 5000, 32)
    # the idle timeout (1 ms) stays below the publish wait (20 ms), so an idle
    # executor is asked to leave before its own waits could expire
    with cc.Server(GB, publish_wait_us=20000, fault_hold_publish_us=500000, idle_timeout_us=1000) as srv:
        t, gid = srv.new_graph(n, dev(base))
        assert srv.wait(t, 60) == cc.CC_OK  # admission runs on a side stream, not on the executor
        # the first executor request: its tiles reach the ring 500 ms late, the
        # executor gives up after 20 ms, leaves, and the host fails the request
        st, _ = query(srv, gid, q)
        assert st == cc.CC_ERR_TIMEOUT
        stats = srv.stats()
        assert stats["executor_timeouts"] >= 1 and stats["failed"] >= 1
        # later requests relaunch the executor and are served correctly
        L = oracle.min_labels(n, base)
        st, out = query(srv, gid, q)
        assert st == cc.CC_OK
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.connected(L, q))
        extra = graphgen.pairs(n, 3000, 33)
        t = srv.insert(gid, dev(extra))
        assert srv.wait(t, 60) == cc.CC_OK
        L2 = oracle.min_labels(n, np.concatenate([base, extra]))
        st, out = query(srv, gid, q)
        assert st == cc.CC_OK
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.connected(L2, q))
        st, got = snapshot(srv, gid, n)
        assert st == cc.CC_OK
        np.testing.assert_array_equal(got, L2)


def test_insert_gate_wait_times_out_and_leaves_a_consistent_forest():
    n = 1 << 15
    base = graphgen.rmat(15, 1 << 17, 41, scramble=True)
    big = graphgen.pairs(n, 200000, 42)  # below the side-insert size: validate tiles, then gated apply tiles
    q = graphgen.pairs(n, 4000, 43)
    with cc.Server(GB, gate_wait_us=1) as srv:
        t, gid = srv.new_graph(n, dev(base))
        assert srv.wait(t, 60) == cc.CC_OK
        t = srv.insert(gid, dev(big))
        # apply tiles claimed while validation still runs give up after 1 us
        assert srv.wait(t, 60) == cc.CC_ERR_TIMEOUT
        st, L = snapshot(srv, gid, n)
        assert st == cc.CC_OK
        # the forest holds the base edges plus some subset A of the batch:
        # with S the batch edges inside one label class (S contains A, and
        # adds no join beyond A's), the labels are exactly the oracle's on
        # base + S, and a refinement of the oracle's on base + batch
        S = big[L[big[:, 0]] == L[big[:, 1]]]
        np.testing.assert_array_equal(L, oracle.min_labels(n, np.concatenate([base, S])))
        U = oracle.min_labels(n, np.concatenate([base, big]))
        assert (U[L] == U).all()
        # queries (ungated) still run and agree with the snapshot
        st, out = query(srv, gid, q)
        assert st == cc.CC_OK
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.connected(L, q))


def test_batched_barrier_wait_times_out_then_a_default_run_matches_the_oracle():
    b = graphgen.batch(256, 51)
    want = oracle.batch_min_labels(b.edges, b.vtx_off, b.edge_off)
    G = len(b.vtx_off) - 1
    vo = torch.from_numpy(b.vtx_off.astype(np.uint64).view(np.int64)).cuda()
    eo = torch.from_numpy(b.edge_off.astype(np.uint64).view(np.int64)).cuda()
    e = dev(b.edges.astype(np.uint32).reshape(-1, 2))
    L = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
    with cc.Batch(G) as bt:
        # the first barrier waits while one block checks 256 graphs' offsets
        cc.cc_batch_set_config(bt.h, barrier_wait_us=1)
        bt.run(G, vo, eo, e, L)
        assert cc.cc_batch_sync_status(bt.h) == cc.CC_ERR_TIMEOUT
        cc.cc_batch_set_config(bt.h, barrier_wait_us=0)  # the default, 4 s
        L.fill_(-1)
        bt.run(G, vo, eo, e, L)
        assert cc.cc_batch_sync_status(bt.h) == cc.CC_OK
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)

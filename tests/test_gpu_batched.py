"""Batched connected components (include/cc_batch.h) against the CPU oracle:
every graph of the concatenated batch gets its own min-id labels, bit for
bit, under every kernel configuration the autotuner can pick, through CUDA
graph capture, and with malformed input reported, not crashing."""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def run_batch(edges, vtx_off, edge_off, **cfg):
    n_graphs = len(vtx_off) - 1
    with cc.Batch(max(n_graphs, 1)) as b:
        if cfg:
            cc.cc_batch_set_config(b.h, **cfg)
        L = torch.full((max(int(vtx_off[-1]), 1),), -7, dtype=torch.int32, device="cuda")
        e = dev(edges.astype(np.uint32).reshape(-1, 2), np.int32) if len(edges) else torch.empty((0, 2), dtype=torch.int32, device="cuda")
        b.run(n_graphs, dev(vtx_off.astype(np.uint64), np.int64), dev(edge_off.astype(np.uint64), np.int64), e, L)
        status = cc.cc_batch_sync_status(b.h)
        return L[: int(vtx_off[-1])].cpu().numpy().view(np.uint32), status


@pytest.fixture(scope="module")
def small_batch():
    b = graphgen.batch(96, 21)
    return b, oracle.batch_min_labels(b.edges, b.vtx_off, b.edge_off)


CONFIGS = [dict(block_size=bs, edges_per_thread=ept, filter=f, tile_edges=te, tile_vertices=tv)
           for bs in (256, 512) for ept in (1, 2, 4) for f in (0, 1)
           for te, tv in ((256, 256), (16384, 4096))]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "-".join(str(v) for v in c.values()))
def test_every_config(small_batch, cfg):
    b, want = small_batch
    got, st = run_batch(b.edges, b.vtx_off, b.edge_off, **cfg)
    assert st == cc.CC_OK
    np.testing.assert_array_equal(got, want)


def test_degenerate_graphs():
    # graphs with no edges, single vertices, self-loops only, one with all
    # edges, and an empty graph in the middle (zero vertices, zero edges)
    parts = [
        (1, []), (5, []), (4, [[0, 1], [2, 3]]), (0, []), (3, [[2, 2], [1, 1]]),
        (7, [[6, 0], [0, 5], [5, 4], [4, 3]]), (2, [[1, 0]] * 50),
    ]
    vtx, edg, es = [0], [0], []
    for nv, e in parts:
        vtx.append(vtx[-1] + nv)
        edg.append(edg[-1] + len(e))
        es.extend(e)
    edges = np.array(es, dtype=np.uint32).reshape(-1, 2)
    want = oracle.batch_min_labels(edges, np.array(vtx), np.array(edg))
    for cfg in ({}, dict(filter=0, edges_per_thread=1)):
        got, st = run_batch(edges, np.array(vtx), np.array(edg), **cfg)
        assert st == cc.CC_OK
        np.testing.assert_array_equal(got, want)


def test_out_of_range_and_bad_offsets_are_reported():
    vtx = np.array([0, 4, 8], np.uint64)
    edg = np.array([0, 2, 3], np.uint64)
    edges = np.array([[0, 1], [2, 9], [3, 2]], np.uint32)  # 9 is not in graph 0
    got, st = run_batch(edges, vtx, edg)
    assert st == cc.CC_ERR_OUT_OF_RANGE
    np.testing.assert_array_equal(got, [0, 0, 2, 3, 0, 1, 2, 2])  # the bad edge is skipped
    bad = np.array([0, 6, 5], np.uint64)  # decreasing vertex offsets
    _, st = run_batch(edges, bad, edg)
    assert st == cc.CC_ERR_INVALID_ARGUMENT


def test_tune_then_run(small_batch):
    b, want = small_batch
    with cc.Batch(b.n_graphs) as bt:
        L = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
        args = (b.n_graphs, dev(b.vtx_off, np.int64), dev(b.edge_off, np.int64), dev(b.edges, np.int32), L)
        assert cc.cc_batch_tune_results(bt.h) == []
        best, ms = bt.tune(*args)
        assert ms > 0 and best["block_size"] in (256, 512)
        assert cc.cc_batch_get_config(bt.h) == best
        # the candidate table: every block size x edges per thread x filter x
        # tile size, the kept one being the fastest
        table = cc.cc_batch_tune_results(bt.h)
        assert len(table) == 2 * 3 * 2 * 4
        assert min(t for _, t in table) == ms
        assert [c for c, t in table if t == ms][0] == best
        L.fill_(-1)
        bt.run(*args)
        bt.sync()
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)


def test_cuda_graph_capture_and_replay(small_batch):
    b, want = small_batch
    with cc.Batch(b.n_graphs) as bt:
        L = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
        vo, eo, e = dev(b.vtx_off, np.int64), dev(b.edge_off, np.int64), dev(b.edges, np.int32)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            bt.run(b.n_graphs, vo, eo, e, L, stream=s)  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.run(b.n_graphs, vo, eo, e, L, stream=s)
        for _ in range(3):
            L.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), want)
        assert cc.cc_batch_sync_status(bt.h) == cc.CC_OK


def test_device_generator_matches_host():
    h = graphgen.batch(64, 33)
    d = graphgen.batch_dev(64, 33)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.edges.cpu().numpy().view(np.uint32), h.edges)


def test_full_batch_against_oracle_values():
    with open(os.path.join(GOLDEN, "batch4096.json")) as f:
        gold = json.load(f)
    d = graphgen.batch_dev(gold["n_graphs"], gold["seed"])
    torch.cuda.synchronize()
    assert d.edges.shape[0] == gold["n_edges"]
    assert hashlib.sha256(d.edges.cpu().numpy().view(np.uint8)).hexdigest() == gold["edges_sha256"]
    with cc.Batch(d.n_graphs) as bt:
        L = torch.empty(int(d.vtx_off_host[-1]), dtype=torch.int32, device="cuda")
        bt.run(d.n_graphs, d.vtx_off, d.edge_off, d.edges, L)
        bt.sync()
        assert hashlib.sha256(L.cpu().numpy().view(np.uint8)).hexdigest() == gold["labels_sha256"]

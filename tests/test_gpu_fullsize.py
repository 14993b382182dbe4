"""Full-size parity: the two single-graph workloads (R-MAT scale 24 with edge
factor 16, and the 8192 x 8192 grid kept with p = 0.9), run on the GPU in the
launch configuration the benchmark times, compared bit for bit with stored
expected values that tests/golden/make_golden.py wrote from the CPU oracle.
The device-generated input is first checked to be the exact edge array the
oracle saw. Properties that hold at any size are checked on the device too."""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")
import bench  # noqa: E402  (the benchmark's launch configuration)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sha_tensor(t) -> str:
    return hashlib.sha256(t.contiguous().cpu().numpy().view(np.uint8)).hexdigest()


@pytest.mark.parametrize("name", ["rmat24_ef16", "grid8192x8192_p0.9", "rmat24_ef16_u"])
def test_fullsize_against_oracle_values(name):
    with open(os.path.join(GOLDEN, f"{name}.json")) as f:
        gold = json.load(f)
    w = graphgen.WORKLOADS[name]
    n = w.n_vertices
    e = w.device_edges()
    torch.cuda.synchronize()
    assert e.shape[0] == gold["n_edges"]
    assert sha_tensor(e) == gold["edges_sha256"], "device generator drifted from the host generator"
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    with cc.Graph(n, **bench.BENCH_OPTIONS) as g:
        for _ in range(2):  # the second run reuses the handle, as the benchmark does
            g.run(e, L)
            g.sync()
            assert sha_tensor(L) == gold["labels_min_id_sha256"]
            assert g.num_components() == gold["num_components"]
            assert g.root_vertex() == gold["max_degree_vertex"]
        sample = torch.tensor(gold["sample_vertices"], dtype=torch.int64, device="cuda")
        assert L[sample].cpu().tolist() == gold["sample_min_id_labels"]
        # properties at any size: every edge inside one label class, L_v <= v,
        # L[L_v] == L_v, and each label is the smallest vertex of its class
        Ll = L.long()
        ev = e.long()
        assert bool((Ll[ev[:, 0]] == Ll[ev[:, 1]]).all())
        ar = torch.arange(n, device="cuda")
        assert bool((Ll <= ar).all())
        assert bool((Ll[Ll] == Ll).all())
        # connected() on the live P agrees with the labels
        q = graphgen.pairs_dev(n, 1 << 20, 77)
        out = torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")
        g.connected(q, out)
        g.sync()
        ql = q.long()
        assert bool((out.bool() == (Ll[ql[:, 0]] == Ll[ql[:, 1]])).all())
    opts = dict(bench.BENCH_OPTIONS, label_space=cc.CC_LABEL_ROOT_VALUE)
    with cc.Graph(n, **opts) as g:
        g.run(e, L)
        g.sync()
        assert sha_tensor(L) == gold["labels_root_value_sha256"]
    opts = dict(bench.BENCH_OPTIONS, mode=cc.CC_ROOT_IDENTITY)
    with cc.Graph(n, **opts) as g:
        g.run(e, L)
        g.sync()
        assert sha_tensor(L) == gold["labels_min_id_sha256"]


def sha_chunked(t, rows=1 << 27) -> str:
    """SHA-256 of a large device tensor, copied to the host in pieces."""
    h = hashlib.sha256()
    for i in range(0, t.shape[0], rows):
        h.update(t[i:i + rows].contiguous().cpu().numpy().view(np.uint8))
    return h.hexdigest()


def test_fullsize_rmat28_against_oracle_values():
    """R-MAT scale 28, edge factor 16: 2^32 edges (34.4 GB, 64-bit edge counts,
    64-bit root-selection counters), run as the benchmark runs it."""
    path = os.path.join(GOLDEN, "rmat28_ef16.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/rmat28_ef16.json not generated")
    with open(path) as f:
        gold = json.load(f)
    w = graphgen.WORKLOADS["rmat28_ef16"]
    n = w.n_vertices
    need = 8 * w.n_edges + 24 * n + (4 << 30)
    if torch.cuda.get_device_properties(0).total_memory < need:
        pytest.skip("needs about 45 GB of device memory")
    e = w.device_edges()
    torch.cuda.synchronize()
    assert e.shape[0] == gold["n_edges"] == 1 << 32
    assert sha_chunked(e) == gold["edges_sha256"], "device generator drifted from the host generator"
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    with cc.Graph(n, **bench.BENCH_OPTIONS) as g:
        for _ in range(2):
            g.run(e, L)
            g.sync()
            assert sha_chunked(L) == gold["labels_min_id_sha256"]
            assert g.num_components() == gold["num_components"]
            assert g.root_vertex() == gold["max_degree_vertex"]
        sample = torch.tensor(gold["sample_vertices"], dtype=torch.int64, device="cuda")
        assert L[sample].cpu().tolist() == gold["sample_min_id_labels"]
        Ll = L.long()
        for i in range(0, e.shape[0], 1 << 28):  # every edge inside one class, in pieces
            ev = e[i:i + (1 << 28)].long()
            assert bool((Ll[ev[:, 0]] == Ll[ev[:, 1]]).all())
            del ev
        ar = torch.arange(n, device="cuda")
        assert bool((Ll <= ar).all())
        assert bool((Ll[Ll] == Ll).all())
        del ar
        q = graphgen.pairs_dev(n, 1 << 20, 78)
        out = torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")
        g.connected(q, out)
        g.sync()
        ql = q.long()
        assert bool((out.bool() == (Ll[ql[:, 0]] == Ll[ql[:, 1]])).all())
        del Ll
    opts = dict(bench.BENCH_OPTIONS, label_space=cc.CC_LABEL_ROOT_VALUE)
    with cc.Graph(n, **opts) as g:
        g.run(e, L)
        g.sync()
        assert sha_chunked(L) == gold["labels_root_value_sha256"]


def test_fullsize_csr_rmat24_equals_coo_labels():
    """The CSR of R-MAT scale 24 (rows sorted by source, built on the device)
    stands for the same edges, so its min-id labels equal the stored COO
    values, whatever vertex the longest row plants."""
    with open(os.path.join(GOLDEN, "rmat24_ef16.json")) as f:
        gold = json.load(f)
    w = graphgen.WORKLOADS["rmat24_ef16"]
    n = w.n_vertices
    e = w.device_edges()
    off, nb = bench.device_csr(e, n)
    del e
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    with cc.Graph(n, **bench.BENCH_OPTIONS) as g:
        cc.cc_run_csr(g.h, off, nb, nb.shape[0], L)
        g.sync()
        assert sha_tensor(L) == gold["labels_min_id_sha256"]
        assert g.num_components() == gold["num_components"]
        lens = (off[1:] - off[:-1])
        assert g.root_vertex() == int(torch.argmax(lens).item())  # first index of the maximum



def test_fullsize_serving_rmat26_against_oracle_values():
    """The serving configuration at full size: resident R-MAT scale 26 (1.07G
    edges) in the bench's server setup, then the bench's executor insert burst
    (512 batches of 2^17 pairs, one submission call) and four side-path
    inserts of 2^20 pairs; a snapshot must equal the oracle's labels of the
    union, bit for bit, and queries must agree with the snapshot."""
    path = os.path.join(GOLDEN, "serving_rmat26.json")
    with open(path) as f:
        gold = json.load(f)
    w = graphgen.RMAT26
    n = w.n_vertices
    e = w.device_edges()
    pool = graphgen.pairs_dev(n, gold["pool_pairs"], gold["pool_seed"])
    torch.cuda.synchronize()
    assert e.shape[0] == gold["n_edges"]
    assert sha_chunked(e) == gold["edges_sha256"], "device generator drifted from the host generator"
    assert sha_tensor(pool) == gold["pool_sha256"]
    batches = [pool[o:o + c] for o, c in gold["inserts"]]
    with cc.Server(24 << 30, idle_timeout_us=200000) as srv:
        t, gid = srv.new_graph(n, e)
        assert srv.wait(t, 120) == cc.CC_OK
        small = [b for b in batches if b.shape[0] < (1 << 18)]
        large = [b for b in batches if b.shape[0] >= (1 << 18)]
        assert len(small) == 512 and len(large) == 4
        tickets = srv.insert_many(gid, small) + [srv.insert(gid, b) for b in large]
        for tk in tickets:
            assert srv.wait(tk, 120) == cc.CC_OK
        L = torch.empty(n, dtype=torch.int32, device="cuda")
        t = srv.snapshot(gid, L)
        assert srv.wait(t, 120) == cc.CC_OK
        assert sha_tensor(L) == gold["labels_min_id_sha256"]
        sample = torch.tensor(gold["sample_vertices"], dtype=torch.int64, device="cuda")
        assert L[sample].cpu().tolist() == gold["sample_min_id_labels"]
        q = graphgen.pairs_dev(n, 1 << 20, 78)
        out = torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")
        t = srv.query(gid, q, out)
        assert srv.wait(t, 120) == cc.CC_OK
        Ll, ql = L.long(), q.long()
        assert bool((out.bool() == (Ll[ql[:, 0]] == Ll[ql[:, 1]])).all())
        assert srv.stats()["executor_timeouts"] == 0
    del e, pool, batches, L
    torch.cuda.empty_cache()

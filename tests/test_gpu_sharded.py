"""Edge sharding with one Reducer step (Section III, Algorithm 2) on the GPU.

cc_forest_pairs turns a parent array into the pairs (v, parent of v) that a
machine sends to the Reducer; they must have exactly the components of the
edges applied so far. The sharded pipeline (each slice's pass on a private
parent array, the forests gathered, the Reducer's pass over them) must give
the oracle's labels of the whole graph. On one GPU the ranks' passes run one
after another, with no kernel waiting on another."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")
from paper_2507_03695_gb300 import sharded  # noqa: E402


def dev(e):
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.uint32).reshape(-1, 2).view(np.int32)).cuda()


@pytest.mark.parametrize("mode", [cc.CC_ROOT_MAXDEG, cc.CC_ROOT_IDENTITY])
@pytest.mark.parametrize("compressed", [True, False])
def test_forest_pairs_have_the_components_of_the_edges(mode, compressed):
    n = 1 << 16
    e = graphgen.rmat(16, 1 << 19, 41, scramble=True)
    extra = graphgen.pairs(n, 5000, 42)
    want = oracle.min_labels(n, np.concatenate([e, extra]))
    with cc.Graph(n, mode=mode) as g:
        g.run(dev(e), None)
        g.insert(dev(extra))  # the inserted edges leave P uncompressed
        if compressed:
            g.labels(torch.empty(n, dtype=torch.int32, device="cuda"))
        p = g.forest_pairs()
        g.sync()
        pairs = p.cpu().numpy().view(np.uint32)
        assert len(pairs) == n - oracle.num_components(want)
        assert (pairs[:, 0] != pairs[:, 1]).all() and (pairs < n).all()
        assert len(np.unique(pairs[:, 0])) == len(pairs)  # one pair per non-root vertex
        np.testing.assert_array_equal(oracle.min_labels(n, pairs), want)
        if compressed:  # after pointer jumping every pair names a root
            roots = set(pairs[:, 0].tolist())
            assert not any(int(r) in roots for r in pairs[:, 1])
        # a buffer that is too small: the status says so and gives the count
        small = torch.empty((10, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(cc.CCError) as ex:
            cc.cc_forest_pairs(g.h, small)
        assert ex.value.status == cc.CC_ERR_TOO_LARGE and ex.value.count == len(pairs)


def test_forest_pairs_of_an_edgeless_graph_are_empty():
    with cc.Graph(100) as g:
        g.run(torch.empty((0, 2), dtype=torch.int32, device="cuda"), None)
        assert g.forest_pairs().shape[0] == 0


@pytest.mark.parametrize("world", [1, 3, 4])
def test_sharded_pipeline_equals_the_oracle(world):
    n = 1 << 20
    e = graphgen.rmat(20, 1 << 23, 43, scramble=True)
    e_dev = dev(e)
    forests = []
    for r in range(world):
        a, b = sharded.edge_range(len(e), r, world)
        forests.append(sharded.shard_forest(n, e_dev[a:b]))
    pairs_all = torch.cat(forests)
    assert pairs_all.shape[0] <= min(len(e), world * n)  # the exchange volume bound (Section V)
    L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sharded.reduce_forests(n, pairs_all, L)
    np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), oracle.min_labels(n, e))


def test_run_sharded_through_a_one_rank_nccl_group():
    import os
    import socket
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        n = 1 << 18
        e = graphgen.rmat(18, 1 << 21, 44, scramble=True)
        L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        out = sharded.run_sharded(n, dev(e), dist, L)
        assert out is L
        np.testing.assert_array_equal(L.cpu().numpy().view(np.uint32), oracle.min_labels(n, e))
    finally:
        dist.destroy_process_group()

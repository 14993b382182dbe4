"""Edge sharding with one Reducer step (Section III, Algorithm 2), host side,
on CPU: the edge-balanced slices, and the exchange of the per-rank forests to
the Reducer over two gloo ranks. Each rank's forest comes from the CPU oracle
here (the (v, L_v) pairs of its slice's min-id labels: a valid forest of the
slice); the Reducer's labels over the gathered pairs must equal the oracle's
labels of the whole edge list."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen
import oracle
from paper_2507_03695_gb300 import sharded

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("E,world", [(0, 1), (1, 2), (7, 3), (10, 4), (1000003, 8), (64, 64), (5, 8)])
def test_edge_ranges_partition_the_edges(E, world):
    spans = [sharded.edge_range(E, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == E
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in spans]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.edge_range(E, world, world)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch
    sys.path.insert(0, ROOT)
    import graphgen as gg
    import oracle as orc
    from paper_2507_03695_gb300 import sharded as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 1 << 12
    e = gg.rmat(12, 5 * n + 3, 31, scramble=True)
    a, b = sh.edge_range(len(e), rank, world)
    L = orc.min_labels(n, e[a:b])
    v = np.flatnonzero(L != np.arange(n, dtype=np.uint32)).astype(np.uint32)
    if rank == 1:
        v = v[:0]  # an empty forest on one rank: padding and trimming still agree
    pairs = torch.from_numpy(np.stack([v, L[v]], 1).astype(np.uint32).view(np.int32))
    got = sh.gather_to_reducer(pairs, dist, reducer=0)
    if rank == 0:
        g = got.numpy().view(np.uint32)
        # rank 1 sent nothing: the Reducer sees rank 0's forest only
        want = orc.min_labels(n, e[a:b])
        q.put((rank, np.array_equal(orc.min_labels(n, g), want), int(got.shape[0]), len(v)))
    else:
        q.put((rank, got is None, 0, 0))
    dist.barrier()
    dist.destroy_process_group()


def _rank_full(rank, world, port, q):
    import torch
    sys.path.insert(0, ROOT)
    import graphgen as gg
    import oracle as orc
    from paper_2507_03695_gb300 import sharded as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 1 << 14
    e = gg.rmat(14, 6 * n + 1, 32, scramble=True)
    a, b = sh.edge_range(len(e), rank, world)
    L = orc.min_labels(n, e[a:b])
    v = np.flatnonzero(L != np.arange(n, dtype=np.uint32)).astype(np.uint32)
    pairs = torch.from_numpy(np.stack([v, L[v]], 1).astype(np.uint32).view(np.int32))
    got = sh.gather_to_reducer(pairs, dist, reducer=1)  # the Reducer need not be rank 0
    if rank == 1:
        g = got.numpy().view(np.uint32)
        ok = np.array_equal(orc.min_labels(n, g), orc.min_labels(n, e))
        # the exchange volume bound of Section V: at most min(E, ranks * n) pairs
        q.put((rank, ok and len(g) <= min(len(e), world * n), int(len(g)), 0))
    else:
        q.put((rank, got is None, 0, 0))
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {r: rest for r, *rest in (q.get(timeout=120) for _ in procs)}
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return res


def test_gather_to_reducer_two_gloo_ranks_with_an_empty_forest():
    res = _spawn(_rank, 2)
    assert res[0][0] and res[1][0]
    assert res[0][1] == res[0][2]  # nothing but rank 0's pairs arrived


def test_sharded_labels_equal_the_whole_graph_two_gloo_ranks():
    res = _spawn(_rank_full, 2)
    assert res[0][0] and res[1][0]
    assert res[1][1] > 0

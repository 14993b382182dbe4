"""cc_max_degree_vertex_noalloc: the maximum-degree vertex for callers that
cannot allocate device memory -- code running inside another framework's
allocator or pool callbacks, services whose device memory is fixed at
start-up, code that must not risk the device synchronisation of cudaMalloc.
Its scratch is a fixed static device array inside the library.

Called through the C ABI, it must give the vertex the CPU oracle computes
(oracle.max_degree_vertex: endpoint occurrences, a self-loop twice, ties to
the smaller id) and the same vertex as the existing entry point (cc_run in
f = R mode with exact root selection, then cc_root_vertex), on consecutive
calls whose inputs differ, so counts left in the shared array by one call
cannot leak into the next.

Collected last on purpose: run it alone in a fresh process, or after the
other GPU tests."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")

MAX_V = 1 << 22  # CC_NOALLOC_MAX_VERTICES


def existing_entry_point(n, e_dev):
    with cc.Graph(n, mode=cc.CC_ROOT_MAXDEG, root_select=cc.CC_ROOT_SELECT_EXACT) as g:
        g.run(e_dev, None)
        g.sync()
        return g.root_vertex()


def noalloc(n, e_dev, n_edges=None):
    m_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    cc.cc_max_degree_vertex_noalloc(e_dev, n, m_out, n_edges=n_edges)
    torch.cuda.synchronize()
    return int(m_out.item())


def to_dev(e):
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.uint32).reshape(-1, 2).view(np.int32)).cuda()


def test_noalloc_matches_oracle_and_existing_entry_point_on_consecutive_calls():
    n = 1 << 16
    a = graphgen.rmat(16, 1 << 20, 1, scramble=False)   # hub at vertex 0, degree ~26K
    b = np.stack([np.full(1000, 5), np.arange(1000, 2000)], 1).astype(np.uint32)  # star: vertex 5, degree 1000
    c = graphgen.rmat(16, 1 << 19, 3, scramble=True)     # hub elsewhere
    inputs = (a, b, c, a)
    want = [oracle.max_degree_vertex(n, x) for x in inputs]
    assert want[1] == 5 and want[0] != want[1] != want[2]
    assert [existing_entry_point(n, to_dev(x)) for x in inputs] == want
    got = [noalloc(n, to_dev(x)) for x in inputs]   # four calls in a row, no clearing in between
    assert got == want


def test_noalloc_near_the_size_limit_and_misaligned_input():
    n = MAX_V
    e = graphgen.rmat(22, 1 << 24, 8, scramble=True)
    want = oracle.max_degree_vertex(n, e)
    assert existing_entry_point(n, to_dev(e)) == want
    assert noalloc(n, to_dev(e)) == want
    buf = torch.empty((len(e) + 1, 2), dtype=torch.int32, device="cuda")
    buf[1:] = to_dev(e)
    assert buf[1:].data_ptr() % 16 == 8
    assert noalloc(n, buf[1:]) == want
    # a smaller graph right after the large one
    small = graphgen.rmat(12, 1 << 14, 2, scramble=True)
    assert noalloc(1 << 12, to_dev(small)) == oracle.max_degree_vertex(1 << 12, small)


def test_noalloc_empty_edge_list_and_out_of_range_ids():
    # an edgeless graph: every degree is 0, the smallest id wins
    empty = torch.empty((0, 2), dtype=torch.int32, device="cuda")
    assert noalloc(100, empty) == oracle.max_degree_vertex(100, np.empty((0, 2), np.uint32)) == 0
    # after a call that left counts behind, an edgeless call still gives 0
    star = np.stack([np.full(50, 7), np.arange(10, 60)], 1).astype(np.uint32)
    assert noalloc(100, to_dev(star)) == 7
    assert noalloc(100, empty) == 0
    # endpoints >= n are not counted, the other endpoint of such an edge is:
    # k edges (x, bad) add k to x, which the oracle sees as k / 2 self-loops
    # on x; edges with both endpoints bad add nothing
    n, bad = 64, 1000
    rng = np.random.default_rng(4)
    valid = rng.integers(0, n, size=(300, 2)).astype(np.uint32)
    x, k = 41, 40
    odd = np.concatenate([valid, np.stack([np.full(k, x), np.full(k, bad)], 1),
                          np.full((25, 2), bad)]).astype(np.uint32)
    rng.shuffle(odd)
    same = np.concatenate([valid, np.full((k // 2, 2), x)]).astype(np.uint32)
    want = oracle.max_degree_vertex(n, same)
    assert want == x  # the extra half-edges make x the maximum
    assert noalloc(n, to_dev(odd)) == want
    assert noalloc(n, to_dev(valid)) == oracle.max_degree_vertex(n, valid)


def test_noalloc_rejects_sizes_over_the_limit():
    e = to_dev(np.array([[0, 1]], np.uint32))
    m_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as ex:
        cc.cc_max_degree_vertex_noalloc(e, MAX_V + 1, m_out)
    assert ex.value.status == cc.CC_ERR_TOO_LARGE
    with pytest.raises(cc.CCError) as ex:
        cc.cc_max_degree_vertex_noalloc(e, 0, m_out)
    assert ex.value.status == cc.CC_ERR_INVALID_ARGUMENT
    # 2^31 edges would overflow the 32-bit counters: rejected on the host,
    # before any device memory is touched
    with pytest.raises(cc.CCError) as ex:
        cc.cc_max_degree_vertex_noalloc(e, 16, m_out, n_edges=1 << 31)
    assert ex.value.status == cc.CC_ERR_TOO_LARGE
    assert int(m_out.item()) == 0  # untouched by the rejected calls

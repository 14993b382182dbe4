"""cc_max_degree_vertex_noalloc: the maximum-degree vertex for callers that
cannot allocate device memory (its scratch is a fixed static device array
inside the library). Called through the C ABI, it must give the same vertex
as the existing entry point (cc_run in f = R mode with exact root selection,
then cc_root_vertex), on consecutive calls whose inputs differ, so counts
left in the shared array by one call cannot leak into the next.

Collected last on purpose: run it alone in a fresh process, or after the
other GPU tests."""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cc = pytest.importorskip("paper_2507_03695_gb300")

MAX_V = 1 << 22  # CC_NOALLOC_MAX_VERTICES


def existing_entry_point(n, e_dev):
    with cc.Graph(n, mode=cc.CC_ROOT_MAXDEG, root_select=cc.CC_ROOT_SELECT_EXACT) as g:
        g.run(e_dev, None)
        g.sync()
        return g.root_vertex()


def noalloc(n, e_dev):
    m_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    cc.cc_max_degree_vertex_noalloc(e_dev, n, m_out)
    torch.cuda.synchronize()
    return int(m_out.item())


def to_dev(e):
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.uint32).view(np.int32)).cuda()


def test_noalloc_matches_existing_entry_point_on_consecutive_calls():
    n = 1 << 16
    a = to_dev(graphgen.rmat(16, 1 << 20, 1, scramble=False))   # hub at vertex 0, degree ~26K
    star = np.stack([np.full(1000, 5), np.arange(1000, 2000)], 1)  # vertex 5, degree 1000
    b = to_dev(star)
    c = to_dev(graphgen.rmat(16, 1 << 19, 3, scramble=True))     # hub elsewhere
    want = [existing_entry_point(n, x) for x in (a, b, c, a)]
    assert want[1] == 5 and want[0] != want[1] != want[2]
    got = [noalloc(n, x) for x in (a, b, c, a)]   # four calls in a row, no clearing in between
    assert got == want


def test_noalloc_near_the_size_limit_and_misaligned_input():
    n = MAX_V
    e = graphgen.rmat(22, 1 << 24, 8, scramble=True)
    want = existing_entry_point(n, to_dev(e))
    assert noalloc(n, to_dev(e)) == want
    buf = torch.empty((len(e) + 1, 2), dtype=torch.int32, device="cuda")
    buf[1:] = to_dev(e)
    assert buf[1:].data_ptr() % 16 == 8
    assert noalloc(n, buf[1:]) == want
    # a smaller graph right after the large one
    small = graphgen.rmat(12, 1 << 14, 2, scramble=True)
    assert noalloc(1 << 12, to_dev(small)) == existing_entry_point(1 << 12, to_dev(small))


def test_noalloc_rejects_sizes_over_the_limit():
    e = to_dev(np.array([[0, 1]], np.uint32))
    m_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as ex:
        cc.cc_max_degree_vertex_noalloc(e, MAX_V + 1, m_out)
    assert ex.value.status == cc.CC_ERR_TOO_LARGE
    with pytest.raises(cc.CCError) as ex:
        cc.cc_max_degree_vertex_noalloc(e, 0, m_out)
    assert ex.value.status == cc.CC_ERR_INVALID_ARGUMENT
    assert int(m_out.item()) == 0  # untouched by the rejected calls

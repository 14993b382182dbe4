"""The largest vertex count the library accepts, n = 2^31 - 1 (Eq. 1's root
value v + 1 must fit the int32 parent array): P and the labels are 8 GiB
each, the zero-tree bitmap 256 MiB, and the top vertex's root value is
exactly INT32_MAX.

The oracle runs on the touched vertices only, renumbered in increasing order.
Renumbering that keeps the order keeps every component's smallest member, so
the oracle's labels map back to the original ids; every untouched vertex is a
component of its own (L_v = v)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2507_03695_gb300 as cc

pytestmark = pytest.mark.gpu

N_MAX = (1 << 31) - 1


def _edges():
    rng = np.random.default_rng(31)
    n = N_MAX
    hub = n - 5
    pool = np.unique(np.concatenate([
        rng.integers(0, n - 1, size=400_000, dtype=np.int64),
        np.array([0, 1, 2, 3, n - 2, n - 3, n - 4, n - 5, n - 6], dtype=np.int64)]))
    spokes = rng.choice(pool, size=50_000, replace=False)
    star = np.stack([np.full(spokes.size, hub), spokes], axis=1)          # the planted vertex
    rand = pool[rng.integers(0, pool.size, size=(200_000, 2))]             # random pairs
    # the top vertex n - 1 only in a self-loop: a component of its own whose
    # root value (Eq. 1) is n = INT32_MAX; a chain from the top to a low id;
    # a duplicate edge
    top = np.array([[n - 1, n - 1], [n - 2, n - 3], [n - 3, 3], [n - 2, n - 3], [n - 4, n - 6]],
                   dtype=np.int64)
    e = np.concatenate([star, rand, top]).astype(np.uint32)
    return e, hub


def _oracle_labels(e: np.ndarray):
    """(touched ids, their min-id labels, the max-degree vertex)."""
    ids, inv = np.unique(e.astype(np.int64), return_inverse=True)
    ec = inv.reshape(-1, 2).astype(np.uint32)
    Lc = oracle.min_labels(int(ids.size), ec)
    mc = oracle.max_degree_vertex(int(ids.size), ec)
    return ids, ids[Lc.astype(np.int64)], int(ids[mc])


def test_max_vertex_count_matches_the_oracle():
    n = N_MAX
    e, hub = _edges()
    ids, L_touched, m = _oracle_labels(e)
    assert m == hub
    n_comp_touched = int(np.unique(L_touched).size)
    e_dev = torch.from_numpy(e.view(np.int32)).cuda()
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    ids_dev = torch.from_numpy(ids).cuda()
    with cc.Graph(n) as g:                                # f = R, exact selection, min-id labels
        g.run(e_dev, L)
        g.sync()
        assert g.root_vertex() == m
        assert g.num_components() == n - ids.size + n_comp_touched
        assert np.array_equal(L[ids_dev].cpu().numpy().astype(np.int64), L_touched)
        # untouched vertices keep their own id; checked in slices to bound the scratch
        touched = torch.zeros(n, dtype=torch.bool, device="cuda")
        touched[ids_dev] = True
        step = 1 << 28
        for a in range(0, n, step):
            b = min(n, a + step)
            ar = torch.arange(a, b, dtype=torch.int32, device="cuda")
            keep = ~touched[a:b]
            assert bool((L[a:b][keep] == ar[keep]).all())
        del touched
        # connected() on the live P at the top of the id range
        q = torch.tensor([[n - 1, 3], [n - 2, 3], [n - 4, n - 6], [n - 1, n - 1], [n - 1, n - 2]],
                         dtype=torch.int32, device="cuda")
        out = torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")
        g.connected(q, out)
        g.sync()
        Lt = dict(zip(ids.tolist(), L_touched.tolist()))
        assert Lt[n - 1] == n - 1 and Lt[n - 2] == Lt[3]
        expect = [Lt[u] == Lt[v] for u, v in q.cpu().tolist()]
        assert out.cpu().tolist() == [int(x) for x in expect]
    # root-value labels (Eq. 1): 0 in m's component, else the min-id label + 1;
    # the top vertex's is n = 2^31 - 1, the largest int32
    with cc.Graph(n, label_space=cc.CC_LABEL_ROOT_VALUE) as g:
        g.run(e_dev, L)
        g.sync()
        assert g.root_vertex() == m
        expect_rv = np.where(L_touched == Lt[m], 0, L_touched + 1)
        assert np.array_equal(L[ids_dev].cpu().numpy().astype(np.int64), expect_rv)
        assert int(L[n - 1].item()) == (1 << 31) - 1
        v = next(v for v in range(n - 7, 0, -1) if v not in Lt)  # an untouched vertex: its own root
        assert int(L[v].item()) == v + 1
    del L, e_dev
    torch.cuda.empty_cache()


def test_wide_histogram_without_a_hub():
    """2^31 + 5 edges (i mod n, (i + 1) mod n) on n = 2^20 vertices: a cycle
    wound 2048 times. No vertex stands out in the sample, so the certificate
    finds no candidate and the exact selection falls back to the full
    histogram, in 64-bit counters (2^31 edges or more). Closed form, pinned
    against the oracle in tests/test_oracle_pins.py::test_wound_cycle_closed_form:
    vertices 1 .. 4 have the largest degree, so m = 1; one component, min-id
    label 0 (root value 0 under f = R)."""
    n = 1 << 20
    E = (1 << 31) + 5
    e = torch.empty((E, 2), dtype=torch.int32, device="cuda")
    step = 1 << 28
    for a in range(0, E, step):
        b = min(E, a + step)
        i = torch.arange(a, b, dtype=torch.int64, device="cuda")
        e[a:b, 0] = (i % n).to(torch.int32)
        e[a:b, 1] = ((i + 1) % n).to(torch.int32)
        del i
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    for label_space in (cc.CC_LABEL_MIN_ID, cc.CC_LABEL_ROOT_VALUE):
        with cc.Graph(n, label_space=label_space) as g:
            g.run(e, L)
            g.sync()
            assert g.root_vertex() == 1
            assert g.num_components() == 1
            assert int(L.min().item()) == 0 and int(L.max().item()) == 0
    # the same edges from pinned host memory: the chunked selection of
    # cc_run_host sees no hub in its first chunk and builds the full
    # histogram, 64-bit, chunk by chunk
    h = torch.empty((E, 2), dtype=torch.int32, pin_memory=True)
    h.copy_(e)
    del e, L
    torch.cuda.empty_cache()
    Lh = torch.full((n,), -1, dtype=torch.int32, pin_memory=True)
    with cc.Graph(n, E) as g:
        cc.cc_run_host(g.h, h, E, Lh)
        assert g.root_vertex() == 1
        assert g.num_components() == 1
        assert int(Lh.min().item()) == 0 and int(Lh.max().item()) == 0
    del h, Lh
    torch.cuda.empty_cache()

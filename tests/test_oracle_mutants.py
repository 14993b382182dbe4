"""Planted mistakes in the oracle (CPU only): each mutant of cc_oracle.c --
a dropped term, a wrong comparison, a transposed operand, a wrong index --
must fail at least one of the pins that guard the real oracle."""
import ctypes
import itertools
import multiprocessing
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "cc_oracle.c")

MUTANTS = {
    "union_larger_root_wins": ("    if (ra < rb)\n      parent[rb] = ra;", "    if (ra > rb)\n      parent[rb] = ra;"),
    "labels_without_find": ("L[v] = uf_find(h->parent, (uint32_t)v);", "L[v] = h->parent[v];"),
    "R_drops_plus_one": ("return v == m ? 0 : v + 1;", "return v == m ? 0 : v;"),
    "R_compare_flipped": ("if (R_of(ra, m) < R_of(rb, m))", "if (R_of(ra, m) > R_of(rb, m))"),
    "bfs_one_direction": ("    adj[fill[b]++] = a;\n", "\n"),
    "bfs_label_by_parent": ("          L[y] = (uint32_t)s;", "          L[y] = x;"),
    "degree_tie_to_larger": ("if (deg[v] > deg[best]) best = v;", "if (deg[v] >= deg[best]) best = v;"),
    "edge_index_transposed": ("uint32_t a = edges[2 * i], b = edges[2 * i + 1];\n    if (a >= h->n",
                              "uint32_t a = edges[2 * i], b = edges[2 * i];\n    if (a >= h->n"),
    "rfjt_hook_wrong_direction": ("      P[v] = (uint32_t)f_of(use_r, m, u);\n    else\n      P[u] = (uint32_t)f_of(use_r, m, v);",
                                  "      P[u] = (uint32_t)f_of(use_r, m, v);\n    else\n      P[v] = (uint32_t)f_of(use_r, m, u);"),
    "rfjt_inverse_off_by_one": ("return c == 0 ? m : c - 1; /* Eq. 2 */", "return c == 0 ? m : c; /* Eq. 2 */"),
    "pointer_jump_keeps_parent": ("    P[v] = P[u];\n  }", "    P[v] = P[v];\n  }"),
    "csr_row_tie_to_larger": ("if (len > best_len) {", "if (len >= best_len) {"),
    "csr_row_len_dropped_term": ("const uint64_t len = offsets[v + 1] - offsets[v];",
                                 "const uint64_t len = offsets[v + 1];"),
    "degree_add_counts_only_u": ("  for (uint64_t i = 0; i < 2 * n_edges; ++i) {\n    if (edges[i] >= n) return -1;",
                                 "  for (uint64_t i = 0; i < 2 * n_edges; i += 2) {\n    if (edges[i] >= n) return -1;"),
    "degree_add_first_half_only": ("  for (uint64_t i = 0; i < 2 * n_edges; ++i) {\n    if (edges[i] >= n) return -1;",
                                   "  for (uint64_t i = 0; i < n_edges; ++i) {\n    if (edges[i] >= n) return -1;"),
    "degree_add_no_range_check": ("    if (edges[i] >= n) return -1;\n    deg[edges[i]]++;", "    deg[edges[i]]++;"),
}


def _build(tmp_path, name, src) -> str:
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c)])
    return str(so)


def _load(so):
    lib = ctypes.CDLL(so)
    u64, i32, p = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_min_labels.argtypes = [u64, p, u64, p]
    lib.oracle_bfs_labels.argtypes = [u64, p, u64, p]
    lib.oracle_root_value_labels.argtypes = [u64, p, u64, u64, p]
    lib.oracle_max_degree_vertex.argtypes = [u64, p, u64, p]
    lib.oracle_max_degree_vertex.restype = ctypes.c_int64
    lib.oracle_csr_max_row_vertex.argtypes = [u64, p]
    lib.oracle_csr_max_row_vertex.restype = ctypes.c_int64
    lib.oracle_rfjt_init.argtypes = [u64, i32, u64, p]
    lib.oracle_rfjt_hook.argtypes = [u64, i32, u64, p, u64, p]
    lib.oracle_rfjt_pointer_jump.argtypes = [u64, i32, u64, p]
    lib.oracle_degree_add.argtypes = [u64, p, u64, p]
    lib.oracle_degree_add.restype = i32
    return lib


def _pins_pass(lib) -> bool:
    """A compact copy of the pin suite run against a given build."""
    def labels(fn, n, e, *extra):
        L = np.empty(n, np.uint32)
        fn(n, e.ctypes.data, len(e), *extra, L.ctypes.data)
        return L

    n = 5
    cand = [(a, b) for a in range(n) for b in range(a + 1, n)]
    rng = np.random.default_rng(3)
    for mask in range(1 << len(cand)):
        e = np.array([cand[i] for i in range(len(cand)) if mask >> i & 1], np.uint32).reshape(-1, 2)
        e = np.where(rng.random((len(e), 1)) < 0.5, e[:, ::-1], e).astype(np.uint32).copy()
        ref = oracle.closure_labels(n, e)
        if not (labels(lib.oracle_min_labels, n, e) == ref).all():
            return False
        if not (labels(lib.oracle_bfs_labels, n, e) == ref).all():
            return False
        for m in range(n):
            if not (labels(lib.oracle_root_value_labels, n, e, m) == np.where(ref == ref[m], 0, ref + 1)).all():
                return False
    # the tie rule of the degree argmax
    e = np.array([[1, 1], [2, 3], [2, 4], [0, 5]], np.uint32)
    if lib.oracle_max_degree_vertex(6, e.ctypes.data, len(e), None) != 1:
        return False
    # the streaming degree count, fed in uneven chunks, against bincount of
    # both endpoint columns; an out-of-range id is rejected
    for trial in range(10):
        n = int(rng.integers(1, 60))
        e = rng.integers(0, n, size=(int(rng.integers(1, 200)), 2)).astype(np.uint32)
        deg = np.zeros(n, np.uint64)
        for chunk in np.array_split(e, int(rng.integers(1, 5))):
            chunk = np.ascontiguousarray(chunk)
            if lib.oracle_degree_add(n, chunk.ctypes.data, len(chunk), deg.ctypes.data) != 0:
                return False
        if not (deg == np.bincount(e.ravel(), minlength=n)).all():
            return False
    deg = np.zeros(8, np.uint64)
    e = np.array([[0, 1], [2, 9]], np.uint32)
    if lib.oracle_degree_add(4, e.ctypes.data, len(e), deg.ctypes.data) != -1:
        return False
    # CSR rows: on a symmetric graph without self-loops the longest row is
    # the vertex of largest degree (same tie rule); ties and empty rows
    for trial in range(20):
        k = int(rng.integers(1, 12))
        e = rng.integers(0, 8, size=(k, 2)).astype(np.uint32)
        e = e[e[:, 0] != e[:, 1]]
        sym = np.concatenate([e, e[:, ::-1]]).astype(np.uint32)
        off = np.zeros(9, np.uint64)
        np.cumsum(np.bincount(sym[:, 0], minlength=8), out=off[1:])
        want = lib.oracle_max_degree_vertex(8, np.ascontiguousarray(e).ctypes.data, len(e), None) if len(e) else 0
        if lib.oracle_csr_max_row_vertex(8, off.ctypes.data) != want:
            return False
    off = np.array([0, 0, 2, 2, 4, 5], np.uint64)  # rows 1 and 3 tie at 2
    if lib.oracle_csr_max_row_vertex(5, off.ctypes.data) != 1:
        return False
    # sequential Algorithm 3, both root functions, every order of small cases
    for trial in range(6):
        k = 4
        e0 = rng.integers(0, 6, size=(k, 2)).astype(np.uint32)
        ref = oracle.closure_labels(6, e0)
        for use_r, m in ((0, 0), (1, int(rng.integers(0, 6)))):
            for perm in itertools.permutations(range(k)):
                e = e0[list(perm)].copy()
                P = np.empty(6, np.uint32)
                lib.oracle_rfjt_init(6, use_r, m, P.ctypes.data)
                lib.oracle_rfjt_hook(6, use_r, m, e.ctypes.data, k, P.ctypes.data)
                lib.oracle_rfjt_pointer_jump(6, use_r, m, P.ctypes.data)
                want = np.where(ref == ref[m], 0, ref + 1) if use_r else ref
                if not (P == want).all():
                    return False
    # Fig. 1 trace
    P = np.empty(5, np.uint32)
    lib.oracle_rfjt_init(5, 0, 0, P.ctypes.data)
    for edge, expect in (([3, 2], {3: 2}), ([3, 1], {2: 1, 3: 2})):
        e = np.array([edge], np.uint32)
        lib.oracle_rfjt_hook(5, 0, 0, e.ctypes.data, 1, P.ctypes.data)
        if any(P[k] != v for k, v in expect.items()):
            return False
    return True


def _child(so):
    raise SystemExit(0 if _pins_pass(_load(so)) else 1)


def _pins_pass_isolated(so) -> bool:
    """Run the pins in a fresh process: a mutant may crash or loop forever,
    which counts as caught."""
    ctx = multiprocessing.get_context("spawn")
    proc = ctx.Process(target=_child, args=(so,))
    proc.start()
    proc.join(120)
    if proc.is_alive():
        proc.kill()
        proc.join()
        return False
    return proc.exitcode == 0


def test_unmutated_oracle_passes_compact_pins(tmp_path):
    assert _pins_pass_isolated(_build(tmp_path, "orig", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    so = _build(tmp_path, name, src.replace(old, new))
    assert not _pins_pass_isolated(so), f"planted mistake {name} was not caught by the pins"

"""The CPU oracle for connected-components labels.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. It shares no code with the
CUDA path and never imports it.

Plain, slow, sequential. The arithmetic is in ``cc_oracle.c`` (single-threaded
C, built with gcc); this module loads it with ctypes and adds the brute-force
transitive closure used to pin it on tiny graphs. What each function computes,
with the passage of the paper it follows:

* :func:`min_labels` -- ``L[v] = min{w : w ~ v}`` (Section II, terminology:
  ``L_u = L_v`` iff u, v share a component; the JT description identifies each
  component by its lowest vertex id).
* :func:`root_value_labels` -- ``L[v] = min{R(w) : w ~ v}``, the value that the
  pointer jumping of Algorithm 3 leaves in ``P`` when ``f = R`` (Eq. 1).
* :func:`bfs_labels` -- the same min-id labels by search-based CC (Section II,
  related work), a different algorithm, used to pin :func:`min_labels`.
* :func:`closure_labels` -- the definition itself on tiny graphs: a
  transitive-closure (Warshall) matrix, then the minimum of each row.
* :func:`max_degree_vertex` -- ``m`` of Eq. 1 (Algorithm 4, ``max_degree()``):
  endpoint occurrences, ties to the smaller id.
* :func:`degree_add` -- the same endpoint counts accumulated chunk by chunk,
  for inputs too large to hold at once.
* :func:`rfjt_init`, :func:`rfjt_hook`, :func:`rfjt_pointer_jump` --
  Algorithm 3 (Algorithm 1 when ``use_r=False``) run sequentially.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SRC = os.path.join(_HERE, "cc_oracle.c")
_LOCK = threading.Lock()
_lib = None

_u64, _i64, _i32, _ptr = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, single-threaded)."""
    with _LOCK:
        fresh = os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
        if force or not fresh:
            os.makedirs(os.path.dirname(_SO), exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-fvisibility=hidden", "-o", tmp, _SRC])
            os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_uf_new.argtypes = [_u64]
        lib.oracle_uf_new.restype = _ptr
        lib.oracle_uf_free.argtypes = [_ptr]
        lib.oracle_uf_free.restype = None
        lib.oracle_uf_add.argtypes = [_ptr, _ptr, _u64]
        lib.oracle_uf_add.restype = _i32
        lib.oracle_uf_min_labels.argtypes = [_ptr, _ptr]
        lib.oracle_uf_min_labels.restype = None
        lib.oracle_min_labels.argtypes = [_u64, _ptr, _u64, _ptr]
        lib.oracle_min_labels.restype = _i32
        lib.oracle_root_value_labels.argtypes = [_u64, _ptr, _u64, _u64, _ptr]
        lib.oracle_root_value_labels.restype = _i32
        lib.oracle_bfs_labels.argtypes = [_u64, _ptr, _u64, _ptr]
        lib.oracle_bfs_labels.restype = _i32
        lib.oracle_max_degree_vertex.argtypes = [_u64, _ptr, _u64, _ptr]
        lib.oracle_max_degree_vertex.restype = _i64
        lib.oracle_csr_max_row_vertex.argtypes = [_u64, _ptr]
        lib.oracle_csr_max_row_vertex.restype = _i64
        lib.oracle_degree_add.argtypes = [_u64, _ptr, _u64, _ptr]
        lib.oracle_degree_add.restype = _i32
        lib.oracle_num_components.argtypes = [_u64, _ptr]
        lib.oracle_num_components.restype = _u64
        lib.oracle_connected.argtypes = [_u64, _ptr, _ptr, _u64, _ptr]
        lib.oracle_connected.restype = _i32
        lib.oracle_rfjt_init.argtypes = [_u64, _i32, _u64, _ptr]
        lib.oracle_rfjt_init.restype = None
        lib.oracle_rfjt_hook.argtypes = [_u64, _i32, _u64, _ptr, _u64, _ptr]
        lib.oracle_rfjt_hook.restype = _i32
        lib.oracle_rfjt_pointer_jump.argtypes = [_u64, _i32, _u64, _ptr]
        lib.oracle_rfjt_pointer_jump.restype = None
        _lib = lib
    return _lib


def _edges(edges) -> np.ndarray:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
    return e


def _ok(rc: int, what: str) -> None:
    if rc == -1:
        raise ValueError(f"{what}: vertex id out of range")
    if rc < 0:
        raise MemoryError(f"{what}: allocation failed")


def min_labels(n: int, edges) -> np.ndarray:
    """L[v] = min{w : w ~ v} by sequential union-find (smaller root wins)."""
    e = _edges(edges)
    L = np.empty(n, dtype=np.uint32)
    _ok(_L().oracle_min_labels(n, e.ctypes.data, len(e), L.ctypes.data), "min_labels")
    return L


def bfs_labels(n: int, edges) -> np.ndarray:
    """L[v] = min{w : w ~ v} by breadth-first search in increasing start order."""
    e = _edges(edges)
    L = np.empty(n, dtype=np.uint32)
    _ok(_L().oracle_bfs_labels(n, e.ctypes.data, len(e), L.ctypes.data), "bfs_labels")
    return L


def root_value_labels(n: int, edges, m: int) -> np.ndarray:
    """L[v] = min{R(w) : w ~ v} with R(m) = 0, R(x) = x + 1 otherwise (Eq. 1)."""
    e = _edges(edges)
    L = np.empty(n, dtype=np.uint32)
    _ok(_L().oracle_root_value_labels(n, e.ctypes.data, len(e), m, L.ctypes.data),
        "root_value_labels")
    return L


def csr_max_row_vertex(n: int, offsets) -> int:
    """CSR input: the vertex with the longest row, smallest id on ties."""
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    if len(off) != n + 1:
        raise ValueError("offsets must hold n + 1 entries")
    m = _L().oracle_csr_max_row_vertex(n, off.ctypes.data)
    _ok(int(m), "csr_max_row_vertex")
    return int(m)


def csr_edges(offsets, neighbors) -> np.ndarray:
    """The (u, v) pairs a CSR graph stands for, in storage order."""
    off = np.asarray(offsets, dtype=np.int64)
    u = np.repeat(np.arange(len(off) - 1, dtype=np.uint32), np.diff(off))
    return np.stack([u, np.asarray(neighbors, dtype=np.uint32)], axis=1)


def max_degree_vertex(n: int, edges, return_degrees: bool = False):
    """Smallest vertex of maximum endpoint count (a self-loop counts twice)."""
    e = _edges(edges)
    deg = np.empty(n, dtype=np.uint64) if return_degrees else None
    m = _L().oracle_max_degree_vertex(n, e.ctypes.data, len(e),
                                      deg.ctypes.data if deg is not None else None)
    _ok(int(m), "max_degree_vertex")
    return (int(m), deg) if return_degrees else int(m)


def degree_add(n: int, edges, deg: np.ndarray) -> np.ndarray:
    """Adds the endpoint occurrences of one chunk of edges to deg (uint64[n],
    in place, and returned): deg[x] += number of times x occurs as u or v."""
    assert deg.dtype == np.uint64 and deg.flags.c_contiguous and len(deg) == n
    e = _edges(edges)
    _ok(_L().oracle_degree_add(n, e.ctypes.data, len(e), deg.ctypes.data), "degree_add")
    return deg


def num_components(L: np.ndarray) -> int:
    L = np.ascontiguousarray(L, dtype=np.uint32)
    return int(_L().oracle_num_components(len(L), L.ctypes.data))


def connected(L: np.ndarray, pairs) -> np.ndarray:
    """out[i] = (L[u_i] == L[v_i])."""
    L = np.ascontiguousarray(L, dtype=np.uint32)
    p = _edges(pairs)
    out = np.empty(len(p), dtype=np.uint8)
    _ok(_L().oracle_connected(len(L), L.ctypes.data, p.ctypes.data, len(p), out.ctypes.data),
        "connected")
    return out


class StreamingUnionFind:
    """The min-id union-find fed in chunks (inputs too large to hold at once,
    and the union of incremental batches)."""

    def __init__(self, n: int):
        self.n = n
        self._h = _L().oracle_uf_new(n)
        if not self._h:
            raise MemoryError("oracle_uf_new")

    def add(self, edges) -> None:
        e = _edges(edges)
        _ok(_L().oracle_uf_add(self._h, e.ctypes.data, len(e)), "StreamingUnionFind.add")

    def min_labels(self) -> np.ndarray:
        L = np.empty(self.n, dtype=np.uint32)
        _L().oracle_uf_min_labels(self._h, L.ctypes.data)
        return L

    def close(self) -> None:
        if self._h:
            _L().oracle_uf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_min_labels(edges, vtx_off, edge_off) -> np.ndarray:
    """Graph-local min-id labels of each graph of a concatenated batch."""
    e = _edges(edges)
    vtx_off = np.asarray(vtx_off, dtype=np.uint64)
    edge_off = np.asarray(edge_off, dtype=np.uint64)
    out = np.empty(int(vtx_off[-1]), dtype=np.uint32)
    for g in range(len(vtx_off) - 1):
        v0, v1 = int(vtx_off[g]), int(vtx_off[g + 1])
        e0, e1 = int(edge_off[g]), int(edge_off[g + 1])
        out[v0:v1] = min_labels(v1 - v0, e[e0:e1])
    return out


def closure_labels(n: int, edges) -> np.ndarray:
    """The definition on tiny graphs: reach[u][v] from the edge set taken as
    unordered pairs plus reflexivity, closed by Warshall's algorithm; then
    L[v] = min{w : reach[v][w]}."""
    reach = [[u == v for v in range(n)] for u in range(n)]
    for a, b in _edges(edges).tolist():
        if a >= n or b >= n:
            raise ValueError("closure_labels: vertex id out of range")
        reach[a][b] = True
        reach[b][a] = True
    for k in range(n):
        for i in range(n):
            if reach[i][k]:
                row_k = reach[k]
                row_i = reach[i]
                for j in range(n):
                    if row_k[j]:
                        row_i[j] = True
    return np.array([min(w for w in range(n) if reach[v][w]) for v in range(n)], dtype=np.uint32)


def rfjt_init(n: int, use_r: bool = False, m: int = 0) -> np.ndarray:
    """P[v] = f(v) (Algorithm 3, initialisation)."""
    P = np.empty(n, dtype=np.uint32)
    _L().oracle_rfjt_init(n, int(use_r), m, P.ctypes.data)
    return P


def rfjt_hook(P: np.ndarray, edges, use_r: bool = False, m: int = 0) -> np.ndarray:
    """Sequential hooking of Algorithm 3 applied to P in place (and returned)."""
    assert P.dtype == np.uint32 and P.flags.c_contiguous
    e = _edges(edges)
    _ok(_L().oracle_rfjt_hook(len(P), int(use_r), m, e.ctypes.data, len(e), P.ctypes.data),
        "rfjt_hook")
    return P


def rfjt_pointer_jump(P: np.ndarray, use_r: bool = False, m: int = 0) -> np.ndarray:
    """Pointer jumping of Algorithm 3: P[v] <- P[root(v)] (in place)."""
    assert P.dtype == np.uint32 and P.flags.c_contiguous
    _L().oracle_rfjt_pointer_jump(len(P), int(use_r), m, P.ctypes.data)
    return P

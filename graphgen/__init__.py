"""Seeded synthetic graph inputs shared by the tests, the benchmark and the
stored expected values.

This module holds no connected-components arithmetic. Both the CPU oracle's
tests and the CUDA path's tests draw their inputs from here; the generators
themselves live in ``gg_core.h`` (pure integer arithmetic) and are compiled
twice, for the host (``gg_host.c``, C + OpenMP) and for the GPU
(``gg_device.cu``), producing identical bits.

Edges are returned as ``uint32`` arrays of shape ``(E, 2)`` (row ``i`` is the
pair ``(u_i, v_i)``), i.e. the interleaved COO layout ``u0, v0, u1, v1, ...``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_HOST_SO = os.path.join(_BUILD, "libgg_host.so")
_DEV_SO = os.path.join(_BUILD, "libgg_device.so")
_LOCK = threading.Lock()

P90 = 3865470566  # round(0.9 * 2^32): keep threshold of the grid workloads

KIND_ER, KIND_RMAT, KIND_GRID = 0, 1, 2


def _newer(target: str, *sources: str) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(s) <= t for s in sources)


def build_host(force: bool = False) -> str:
    """Compile the host generator library with gcc (OpenMP)."""
    src = os.path.join(_HERE, "gg_host.c")
    hdr = os.path.join(_HERE, "gg_core.h")
    with _LOCK:
        if force or not _newer(_HOST_SO, src, hdr):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _HOST_SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                   "-fvisibility=hidden", "-o", tmp, src])
            os.replace(tmp, _HOST_SO)
    return _HOST_SO


def build_device(force: bool = False, arch: str = "103a") -> str:
    """Compile the device generator library with nvcc for sm_103a."""
    src = os.path.join(_HERE, "gg_device.cu")
    hdr = os.path.join(_HERE, "gg_core.h")
    with _LOCK:
        if force or not _newer(_DEV_SO, src, hdr):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _DEV_SO + f".tmp{os.getpid()}"
            subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                                   "-Xcompiler", "-fvisibility=hidden",
                                   f"-gencode=arch=compute_{arch},code=sm_{arch}", "-o", tmp, src])
            os.replace(tmp, _DEV_SO)
    return _DEV_SO


def build(force: bool = False) -> None:
    build_host(force)
    build_device(force)


_host_lib = None
_dev_lib = None
_u64, _u32, _i32, _ptr = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p


def _host():
    global _host_lib
    if _host_lib is None:
        lib = ctypes.CDLL(build_host())
        lib.gg_rmat.argtypes = [_u64, _i32, _i32, _u64, _u64, _ptr]
        lib.gg_rmat.restype = None
        lib.gg_er.argtypes = [_u64, _u64, _u64, _u64, _ptr]
        lib.gg_er.restype = None
        lib.gg_pairs.argtypes = [_u64, _u64, _u64, _u64, _ptr]
        lib.gg_pairs.restype = None
        lib.gg_grid_count.argtypes = [_u64, _u32, _u32, _u64, _u32]
        lib.gg_grid_count.restype = _u64
        lib.gg_grid.argtypes = [_u64, _u32, _u32, _u64, _u32, _ptr]
        lib.gg_grid.restype = _u64
        lib.gg_batch_plan.argtypes = [_u64, _u32, _ptr, _ptr, _ptr]
        lib.gg_batch_plan.restype = None
        lib.gg_batch_fill.argtypes = [_u64, _u32, _ptr, _ptr]
        lib.gg_batch_fill.restype = None
        _host_lib = lib
    return _host_lib


def _dev():
    global _dev_lib
    if _dev_lib is None:
        if not os.path.exists(_DEV_SO):
            raise RuntimeError(f"{_DEV_SO} is not built; run graphgen.build_device()")
        lib = ctypes.CDLL(_DEV_SO)
        lib.gg_rmat_dev.argtypes = [_u64, _i32, _i32, _u64, _u64, _ptr, _ptr]
        lib.gg_er_dev.argtypes = [_u64, _u64, _u64, _u64, _ptr, _ptr]
        lib.gg_pairs_dev.argtypes = [_u64, _u64, _u64, _u64, _ptr, _ptr]
        lib.gg_grid_dev.argtypes = [_u64, _u32, _u32, _u64, _u32, _ptr, ctypes.POINTER(_u64), _ptr]
        lib.gg_batch_fill_dev.argtypes = [_u64, _u32, _ptr, _u64, _ptr, _ptr]
        for f in (lib.gg_rmat_dev, lib.gg_er_dev, lib.gg_pairs_dev, lib.gg_grid_dev, lib.gg_batch_fill_dev):
            f.restype = ctypes.c_int
        _dev_lib = lib
    return _dev_lib


def _pairs_out(count: int, out=None) -> np.ndarray:
    if out is None:
        out = np.empty((count, 2), dtype=np.uint32)
    assert out.dtype == np.uint32 and out.flags.c_contiguous and out.size >= 2 * count
    return out


# ----------------------------------------------------------------- host side

def rmat(scale: int, n_edges: int, seed: int, scramble: bool = True, e_begin: int = 0,
         e_end: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Edges [e_begin, e_end) of R-MAT(scale, seed) with a=.57, b=.19, c=.19, d=.05."""
    if e_end is None:
        e_end = n_edges
    out = _pairs_out(e_end - e_begin, out)
    if e_end > e_begin:
        _host().gg_rmat(seed, scale, int(bool(scramble)), e_begin, e_end, out.ctypes.data)
    return out


def er(n: int, m: int, seed: int, e_begin: int = 0, e_end: int | None = None) -> np.ndarray:
    """Pairs of G(n, m): independent uniform (u, v), self-loops and duplicates kept."""
    if e_end is None:
        e_end = m
    out = _pairs_out(e_end - e_begin)
    if e_end > e_begin:
        _host().gg_er(seed, n, e_begin, e_end, out.ctypes.data)
    return out


def pairs(n: int, count: int, seed: int, tag: int = 0) -> np.ndarray:
    """count uniform pairs on [0, n) (insert and query batches)."""
    out = _pairs_out(count)
    if count:
        _host().gg_pairs(seed, tag, n, count, out.ctypes.data)
    return out


def grid(W: int, H: int, seed: int, p_thresh: int = P90, n_limit: int | None = None) -> np.ndarray:
    """4-neighbour W x H grid, vertex id r*W + c, each candidate kept with
    probability p_thresh / 2^32, in row-major order (right, then down)."""
    if n_limit is None:
        n_limit = W * H
    lib = _host()
    cnt = lib.gg_grid_count(seed, W, H, n_limit, p_thresh)
    out = _pairs_out(cnt)
    got = lib.gg_grid(seed, W, H, n_limit, p_thresh, out.ctypes.data)
    assert got == cnt
    return out


@dataclass
class Batch:
    edges: np.ndarray      # (E, 2) uint32, graph-local ids, graphs concatenated
    vtx_off: np.ndarray    # (G+1,) uint64
    edge_off: np.ndarray   # (G+1,) uint64
    kinds: np.ndarray      # (G,) uint32: 0 G(n,m), 1 R-MAT, 2 grid

    @property
    def n_graphs(self) -> int:
        return len(self.kinds)


def batch_plan(n_graphs: int, seed: int):
    kinds = np.empty(n_graphs, dtype=np.uint32)
    vtx_off = np.empty(n_graphs + 1, dtype=np.uint64)
    edge_off = np.empty(n_graphs + 1, dtype=np.uint64)
    _host().gg_batch_plan(seed, n_graphs, kinds.ctypes.data, vtx_off.ctypes.data,
                          edge_off.ctypes.data)
    return kinds, vtx_off, edge_off


def batch(n_graphs: int, seed: int) -> Batch:
    """The mixed batch: 40% G(n,m), 40% R-MAT, 20% grid (p = 0.9); |V| piecewise
    log-uniform on [2^8, 2^18); average degree in [2, 32]."""
    kinds, vtx_off, edge_off = batch_plan(n_graphs, seed)
    edges = np.empty((int(edge_off[-1]), 2), dtype=np.uint32)
    _host().gg_batch_fill(seed, n_graphs, edge_off.ctypes.data, edges.ctypes.data)
    return Batch(edges, vtx_off, edge_off, kinds)


# --------------------------------------------------------------- device side

def _stream_ptr(stream) -> int:
    return 0 if stream is None else int(stream.cuda_stream)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what} failed with CUDA error {rc}")


def to_csr(n: int, edges: np.ndarray):
    """CSR layout of a COO edge list for cc_run_csr: offsets (uint64[n + 1])
    and neighbors (uint32), row u holding the v of every pair (u, v) in input
    order (a stable sort by u). No symmetrisation."""
    e = np.ascontiguousarray(edges, dtype=np.uint32).reshape(-1, 2)
    order = np.argsort(e[:, 0], kind="stable")
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(e[:, 0], minlength=n), out=offsets[1:])
    return offsets, np.ascontiguousarray(e[order, 1])


def pack_ids(edges: np.ndarray, id_bytes: int = 3) -> np.ndarray:
    """The compact host layout of cc_run_host_packed: every id in id_bytes
    little-endian bytes, u then v, no padding (uint8[2 * id_bytes * E])."""
    e = np.ascontiguousarray(edges, dtype=np.uint32).reshape(-1)
    if id_bytes == 4:
        return e.view(np.uint8).copy()
    if id_bytes != 3 or (len(e) and int(e.max()) >= 1 << 24):
        raise ValueError("3-byte ids hold values below 2^24")
    return e.view(np.uint8).reshape(-1, 4)[:, :3].reshape(-1).copy()


def rmat_dev(scale: int, n_edges: int, seed: int, scramble: bool = True, out=None,
             e_begin: int = 0, e_end: int | None = None, stream=None):
    """R-MAT edges generated directly in HBM; returns a (E, 2) uint32-valued
    int32 torch tensor on the current device (same bits as :func:`rmat`)."""
    import torch
    if e_end is None:
        e_end = n_edges
    cnt = e_end - e_begin
    if out is None:
        out = torch.empty((cnt, 2), dtype=torch.int32, device="cuda")
    _check(_dev().gg_rmat_dev(seed, scale, int(bool(scramble)), e_begin, e_end, out.data_ptr(),
                              _stream_ptr(stream)), "gg_rmat_dev")
    return out


def er_dev(n: int, m: int, seed: int, stream=None):
    import torch
    out = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    _check(_dev().gg_er_dev(seed, n, 0, m, out.data_ptr(), _stream_ptr(stream)), "gg_er_dev")
    return out


def pairs_dev(n: int, count: int, seed: int, tag: int = 0, stream=None):
    import torch
    out = torch.empty((count, 2), dtype=torch.int32, device="cuda")
    _check(_dev().gg_pairs_dev(seed, tag, n, count, out.data_ptr(), _stream_ptr(stream)),
           "gg_pairs_dev")
    return out


def grid_dev(W: int, H: int, seed: int, p_thresh: int = P90, n_limit: int | None = None,
             stream=None):
    import torch
    if n_limit is None:
        n_limit = W * H
    cap = 2 * W * H
    buf = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    cnt = _u64(0)
    _check(_dev().gg_grid_dev(seed, W, H, n_limit, p_thresh, buf.data_ptr(), ctypes.byref(cnt),
                              _stream_ptr(stream)), "gg_grid_dev")
    return buf[: cnt.value].clone()


@dataclass
class DeviceBatch:
    edges: "object"        # (E, 2) int32 torch tensor on the GPU, graph-local ids
    vtx_off: "object"      # (G+1,) int64 torch tensor on the GPU
    edge_off: "object"     # (G+1,) int64 torch tensor on the GPU
    vtx_off_host: np.ndarray
    edge_off_host: np.ndarray
    kinds: np.ndarray

    @property
    def n_graphs(self) -> int:
        return len(self.kinds)


def batch_dev(n_graphs: int, seed: int, stream=None) -> DeviceBatch:
    """The mixed batch generated in HBM (same bits as :func:`batch`)."""
    import torch
    kinds, vtx_off, edge_off = batch_plan(n_graphs, seed)
    total = int(edge_off[-1])
    eo = torch.from_numpy(edge_off.view(np.int64)).cuda()
    vo = torch.from_numpy(vtx_off.view(np.int64)).cuda()
    edges = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    _check(_dev().gg_batch_fill_dev(seed, n_graphs, eo.data_ptr(), total, edges.data_ptr(), _stream_ptr(stream)),
           "gg_batch_fill_dev")
    return DeviceBatch(edges, vo, eo, vtx_off, edge_off, kinds)


# ---------------------------------------------------------------- workloads

@dataclass(frozen=True)
class Workload:
    """A named single-graph workload: what it is, with its sizes."""
    name: str
    kind: str           # "rmat" | "grid"
    n_vertices: int
    n_edges: int | None  # None: decided by the generator (grid)
    seed: int
    scale: int = 0
    scramble: bool = False
    grid_w: int = 0
    grid_h: int = 0

    def host_edges(self) -> np.ndarray:
        if self.kind == "rmat":
            return rmat(self.scale, self.n_edges, self.seed, self.scramble)
        return grid(self.grid_w, self.grid_h, self.seed)

    def device_edges(self, stream=None):
        if self.kind == "rmat":
            return rmat_dev(self.scale, self.n_edges, self.seed, self.scramble, stream=stream)
        return grid_dev(self.grid_w, self.grid_h, self.seed, stream=stream)


def rmat_workload(name: str, scale: int, edge_factor: int, seed: int, scramble: bool) -> Workload:
    n = 1 << scale
    return Workload(name, "rmat", n, edge_factor * n, seed, scale=scale, scramble=scramble)


def grid_workload(name: str, W: int, H: int, seed: int) -> Workload:
    return Workload(name, "grid", W * H, None, seed, grid_w=W, grid_h=H)


# The five configurations: one small R-MAT; R-MAT scale 24 and the 8192^2 grid;
# R-MAT scale 28; the 4096-graph mixed batch; the resident scale-26 serving graph.
RMAT16 = rmat_workload("rmat16_ef16", 16, 16, 1, scramble=False)
RMAT24 = rmat_workload("rmat24_ef16", 24, 16, 2, scramble=True)
GRID8K = grid_workload("grid8192x8192_p0.9", 8192, 8192, 3)
RMAT28 = rmat_workload("rmat28_ef16", 28, 16, 4, scramble=True)
BATCH_GRAPHS, BATCH_SEED = 4096, 5
RMAT26 = rmat_workload("rmat26_ef16", 26, 16, 6, scramble=True)
# A profiling case for the zero-tree edge pass: the parent array (268 MB) is
# larger than L2 while the edges (2.1 GB) stay a few GB.
RMAT26_EF4 = rmat_workload("rmat26_ef4", 26, 4, 7, scramble=True)
# R-MAT scale 24 as generated, without the id scramble: the hubs keep low ids,
# which changes the parent array's cache locality (a secondary row of C2).
RMAT24_U = rmat_workload("rmat24_ef16_u", 24, 16, 2, scramble=False)

WORKLOADS = {w.name: w for w in (RMAT16, RMAT24, GRID8K, RMAT28, RMAT26, RMAT26_EF4, RMAT24_U)}

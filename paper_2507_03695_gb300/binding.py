"""ctypes binding of libcc.so (include/cc.h): same names as the C ABI,
argument marshalling only. Every step of the computation runs in the CUDA
kernels of the library; there is no Python or CPU fallback. If the library is
not built, the first call raises.

Buffers may be torch tensors (device pointers are taken with ``data_ptr()``;
edge tensors of shape (E, 2) give ``n_edges = E``) or plain integers
(addresses). ``stream=None`` means torch's current stream on the current
device.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_u64, _u32, _i32, _ptr = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p
CC_ROOT_AUTO = 0xFFFFFFFFFFFFFFFF

# cc_status
CC_OK = 0
CC_ERR_INVALID_ARGUMENT = 1
CC_ERR_TOO_LARGE = 2
CC_ERR_OOM = 3
CC_ERR_OUT_OF_RANGE = 4
CC_ERR_TIMEOUT = 5
CC_ERR_CUDA = 6
CC_ERR_INTERNAL = 7
CC_ERR_NOT_READY = 8
# cc_root_mode / cc_root_select / cc_filter / cc_label_space
CC_ROOT_IDENTITY, CC_ROOT_MAXDEG = 0, 1
CC_ROOT_SELECT_EXACT, CC_ROOT_SELECT_SAMPLED = 0, 1
CC_FILTER_AUTO, CC_FILTER_ON, CC_FILTER_OFF, CC_FILTER_BITMAP = 0, 1, 2, 3
CC_PUSH_AUTO, CC_PUSH_ON, CC_PUSH_OFF = 0, 1, 2
CC_LABEL_MIN_ID, CC_LABEL_ROOT_VALUE = 0, 1


class cc_options(ctypes.Structure):
    _fields_ = [
        ("mode", _i32), ("root_select", _i32), ("root_hint", _u64), ("filter", _i32),
        ("label_space", _i32), ("block_size", _i32), ("edges_per_thread", _i32),
        ("sample_stride", _i32), ("timing", _i32), ("hbm_budget_bytes", _u64),
        ("initial_push", _i32), ("reserved32", _i32), ("reserved", _u64 * 3),
    ]


class cc_batch_config(ctypes.Structure):
    _fields_ = [
        ("block_size", _i32), ("edges_per_thread", _i32), ("filter", _i32), ("tile_edges", _u32),
        ("tile_vertices", _u32), ("barrier_wait_us", _u32), ("reserved", _i32 * 2),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class cc_request(ctypes.Structure):
    _fields_ = [
        ("kind", _i32), ("graph", _u32), ("n_vertices", _u64), ("edges_dev", _ptr), ("n_edges", _u64),
        ("pairs_dev", _ptr), ("n_pairs", _u64), ("out_dev", _ptr), ("labels_dev", _ptr),
    ]


class cc_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", _u64), ("max_graphs", _u32), ("executor_blocks_per_sm", _u32),
        ("tile_edges", _u32), ("idle_timeout_us", _u32), ("mode", _i32), ("label_space", _i32),
        ("publish_wait_us", _u32), ("gate_wait_us", _u32), ("fault_hold_publish_us", _u32), ("reserved", _i32 * 1),
    ]


class cc_server_stats(ctypes.Structure):
    _fields_ = [(k, _u64) for k in ("submitted", "completed", "failed", "resident_graphs", "arena_bytes_used",
                                    "arena_bytes", "executor_launches", "tiles_run", "side_drains",
                                    "executor_timeouts", "snapshot_overlaps")]


CC_REQ_NEW_GRAPH, CC_REQ_INSERT, CC_REQ_QUERY, CC_REQ_SNAPSHOT, CC_REQ_DROP_GRAPH = 1, 2, 3, 4, 5


class CCError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {cc_status_string(status)}")


_lib = None


def lib():
    """The loaded libcc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is not built: run paper_2507_03695_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(_build.LIB)
        P = ctypes.POINTER
        sigs = {
            "cc_options_init": (None, [P(cc_options)]),
            "cc_create": (_i32, [_u64, _u64, P(cc_options), P(_ptr)]),
            "cc_run": (_i32, [_ptr, _ptr, _u64, _ptr, _ptr]),
            "cc_run_host": (_i32, [_ptr, _ptr, _u64, _ptr, _ptr]),
            "cc_run_host_packed": (_i32, [_ptr, _ptr, _u64, _i32, _ptr, _ptr]),
            "cc_run_host_async": (_i32, [_ptr, _ptr, _u64, _ptr, _ptr]),
            "cc_run_host_packed_async": (_i32, [_ptr, _ptr, _u64, _i32, _ptr, _ptr]),
            "cc_run_csr": (_i32, [_ptr, _ptr, _ptr, _u64, _ptr, _ptr]),
            "cc_stream_insert": (_i32, [_ptr, _ptr, _u64, _ptr]),
            "cc_labels": (_i32, [_ptr, _ptr, _ptr]),
            "cc_connected": (_i32, [_ptr, _ptr, _u64, _ptr, _ptr]),
            "cc_connected1": (_i32, [_ptr, _u64, _u64, P(ctypes.c_int)]),
            "cc_forest_pairs": (_i32, [_ptr, _ptr, _u64, P(_u64), _ptr]),
            "cc_num_components": (_i32, [_ptr, P(_u64)]),
            "cc_root_vertex": (_i32, [_ptr, P(_u64)]),
            "cc_sync": (_i32, [_ptr]),
            "cc_phase_times": (_i32, [_ptr, P(ctypes.c_float)]),
            "cc_phase_times_total": (_i32, [_ptr, P(ctypes.c_float), P(_u64)]),
            "cc_kernel_launches": (_u64, []),
            "cc_max_degree_vertex_noalloc": (_i32, [_ptr, _u64, _u64, _ptr, _ptr]),
            "cc_measure_random_loads": (_i32, [_u64, P(ctypes.c_double)]),
            "cc_checkpoint_size": (_i32, [_ptr, P(_u64)]),
            "cc_checkpoint": (_i32, [_ptr, _ptr, _u64]),
            "cc_restore": (_i32, [_ptr, _ptr, _u64]),
            "cc_device_bytes": (_i32, [_ptr, P(_u64)]),
            "cc_destroy": (None, [_ptr]),
            "cc_status_string": (ctypes.c_char_p, [_i32]),
            "cc_batch_create": (_i32, [_u32, P(_ptr)]),
            "cc_run_batched": (_i32, [_ptr, _u32, _ptr, _ptr, _ptr, _ptr, _ptr]),
            "cc_batch_tune": (_i32, [_ptr, _u32, _ptr, _ptr, _ptr, _ptr, _ptr, P(cc_batch_config),
                                     P(ctypes.c_float)]),
            "cc_batch_set_config": (_i32, [_ptr, P(cc_batch_config)]),
            "cc_batch_tune_results": (_i32, [_ptr, P(cc_batch_config), P(ctypes.c_float), _u32, P(_u32)]),
            "cc_batch_get_config": (_i32, [_ptr, P(cc_batch_config)]),
            "cc_batch_sync": (_i32, [_ptr]),
            "cc_batch_destroy": (None, [_ptr]),
            "cc_server_config_init": (None, [P(cc_server_config)]),
            "cc_server_create": (_i32, [P(cc_server_config), P(_ptr)]),
            "cc_server_submit": (_i32, [_ptr, P(cc_request), P(_u64)]),
            "cc_server_submit_many": (_i32, [_ptr, P(cc_request), _u32, P(_u64), P(_u32)]),
            "cc_server_poll": (_i32, [_ptr, _u64, P(_i32)]),
            "cc_server_wait": (_i32, [_ptr, _u64, _u64, P(_i32)]),
            "cc_server_result_graph": (_i32, [_ptr, _u64, P(_u32)]),
            "cc_server_latency_ns": (_i32, [_ptr, _u64, P(_u64)]),
            "cc_server_get_stats": (_i32, [_ptr, P(cc_server_stats)]),
            "cc_server_destroy": (None, [_ptr]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str) -> None:
    if st != CC_OK:
        raise CCError(st, what)


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _count_pairs(x, n) -> int:
    if n is not None:
        return int(n)
    if hasattr(x, "numel"):
        return int(x.numel()) // 2
    if hasattr(x, "size"):
        return int(x.size) // 2
    raise TypeError("pass the number of pairs explicitly")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def cc_status_string(status: int) -> str:
    s = lib().cc_status_string(int(status))
    return s.decode() if s else f"status {status}"


def cc_options_init(**overrides) -> cc_options:
    o = cc_options()
    lib().cc_options_init(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"cc_options has no field {k!r}")
        setattr(o, k, v)
    return o


def cc_create(n_vertices: int, n_edges_capacity: int = 0, opt: cc_options | None = None) -> int:
    h = _ptr()
    _check(lib().cc_create(n_vertices, n_edges_capacity, ctypes.byref(opt) if opt is not None else None,
                           ctypes.byref(h)), "cc_create")
    return h.value


def cc_run(g: int, edges, n_edges: int | None = None, L_out=None, stream=None) -> None:
    _check(lib().cc_run(g, _addr(edges), _count_pairs(edges, n_edges), _addr(L_out), _stream(stream)),
           "cc_run")


def cc_run_csr(g: int, offsets, neighbors, n_entries: int | None = None, L_out=None, stream=None) -> None:
    """offsets: uint64[n + 1] on the device (an int64 tensor), neighbors: uint32[n_entries]."""
    if n_entries is None:
        n_entries = int(neighbors.numel()) if hasattr(neighbors, "numel") else int(neighbors.size)
    _check(lib().cc_run_csr(g, _addr(offsets), _addr(neighbors), int(n_entries), _addr(L_out), _stream(stream)),
           "cc_run_csr")


def cc_run_host_packed(g: int, edges_host, n_edges: int, id_bytes: int, L_out_host=None, stream=None) -> None:
    """edges_host: a host buffer of 2 * id_bytes * n_edges bytes (pinned for speed)."""
    _check(lib().cc_run_host_packed(g, _addr(edges_host), int(n_edges), int(id_bytes), _addr(L_out_host),
                                    _stream(stream)), "cc_run_host_packed")


def cc_run_host(g: int, edges_host, n_edges: int | None = None, L_out_host=None, stream=None) -> None:
    _check(lib().cc_run_host(g, _addr(edges_host), _count_pairs(edges_host, n_edges), _addr(L_out_host),
                             _stream(stream)), "cc_run_host")


def cc_run_host_async(g: int, edges_host, n_edges: int | None = None, L_out_host=None, stream=None) -> None:
    """As cc_run_host without the final wait: keep edges_host and L_out_host
    untouched until cc_sync(g) has returned."""
    _check(lib().cc_run_host_async(g, _addr(edges_host), _count_pairs(edges_host, n_edges), _addr(L_out_host),
                                   _stream(stream)), "cc_run_host_async")


def cc_run_host_packed_async(g: int, edges_host, n_edges: int, id_bytes: int, L_out_host=None,
                             stream=None) -> None:
    _check(lib().cc_run_host_packed_async(g, _addr(edges_host), int(n_edges), int(id_bytes), _addr(L_out_host),
                                          _stream(stream)), "cc_run_host_packed_async")


def cc_stream_insert(g: int, edges, n_edges: int | None = None, stream=None) -> None:
    _check(lib().cc_stream_insert(g, _addr(edges), _count_pairs(edges, n_edges), _stream(stream)),
           "cc_stream_insert")


def cc_labels(g: int, L_out, stream=None) -> None:
    _check(lib().cc_labels(g, _addr(L_out), _stream(stream)), "cc_labels")


def cc_connected(g: int, pairs, out, n_pairs: int | None = None, stream=None) -> None:
    _check(lib().cc_connected(g, _addr(pairs), _count_pairs(pairs, n_pairs), _addr(out), _stream(stream)),
           "cc_connected")


def cc_connected1(g: int, u: int, v: int) -> bool:
    r = ctypes.c_int(0)
    _check(lib().cc_connected1(g, u, v, ctypes.byref(r)), "cc_connected1")
    return bool(r.value)


def cc_forest_pairs(g: int, pairs_out, capacity: int | None = None, stream=None) -> int:
    """Writes the forest of P as (v, parent) pairs into pairs_out (an (m, 2)
    int32 device tensor or an address with `capacity` pairs); returns the
    number of non-root vertices. Raises CCError(CC_ERR_TOO_LARGE) when the
    buffer is too small (the exception's `count` holds the number needed)."""
    cap = _count_pairs(pairs_out, capacity) if pairs_out is not None else 0
    cnt = _u64(0)
    st = lib().cc_forest_pairs(g, _addr(pairs_out), cap, ctypes.byref(cnt), _stream(stream))
    if st != CC_OK:
        err = CCError(st, "cc_forest_pairs")
        err.count = int(cnt.value)
        raise err
    return int(cnt.value)


def cc_num_components(g: int) -> int:
    r = _u64(0)
    _check(lib().cc_num_components(g, ctypes.byref(r)), "cc_num_components")
    return int(r.value)


def cc_root_vertex(g: int) -> int:
    r = _u64(0)
    _check(lib().cc_root_vertex(g, ctypes.byref(r)), "cc_root_vertex")
    return int(r.value)


def cc_sync(g: int) -> None:
    _check(lib().cc_sync(g), "cc_sync")


def cc_sync_status(g: int) -> int:
    """cc_sync returning the status instead of raising."""
    return int(lib().cc_sync(g))


def cc_phase_times(g: int) -> list[float]:
    ms = (ctypes.c_float * 5)()
    _check(lib().cc_phase_times(g, ms), "cc_phase_times")
    return list(ms)


def cc_phase_times_total(g: int) -> tuple[list[float], int]:
    """Summed per-phase times since the previous call, and the run count."""
    ms = (ctypes.c_float * 5)()
    runs = _u64(0)
    _check(lib().cc_phase_times_total(g, ms, ctypes.byref(runs)), "cc_phase_times_total")
    return list(ms), int(runs.value)


def cc_kernel_launches() -> int:
    return int(lib().cc_kernel_launches())


def cc_max_degree_vertex_noalloc(edges, n_vertices: int, m_out, n_edges: int | None = None,
                                 stream=None) -> None:
    """Maximum-degree vertex into the device uint32 m_out, allocating nothing."""
    _check(lib().cc_max_degree_vertex_noalloc(_addr(edges), _count_pairs(edges, n_edges), n_vertices,
                                              _addr(m_out), _stream(stream)),
           "cc_max_degree_vertex_noalloc")


def cc_measure_random_loads(array_bytes: int) -> float:
    """Random 4-byte loads per second from an array of array_bytes bytes on
    the current device (a power of two in [2^16, 2^32])."""
    r = ctypes.c_double()
    _check(lib().cc_measure_random_loads(array_bytes, ctypes.byref(r)), "cc_measure_random_loads")
    return r.value


def cc_checkpoint_size(g: int) -> int:
    r = _u64(0)
    _check(lib().cc_checkpoint_size(g, ctypes.byref(r)), "cc_checkpoint_size")
    return int(r.value)


def cc_checkpoint(g: int) -> bytearray:
    buf = bytearray(cc_checkpoint_size(g))
    c = (ctypes.c_char * len(buf)).from_buffer(buf)
    _check(lib().cc_checkpoint(g, ctypes.addressof(c), len(buf)), "cc_checkpoint")
    return buf


def cc_restore(g: int, buf) -> None:
    b = bytes(buf)
    _check(lib().cc_restore(g, b, len(b)), "cc_restore")


def cc_device_bytes(g: int) -> int:
    r = _u64(0)
    _check(lib().cc_device_bytes(g, ctypes.byref(r)), "cc_device_bytes")
    return int(r.value)


def cc_destroy(g: int) -> None:
    if g:
        lib().cc_destroy(g)


class Graph:
    """Owning wrapper of a cc_graph handle (context manager)."""

    def __init__(self, n_vertices: int, n_edges_capacity: int = 0, **options):
        self.n = n_vertices
        self.opt = cc_options_init(**options)
        self.h = cc_create(n_vertices, n_edges_capacity, self.opt)

    def run(self, edges, L_out=None, stream=None):
        cc_run(self.h, edges, None, L_out, stream)
        return L_out

    def labels(self, L_out, stream=None):
        cc_labels(self.h, L_out, stream)
        return L_out

    def insert(self, edges, stream=None):
        cc_stream_insert(self.h, edges, None, stream)

    def connected(self, pairs, out, stream=None):
        cc_connected(self.h, pairs, out, None, stream)
        return out

    def forest_pairs(self, stream=None):
        """The forest of P as an (count, 2) int32 device tensor of (v, parent)
        pairs: a view of one device buffer of n pairs kept with the handle and
        rewritten by the next call (see cc_forest_pairs)."""
        import torch
        buf = getattr(self, "_pairs_buf", None)
        if buf is None:
            buf = self._pairs_buf = torch.empty((max(self.n, 1), 2), dtype=torch.int32, device="cuda")
        count = cc_forest_pairs(self.h, buf, self.n, stream)
        return buf[:count]

    def num_components(self) -> int:
        return cc_num_components(self.h)

    def root_vertex(self) -> int:
        return cc_root_vertex(self.h)

    def sync(self):
        cc_sync(self.h)

    def close(self):
        if self.h:
            cc_destroy(self.h)
            self.h = 0
        self._pairs_buf = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched

def cc_batch_create(max_graphs: int) -> int:
    h = _ptr()
    _check(lib().cc_batch_create(max_graphs, ctypes.byref(h)), "cc_batch_create")
    return h.value


def cc_run_batched(b: int, n_graphs: int, vtx_off, edge_off, edges, L_out, stream=None) -> None:
    _check(lib().cc_run_batched(b, n_graphs, _addr(vtx_off), _addr(edge_off), _addr(edges), _addr(L_out),
                                _stream(stream)), "cc_run_batched")


def cc_batch_tune(b: int, n_graphs: int, vtx_off, edge_off, edges, L_out, stream=None):
    """Autotune; returns (best config as a dict, its time in ms)."""
    cfg = cc_batch_config()
    ms = ctypes.c_float(0)
    _check(lib().cc_batch_tune(b, n_graphs, _addr(vtx_off), _addr(edge_off), _addr(edges), _addr(L_out),
                               _stream(stream), ctypes.byref(cfg), ctypes.byref(ms)), "cc_batch_tune")
    return cfg.as_dict(), float(ms.value)


def cc_batch_tune_results(b: int) -> list:
    """[(config dict, best ms)] of every candidate of the last cc_batch_tune."""
    cfgs = (cc_batch_config * 64)()
    ms = (ctypes.c_float * 64)()
    count = _u32(0)
    _check(lib().cc_batch_tune_results(b, cfgs, ms, 64, ctypes.byref(count)), "cc_batch_tune_results")
    return [(cfgs[i].as_dict(), float(ms[i])) for i in range(min(count.value, 64))]


def cc_batch_set_config(b: int, **cfg) -> None:
    c = cc_batch_config()
    _check(lib().cc_batch_get_config(b, ctypes.byref(c)), "cc_batch_get_config")
    for k, v in cfg.items():
        setattr(c, k, v)
    _check(lib().cc_batch_set_config(b, ctypes.byref(c)), "cc_batch_set_config")


def cc_batch_get_config(b: int) -> dict:
    c = cc_batch_config()
    _check(lib().cc_batch_get_config(b, ctypes.byref(c)), "cc_batch_get_config")
    return c.as_dict()


def cc_batch_sync(b: int) -> None:
    _check(lib().cc_batch_sync(b), "cc_batch_sync")


def cc_batch_sync_status(b: int) -> int:
    return int(lib().cc_batch_sync(b))


def cc_batch_destroy(b: int) -> None:
    if b:
        lib().cc_batch_destroy(b)


class Batch:
    """Owning wrapper of a cc_batch context."""

    def __init__(self, max_graphs: int):
        self.h = cc_batch_create(max_graphs)

    def run(self, n_graphs, vtx_off, edge_off, edges, L_out, stream=None):
        cc_run_batched(self.h, n_graphs, vtx_off, edge_off, edges, L_out, stream)
        return L_out

    def tune(self, n_graphs, vtx_off, edge_off, edges, L_out, stream=None):
        return cc_batch_tune(self.h, n_graphs, vtx_off, edge_off, edges, L_out, stream)

    def sync(self):
        cc_batch_sync(self.h)

    def close(self):
        if self.h:
            cc_batch_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def cc_server_config_init(**overrides) -> cc_server_config:
    c = cc_server_config()
    lib().cc_server_config_init(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def cc_server_create(cfg: cc_server_config) -> int:
    h = _ptr()
    _check(lib().cc_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cc_server_create")
    return h.value


def cc_server_submit(srv: int, req: cc_request) -> int:
    t = _u64(0)
    _check(lib().cc_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), "cc_server_submit")
    return int(t.value)


def _request_dtype():
    """numpy view of cc_request: the same field offsets, pointers as uint64."""
    import numpy as np
    kinds = {_i32: np.int32, _u32: np.uint32, _u64: np.uint64, _ptr: np.uint64}
    names = [f[0] for f in cc_request._fields_]
    return np.dtype({"names": names, "formats": [kinds[f[1]] for f in cc_request._fields_],
                     "offsets": [getattr(cc_request, nm).offset for nm in names],
                     "itemsize": ctypes.sizeof(cc_request)})


def cc_server_submit_many(srv: int, reqs) -> tuple[list, int]:
    """Queues a ctypes array of cc_request in order; returns (tickets of the
    queued requests, status of the first refused one or CC_OK)."""
    count = len(reqs)
    tickets = (_u64 * max(count, 1))()
    queued = _u32(0)
    st = lib().cc_server_submit_many(srv, reqs, count, tickets, ctypes.byref(queued))
    return list(tickets[:queued.value]), int(st)


def cc_server_poll(srv: int, ticket: int):
    """None while running, else the request's status."""
    r = _i32(0)
    st = lib().cc_server_poll(srv, ticket, ctypes.byref(r))
    if st == CC_ERR_NOT_READY:
        return None
    _check(st, "cc_server_poll")
    return int(r.value)


def cc_server_wait(srv: int, ticket: int, timeout_s: float = 60.0) -> int:
    r = _i32(0)
    _check(lib().cc_server_wait(srv, ticket, int(timeout_s * 1e9), ctypes.byref(r)), "cc_server_wait")
    return int(r.value)


def cc_server_result_graph(srv: int, ticket: int) -> int:
    g = _u32(0)
    _check(lib().cc_server_result_graph(srv, ticket, ctypes.byref(g)), "cc_server_result_graph")
    return int(g.value)


def cc_server_latency_ns(srv: int, ticket: int) -> int:
    v = _u64(0)
    _check(lib().cc_server_latency_ns(srv, ticket, ctypes.byref(v)), "cc_server_latency_ns")
    return int(v.value)


def cc_server_get_stats(srv: int) -> dict:
    st = cc_server_stats()
    _check(lib().cc_server_get_stats(srv, ctypes.byref(st)), "cc_server_get_stats")
    return {k: int(getattr(st, k)) for k, _ in st._fields_}


def cc_server_destroy(srv: int) -> None:
    if srv:
        lib().cc_server_destroy(srv)


class Server:
    """Owning wrapper of a cc_server. Request buffers (torch tensors) are kept
    referenced until the request is waited for."""

    def __init__(self, hbm_budget_bytes: int, **cfg):
        self.h = cc_server_create(cc_server_config_init(hbm_budget_bytes=hbm_budget_bytes, **cfg))
        self._keep = {}

    def _submit(self, keep, **fields) -> int:
        req = cc_request()
        for k, v in fields.items():
            setattr(req, k, v)
        t = cc_server_submit(self.h, req)
        self._keep[t] = keep
        return t

    def new_graph(self, n_vertices: int, edges, labels=None) -> tuple[int, int]:
        t = self._submit((edges, labels), kind=CC_REQ_NEW_GRAPH, n_vertices=n_vertices,
                         edges_dev=_addr(edges), n_edges=_count_pairs(edges, None), labels_dev=_addr(labels))
        return t, cc_server_result_graph(self.h, t)

    def insert(self, graph: int, edges) -> int:
        return self._submit((edges,), kind=CC_REQ_INSERT, graph=graph, edges_dev=_addr(edges),
                            n_edges=_count_pairs(edges, None))

    def _submit_many(self, kind: int, graph: int, bufs, counts, keeps, **ptr_fields) -> list:
        """One cc_server_submit_many call for requests that differ only in
        their buffers (ptr_fields: field name -> list of addresses)."""
        import numpy as np
        n = len(counts)
        arr = (cc_request * n)()
        view = np.frombuffer(arr, dtype=_request_dtype(), count=n)  # fields filled column-wise
        view["kind"] = kind
        view["graph"] = graph
        view["n_edges" if kind == CC_REQ_INSERT else "n_pairs"] = np.asarray(counts, dtype=np.uint64)
        for name, addrs in ptr_fields.items():
            view[name] = np.asarray(addrs, dtype=np.uint64)
        tickets, st = cc_server_submit_many(self.h, arr)
        for t, keep in zip(tickets, keeps):
            self._keep[t] = keep
        if st != CC_OK:
            err = CCError(st, f"cc_server_submit_many (request {len(tickets)} of {n})")
            err.tickets = tickets  # the requests before the refused one are queued
            raise err
        return tickets

    def insert_many(self, graph: int, edge_batches) -> list:
        """Insert batches (each a (k, 2) int32 device tensor) queued in one call."""
        return self._submit_many(CC_REQ_INSERT, graph, edge_batches,
                                 [_count_pairs(e, None) for e in edge_batches], [(e,) for e in edge_batches],
                                 edges_dev=[_addr(e) for e in edge_batches])

    def query_many(self, graph: int, pair_batches, outs) -> list:
        """Query batches with their uint8 output tensors, queued in one call."""
        return self._submit_many(CC_REQ_QUERY, graph, pair_batches,
                                 [_count_pairs(p, None) for p in pair_batches],
                                 [(p, o) for p, o in zip(pair_batches, outs)],
                                 pairs_dev=[_addr(p) for p in pair_batches], out_dev=[_addr(o) for o in outs])

    def query(self, graph: int, pairs, out) -> int:
        return self._submit((pairs, out), kind=CC_REQ_QUERY, graph=graph, pairs_dev=_addr(pairs),
                            n_pairs=_count_pairs(pairs, None), out_dev=_addr(out))

    def snapshot(self, graph: int, labels) -> int:
        return self._submit((labels,), kind=CC_REQ_SNAPSHOT, graph=graph, labels_dev=_addr(labels))

    def drop(self, graph: int) -> int:
        return self._submit((), kind=CC_REQ_DROP_GRAPH, graph=graph)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        st = cc_server_wait(self.h, ticket, timeout_s)
        self._keep.pop(ticket, None)
        return st

    def poll(self, ticket: int):
        return cc_server_poll(self.h, ticket)

    def latency_ns(self, ticket: int) -> int:
        return cc_server_latency_ns(self.h, ticket)

    def stats(self) -> dict:
        return cc_server_get_stats(self.h)

    def close(self):
        if self.h:
            cc_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


"""bench.py's host-side helpers, without a GPU: the request roofline's
arithmetic and which graphs it covers, the lookup-array rule, the lookup of
profiled DRAM traffic by kernel-source hash, and the host-memory probe."""
import os

import pytest

import bench
import graphgen


class FakeCC:
    """Stands in for the library's random-load measurement."""
    calls = []

    @classmethod
    def cc_measure_random_loads(cls, size):
        cls.calls.append(size)
        return 3.0e11


def test_lookup_array_rule():
    # R-MAT graphs from a 128 MiB parent array up read the zero-tree bitmap
    assert bench.lookup_array_bytes("rmat28_ef16", 1 << 28) == (1 << 25, "zero-tree bitmap")
    assert bench.lookup_array_bytes("rmat24_ef16", 1 << 24) == (1 << 26, "parent array P")
    assert bench.lookup_array_bytes("grid8192x8192_p0.9", 1 << 26)[1] == "parent array P"


def test_request_roofline_covers_rmat_graphs_only():
    FakeCC.calls = []
    r24, grid = graphgen.WORKLOADS["rmat24_ef16"], graphgen.WORKLOADS["grid8192x8192_p0.9"]
    graphs = [(r24, None, 1 << 28), (grid, None, 120776866)]
    phases = [[0, 0, 2.0, 0, 0], [0, 0, 1.0, 0, 0]]
    out = bench.request_roofline(FakeCC, graphs, phases, {})
    # 2 lookups per edge over the R-MAT graph's edge-pass time only
    assert out["achieved"] == pytest.approx(2 * (1 << 28) / 2.0e-3 / 1e9)
    assert out["peak"] == pytest.approx(300.0)
    assert out["frac"] == pytest.approx(out["achieved"] / 300.0)
    assert "excluded" in out["by_graph"][grid.name]
    assert FakeCC.calls == [1 << 26]  # P of R-MAT 24, a power of two already
    only_grid = bench.request_roofline(FakeCC, graphs[1:], phases[1:], {})
    assert only_grid["frac"] is None


def test_request_roofline_measures_each_size_once():
    FakeCC.calls = []
    r24 = graphgen.WORKLOADS["rmat24_ef16"]
    cache = {}
    bench.request_roofline(FakeCC, [(r24, None, 100)], [[0, 0, 1.0, 0, 0]], cache)
    bench.request_roofline(FakeCC, [(r24, None, 100)], [[0, 0, 1.0, 0, 0]], cache)
    assert FakeCC.calls == [1 << 26]


def test_profiled_traffic_follows_the_kernel_source():
    # the committed summaries carry the current source hash (else the bench
    # reports traffic as null, which this test would flag)
    t = bench.profiled_traffic("rmat28", ["rmat28_ef16"])
    assert t is not None and t["rmat28_ef16"] > 34e9
    t2 = bench.profiled_traffic("rmat24+grid8192", ["rmat24_ef16", "grid8192x8192_p0.9"])
    assert t2 is not None and set(t2) == {"rmat24_ef16", "grid8192x8192_p0.9"}
    assert bench.profiled_traffic("rmat28", ["not_a_graph"]) is None
    ex = bench.profiled_executor_traffic()
    assert ex is not None and ex["insert"] > 8 and ex["query"] > 9


def test_host_memory_available():
    m = bench.host_memory_available()
    assert m is None or m > 0


def test_guarded_reports_a_failing_leg():
    assert bench.guarded(lambda: {"ok": 1}) == {"ok": 1}

    def bad():
        raise ValueError("leg failed")
    out = bench.guarded(bad)
    assert out == {"error": "ValueError: leg failed"}

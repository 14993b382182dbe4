"""The C ABI without a GPU: the library loads, exports every function that
include/*.h declares, agrees with the header on struct layout, and its
host-side argument checks return the documented status codes."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_2507_03695_gb300 import build as ccbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ccbuild.build()
    import paper_2507_03695_gb300 as cc
    return cc


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"CC_API\s+[\w\s\*]+?\b(cc_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    so = ctypes.CDLL(ccbuild.LIB)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, f"declared but not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", ccbuild.LIB], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported


def test_options_layout_matches_header(tmp_path, lib):
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cc.h"\nint main(void){'
                 'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(cc_options), offsetof(cc_options, root_hint),'
                 'offsetof(cc_options, filter), offsetof(cc_options, timing),'
                 'offsetof(cc_options, hbm_budget_bytes), offsetof(cc_options, reserved));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    o = lib.cc_options
    assert got == [ctypes.sizeof(o), o.root_hint.offset, o.filter.offset, o.timing.offset,
                   o.hbm_budget_bytes.offset, o.reserved.offset]


def test_batch_and_server_layouts_match_headers(tmp_path, lib):
    c = tmp_path / "layout2.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cc_batch.h"\n#include "cc_server.h"\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cc_batch_config),'
                 'offsetof(cc_batch_config, tile_vertices), sizeof(cc_request), offsetof(cc_request, labels_dev),'
                 'sizeof(cc_server_config), offsetof(cc_server_config, label_space), sizeof(cc_server_stats),'
                 'offsetof(cc_batch_config, barrier_wait_us), offsetof(cc_server_config, publish_wait_us),'
                 'offsetof(cc_server_config, fault_hold_publish_us), offsetof(cc_server_stats, snapshot_overlaps));'
                 'return 0;}\n')
    exe = tmp_path / "layout2"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(lib.cc_batch_config), lib.cc_batch_config.tile_vertices.offset,
                   ctypes.sizeof(lib.cc_request), lib.cc_request.labels_dev.offset,
                   ctypes.sizeof(lib.cc_server_config), lib.cc_server_config.label_space.offset,
                   ctypes.sizeof(lib.cc_server_stats), lib.cc_batch_config.barrier_wait_us.offset,
                   lib.cc_server_config.publish_wait_us.offset, lib.cc_server_config.fault_hold_publish_us.offset,
                   lib.cc_server_stats.snapshot_overlaps.offset]


def test_defaults_and_status_strings(lib):
    o = lib.cc_options_init()
    assert o.mode == lib.CC_ROOT_MAXDEG and o.root_select == lib.CC_ROOT_SELECT_EXACT
    assert o.root_hint == lib.CC_ROOT_AUTO and o.label_space == lib.CC_LABEL_MIN_ID
    for s in range(0, 9):
        assert lib.cc_status_string(s).startswith("CC_")
    assert "unknown" in lib.cc_status_string(99)


def test_host_side_errors(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    # too many vertices for int32 root values (Eq. 1 needs v + 1)
    assert L.cc_create(1 << 31, 0, None, ctypes.byref(h)) == lib.CC_ERR_TOO_LARGE
    # invalid options
    bad = lib.cc_options_init(mode=7)
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    bad = lib.cc_options_init(edges_per_thread=3)
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    bad = lib.cc_options_init(root_hint=10)
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    bad = lib.cc_options_init()
    bad.reserved[2] = 1
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    bad = lib.cc_options_init(initial_push=3)
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    bad = lib.cc_options_init()
    bad.reserved32 = 1
    assert L.cc_create(10, 0, ctypes.byref(bad), ctypes.byref(h)) == lib.CC_ERR_INVALID_ARGUMENT
    # the HBM budget refuses before any allocation
    small = lib.cc_options_init(hbm_budget_bytes=1 << 20)
    assert L.cc_create(1 << 20, 0, ctypes.byref(small), ctypes.byref(h)) == lib.CC_ERR_OOM
    assert h.value is None
    assert L.cc_create(10, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    # the random-load measurement checks its arguments before touching a GPU
    r = ctypes.c_double()
    for bad_bytes in (0, 1 << 15, (1 << 20) + 4, 3 << 20, 1 << 33):
        assert L.cc_measure_random_loads(bad_bytes, ctypes.byref(r)) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_measure_random_loads(1 << 20, None) == lib.CC_ERR_INVALID_ARGUMENT
    nq = ctypes.c_uint32(7)
    assert L.cc_server_submit_many(None, None, 0, None, ctypes.byref(nq)) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_server_submit_many(None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    # NULL handles
    assert L.cc_run(None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_stream_insert(None, None, 0, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_labels(None, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_connected(None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_sync(None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_run_host(None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_run_host_async(None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_run_host_packed(None, None, 0, 3, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_run_host_packed_async(None, None, 0, 3, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    assert L.cc_run_csr(None, None, None, 0, None, None) == lib.CC_ERR_INVALID_ARGUMENT
    out = ctypes.c_uint64()
    assert L.cc_num_components(None, ctypes.byref(out)) == lib.CC_ERR_INVALID_ARGUMENT
    L.cc_destroy(None)


def test_build_entry_point_builds_everything():
    __graft_entry__.build()
    for so in (ccbuild.LIB,
               os.path.join(ROOT, "graphgen", "_build", "libgg_host.so"),
               os.path.join(ROOT, "graphgen", "_build", "libgg_device.so"),
               os.path.join(ROOT, "oracle", "_build", "liboracle.so")):
        assert os.path.exists(so), so


def test_product_path_does_not_import_the_oracle():
    """The library and its binding never load the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2507_03695_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "liboracle" not in src and "cc_oracle" not in src, f

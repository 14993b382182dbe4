"""Every global name that a function of the committed Python files reads is
defined at module level or is a builtin (a static check: a misspelled or
out-of-scope name would otherwise surface only when that branch runs, e.g. a
benchmark section on the GPU)."""
import builtins
import glob
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(
    [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    + glob.glob(os.path.join(ROOT, "paper_2507_03695_gb300", "*.py"))
    + glob.glob(os.path.join(ROOT, "graphgen", "*.py"))
    + glob.glob(os.path.join(ROOT, "oracle", "*.py"))
    + glob.glob(os.path.join(ROOT, "tests", "golden", "*.py")))


def undefined_globals(path):
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    if "*" in src and "import *" in src:
        return []  # star imports define names the table cannot see
    known = module_names | set(dir(builtins)) | {"__file__", "__name__", "__doc__", "__spec__"}
    bad = []

    def walk(t):
        for c in t.get_children():
            if c.get_type() in ("function", "class"):
                for s in c.get_symbols():
                    if s.is_referenced() and s.is_global() and s.get_name() not in known:
                        bad.append(f"{c.get_name()}: {s.get_name()}")
            walk(c)

    walk(top)
    return bad


@pytest.mark.parametrize("path", FILES, ids=[os.path.relpath(f, ROOT) for f in FILES])
def test_no_undefined_globals(path):
    assert undefined_globals(path) == []

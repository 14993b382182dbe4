"""Builds libcc.so (the CUDA kernels + C ABI) in-tree for sm_103a with nvcc.

Each translation unit is compiled to an object in parallel, then linked into
``_build/libcc.so``; rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcc.so")
ARCH = "103a"
_LOCK = threading.Lock()

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
    "-I", os.path.join(ROOT, "include"),
]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          defines: tuple[str, ...] = (), out_dir: str | None = None) -> str:
    """Compile and link libcc.so. `defines` adds -D build options and
    `out_dir` builds into another folder (the default is the in-tree _build)."""
    bdir = out_dir or BUILD
    lib = os.path.join(bdir, "libcc.so")
    with _LOCK:
        if not force and not defines and not _stale(lib):
            return lib
        os.makedirs(bdir, exist_ok=True)
        extra = ["-Xptxas", "-v"] if ptxas_info else []
        extra += [f"-D{d}" for d in defines]

        def compile_one(src: str) -> str:
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            cmd = ["nvcc", *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            if ptxas_info or verbose:
                sys.stderr.write(r.stderr)
            return obj

        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            objs = list(ex.map(compile_one, sources()))
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["nvcc", "-shared", f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)

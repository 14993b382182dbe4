"""GB300 (sm_103a) connected components: Root-Function Jayanti-Tarjan
union-find with one edge pass and a flatten pass, behind the C ABI of
include/cc.h. This package holds the CUDA sources (csrc/), the in-tree build
(build.py) and the ctypes binding (binding.py)."""
from .binding import *  # noqa: F401,F403
from .binding import Batch, CCError, Graph, Server, lib  # noqa: F401

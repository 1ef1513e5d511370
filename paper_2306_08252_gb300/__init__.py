"""GraphVine on GB300: a device-resident dynamic graph behind a C ABI.

The CUDA library (libgraphvine.so, built from csrc/ by build.py) holds the
data structure and every kernel; `graphvine` is its ctypes binding.
"""
from .graphvine import *  # noqa: F401,F403
from .graphvine import Graph, GraphVineError, load, LIB_PATH  # noqa: F401

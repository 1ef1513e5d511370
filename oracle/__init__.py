"""ctypes wrapper of the CPU oracle (gv_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The GPU library never loads it.  The same
library carries the parallel CPU baseline (gv_cpu_parallel.c: the oracle's
algorithm over all host cores with OpenMP), used only to time a multi-core
CPU beside the GPU path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gv_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "gv_cpu_parallel.c")]
_DEPS = _SRCS + [os.path.join(_HERE, "gv_oracle_internal.h")]
_LIB = os.path.join(_HERE, "libgv_oracle.so")
_lock = threading.Lock()
_lib = None

DEDUP = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _DEPS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
            sig = {
                "orc_create": ([u32, u32], p),
                "orc_destroy": ([p], None),
                "orc_insert_edges": ([p, p, p, u64, p, p], None),
                "orc_delete_edges": ([p, p, p, u64, p, p], None),
                "orc_query_edges": ([p, p, p, u64, p], None),
                "orc_insert_vertices": ([p, u32, p], u32),
                "orc_delete_vertices": ([p, p, u32], u32),
                "orc_num_vertices": ([p], u32),
                "orc_num_edges": ([p], u64),
                "orc_degrees": ([p, p], None),
                "orc_alive": ([p, p], None),
                "orc_neighbors": ([p, p, u32, p, p, u64], u64),
                "orc_export_csr": ([p, p, p], None),
                "orc_dictionary_capacity": ([u64], u64),
                "orc_blocks_for_degree": ([u64, u32], u64),
                "orc_block_capacity_rule": ([p, u32], u32),
                "orc_min_footprint_capacity": ([p, u32, ctypes.c_int], u32),
                "orc_cbt_path": ([u64, ctypes.c_char_p], u32),
                "orc_pop_ranges": ([p, u32, p, p], None),
                "orc_insert_block_demand": ([u64, u64, u32], u64),
                "orc_bfs": ([p, u32, p], u32),
                "orc_insert_edges_weighted": ([p, p, p, p, u64, p, p], None),
                "orc_neighbors_weighted": ([p, p, u32, p, p, p, u64], u64),
                "orc_pagerank": ([p, u32, ctypes.c_double, p], None),
                "orc_sssp": ([p, u32, ctypes.c_int, p], u32),
                "orc_par_insert_edges": ([p, p, p, u64, ctypes.c_int, p, p], None),
                "orc_par_delete_edges": ([p, p, p, u64, ctypes.c_int, p, p], None),
                "orc_par_query_edges": ([p, p, p, u64, ctypes.c_int, p], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


class OracleGraph:
    """The plain CPU model of the dynamic graph (one operation at a time)."""

    def __init__(self, nv: int, flags: int = 0):
        self._lib = _get()
        self._g = self._lib.orc_create(nv, flags)
        self.flags = flags

    def close(self):
        if self._g:
            self._lib.orc_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_vertices(self) -> int:
        return int(self._lib.orc_num_vertices(self._g))

    @property
    def num_edges(self) -> int:
        return int(self._lib.orc_num_edges(self._g))

    def insert_edges(self, src, dst):
        s, d = _u32(src), _u32(dst)
        a = np.zeros(2, dtype=np.uint64)
        self._lib.orc_insert_edges(self._g, s.ctypes.data, d.ctypes.data, s.size,
                                   a[0:].ctypes.data, a[1:].ctypes.data)
        return int(a[0]), int(a[1])

    def insert_edges_weighted(self, src, dst, w):
        s, d, ww = _u32(src), _u32(dst), _u32(w)
        a = np.zeros(2, dtype=np.uint64)
        self._lib.orc_insert_edges_weighted(self._g, s.ctypes.data, d.ctypes.data, ww.ctypes.data, s.size,
                                            a[0:].ctypes.data, a[1:].ctypes.data)
        return int(a[0]), int(a[1])

    def neighbors_weighted(self, vids):
        """(offsets, nbrs, weights) in canonical (v, w) order per vertex."""
        v = _u32(vids)
        off = np.zeros(v.size + 1, dtype=np.uint64)
        tot = int(self._lib.orc_neighbors_weighted(self._g, v.ctypes.data, v.size, off.ctypes.data, None, None, 0))
        nb = np.zeros(max(tot, 1), dtype=np.uint32)
        wt = np.zeros(max(tot, 1), dtype=np.uint32)
        self._lib.orc_neighbors_weighted(self._g, v.ctypes.data, v.size, off.ctypes.data, nb.ctypes.data,
                                         wt.ctypes.data, tot)
        return off, nb[:tot], wt[:tot]

    def bulk_build(self, src, dst):
        return self.insert_edges(src, dst)

    def delete_edges(self, src, dst):
        s, d = _u32(src), _u32(dst)
        a = np.zeros(2, dtype=np.uint64)
        self._lib.orc_delete_edges(self._g, s.ctypes.data, d.ctypes.data, s.size,
                                   a[0:].ctypes.data, a[1:].ctypes.data)
        return int(a[0]), int(a[1])

    def query_edges(self, src, dst) -> np.ndarray:
        s, d = _u32(src), _u32(dst)
        out = np.zeros(s.size, dtype=np.uint8)
        self._lib.orc_query_edges(self._g, s.ctypes.data, d.ctypes.data, s.size, out.ctypes.data)
        return out

    # parallel CPU baseline: the same results over `threads` host cores
    def par_insert_edges(self, src, dst, threads: int):
        s, d = _u32(src), _u32(dst)
        a = np.zeros(2, dtype=np.uint64)
        self._lib.orc_par_insert_edges(self._g, s.ctypes.data, d.ctypes.data, s.size, threads,
                                       a[0:].ctypes.data, a[1:].ctypes.data)
        return int(a[0]), int(a[1])

    def par_delete_edges(self, src, dst, threads: int):
        s, d = _u32(src), _u32(dst)
        a = np.zeros(2, dtype=np.uint64)
        self._lib.orc_par_delete_edges(self._g, s.ctypes.data, d.ctypes.data, s.size, threads,
                                       a[0:].ctypes.data, a[1:].ctypes.data)
        return int(a[0]), int(a[1])

    def par_query_edges(self, src, dst, threads: int) -> np.ndarray:
        s, d = _u32(src), _u32(dst)
        out = np.zeros(s.size, dtype=np.uint8)
        self._lib.orc_par_query_edges(self._g, s.ctypes.data, d.ctypes.data, s.size, threads, out.ctypes.data)
        return out

    def insert_vertices(self, k: int) -> np.ndarray:
        ids = np.zeros(max(k, 1), dtype=np.uint32)
        self._lib.orc_insert_vertices(self._g, k, ids.ctypes.data)
        return ids[:k]

    def delete_vertices(self, ids) -> int:
        a = _u32(ids)
        return int(self._lib.orc_delete_vertices(self._g, a.ctypes.data, a.size))

    def degrees(self) -> np.ndarray:
        out = np.zeros(max(self.num_vertices, 1), dtype=np.uint32)
        self._lib.orc_degrees(self._g, out.ctypes.data)
        return out[:self.num_vertices]

    def alive(self) -> np.ndarray:
        out = np.zeros(max(self.num_vertices, 1), dtype=np.uint8)
        self._lib.orc_alive(self._g, out.ctypes.data)
        return out[:self.num_vertices]

    def neighbors(self, vids):
        v = _u32(vids)
        off = np.zeros(v.size + 1, dtype=np.uint64)
        tot = int(self._lib.orc_neighbors(self._g, v.ctypes.data, v.size, off.ctypes.data, None, 0))
        nb = np.zeros(max(tot, 1), dtype=np.uint32)
        self._lib.orc_neighbors(self._g, v.ctypes.data, v.size, off.ctypes.data, nb.ctypes.data, tot)
        return off, nb[:tot]

    def bfs(self, source: int):
        """(dist[nv] uint32, levels); unreached = 0xFFFFFFFF."""
        dist = np.zeros(max(self.num_vertices, 1), dtype=np.uint32)
        lv = int(self._lib.orc_bfs(self._g, source, dist.ctypes.data))
        return dist[:self.num_vertices], lv

    def pagerank(self, iterations: int, damping: float = 0.85) -> np.ndarray:
        r = np.zeros(max(self.num_vertices, 1), dtype=np.float64)
        self._lib.orc_pagerank(self._g, iterations, damping, r.ctypes.data)
        return r[:self.num_vertices]

    def sssp(self, source: int, weighted: bool = False):
        """(dist[nv] uint64, reached); entry length = payload if weighted
        else 1; unreached = 2^64 - 1."""
        dist = np.zeros(max(self.num_vertices, 1), dtype=np.uint64)
        r = int(self._lib.orc_sssp(self._g, source, 1 if weighted else 0, dist.ctypes.data))
        return dist[:self.num_vertices], r

    def export_csr(self):
        nv = self.num_vertices
        off = np.zeros(nv + 1, dtype=np.uint64)
        nb = np.zeros(max(self.num_edges, 1), dtype=np.uint32)
        self._lib.orc_export_csr(self._g, off.ctypes.data, nb.ctypes.data)
        return off, nb[:self.num_edges]


# ---------------------------------------------------------- structural rules

def dictionary_capacity(n: int) -> int:
    return int(_get().orc_dictionary_capacity(n))


def blocks_for_degree(deg: int, C: int) -> int:
    return int(_get().orc_blocks_for_degree(deg, C))


def block_capacity_rule(deg) -> int:
    d = _u32(deg)
    return int(_get().orc_block_capacity_rule(d.ctypes.data, d.size))


def min_footprint_capacity(deg, weighted: bool = False) -> int:
    d = _u32(deg)
    return int(_get().orc_min_footprint_capacity(d.ctypes.data, d.size, 1 if weighted else 0))


def cbt_path(k: int) -> str:
    buf = ctypes.create_string_buffer(80)
    _get().orc_cbt_path(k, buf)
    return buf.value.decode()


def pop_ranges(need):
    n = _u32(need)
    b = np.zeros(n.size, dtype=np.uint64)
    e = np.zeros(n.size, dtype=np.uint64)
    _get().orc_pop_ranges(n.ctypes.data, n.size, b.ctypes.data, e.ctypes.data)
    return b, e


def insert_block_demand(deg: int, cnt: int, C: int) -> int:
    return int(_get().orc_insert_block_demand(deg, cnt, C))

"""Thin Python binding of libgraphvine.so (include/graphvine.h).

Argument marshalling only: every step of every operation runs in the CUDA
kernels of the library.  Functions keep the C names (gv_create,
gv_insert_edges, ...); `Graph` is a small convenience wrapper over them that
accepts torch tensors (CUDA or CPU) and numpy arrays.  There is no CPU
fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgraphvine.so")

GV_OK = 0
GV_ERR_INVALID_ARG = 1
GV_ERR_OUT_OF_MEMORY = 2
GV_ERR_CUDA = 3
GV_ERR_TIMEOUT = 4
GV_ERR_STATE = 5
GV_DEDUP = 1
GV_GROW = 2
GV_WEIGHTED = 4
GV_RADIX_GROUPING = 8
GV_REBLOCK_MIN_FOOTPRINT = 1  # gv_reblock: the block size of least pool footprint

c_u32, c_u64, c_vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p


class gv_config(ctypes.Structure):
    _fields_ = [
        ("block_capacity", c_u32),
        ("flags", c_u32),
        ("pool_bytes", c_u64),
        ("pool_mem", c_vp),
        ("vertex_capacity", c_u32),
        ("item_blocks", c_u32),
        ("dense_shift", c_u32),
        ("hub_shift", c_u32),
        ("hub_degree", c_u32),
        ("hub_percent", c_u32),
        ("reserved", c_u32),
    ]


class gv_serve_request(ctypes.Structure):
    _fields_ = [
        ("kind", c_u32),
        ("status", ctypes.c_int32),
        ("n", c_u64),
        ("src", c_vp),
        ("dst", c_vp),
        ("answers", c_vp),
        ("arrival", ctypes.c_double),
        ("done", ctypes.c_double),
        ("counts", c_u64 * 2),
    ]


class gv_serve_config(ctypes.Structure):
    _fields_ = [
        ("slots", c_u32),
        ("max_reqs", c_u32),
        ("merge_pairs", c_u64),
        ("realtime", c_u32),
        ("reserved", c_u32),
    ]


class gv_stats_t(ctypes.Structure):
    _fields_ = [
        ("num_vertices", c_u32),
        ("vertex_capacity", c_u32),
        ("block_capacity", c_u32),
        ("flags", c_u32),
        ("num_edges", c_u64),
        ("pool_blocks", c_u64),
        ("pool_blocks_used", c_u64),
        ("pool_blocks_free", c_u64),
        ("pool_bytes", c_u64),
        ("device_bytes", c_u64),
        ("total_inserted", c_u64),
        ("total_deleted", c_u64),
        ("total_rejected", c_u64),
        ("device_status", c_u32),
        ("hub_shift", c_u32),
        ("pool_runs", c_u64),
        ("pool_runs_free", c_u64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# name -> (argtypes, restype); every symbol include/graphvine.h declares.
SIGNATURES = {
    "gv_create": ([ctypes.POINTER(gv_config), c_u32, c_vp, ctypes.POINTER(c_vp)], ctypes.c_int),
    "gv_destroy": ([c_vp], ctypes.c_int),
    "gv_bulk_build": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp], ctypes.c_int),
    "gv_insert_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp], ctypes.c_int),
    "gv_delete_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp], ctypes.c_int),
    "gv_query_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp], ctypes.c_int),
    "gv_neighbors": ([c_vp, c_vp, c_u32, c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp], ctypes.c_int),
    "gv_insert_vertices": ([c_vp, c_u32, c_vp, c_vp], ctypes.c_int),
    "gv_delete_vertices": ([c_vp, c_vp, c_u32, c_vp], ctypes.c_int),
    "gv_export_csr": ([c_vp, c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp], ctypes.c_int),
    "gv_degrees": ([c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "gv_bfs": ([c_vp, c_u32, c_vp, ctypes.POINTER(c_u32), c_vp], ctypes.c_int),
    "gv_sssp": ([c_vp, c_u32, c_vp, ctypes.POINTER(c_u32), c_vp], ctypes.c_int),
    "gv_reblock": ([c_vp, c_u32, ctypes.POINTER(c_u32), c_vp], ctypes.c_int),
    "gv_pagerank": ([c_vp, c_u32, ctypes.c_double, c_vp, c_vp], ctypes.c_int),
    "gv_reserve": ([c_vp, c_u64], ctypes.c_int),
    "gv_sync": ([c_vp], ctypes.c_int),
    "gv_stats": ([c_vp, ctypes.POINTER(gv_stats_t)], ctypes.c_int),
    "gv_validate": ([c_vp, ctypes.POINTER(c_u64), c_vp], ctypes.c_int),
    "gv_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gv_serve": ([c_vp, ctypes.POINTER(gv_serve_request), c_u64, ctypes.POINTER(gv_serve_config), c_vp, c_vp],
                 ctypes.c_int),
    "gv_profile": ([c_vp, ctypes.c_int], ctypes.c_int),
    "gv_profile_read": ([c_vp, c_vp, c_vp, c_u32], ctypes.c_int),
    "gv_profile_num_phases": ([], c_u32),
    "gv_profile_phase_name": ([c_u32], ctypes.c_char_p),
    "gv_degree_offsets_noalloc": ([c_vp, c_vp, c_u32, c_vp, c_vp], ctypes.c_int),
    "gv_insert_edges_segmented": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_u32, c_vp, c_vp], ctypes.c_int),
    "gv_delete_edges_segmented": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_u32, c_vp, c_vp], ctypes.c_int),
    "gv_insert_edges_weighted": ([c_vp, c_vp, c_vp, c_vp, c_u64, c_vp, c_vp], ctypes.c_int),
    "gv_neighbors_weighted": ([c_vp, c_vp, c_u32, c_vp, c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp],
                              ctypes.c_int),
    "gv_set_create": ([ctypes.POINTER(gv_config), c_u32, c_vp, c_vp, ctypes.POINTER(c_vp)], ctypes.c_int),
    "gv_set_insert_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp, c_vp], ctypes.c_int),
    "gv_set_delete_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp, c_vp], ctypes.c_int),
    "gv_set_query_edges": ([c_vp, c_vp, c_vp, c_u64, c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "gv_set_member_neighbors": ([c_vp, c_u32, c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp], ctypes.c_int),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


class GraphVineError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().gv_status_string(code)
        super().__init__(f"{where}: {msg.decode() if msg else code}")


def check(code, where=""):
    if code != GV_OK:
        raise GraphVineError(code, where)
    return code


# ------------------------------------------------------------- marshalling

def ptr(a):
    """Address of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _len(a):
    if hasattr(a, "numel"):
        return int(a.numel())
    return int(np.asarray(a).size)


def _check_u32(a, name):
    item = a.element_size() if hasattr(a, "element_size") else a.itemsize
    if item != 4:
        raise TypeError(f"{name} must hold 32-bit ids")


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


# -------------------------------------------------------- C-named wrappers

def gv_create(num_vertices, block_capacity=0, pool_bytes=0, pool_mem=None, flags=0, vertex_capacity=0,
              stream=None, item_blocks=0, dense_shift=0, hub_shift=0, hub_degree=0, hub_percent=0):
    cfg = gv_config(block_capacity, flags, pool_bytes, ptr(pool_mem), vertex_capacity, item_blocks, dense_shift,
                    hub_shift, hub_degree, hub_percent, 0)
    h = c_vp()
    check(load().gv_create(ctypes.byref(cfg), num_vertices, stream, ctypes.byref(h)), "gv_create")
    return h.value


def gv_destroy(g):
    return check(load().gv_destroy(g), "gv_destroy")


def gv_bulk_build(g, src, dst, counts=None, stream=None):
    _check_u32(src, "src")
    _check_u32(dst, "dst")
    return check(load().gv_bulk_build(g, ptr(src), ptr(dst), _len(src), ptr(counts), stream), "gv_bulk_build")


def gv_insert_edges(g, src, dst, counts=None, stream=None):
    _check_u32(src, "src")
    _check_u32(dst, "dst")
    return check(load().gv_insert_edges(g, ptr(src), ptr(dst), _len(src), ptr(counts), stream), "gv_insert_edges")


def gv_delete_edges(g, src, dst, counts=None, stream=None):
    _check_u32(src, "src")
    _check_u32(dst, "dst")
    return check(load().gv_delete_edges(g, ptr(src), ptr(dst), _len(src), ptr(counts), stream), "gv_delete_edges")


def gv_query_edges(g, src, dst, out, stream=None):
    _check_u32(src, "src")
    _check_u32(dst, "dst")
    return check(load().gv_query_edges(g, ptr(src), ptr(dst), _len(src), ptr(out), stream), "gv_query_edges")


def gv_neighbors(g, vids, offsets, nbrs, nbr_capacity, stream=None):
    total = c_u64(0)
    code = load().gv_neighbors(g, ptr(vids), _len(vids), ptr(offsets), ptr(nbrs), nbr_capacity,
                               ctypes.byref(total), stream)
    return code, total.value


def gv_insert_vertices(g, k, new_ids=None, stream=None):
    return check(load().gv_insert_vertices(g, k, ptr(new_ids), stream), "gv_insert_vertices")


def gv_delete_vertices(g, ids, stream=None):
    _check_u32(ids, "ids")
    return check(load().gv_delete_vertices(g, ptr(ids), _len(ids), stream), "gv_delete_vertices")


def gv_export_csr(g, offsets, nbrs, nbr_capacity, stream=None):
    total = c_u64(0)
    code = load().gv_export_csr(g, ptr(offsets), ptr(nbrs), nbr_capacity, ctypes.byref(total), stream)
    return code, total.value


def gv_bfs(g, source, dist, stream=None):
    """Distances from `source` into `dist` (uint32 per vertex); returns the
    number of levels."""
    levels = c_u32(0)
    check(load().gv_bfs(g, source, ptr(dist), ctypes.byref(levels), stream), "gv_bfs")
    return levels.value


def gv_reblock(g, block_capacity=0, stream=None):
    """Re-block every adjacency at `block_capacity` (0: the paper's rule over
    the current degrees); returns the block capacity now in use."""
    c = c_u32(0)
    check(load().gv_reblock(g, block_capacity, ctypes.byref(c), stream), "gv_reblock")
    return c.value


def gv_sssp(g, source, dist, stream=None):
    """Shortest path lengths from `source` into `dist` (uint64 per vertex);
    returns the number of relaxation rounds."""
    rounds = c_u32(0)
    check(load().gv_sssp(g, source, ptr(dist), ctypes.byref(rounds), stream), "gv_sssp")
    return rounds.value


def gv_pagerank(g, iterations, damping, rank, stream=None):
    return check(load().gv_pagerank(g, iterations, damping, ptr(rank), stream), "gv_pagerank")


def gv_degrees(g, deg, alive=None, stream=None):
    return check(load().gv_degrees(g, ptr(deg), ptr(alive), stream), "gv_degrees")


def gv_reserve(g, max_batch):
    return check(load().gv_reserve(g, max_batch), "gv_reserve")


def gv_sync(g):
    return load().gv_sync(g)


def gv_stats(g):
    st = gv_stats_t()
    code = load().gv_stats(g, ctypes.byref(st))
    return code, st.as_dict()


def gv_validate(g, stream=None):
    v = c_u64(0)
    check(load().gv_validate(g, ctypes.byref(v), stream), "gv_validate")
    return v.value


def gv_degree_offsets_noalloc(g, d_vids, d_offsets, stream=None):
    """Degree offsets of the listed vertices with no allocation (device arrays only)."""
    return load().gv_degree_offsets_noalloc(g, ptr(d_vids), _len(d_vids), ptr(d_offsets), stream)


def gv_insert_edges_segmented(g, d_src, d_dst, d_offsets, nseg, d_counts, stream=None):
    return check(load().gv_insert_edges_segmented(g, ptr(d_src), ptr(d_dst), _len(d_src), ptr(d_offsets), nseg,
                                                  ptr(d_counts), stream), "gv_insert_edges_segmented")


def gv_insert_edges_weighted(g, src, dst, w, counts=None, stream=None):
    _check_u32(src, "src")
    _check_u32(dst, "dst")
    _check_u32(w, "w")
    return check(load().gv_insert_edges_weighted(g, ptr(src), ptr(dst), ptr(w), _len(src), ptr(counts), stream),
                 "gv_insert_edges_weighted")


def gv_neighbors_weighted(g, vids, offsets, nbrs, weights, nbr_capacity, stream=None):
    total = c_u64(0)
    code = load().gv_neighbors_weighted(g, ptr(vids), _len(vids), ptr(offsets), ptr(nbrs), ptr(weights),
                                        nbr_capacity, ctypes.byref(total), stream)
    return code, total.value


def gv_delete_edges_segmented(g, d_src, d_dst, d_offsets, nseg, d_counts, stream=None):
    return check(load().gv_delete_edges_segmented(g, ptr(d_src), ptr(d_dst), _len(d_src), ptr(d_offsets), nseg,
                                                  ptr(d_counts), stream), "gv_delete_edges_segmented")


def gv_profile(g, enable):
    return check(load().gv_profile(g, 1 if enable else 0), "gv_profile")


def gv_profile_read(g):
    """{phase name: (device ms, launches)} since the previous read."""
    lib = load()
    n = lib.gv_profile_num_phases()
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.uint64)
    check(lib.gv_profile_read(g, ms.ctypes.data, cnt.ctypes.data, n), "gv_profile_read")
    return {lib.gv_profile_phase_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}


class GraphSet:
    """Many member graphs in one device structure (gv_set_*)."""

    def __init__(self, num_vertices, block_capacity, pool_bytes=0, stream=None, item_blocks=0, dense_shift=0):
        nv = np.ascontiguousarray(num_vertices, dtype=np.uint32)
        self.num_vertices = nv
        self.stream = stream
        cfg = gv_config(block_capacity, 0, pool_bytes, None, 0, item_blocks, dense_shift, 0, 0, 0, 0)
        h = c_vp()
        check(load().gv_set_create(ctypes.byref(cfg), nv.size, nv.ctypes.data, self._s(), ctypes.byref(h)),
              "gv_set_create")
        self.handle = h.value

    def _s(self):
        return self.stream if self.stream is not None else current_stream()

    def close(self):
        if getattr(self, "handle", None):
            gv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert_edges(self, d_src, d_dst, d_offsets, d_counts):
        check(load().gv_set_insert_edges(self.handle, ptr(d_src), ptr(d_dst), _len(d_src), ptr(d_offsets),
                                         ptr(d_counts), self._s()), "gv_set_insert_edges")

    def delete_edges(self, d_src, d_dst, d_offsets, d_counts):
        check(load().gv_set_delete_edges(self.handle, ptr(d_src), ptr(d_dst), _len(d_src), ptr(d_offsets),
                                         ptr(d_counts), self._s()), "gv_set_delete_edges")

    def query_edges(self, d_src, d_dst, d_offsets, d_counts, d_out):
        check(load().gv_set_query_edges(self.handle, ptr(d_src), ptr(d_dst), _len(d_src), ptr(d_offsets),
                                        ptr(d_counts), ptr(d_out), self._s()), "gv_set_query_edges")

    def member_csr(self, member):
        nv = int(self.num_vertices[member])
        off = np.zeros(nv + 1, dtype=np.uint64)
        total = c_u64(0)
        lib = load()
        code = lib.gv_set_member_neighbors(self.handle, member, off.ctypes.data, None, 0, ctypes.byref(total),
                                           self._s())
        nb = np.zeros(max(total.value, 1), dtype=np.uint32)
        check(lib.gv_set_member_neighbors(self.handle, member, off.ctypes.data, nb.ctypes.data, nb.size,
                                          ctypes.byref(total), self._s()), "gv_set_member_neighbors")
        return off, nb[:total.value]

    def reserve(self, max_batch):
        gv_reserve(self.handle, max_batch)

    def sync(self):
        return check(gv_sync(self.handle), "device status")

    def stats(self):
        code, st = gv_stats(self.handle)
        check(code, "device status")
        return st

    def validate(self):
        return gv_validate(self.handle, self._s())

    def profile(self, enable=True):
        gv_profile(self.handle, enable)

    def profile_read(self):
        return gv_profile_read(self.handle)


# -------------------------------------------------------------- convenience

class Graph:
    """A device-resident GraphVine graph (see include/graphvine.h)."""

    def __init__(self, num_vertices, block_capacity=0, pool_bytes=0, pool_mem=None, flags=0,
                 vertex_capacity=0, stream=None, item_blocks=0, dense_shift=0, hub_shift=0, hub_degree=0,
                 hub_percent=0):
        self.stream = stream
        self._pool_ref = pool_mem  # keep a caller-owned pool alive
        self.handle = gv_create(num_vertices, block_capacity, pool_bytes, pool_mem, flags, vertex_capacity,
                                self._s(), item_blocks, dense_shift, hub_shift, hub_degree, hub_percent)

    def _s(self):
        if self.stream is not None:
            return self.stream
        return current_stream()

    def close(self):
        if getattr(self, "handle", None):
            gv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- operations (arrays: torch CUDA/CPU tensors or numpy)
    def bulk_build(self, src, dst, counts=None):
        gv_bulk_build(self.handle, src, dst, counts, self._s())

    def insert_edges(self, src, dst, counts=None):
        gv_insert_edges(self.handle, src, dst, counts, self._s())

    def delete_edges(self, src, dst, counts=None):
        gv_delete_edges(self.handle, src, dst, counts, self._s())

    def query_edges(self, src, dst, out):
        gv_query_edges(self.handle, src, dst, out, self._s())

    def insert_vertices(self, k, new_ids=None):
        gv_insert_vertices(self.handle, k, new_ids, self._s())

    def delete_vertices(self, ids):
        gv_delete_vertices(self.handle, ids, self._s())

    def reserve(self, max_batch):
        gv_reserve(self.handle, max_batch)

    def sync(self):
        return check(gv_sync(self.handle), "device status")

    def stats(self):
        code, st = gv_stats(self.handle)
        check(code, "device status")
        return st

    def validate(self):
        return gv_validate(self.handle, self._s())

    def profile(self, enable=True):
        gv_profile(self.handle, enable)

    def profile_read(self):
        return gv_profile_read(self.handle)

    # ---- host-side results (numpy), for tests and tools
    def degrees(self):
        st = self.stats()
        nv = st["num_vertices"]
        deg = np.zeros(max(nv, 1), dtype=np.uint32)
        alive = np.zeros(max(nv, 1), dtype=np.uint8)
        gv_degrees(self.handle, deg, alive, self._s())
        return deg[:nv], alive[:nv]

    def neighbors(self, vids):
        vids = np.ascontiguousarray(vids, dtype=np.uint32)
        off = np.zeros(vids.size + 1, dtype=np.uint64)
        code, total = gv_neighbors(self.handle, vids, off, None, 0, self._s())
        nb = np.zeros(max(total, 1), dtype=np.uint32)
        code, total = gv_neighbors(self.handle, vids, off, nb, nb.size, self._s())
        check(code, "gv_neighbors")
        return off, nb[:total]

    def insert_edges_weighted(self, src, dst, w, counts=None):
        return gv_insert_edges_weighted(self.handle, src, dst, w, counts, self._s())

    def neighbors_weighted(self, vids):
        """(offsets, nbrs, weights) of the listed vertices, storage order."""
        vids = np.ascontiguousarray(vids, dtype=np.uint32)
        off = np.zeros(vids.size + 1, dtype=np.uint64)
        code, total = gv_neighbors_weighted(self.handle, vids, off, None, None, 0, self._s())
        nb = np.zeros(max(total, 1), dtype=np.uint32)
        wt = np.zeros(max(total, 1), dtype=np.uint32)
        code, total = gv_neighbors_weighted(self.handle, vids, off, nb, wt, nb.size, self._s())
        check(code, "gv_neighbors_weighted")
        return off, nb[:total], wt[:total]

    def bfs(self, source, dist=None):
        """(dist, levels): uint32 distances (0xFFFFFFFF = unreached); `dist`
        may be a device tensor or host array of vertex-count entries."""
        if dist is None:
            dist = np.zeros(max(self.stats()["num_vertices"], 1), dtype=np.uint32)
        levels = gv_bfs(self.handle, source, dist, self._s())
        return dist, levels

    def reblock(self, block_capacity=0):
        """Change the edge-block size in place (0: the paper's rule over the
        current degrees); returns the new block capacity."""
        return gv_reblock(self.handle, block_capacity, self._s())

    def sssp(self, source, dist=None):
        """(dist, rounds): uint64 path lengths (2^64 - 1 = unreached); entry
        length = payload on a weighted graph, else 1."""
        if dist is None:
            dist = np.zeros(max(self.stats()["num_vertices"], 1), dtype=np.uint64)
        rounds = gv_sssp(self.handle, source, dist, self._s())
        return dist, rounds

    def pagerank(self, iterations, damping=0.85, rank=None):
        if rank is None:
            rank = np.zeros(max(self.stats()["num_vertices"], 1), dtype=np.float64)
        gv_pagerank(self.handle, iterations, damping, rank, self._s())
        return rank

    def export_csr(self):
        st = self.stats()
        nv = st["num_vertices"]
        off = np.zeros(nv + 1, dtype=np.uint64)
        cap = st["num_edges"]
        nb = np.zeros(max(cap, 1), dtype=np.uint32)
        code, total = gv_export_csr(self.handle, off, nb, nb.size, self._s())
        check(code, "gv_export_csr")
        return off, nb[:total]


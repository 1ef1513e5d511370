"""Seeded synthetic workloads for the dynamic-graph hot path.

This module only draws random numbers (through ``gvgen.c``) and filters pair
keys against sets of keys; it holds none of the data structure's arithmetic.
Both the CPU oracle and the GPU path of every test and of the benchmark take
their inputs from here.

The workloads stand in for the DIMACS-10 graphs of the paper's evaluation
(Table 1), which are not shipped: RMAT graphs mirror the skewed co-paper
graphs (G1, G2: high maximum degree, average degree in the tens) and uniform
Erdos-Renyi graphs mirror the low-degree meshes and road networks (G3, G6:
average degree 2 to 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gvgen.c")
_LIB = os.path.join(_HERE, "libgvgen.so")
_lock = threading.Lock()
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile gvgen.c into an in-tree shared library (plain C, gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u32, dbl, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
            lib.gvgen_raw.argtypes = [u64, u64, u64, p]
            lib.gvgen_uniform_pairs.argtypes = [u64, u64, u64, u32, u32, p, p]
            lib.gvgen_uniform_u32.argtypes = [u64, u64, u64, u32, u32, p]
            lib.gvgen_uniform_f64.argtypes = [u64, u64, u64, p]
            lib.gvgen_rmat_pairs.argtypes = [u64, u64, u64, u32, dbl, dbl, dbl, u32, p, p]
            lib.gvgen_shuffle_u64.argtypes = [u64, u64, u64, p]
            lib.gvgen_shuffle_u32.argtypes = [u64, u64, u64, p]
            lib.gvgen_sample_with_replacement.argtypes = [u64, u64, u64, u64, p]
            for f in (lib.gvgen_raw, lib.gvgen_uniform_pairs, lib.gvgen_uniform_u32,
                      lib.gvgen_uniform_f64, lib.gvgen_rmat_pairs, lib.gvgen_shuffle_u64,
                      lib.gvgen_shuffle_u32, lib.gvgen_sample_with_replacement):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- primitives

def raw(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _get().gvgen_raw(seed, stream, n, _ptr(out))
    return out


def uniform_pairs(seed: int, stream: int, n: int, nv: int, lo: int = 0):
    src = np.empty(n, dtype=np.uint32)
    dst = np.empty(n, dtype=np.uint32)
    _get().gvgen_uniform_pairs(seed, stream, n, lo, nv, _ptr(src), _ptr(dst))
    return src, dst


def uniform_u32(seed: int, stream: int, n: int, lo: int, rng: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    _get().gvgen_uniform_u32(seed, stream, n, lo, rng, _ptr(out))
    return out


def uniform_f64(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _get().gvgen_uniform_f64(seed, stream, n, _ptr(out))
    return out


def rmat_pairs(seed: int, stream: int, n: int, scale: int, abcd=RMAT_ABCD, limit: int = 0):
    a, b, c, _ = abcd
    src = np.empty(n, dtype=np.uint32)
    dst = np.empty(n, dtype=np.uint32)
    _get().gvgen_rmat_pairs(seed, stream, n, scale, a, b, c, limit, _ptr(src), _ptr(dst))
    return src, dst


def shuffled(seed: int, stream: int, a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a).copy()
    if a.dtype == np.uint64:
        _get().gvgen_shuffle_u64(seed, stream, a.size, _ptr(a))
    elif a.dtype == np.uint32:
        _get().gvgen_shuffle_u32(seed, stream, a.size, _ptr(a))
    else:
        raise TypeError(a.dtype)
    return a


def sample_indices(seed: int, stream: int, n: int, k: int) -> np.ndarray:
    out = np.empty(k, dtype=np.uint64)
    _get().gvgen_sample_with_replacement(seed, stream, n, k, _ptr(out))
    return out


def keys(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Pack (src, dst) into one uint64 key per pair (src in the high half)."""
    return (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)


def unkey(k: np.ndarray):
    return (k >> np.uint64(32)).astype(np.uint32), (k & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def unique_sorted(a: np.ndarray) -> np.ndarray:
    """The distinct values of ``a`` in increasing order (what np.unique
    returns), by one sort and a comparison of neighbours."""
    a = np.sort(np.asarray(a), kind="stable")
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def in_sorted(a: np.ndarray, table: np.ndarray) -> np.ndarray:
    """Membership of every value of ``a`` in the sorted distinct ``table``."""
    if table.size == 0:
        return np.zeros(a.size, dtype=bool)
    pos = np.searchsorted(table, a)
    pos[pos == table.size] = 0
    return table[pos] == a


def absent_pairs(seed: int, stream: int, n: int, nv: int, exclude_keys: np.ndarray, lo: int = 0):
    """n uniform pairs whose keys are not in ``exclude_keys`` (sorted or not)."""
    excl = unique_sorted(exclude_keys)
    got = []
    have = 0
    rnd = 0
    while have < n:
        s, d = uniform_pairs(seed, stream * 1000 + rnd, max(2 * (n - have), 64), nv, lo)
        k = keys(s, d)
        k = k[~in_sorted(k, excl)]
        got.append(k)
        have += k.size
        rnd += 1
    k = np.concatenate(got)[:n]
    return unkey(k)


# ------------------------------------------------------------ configurations

class Batch:
    """One operation of a workload: kind in {insert, delete, query, vdel, vins}."""

    def __init__(self, kind, src=None, dst=None, ids=None, k=0):
        self.kind = kind
        self.src = src
        self.dst = dst
        self.ids = ids
        self.k = k

    def __len__(self):
        if self.src is not None:
            return int(self.src.size)
        if self.ids is not None:
            return int(self.ids.size)
        return int(self.k)


def tiny_uniform(seed: int = 1, nv: int = 1024, base_edges: int = 8192, rounds: int = 10,
                 batch: int = 1024):
    """Uniform directed multigraph on nv vertices, bulk build of base_edges,
    then ``rounds`` rounds of ``batch`` uniform inserts followed by ``batch``
    deletes: half are distinct pairs of the base graph (disjoint slices of a
    seeded permutation, so each is present when deleted), half are pairs never
    inserted so far (absent)."""
    bs, bd = uniform_pairs(seed, 0, base_edges, nv)
    base_keys = unique_sorted(keys(bs, bd))
    perm = shuffled(seed, 1, base_keys)
    seen = [keys(bs, bd)]
    ops = []
    half = batch // 2
    for r in range(rounds):
        s, d = uniform_pairs(seed, 10 + r, batch, nv)
        ops.append(Batch("insert", s, d))
        seen.append(keys(s, d))
        ex = perm[r * half:(r + 1) * half]
        es, ed = unkey(ex)
        as_, ad = absent_pairs(seed, 100 + r, batch - half, nv, np.concatenate(seen))
        ds = np.concatenate([es, as_])
        dd = np.concatenate([ed, ad])
        order = shuffled(seed, 200 + r, np.arange(ds.size, dtype=np.uint32))
        ops.append(Batch("delete", ds[order], dd[order]))
    return {"nv": nv, "bulk": (bs, bd), "ops": ops, "block_capacity": 16}


def rmat_graph(seed: int = 2, scale: int = 20, edges: int = 16_777_216, abcd=RMAT_ABCD):
    """RMAT base graph (Chakrabarti et al.), ids in [0, 2^scale)."""
    return rmat_pairs(seed, 0, edges, scale, abcd)


def rmat_update(seed: int, scale: int, b: int, round_: int, abcd=RMAT_ABCD):
    """A fresh RMAT insert batch of b edges; the matching delete batch is the
    same pairs (the paper deletes edges inserted by a previous update)."""
    return rmat_pairs(seed, 1000 + round_, b, scale, abcd)


def rmat_queries(seed: int, scale: int, n: int, present_src, present_dst, round_: int,
                 abcd=RMAT_ABCD):
    """n queries: half sampled (with replacement) from the given present pairs,
    half fresh RMAT pairs; interleaved by a seeded permutation."""
    half = n // 2
    idx = sample_indices(seed, 5000 + round_, present_src.size, half)
    ps, pd = present_src[idx], present_dst[idx]
    rs, rd = rmat_pairs(seed, 6000 + round_, n - half, scale, abcd)
    s = np.concatenate([ps, rs])
    d = np.concatenate([pd, rd])
    order = shuffled(seed, 7000 + round_, np.arange(n, dtype=np.uint32))
    return s[order], d[order]


def er_mixed(seed: int = 3, nv: int = 1 << 22, base_edges: int = 16_777_216, rounds: int = 1,
             batch: int = 1_000_000, vdel: int = 65_536, vins: int = 65_536, vins_edges: int = 8):
    """Erdos-Renyi-style uniform multigraph with mixed rounds, then vertex
    deletes of distinct ids and vertex inserts with out-edges to live ids."""
    bs, bd = uniform_pairs(seed, 0, base_edges, nv)
    base_keys = unique_sorted(keys(bs, bd))
    perm = shuffled(seed, 1, base_keys)
    seen = [keys(bs, bd)]
    ops = []
    half = batch // 2
    for r in range(rounds):
        s, d = uniform_pairs(seed, 10 + r, batch, nv)
        ops.append(Batch("insert", s, d))
        seen.append(keys(s, d))
        es, ed = unkey(perm[r * half:(r + 1) * half])
        as_, ad = absent_pairs(seed, 100 + r, batch - half, nv, np.concatenate(seen))
        ds = np.concatenate([es, as_])
        dd = np.concatenate([ed, ad])
        order = shuffled(seed, 200 + r, np.arange(ds.size, dtype=np.uint32))
        ops.append(Batch("delete", ds[order], dd[order]))
    ids = shuffled(seed, 300, np.arange(nv, dtype=np.uint32))[:vdel].copy()
    ops.append(Batch("vdel", ids=ids))
    ops.append(Batch("vins", k=vins))
    dead = np.zeros(nv + vins, dtype=bool)
    dead[ids] = True
    live = np.nonzero(~dead)[0].astype(np.uint32)
    new_ids = np.arange(nv, nv + vins, dtype=np.uint32)
    es = np.repeat(new_ids, vins_edges)
    pick = sample_indices(seed, 400, live.size, es.size)
    ed = live[pick]
    ops.append(Batch("insert", es, ed))
    return {"nv": nv, "bulk": (bs, bd), "ops": ops}


def batched_rmat(seed: int = 4, graphs: int = 256, xlo: float = 10.0, xhi: float = 18.0, avg_degree: int = 8,
                 smax: float = 1e6, abcd=RMAT_ABCD):
    """Many independent RMAT graphs with uneven update batches.

    Member i: x ~ U(xlo, xhi), V = round(2^x) vertices (RMAT at scale
    ceil(x), ids >= V redrawn), E = avg_degree * V base edges; an insert batch
    of s fresh RMAT pairs and a delete batch of s pairs (half distinct pairs
    of the base graph, half pairs absent from it and from the insert batch),
    s = round(exp(U(0, ln smax))).  Returns a list of dicts with member-local
    ids."""
    xs = xlo + (xhi - xlo) * uniform_f64(seed, 0, graphs)
    ls = np.log(smax) * uniform_f64(seed, 1, graphs)

    def member(i):
        x = float(xs[i])
        nv = max(2, int(round(2.0 ** x)))
        scale = int(np.ceil(np.log2(nv)))
        e = avg_degree * nv
        bs, bd = rmat_pairs(seed, 100 + i, e, scale, abcd, limit=nv)
        s = max(1, int(round(np.exp(ls[i]))))
        ins_s, ins_d = rmat_pairs(seed, 100_000 + i, s, scale, abcd, limit=nv)
        base_keys = unique_sorted(keys(bs, bd))
        ex = shuffled(seed, 200_000 + i, base_keys)[:s // 2]
        es, ed = unkey(ex)
        as_, ad = absent_pairs(seed, 300_000 + i, s - es.size, nv,
                               np.concatenate([base_keys, keys(ins_s, ins_d)]))
        ds = np.concatenate([es, as_])
        dd = np.concatenate([ed, ad])
        order = shuffled(seed, 400_000 + i, np.arange(ds.size, dtype=np.uint32))
        return {"nv": nv, "bulk": (bs, bd), "insert": (ins_s, ins_d), "delete": (ds[order], dd[order])}

    # members are independent (each draws from its own streams), so they are
    # generated on host threads (the C generators and numpy's sorts release
    # the interpreter lock); the result does not depend on the thread count
    return _parallel_map(member, range(graphs))


def _parallel_map(fn, items):
    from concurrent.futures import ThreadPoolExecutor
    items = list(items)
    workers = min(len(items), os.cpu_count() or 1)
    if workers <= 1:
        return [fn(i) for i in items]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def concat_member_batches(members, key):
    """Concatenate one batch kind over members: (src, dst, offsets[G+1])."""
    parts = [m[key] for m in members]
    off = np.zeros(len(parts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([p[0].size for p in parts])
    src = np.concatenate([p[0] for p in parts]).astype(np.uint32) if parts else np.zeros(0, np.uint32)
    dst = np.concatenate([p[1] for p in parts]).astype(np.uint32) if parts else np.zeros(0, np.uint32)
    return src, dst, off


def serving_requests(seed: int, base_src, base_dst, scale: int, n_requests: int, smax: float = 1e6,
                     mix=(0.4, 0.4, 0.2), abcd=RMAT_ABCD):
    """Request stream for the serving loop: kinds drawn with probabilities
    mix = (insert, delete, query); sizes s = round(exp(U(0, ln smax)));
    inserts are fresh RMAT pairs, deletes pairs sampled from the base graph
    (present unless an earlier request removed them), queries half base
    pairs, half RMAT pairs.  Also returns unit-mean exponential gaps (scale
    them by 1 / rate for Poisson arrivals)."""
    u = uniform_f64(seed, 0, n_requests)
    ls = np.log(smax) * uniform_f64(seed, 1, n_requests)
    gaps = -np.log(1.0 - uniform_f64(seed, 2, n_requests))

    def request(i):
        s = max(1, int(round(np.exp(ls[i]))))
        if u[i] < mix[0]:
            a, b = rmat_pairs(seed, 10_000 + i, s, scale, abcd)
            return ("insert", a, b)
        if u[i] < mix[0] + mix[1]:
            idx = sample_indices(seed, 20_000 + i, base_src.size, s)
            return ("delete", base_src[idx], base_dst[idx])
        h = s // 2
        idx = sample_indices(seed, 30_000 + i, base_src.size, h)
        a, b = rmat_pairs(seed, 40_000 + i, s - h, scale, abcd)
        return ("query", np.concatenate([base_src[idx], a]), np.concatenate([base_dst[idx], b]))

    reqs = _parallel_map(request, range(n_requests))
    return reqs, gaps

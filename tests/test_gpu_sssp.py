"""GPU single-source shortest paths against the oracle's Dijkstra.

Distances are unique integers (sums of 32-bit lengths in 64 bits), so the
comparison is bit-exact whatever order the GPU's atomic minima take; the
number of relaxation rounds depends on that order and is only bounded.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import Pair, dev_u32

pytestmark = pytest.mark.gpu

INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def _winsert(p, s, d, w):
    import torch
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
    assert tuple(int(x) for x in cnt.cpu().tolist()) == p.o.insert_edges_weighted(s, d, w)


def _check(p, sources, weighted):
    import torch
    nv = p.o.num_vertices
    for s in sources:
        dist, rounds = p.g.sssp(int(s))
        odist, reached = p.o.sssp(int(s), weighted)
        np.testing.assert_array_equal(dist[:nv], odist)
        assert (rounds == 0) == (reached == 0) and rounds <= nv
    d = torch.zeros(nv, dtype=torch.int64, device="cuda")
    p.g.sssp(int(sources[0]), d)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint64), p.o.sssp(int(sources[0]), weighted)[0])
    assert p.g.sync() == 0


@pytest.mark.parametrize("C,wmax", [(4, 1000), (16, 0xFFFFFFFF), (64, 3)])
def test_sssp_weighted_rmat_after_updates(C, wmax):
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    rng = np.random.default_rng(800 + C)
    p = Pair(nv, C=C, pool_bytes=64 << 20, flags=gv.GV_WEIGHTED)
    try:
        bs, bd = W.rmat_pairs(81, 0, 40000, scale)
        bw = rng.integers(0, wmax, bs.size, dtype=np.uint64, endpoint=True).astype(np.uint32)
        _winsert(p, bs, bd, bw)
        _check(p, [0, 1, 77, nv - 1], True)
        s, d = W.rmat_pairs(81, 1, 20000, scale)
        _winsert(p, s, d, rng.integers(0, wmax, s.size, dtype=np.uint64, endpoint=True).astype(np.uint32))
        p.insert(s[:3000], d[:3000])  # unweighted inserts: length 0
        p.delete(bs[:15000], bd[:15000])
        p.vdel(np.array([0, 5, 9, 4000], dtype=np.uint32))
        p.vins(10)
        _winsert(p, np.arange(nv, nv + 10, dtype=np.uint32), np.arange(1, 11, dtype=np.uint32),
                 np.arange(10, dtype=np.uint32))
        p.check()
        _check(p, [0, 1, 2, nv, nv + 9, 100], True)
    finally:
        p.close()


def test_sssp_unweighted_equals_bfs():
    scale, nv = 12, 1 << 12
    bs, bd = W.rmat_pairs(82, 0, 40000, scale)
    p = Pair(nv, C=8, pool_bytes=64 << 20)
    try:
        p.bulk(bs, bd)
        p.delete(bs[:5000], bd[:5000])
        _check(p, [0, 3, 4095], False)
        for s in (0, 3):
            dist, _ = p.g.sssp(s)
            bfs, _ = p.g.bfs(s)
            exp = np.where(bfs[:nv] == 0xFFFFFFFF, INF, bfs[:nv].astype(np.uint64))
            np.testing.assert_array_equal(dist[:nv], exp)
    finally:
        p.close()


@pytest.mark.parametrize("C", [4, 32])
def test_sssp_degenerate(C):
    import paper_2306_08252_gb300 as gv
    p = Pair(100, C=C, pool_bytes=8 << 20, flags=gv.GV_WEIGHTED)
    try:
        _check(p, [0, 99], True)  # no edges
        # a path of maximal lengths (sums past 32 bits), zero-length edges,
        # parallel entries of different lengths, self loops, a hub
        _winsert(p, np.arange(99), np.arange(1, 100), np.full(99, 0xFFFFFFFF, dtype=np.uint32))
        _winsert(p, [5, 5, 5, 7, 0, 0], [5, 6, 6, 7, 50, 50], [0, 9, 2, 1, 3, 0xFFFFFFFF])
        _winsert(p, np.full(300, 50), np.arange(300) % 100, np.arange(300, dtype=np.uint32))
        p.check()
        _check(p, [0, 50, 99], True)
        p.vdel(np.array([50], dtype=np.uint32))
        _check(p, [0, 50, 49], True)  # 50 is dead: reaches nothing
        with pytest.raises(gv.GraphVineError):
            p.g.sssp(100)
    finally:
        p.close()


def test_sssp_full_size_weighted_rmat():
    import paper_2306_08252_gb300 as gv
    bs, bd = W.rmat_graph(2, 20, 1 << 24)
    w = (np.arange(bs.size, dtype=np.uint64) * 2654435761 % 1000).astype(np.uint32)
    p = Pair(1 << 20, C=16, pool_bytes=1 << 30, flags=gv.GV_WEIGHTED)
    try:
        _winsert(p, bs, bd, w)
        p.check(full=False)
        _check(p, [0, 12345], True)
    finally:
        p.close()

"""GPU BFS and PageRank against the oracle on the same graph states.

BFS distances are integers: compared bit-exactly.  PageRank is fp64 with
atomic (unordered) summation on the GPU: a sum of k positive terms in any
order is within (k - 1) u of the exact sum (u = 2^-53), and each iteration
carries the previous error forward scaled by the damping d < 1, so after T
iterations every rank is within about T (k + 2) u relative of the oracle's,
with k the largest number of terms in one sum: the largest in-degree plus
the dangling-mass sum over up to N live vertices; the tests allow 4x that.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import Pair

pytestmark = pytest.mark.gpu

NIL = 0xFFFFFFFF


def _pr_rtol(o, iters):
    off, nb = o.export_csr()
    kmax = int(np.bincount(nb, minlength=o.num_vertices).max()) if nb.size else 0
    n_live = int(o.alive().sum())
    return 4.0 * iters * (kmax + n_live + 2) * 2.0 ** -53


def _check(p, sources, iters=(0, 1, 7, 20)):
    import torch
    for s in sources:
        dist, lv = p.g.bfs(int(s))
        odist, olv = p.o.bfs(int(s))
        np.testing.assert_array_equal(dist[:p.o.num_vertices], odist)
        assert lv == olv
    # device output array
    d = torch.zeros(p.o.num_vertices, dtype=torch.int32, device="cuda")
    p.g.bfs(int(sources[0]), d)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), p.o.bfs(int(sources[0]))[0])
    for it in iters:
        for damp in (0.85, 0.5):
            r = p.g.pagerank(it, damp)
            orr = p.o.pagerank(it, damp)
            np.testing.assert_allclose(r[:orr.size], orr, rtol=_pr_rtol(p.o, max(it, 1)), atol=0)
    assert p.g.sync() == 0


def test_analytics_rmat_after_updates():
    scale, nv = 12, 1 << 12
    bs, bd = W.rmat_pairs(41, 0, 40000, scale)
    p = Pair(nv, C=8, pool_bytes=64 << 20)
    try:
        p.bulk(bs, bd)
        _check(p, [0, 1, 77, nv - 1])
        s, d = W.rmat_pairs(41, 1, 20000, scale)
        p.insert(s, d)
        p.delete(bs[:15000], bd[:15000])
        p.vdel(np.array([0, 5, 9, 4000], dtype=np.uint32))
        p.vins(10)
        p.insert(np.arange(nv, nv + 10, dtype=np.uint32), np.arange(1, 11, dtype=np.uint32))
        p.check()
        _check(p, [0, 1, 2, nv, nv + 9, 100])
    finally:
        p.close()


@pytest.mark.parametrize("C", [4, 64])
def test_analytics_degenerate(C):
    import paper_2306_08252_gb300 as gv
    p = Pair(100, C=C, pool_bytes=8 << 20)
    try:
        # no edges at all
        _check(p, [0, 99], iters=(0, 3))
        # a path, a self loop, parallel edges, a hub
        p.insert(np.arange(99), np.arange(1, 100))
        p.insert([5, 5, 5, 7], [5, 6, 6, 7])
        p.insert(np.full(300, 50), np.arange(300) % 100)
        p.check()
        _check(p, [0, 50, 99], iters=(1, 30))
        with pytest.raises(gv.GraphVineError):
            p.g.bfs(100)
        with pytest.raises(gv.GraphVineError):
            p.g.pagerank(3, 1.5)
    finally:
        p.close()


def test_analytics_full_size_rmat():
    bs, bd = W.rmat_graph(2, 20, 1 << 24)
    p = Pair(1 << 20, C=16, pool_bytes=1 << 30)
    try:
        p.bulk(bs, bd)
        p.check(full=False)
        _check(p, [0, 12345], iters=(10,))
    finally:
        p.close()

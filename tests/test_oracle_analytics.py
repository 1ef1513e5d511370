"""Pins of the oracle's graph analytics (BFS distances, PageRank).

Both are textbook definitions (the paper lists analytics on the structure as
future work).  BFS is pinned to scipy's unweighted shortest paths and to
closed forms; PageRank to closed forms, to the stationary vector of the
dense Google matrix from numpy's eigen-solver, and to mass conservation.
"""
import numpy as np
import pytest

import oracle

NIL = 0xFFFFFFFF


def _random_graph(rng, nv, ne, vdel=0):
    o = oracle.OracleGraph(nv)
    s = rng.integers(0, nv, ne).astype(np.uint32)
    d = rng.integers(0, nv, ne).astype(np.uint32)
    o.insert_edges(s, d)
    if vdel:
        o.delete_vertices(rng.choice(nv, vdel, replace=False).astype(np.uint32))
    return o


def _count_matrix(o):
    off, nb = o.export_csr()
    nv = o.num_vertices
    A = np.zeros((nv, nv))
    for u in range(nv):
        for v in nb[off[u]:off[u + 1]]:
            A[u, v] += 1
    return A


@pytest.mark.parametrize("seed", range(12))
def test_bfs_matches_scipy_shortest_paths(seed):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    rng = np.random.default_rng(seed)
    nv = int(rng.integers(2, 60))
    o = _random_graph(rng, nv, int(rng.integers(0, 3 * nv)), vdel=int(rng.integers(0, nv // 4 + 1)))
    A = _count_matrix(o)
    alive = o.alive()
    for src in rng.choice(nv, min(nv, 5), replace=False):
        dist, levels = o.bfs(int(src))
        if not alive[src]:
            assert (dist == NIL).all() and levels == 0
            continue
        ref = sp.shortest_path(sps.csr_matrix((A > 0).astype(float)), unweighted=True, indices=int(src))
        exp = np.where(np.isinf(ref), NIL, ref).astype(np.int64)
        np.testing.assert_array_equal(dist.astype(np.int64), exp)
        assert levels == int(exp[exp != NIL].max()) + 1
    o.close()


def test_bfs_closed_forms():
    n = 50
    o = oracle.OracleGraph(n)
    # directed path 0 -> 1 -> ... -> n-1, plus a back edge that changes nothing
    o.insert_edges(np.arange(n - 1), np.arange(1, n))
    o.insert_edges([n - 1], [0])
    dist, levels = o.bfs(0)
    np.testing.assert_array_equal(dist, np.arange(n))
    assert levels == n
    dist, _ = o.bfs(n // 2)
    np.testing.assert_array_equal(dist, (np.arange(n) - n // 2) % n)
    assert o.bfs(n)[1] == 0 and (o.bfs(n)[0] == NIL).all()  # out of range source
    o.close()
    # star: hub 0 to every leaf, leaves have no out-edges
    o = oracle.OracleGraph(n)
    o.insert_edges(np.zeros(n - 1), np.arange(1, n))
    dist, levels = o.bfs(0)
    assert dist[0] == 0 and (dist[1:] == 1).all() and levels == 2
    dist, levels = o.bfs(3)
    assert dist[3] == 0 and (np.delete(dist, 3) == NIL).all() and levels == 1
    o.close()


def test_pagerank_closed_forms():
    d = 0.85
    # directed cycle: uniform at every iteration
    n = 17
    o = oracle.OracleGraph(n)
    o.insert_edges(np.arange(n), (np.arange(n) + 1) % n)
    for it in (0, 1, 5, 40):
        np.testing.assert_allclose(o.pagerank(it, d), np.full(n, 1.0 / n), rtol=0, atol=1e-15)
    o.close()
    # two vertices, 0 -> 1, vertex 1 dangling: one step by hand, and the fixed
    # point r0 = 1/(2+d), r1 = (1+d)/(2+d)
    o = oracle.OracleGraph(2)
    o.insert_edges([0], [1])
    r1 = o.pagerank(1, d)
    np.testing.assert_allclose(r1, [(1 - d) / 2 + d * 0.25, (1 - d) / 2 + d * (0.5 + 0.25)], rtol=1e-15)
    np.testing.assert_allclose(o.pagerank(200, d), [1 / (2 + d), (1 + d) / (2 + d)], rtol=1e-12)
    o.close()
    # no vertices alive: all zero
    o = oracle.OracleGraph(3)
    o.delete_vertices(np.arange(3, dtype=np.uint32))
    assert (o.pagerank(3, d) == 0).all()
    o.close()


@pytest.mark.parametrize("seed", range(8))
def test_pagerank_matches_google_matrix_eigenvector(seed):
    rng = np.random.default_rng(100 + seed)
    nv = int(rng.integers(2, 40))
    o = _random_graph(rng, nv, int(rng.integers(1, 4 * nv)), vdel=int(rng.integers(0, nv // 5 + 1)))
    d = float(rng.uniform(0.5, 0.9))
    A = _count_matrix(o)
    alive = o.alive().astype(bool)
    idx = np.nonzero(alive)[0]
    N = idx.size
    A = A[np.ix_(idx, idx)]
    deg = A.sum(1)
    M = np.zeros((N, N))
    for i in range(N):
        M[:, i] = A[i] / deg[i] if deg[i] > 0 else 1.0 / N
    G = d * M + (1 - d) / N
    w, V = np.linalg.eig(G)
    k = int(np.argmin(np.abs(w - 1)))
    pi = np.real(V[:, k])
    pi = pi / pi.sum()
    r = o.pagerank(300, d)
    np.testing.assert_allclose(r[idx], pi, rtol=1e-9, atol=1e-12)
    assert (r[~alive] == 0).all()
    # every iteration keeps the total mass at 1
    for it in (1, 2, 7):
        assert abs(o.pagerank(it, d).sum() - 1.0) < 1e-12
    o.close()

"""Pins of the oracle's single-source shortest paths (Dijkstra).

Pinned to a pure-Python Bellman-Ford over the stored (u, v, w) triples
(a different algorithm, brute force on small graphs), to scipy's Dijkstra
on the min-weight matrix, to the oracle's BFS for unit lengths, and to
closed forms on paths and stars (including sums beyond 32 bits).
"""
import numpy as np
import pytest

import oracle

INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def _weighted_graph(rng, nv, ne, wmax, vdel=0, deletes=0):
    o = oracle.OracleGraph(nv)
    s = rng.integers(0, nv, ne).astype(np.uint32)
    d = rng.integers(0, nv, ne).astype(np.uint32)
    w = rng.integers(0, wmax + 1, ne).astype(np.uint32)
    o.insert_edges_weighted(s, d, w)
    if deletes:
        k = rng.choice(ne, min(ne, deletes), replace=False)
        o.delete_edges(s[k], d[k])
    if vdel:
        o.delete_vertices(rng.choice(nv, vdel, replace=False).astype(np.uint32))
    return o


def _triples(o):
    nv = o.num_vertices
    vids = np.arange(nv, dtype=np.uint32)
    off, nb, w = o.neighbors_weighted(vids)
    out = []
    for u in range(nv):
        for j in range(int(off[u]), int(off[u + 1])):
            out.append((u, int(nb[j]), int(w[j])))
    return out


def _bellman_ford(nv, alive, triples, src, weighted):
    INFP = None
    dist = [INFP] * nv
    if not alive[src]:
        return dist
    dist[src] = 0
    for _ in range(nv):
        changed = False
        for u, v, w in triples:
            if dist[u] is None:
                continue
            nd = dist[u] + (w if weighted else 1)
            if dist[v] is None or nd < dist[v]:
                dist[v] = nd
                changed = True
        if not changed:
            break
    return dist


@pytest.mark.parametrize("seed", range(12))
def test_sssp_matches_bellman_ford(seed):
    rng = np.random.default_rng(900 + seed)
    nv = int(rng.integers(2, 40))
    o = _weighted_graph(rng, nv, int(rng.integers(0, 4 * nv)), wmax=int(rng.choice([0, 1, 5, 1000])),
                        vdel=int(rng.integers(0, nv // 4 + 1)), deletes=int(rng.integers(0, nv)))
    tr = _triples(o)
    alive = o.alive()
    for src in rng.choice(nv, min(nv, 5), replace=False):
        for weighted in (True, False):
            dist, reached = o.sssp(int(src), weighted)
            exp = _bellman_ford(nv, alive, tr, int(src), weighted)
            got = [None if x == INF else int(x) for x in dist]
            assert got == exp
            assert reached == sum(x is not None for x in exp)
    o.close()


@pytest.mark.parametrize("seed", range(6))
def test_sssp_matches_scipy_dijkstra(seed):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(950 + seed)
    nv = int(rng.integers(2, 80))
    # lengths >= 1: a dense matrix entry 0 means "no edge" to scipy
    o = oracle.OracleGraph(nv)
    ne = int(rng.integers(0, 5 * nv))
    s = rng.integers(0, nv, ne).astype(np.uint32)
    d = rng.integers(0, nv, ne).astype(np.uint32)
    w = rng.integers(1, 50, ne).astype(np.uint32)
    o.insert_edges_weighted(s, d, w)
    M = np.zeros((nv, nv))
    for u, v, x in _triples(o):
        M[u, v] = x if M[u, v] == 0 else min(M[u, v], x)
    for src in rng.choice(nv, min(nv, 4), replace=False):
        ref = sp.dijkstra(M, indices=int(src))
        dist, _ = o.sssp(int(src), True)
        exp = np.where(np.isinf(ref), 0, ref).astype(np.uint64)
        exp[np.isinf(ref)] = INF
        np.testing.assert_array_equal(dist, exp)
    o.close()


@pytest.mark.parametrize("seed", range(6))
def test_sssp_unit_lengths_equal_bfs(seed):
    rng = np.random.default_rng(970 + seed)
    nv = int(rng.integers(2, 200))
    o = _weighted_graph(rng, nv, int(rng.integers(0, 3 * nv)), wmax=9, vdel=int(rng.integers(0, nv // 5 + 1)))
    for src in rng.choice(nv, min(nv, 5), replace=False):
        bd, _ = o.bfs(int(src))
        sd, reached = o.sssp(int(src), False)
        exp = np.where(bd == 0xFFFFFFFF, INF, bd.astype(np.uint64))
        np.testing.assert_array_equal(sd, exp)
        assert reached == int((bd != 0xFFFFFFFF).sum())
    o.close()


def test_sssp_closed_forms():
    n = 40
    o = oracle.OracleGraph(n)
    w = (np.arange(n - 1) * 7 + 3).astype(np.uint32)
    o.insert_edges_weighted(np.arange(n - 1), np.arange(1, n), w)
    # a heavier shortcut 0 -> n-1 that never wins, and a zero-length one 0 -> 5
    o.insert_edges_weighted([0], [n - 1], [int(w.sum()) + 1])
    o.insert_edges_weighted([0], [5], [0])
    dist, reached = o.sssp(0, True)
    exp = np.concatenate([[0], np.cumsum(w.astype(np.uint64))])
    exp[5:] -= exp[5]  # from 5 on, the zero-length edge is the start
    np.testing.assert_array_equal(dist, exp)
    assert reached == n
    # deleting vertex 20 cuts the path: 21 .. n-2 unreachable, n-1 via the shortcut
    o.delete_vertices([20])
    dist, reached = o.sssp(0, True)
    assert dist[20] == INF and (dist[21:n - 1] == INF).all() and dist[n - 1] == int(w.sum()) + 1
    assert reached == 21
    d20, r20 = o.sssp(20, True)  # dead source
    assert r20 == 0 and (d20 == INF).all()
    o.close()
    # sums past 32 bits: a path of 2^32 - 1 lengths
    m = 9
    o = oracle.OracleGraph(m)
    o.insert_edges_weighted(np.arange(m - 1), np.arange(1, m), np.full(m - 1, 0xFFFFFFFF, dtype=np.uint32))
    dist, _ = o.sssp(0, True)
    np.testing.assert_array_equal(dist, np.arange(m, dtype=np.uint64) * np.uint64(0xFFFFFFFF))
    o.close()
    # star with parallel entries of different lengths: the lightest copy wins
    o = oracle.OracleGraph(6)
    o.insert_edges_weighted([0, 0, 0, 0, 0, 0], [1, 1, 2, 3, 4, 5], [9, 4, 7, 7, 1, 0])
    dist, reached = o.sssp(0, True)
    np.testing.assert_array_equal(dist, np.array([0, 4, 7, 7, 1, 0], dtype=np.uint64))
    assert reached == 6
    o.close()

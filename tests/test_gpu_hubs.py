"""Hub runs (a per-vertex edge-block size) on the GPU against the oracle.

A vertex whose first allocation takes at least hub_degree entries keeps its
blocks in runs of 2^s contiguous blocks, linked by a tree of run heads.  The
graph's contents must not depend on it: every call is compared with the
oracle as in the plain parity tests.  The structure is checked by
gv_validate (run heads aligned inside the run region, every block owned
once, the last block in the last run) and by the closed form of the blocks
owned (whole runs for hubs), with the hub set tracked by the library's rule
in tests/gpu_util.Pair."""
import numpy as np
import pytest

import workloads as W
from gpu_util import Pair, dev_u32, canon

pytestmark = pytest.mark.gpu


def _hub_ops(p, scale, seed, rounds=3):
    """Skewed RMAT batches: bulk build, then inserts, queries, deletes that
    shrink hubs by whole runs and empty some, vertex deletes of hubs and of
    their neighbours, vertex inserts; checked after every call."""
    nv = 1 << scale
    rng = np.random.default_rng(seed)
    bs, bd = W.rmat_pairs(seed, 0, 40 * nv, scale)
    p.bulk(bs, bd)
    st = p.check()
    assert p.hub.any(), "the workload must produce hubs"
    assert st["pool_runs_free"] < st["pool_runs"]
    deg = p.o.degrees()
    hubs = np.flatnonzero(p.hub[:deg.size]).astype(np.uint32)
    for r in range(rounds):
        s, d = W.rmat_pairs(seed, 1 + r, 10 * nv, scale)
        # a fresh vertex that becomes a hub in one insert
        fresh = np.uint32(nv - 1 - r)
        s = np.concatenate([s, np.full(3000, fresh, dtype=np.uint32)])
        d = np.concatenate([d, rng.integers(0, nv, 3000).astype(np.uint32)])
        p.insert(s, d)
        p.check(full=False)
        qs, qd = W.rmat_queries(seed, scale, 5 * nv, bs, bd, r)
        p.query(qs, qd)
        # deletes: most of one hub's entries (whole runs return), all of
        # another's (it stops being a hub), scattered pairs elsewhere
        off, nb = p.o.neighbors(hubs[r:r + 2])
        h0 = nb[off[0]:off[1]]
        h1 = nb[off[1]:off[2]]
        keep = h0[: max(1, h0.size // 10)]
        gone = np.setdiff1d(h0, keep).astype(np.uint32)
        ds = np.concatenate([np.full(gone.size, hubs[r], dtype=np.uint32),
                             np.full(h1.size, hubs[r + 1], dtype=np.uint32), s[::3]])
        dd = np.concatenate([gone, h1, d[::3]])
        p.delete(ds, dd)
        p.check()
        p.check_sampled(hubs[:8])
    # vertex deletes: a hub and a few vertices that hubs point at
    p.vdel(np.array([hubs[-1], 3, 5, 7], dtype=np.uint32))
    p.check()
    p.vins(nv // 2)  # dictionary doubling keeps the run roots
    s, d = W.rmat_pairs(seed, 50, 5 * nv, scale + 1)
    p.insert(s, d)
    p.check()
    return bs, bd


@pytest.mark.parametrize("C,rs", [(4, 3), (16, 3), (16, 5), (8, 4)])
def test_hub_runs_match_oracle(C, rs):
    from test_gpu_analytics import _check
    p = Pair(1 << 12, C=C, pool_bytes=96 << 20, hub_shift=rs)
    try:
        _hub_ops(p, 12, 900 + C + rs)
        # BFS and PageRank read every adjacency through the tree of run heads
        _check(p, [0, 1, 77], iters=(1, 7))
        dist, _ = p.g.sssp(1)
        np.testing.assert_array_equal(dist[:p.o.num_vertices], p.o.sssp(1, False)[0])
    finally:
        p.close()


def test_hub_runs_small_threshold_and_tiny_sources():
    """hub_degree 1: every vertex's first allocation is a run, so the
    thread-per-source tier, single-item and multi-item compaction all run on
    run adjacencies."""
    p = Pair(1 << 11, C=4, pool_bytes=64 << 20, hub_shift=3, hub_degree=1)
    try:
        _hub_ops(p, 11, 77, rounds=2)
    finally:
        p.close()


def test_hub_runs_results_equal_plain_graph():
    """The same calls on a graph with hub runs and one without give the same
    contents (and both match the oracle)."""
    scale, nv = 12, 1 << 12
    a = Pair(nv, C=16, pool_bytes=64 << 20, hub_shift=4)
    b = Pair(nv, C=16, pool_bytes=64 << 20)
    try:
        for p in (a, b):
            bs, bd = W.rmat_pairs(31, 0, 60000, scale)
            p.bulk(bs, bd)
            s, d = W.rmat_pairs(31, 1, 40000, scale)
            p.insert(s, d)
            p.delete(bs[::2], bd[::2])
            p.check()
        oa, na = a.g.export_csr()
        ob, nb = b.g.export_csr()
        np.testing.assert_array_equal(oa, ob)
        np.testing.assert_array_equal(canon(oa, na), canon(ob, nb))
        sa, sb = a.g.stats(), b.g.stats()
        assert sa["hub_shift"] == 4 and sb["hub_shift"] == 0 and sb["pool_runs"] == 0
    finally:
        a.close()
        b.close()


def test_hub_runs_weighted_payloads_follow_entries():
    import paper_2306_08252_gb300 as gv
    import torch
    scale, nv = 11, 1 << 11
    rng = np.random.default_rng(5)
    p = Pair(nv, C=8, pool_bytes=64 << 20, flags=gv.GV_WEIGHTED, hub_shift=3)
    try:
        for r in range(3):
            s, d = W.rmat_pairs(5, r, 30000, scale)
            w = rng.integers(0, 1 << 32, s.size, dtype=np.uint64).astype(np.uint32)
            before = p.o.degrees().astype(np.int64)
            cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
            p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
            assert tuple(int(x) for x in cnt.cpu().tolist()) == p.o.insert_edges_weighted(s, d, w)
            p._hub_update(before)
            k = rng.integers(0, s.size, 12000)
            p.delete(s[k], d[k])
            p.check()
            vids = np.arange(nv, dtype=np.uint32)
            off, nb, wt = p.g.neighbors_weighted(vids)
            ooff, onb, owt = p.o.neighbors_weighted(vids)
            np.testing.assert_array_equal(off, ooff)
            seg = np.repeat(np.arange(nv), np.diff(off.astype(np.int64)))
            order = np.lexsort((wt, nb, seg))
            np.testing.assert_array_equal(nb[order], onb)
            np.testing.assert_array_equal(wt[order], owt)
        assert p.hub.any()
    finally:
        p.close()


def test_hub_runs_set_semantics():
    import paper_2306_08252_gb300 as gv
    scale, nv = 11, 1 << 11
    p = Pair(nv, C=8, pool_bytes=64 << 20, flags=gv.GV_DEDUP, hub_shift=3)
    try:
        for r in range(3):
            s, d = W.rmat_pairs(6, r, 30000, scale)
            p.insert(np.concatenate([s, s[:5000]]), np.concatenate([d, d[:5000]]))
            p.check()
            p.delete(s[::4], d[::4])
            p.check()
        assert p.hub.any()
    finally:
        p.close()


def test_run_region_exhaustion_is_a_noop():
    """An insert needing more runs than are free fails like an exhausted
    pool: GV_ERR_OUT_OF_MEMORY, counts {0, 0}, nothing changes."""
    import paper_2306_08252_gb300 as gv
    nv = 1024
    # a 2 MiB pool of C = 4 (28 bytes a block), 2% in runs of 8 blocks
    p = Pair(nv, C=4, pool_bytes=2 << 20, hub_shift=3, hub_degree=64, hub_percent=2)
    try:
        st = p.g.stats()
        runs = st["pool_runs"]
        assert runs > 0
        # fill the run region: hubs of 32 blocks (4 runs) each
        nh = runs // 4
        s = np.repeat(np.arange(nh, dtype=np.uint32), 128)
        d = np.tile(np.arange(128, dtype=np.uint32), nh)
        p.insert(s, d)
        st = p.check()
        assert st["pool_runs_free"] == runs - 4 * nh
        before = p.g.export_csr()
        # one more hub than the free runs allow
        s2 = np.full(128 * (st["pool_runs_free"] // 4 + 1) * 4 + 64, nv - 1, dtype=np.uint32)
        d2 = np.arange(s2.size, dtype=np.uint32) % nv
        p.g.insert_edges(dev_u32(s2), dev_u32(d2), p.counts)
        assert gv.gv_sync(p.g.handle) == gv.GV_ERR_OUT_OF_MEMORY
        assert tuple(p.counts.cpu().tolist()) == (0, 0)
        after = p.g.export_csr()
        np.testing.assert_array_equal(before[0], after[0])
        np.testing.assert_array_equal(canon(*before), canon(*after))
        p.check()
        # freeing a hub's runs makes room again
        p.delete(s[:128], d[:128])
        p.check()
        p.insert(s2[:200], d2[:200])
        p.check()
    finally:
        p.close()


def test_hub_config_rejected():
    import paper_2306_08252_gb300 as gv
    for kw in [dict(hub_shift=2), dict(hub_shift=9), dict(hub_shift=3, flags=gv.GV_RADIX_GROUPING),
               dict(hub_shift=3, hub_percent=91)]:
        with pytest.raises(gv.GraphVineError) as e:
            gv.Graph(256, block_capacity=8, pool_bytes=4 << 20, **kw)
        assert e.value.code == gv.GV_ERR_INVALID_ARG


@pytest.mark.parametrize("C,C2,rs", [(16, 16, 3), (8, 32, 4), (32, 4, 3), (16, 0, 5)])
def test_reblock_promotes_grown_vertices_to_runs(C, C2, rs):
    """Vertices that grew past the threshold after their first allocation
    stay plain until gv_reblock, which lays out exactly the vertices of
    degree >= the threshold (at the new C) in runs; the graph keeps working
    (inserts, deletes, queries, vertex deletes) on the new layout."""
    scale, nv = 12, 1 << 12
    p = Pair(nv, C=C, pool_bytes=96 << 20, hub_shift=rs)
    try:
        # many small batches: most vertices' first allocation is small, so
        # they grow past the threshold as plain vertices
        for r in range(6):
            s, d = W.rmat_pairs(41 + C + rs, r, 8 * nv, scale)
            p.insert(s, d)
        p.check()
        deg = p.o.degrees().astype(np.int64)
        T = C << rs
        assert ((deg >= T) & ~p.hub[:deg.size]).any(), "some vertices must have grown past the threshold"
        p.reblock(C2)
        st = p.check()
        d = p.o.degrees().astype(np.int64)[p.hub[:nv]]
        R = 1 << rs
        runs_owned = int((((d + p.C - 1) // p.C + R - 1) // R).sum())
        assert p.hub.any() and st["pool_runs_free"] == st["pool_runs"] - runs_owned
        bs, bd = W.rmat_pairs(41, 20, 6 * nv, scale)
        p.insert(bs, bd)
        p.check()
        qs, qd = W.rmat_queries(41, scale, 4 * nv, bs, bd, 0)
        p.query(qs, qd)
        p.delete(bs[::2], bd[::2])
        p.check()
        hubs = np.flatnonzero(p.hub).astype(np.uint32)
        p.vdel(np.concatenate([hubs[:2], np.array([9, 10], dtype=np.uint32)]))
        p.check()
        p.check_sampled(hubs[2:10])
        # a second resize back to the first size
        p.reblock(C)
        p.check()
        p.delete(bs[1::2], bd[1::2])
        p.check()
    finally:
        p.close()


def test_hub_runs_with_pool_growth():
    """GV_GROW with hub runs: the blocks outside the run region grow (the
    growth rule counts those alone), the run region keeps its size, and the
    graph stays equal to the oracle through growth."""
    import paper_2306_08252_gb300 as gv
    p = Pair(1 << 12, C=8, pool_bytes=4 << 20, flags=gv.GV_GROW, hub_shift=3, hub_percent=90)
    try:
        st0 = p.g.stats()
        _hub_ops(p, 12, 1234, rounds=2)
        st = p.g.stats()
        assert st["pool_blocks"] > st0["pool_blocks"] and st["pool_runs"] == st0["pool_runs"]
    finally:
        p.close()

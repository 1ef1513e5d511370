"""Edge-block resize (gv_reblock) on the GPU against the oracle.

Re-blocking changes only the layout: after it every vertex's entries (and
payloads), degrees, counts and query answers still equal the oracle's, the
structure passes the self-check, C is the requested one (or the paper's
rule, or the size of least footprint, over the current degrees, as the
oracle computes them) and the pool
holds exactly sum_u ceil(deg(u) / C) blocks in use.  Later updates go on
matching the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import Pair, canon, dev_u32

pytestmark = pytest.mark.gpu


def _blocks_used(o, C):
    deg = o.degrees().astype(np.int64)
    return int(((deg + C - 1) // C).sum())


def _check_layout(p, C):
    p.check()
    st = p.g.stats()
    assert st["block_capacity"] == C
    assert st["pool_blocks_used"] == _blocks_used(p.o, C)


def _updates(p, seed, scale, nv, k=6000):
    s, d = W.rmat_pairs(seed, 0, k, scale)
    p.insert(s, d)
    p.query(np.concatenate([s[:2000], d[:2000]]), np.concatenate([d[:2000], s[:2000]]))
    p.delete(s[: k // 2], d[: k // 2])


@pytest.mark.parametrize("C0", [4, 16])
def test_reblock_sequence_keeps_graph(C0):
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    p = Pair(nv, C=C0, pool_bytes=64 << 20)
    try:
        bs, bd = W.rmat_pairs(91, 0, 40000, scale)
        p.bulk(bs, bd)
        for i, C in enumerate([8, 64, 4, 512, 0, 12, gv.GV_REBLOCK_MIN_FOOTPRINT]):
            got = p.g.reblock(C)
            if C == gv.GV_REBLOCK_MIN_FOOTPRINT:
                exp = oracle.min_footprint_capacity(p.o.degrees())
            else:
                exp = C if C else oracle.block_capacity_rule(p.o.degrees())
            assert got == exp
            _check_layout(p, exp)
            _updates(p, 92 + i, scale, nv)
            p.vdel(np.array([i * 7 + 1], dtype=np.uint32))
            _check_layout(p, exp)
    finally:
        p.close()


def test_reblock_weighted_payloads_follow():
    import paper_2306_08252_gb300 as gv
    import torch
    scale, nv = 11, 1 << 11
    rng = np.random.default_rng(93)
    p = Pair(nv, C=8, pool_bytes=64 << 20, flags=gv.GV_WEIGHTED)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    try:
        s, d = W.rmat_pairs(93, 0, 30000, scale)
        w = rng.integers(0, 1 << 32, s.size, dtype=np.uint64).astype(np.uint32)
        p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
        assert tuple(int(x) for x in cnt.cpu().tolist()) == p.o.insert_edges_weighted(s, d, w)
        for C in (32, 4, 0, gv.GV_REBLOCK_MIN_FOOTPRINT):
            got = p.g.reblock(C)
            if C == gv.GV_REBLOCK_MIN_FOOTPRINT:
                assert got == oracle.min_footprint_capacity(p.o.degrees(), weighted=True)
            C = got
            _check_layout(p, C)
            vids = np.arange(nv, dtype=np.uint32)
            off, nb, wt = p.g.neighbors_weighted(vids)
            ooff, onb, owt = p.o.neighbors_weighted(vids)
            np.testing.assert_array_equal(off, ooff)
            seg = np.repeat(np.arange(nv), np.diff(off.astype(np.int64)))
            order = np.lexsort((wt, nb, seg))
            np.testing.assert_array_equal(nb[order], onb)
            np.testing.assert_array_equal(wt[order], owt)
            p.delete(s[:3000], d[:3000])
            s, d, w = s[3000:], d[3000:], w[3000:]
    finally:
        p.close()


def test_reblock_out_of_memory_changes_nothing():
    import paper_2306_08252_gb300 as gv
    nv = 4096
    p = Pair(nv, C=4, pool_bytes=2 << 20)
    try:
        s, d = W.uniform_pairs(94, 0, 60000, nv)
        p.bulk(s, d)  # ~4000 non-empty vertices: at C = 512 they need ~8 MB
        with pytest.raises(gv.GraphVineError) as e:
            p.g.reblock(512)
        assert e.value.code == gv.GV_ERR_OUT_OF_MEMORY
        _check_layout(p, 4)
        _updates(p, 95, 12, nv)
        _check_layout(p, 4)
    finally:
        p.close()


def test_reblock_caller_pool_grown_pool_and_empty():
    import paper_2306_08252_gb300 as gv
    import torch
    nv = 2048
    # caller-owned pool memory
    mem = torch.empty(16 << 20, dtype=torch.uint8, device="cuda")
    g = gv.Graph(nv, block_capacity=8, pool_mem=mem, pool_bytes=mem.numel())
    o = oracle.OracleGraph(nv)
    try:
        s, d = W.rmat_pairs(96, 0, 20000, 11)
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        g.bulk_build(dev_u32(s), dev_u32(d), cnt)
        o.bulk_build(s, d)
        assert g.reblock(20) == 20
        off, nb = g.export_csr()
        ooff, onb = o.export_csr()
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(canon(off, nb), onb)
        assert g.validate() == 0
    finally:
        g.close()
        o.close()
    # a pool that grew (GV_GROW) keeps its grown size through the resize
    p = Pair(nv, C=4, pool_bytes=256 << 10, flags=gv.GV_GROW)
    try:
        for r in range(4):
            s, d = W.rmat_pairs(97, r, 20000, 11)
            p.insert(s, d)
        grown = p.g.stats()["pool_bytes"]
        assert grown > 256 << 10
        C = p.g.reblock(0)
        _check_layout(p, C)
        assert p.g.stats()["pool_bytes"] == grown
        _updates(p, 98, 11, nv)
        _check_layout(p, C)
    finally:
        p.close()
    # no edges yet, C fixed at creation: nothing to move
    p = Pair(64, C=8, pool_bytes=1 << 20)
    try:
        assert p.g.reblock(16) == 16
        _check_layout(p, 16)
        p.insert(np.arange(63), np.arange(1, 64))
        _check_layout(p, 16)
        with pytest.raises(gv.GraphVineError):
            p.g.reblock(6)  # not a multiple of 4
    finally:
        p.close()
    # C not fixed yet (C = 0 at creation, no batch): state error
    g = gv.Graph(64, block_capacity=0, pool_bytes=1 << 20)
    try:
        with pytest.raises(gv.GraphVineError) as e:
            g.reblock(8)
        assert e.value.code == gv.GV_ERR_STATE
    finally:
        g.close()


def test_reblock_full_size_rmat():
    import paper_2306_08252_gb300 as gv
    bs, bd = W.rmat_graph(2, 20, 1 << 24)
    p = Pair(1 << 20, C=16, pool_bytes=1 << 30)
    try:
        p.bulk(bs, bd)
        assert p.g.reblock(gv.GV_REBLOCK_MIN_FOOTPRINT) == oracle.min_footprint_capacity(p.o.degrees())
        C = p.g.reblock(0)
        assert C == oracle.block_capacity_rule(p.o.degrees())
        p.check(full=False)
        st = p.g.stats()
        assert st["block_capacity"] == C and st["pool_blocks_used"] == _blocks_used(p.o, C)
        assert p.g.validate() == 0
        rng = np.random.default_rng(99)
        p.check_sampled(rng.choice(1 << 20, 4096, replace=False))
        s, d = W.rmat_pairs(2, 7, 1_000_000, 20)
        p.insert(s, d)
        p.delete(s[:500_000], d[:500_000])
        p.check(full=False)
        p.check_sampled(np.unique(s[:4096]))
    finally:
        p.close()

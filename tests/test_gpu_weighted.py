"""Weighted entries (GV_WEIGHTED) on the GPU against the oracle: every
entry's 32-bit payload must stay with it through inserts, deletes (in-place
compaction of single-item adjacencies, hole filling of multi-item ones, the
thread-per-source tier), vertex deletes and pool growth; compared per vertex
as sorted (destination, payload) pairs after every call."""
import numpy as np
import pytest

import workloads as W
from gpu_util import Pair, dev_u32

pytestmark = pytest.mark.gpu


def _check_weighted(p):
    p.check()
    nv = p.o.num_vertices
    vids = np.arange(nv, dtype=np.uint32)
    off, nb, wt = p.g.neighbors_weighted(vids)
    ooff, onb, owt = p.o.neighbors_weighted(vids)
    np.testing.assert_array_equal(off, ooff)
    seg = np.repeat(np.arange(nv), np.diff(off.astype(np.int64)))
    order = np.lexsort((wt, nb, seg))  # canonical: by vertex, then (v, w)
    np.testing.assert_array_equal(nb[order], onb)
    np.testing.assert_array_equal(wt[order], owt)


def _winsert(p, s, d, w):
    import torch
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
    exp = p.o.insert_edges_weighted(s, d, w)
    assert tuple(int(x) for x in cnt.cpu().tolist()) == exp


@pytest.mark.parametrize("C,grow", [(4, False), (16, False), (64, False), (8, True)])
def test_weighted_entries_follow_their_pairs(C, grow):
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    rng = np.random.default_rng(71 + C)
    flags = gv.GV_WEIGHTED | (gv.GV_GROW if grow else 0)
    p = Pair(nv, C=C, pool_bytes=(4 << 20) if grow else (64 << 20), flags=flags)
    try:
        bs, bd = W.rmat_pairs(71, 0, 30000, scale)
        p.bulk(bs, bd)  # unweighted: payload 0
        _check_weighted(p)
        hub_d = rng.integers(0, nv, 20000).astype(np.uint32)
        for r in range(4):
            s, d = W.rmat_pairs(71, 1 + r, 15000, scale)
            s = np.concatenate([s, np.zeros(4000, dtype=np.uint32)])  # a hub with many work items
            d = np.concatenate([d, hub_d[r * 4000:(r + 1) * 4000]])
            w = rng.integers(0, 1 << 32, s.size, dtype=np.uint64).astype(np.uint32)
            _winsert(p, s, d, w)
            _check_weighted(p)
            # delete scattered pairs: base ones, hub ones, inserted ones, absent ones
            k = rng.integers(0, s.size, 5000)
            ds = np.concatenate([s[k], bs[r * 3000:(r + 1) * 3000], np.zeros(500, dtype=np.uint32)])
            dd = np.concatenate([d[k], bd[r * 3000:(r + 1) * 3000], hub_d[:500]])
            p.delete(ds, dd)
            _check_weighted(p)
        p.vdel(np.array([0, 3, 17, 1000], dtype=np.uint32))
        _check_weighted(p)
        p.insert(bs[:100], bd[:100])  # plain insert on a weighted graph: payload 0
        _check_weighted(p)
    finally:
        p.close()


def test_weighted_flag_rules():
    import torch
    import paper_2306_08252_gb300 as gv
    with pytest.raises(gv.GraphVineError):
        gv.Graph(100, block_capacity=8, pool_bytes=1 << 20, flags=gv.GV_WEIGHTED | gv.GV_DEDUP)
    g = gv.Graph(100, block_capacity=8, pool_bytes=1 << 20)
    try:
        x = torch.zeros(4, dtype=torch.int32, device="cuda")
        with pytest.raises(gv.GraphVineError):
            g.insert_edges_weighted(x, x, x)
        with pytest.raises(gv.GraphVineError):
            g.neighbors_weighted(np.arange(4, dtype=np.uint32))
    finally:
        g.close()

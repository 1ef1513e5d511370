"""The serving loop: every request's result is the same served in the mix
(continuous batching, merged runs, runs in flight) as applied alone, one
call per request, in arrival order; the final graphs are equal and equal to
the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import canon, dev_u32

pytestmark = pytest.mark.gpu


def _alone(g, o, kind, s, d):
    import torch
    if kind == "insert":
        c = torch.zeros(2, dtype=torch.int64, device="cuda")
        g.insert_edges(dev_u32(s), dev_u32(d), c)
        res = tuple(int(x) for x in c.cpu().tolist())
        assert res == o.insert_edges(s, d)
    elif kind == "delete":
        c = torch.zeros(2, dtype=torch.int64, device="cuda")
        g.delete_edges(dev_u32(s), dev_u32(d), c)
        res = tuple(int(x) for x in c.cpu().tolist())
        assert res == o.delete_edges(s, d)
    else:
        out = torch.zeros(max(len(s), 1), dtype=torch.uint8, device="cuda")
        g.query_edges(dev_u32(s), dev_u32(d), out[:len(s)])
        res = out[:len(s)].cpu().numpy()
        np.testing.assert_array_equal(res, o.query_edges(s, d))
    return res


@pytest.mark.parametrize("realtime,pinned,native", [(False, False, False), (True, False, False), (True, True, False),
                                                    (False, False, True), (True, False, True), (True, True, True)])
def test_served_results_equal_alone(realtime, pinned, native):
    """pinned: the requests live in pinned host memory and are uploaded
    straight from it (serve.pin_requests); native: the loop of the C ABI
    (gv_serve) instead of the Python one."""
    import paper_2306_08252_gb300 as gv
    from paper_2306_08252_gb300 import serve
    scale, C = 12, 8
    bs, bd = W.rmat_pairs(51, 0, 40_000, scale)
    reqs, gaps = W.serving_requests(52 + realtime, bs, bd, scale, 300, smax=3000)
    # a few pairs out of range, to exercise per-request reject counts
    kind, s, d = reqs[3]
    reqs[3] = (kind, np.concatenate([s, [1 << scale]]).astype(np.uint32), np.concatenate([d, [0]]).astype(np.uint32))
    rate = 20_000.0  # requests/s: arrivals faster than service, so requests queue and merge
    arrivals = np.cumsum(gaps) / rate
    served_graph = gv.Graph(1 << scale, block_capacity=C, pool_bytes=64 << 20)
    alone_graph = gv.Graph(1 << scale, block_capacity=C, pool_bytes=64 << 20)
    o = oracle.OracleGraph(1 << scale)
    try:
        served_graph.bulk_build(dev_u32(bs), dev_u32(bd))
        alone_graph.bulk_build(dev_u32(bs), dev_u32(bd))
        o.bulk_build(bs, bd)
        rs = [serve.Request(k, a, b, t) for (k, a, b), t in zip(reqs, arrivals)]
        keep = serve.pin_requests(rs) if pinned else None
        if native:
            st = serve.serve_native(served_graph, rs, slots=3, merge_pairs=20_000, max_reqs=64, realtime=realtime)
            merged, runs = st["merged_requests"], st["runs"]
        else:
            server = serve.Server(served_graph, C, slots=3, merge_pairs=20_000, max_reqs=64)
            server.run(rs, realtime=realtime)
            merged, runs = server.merged_requests, server.runs
        del keep
        assert merged == len(rs)
        assert runs < len(rs)  # some requests were merged
        for r, (kind, s, d) in zip(rs, reqs):
            assert r.status == gv.GV_OK and r.done is not None
            res = _alone(alone_graph, o, kind, s, d)
            if kind == "query":
                np.testing.assert_array_equal(r.result, res)
            else:
                assert r.result == res, (kind, r.result, res)
        a_off, a_nb = served_graph.export_csr()
        b_off, b_nb = alone_graph.export_csr()
        np.testing.assert_array_equal(a_off, b_off)
        np.testing.assert_array_equal(canon(a_off, a_nb), canon(b_off, b_nb))
        o_off, o_nb = o.export_csr()
        np.testing.assert_array_equal(canon(a_off, a_nb), o_nb)
        assert served_graph.validate() == 0
        lat = serve.latency_stats(rs)
        assert lat["p99_ms"] >= lat["p50_ms"] >= 0
    finally:
        served_graph.close()
        alone_graph.close()


@pytest.mark.parametrize("C", [4, 16])
def test_segmented_delete_equals_deletes_in_order(C):
    # one call over several delete batches: per-segment {deleted, rejected}
    # equal those of the batches applied one call each, in order, including
    # pairs named by several segments (credited to the first), pairs named
    # twice inside a segment, absent and invalid pairs, a hub source whose
    # batch set is a global hash set, tiny and multi-item adjacencies
    import torch
    import paper_2306_08252_gb300 as gv
    from gpu_util import Pair
    scale, nv = 12, 1 << 12
    rng = np.random.default_rng(61)
    bs, bd = W.rmat_pairs(61, 0, 50_000, scale)
    hub = rng.integers(0, nv, 20_000).astype(np.uint32)
    bs = np.concatenate([bs, np.zeros_like(hub), bs[:3000]])
    bd = np.concatenate([bd, hub, bd[:3000]])
    p = Pair(nv, C=C, pool_bytes=64 << 20)
    try:
        p.bulk(bs, bd)
        segs = []
        for k in range(7):
            pick = rng.integers(0, bs.size, int(rng.integers(1, 6000)))
            s, d = bs[pick], bd[pick]
            if k == 2:
                s = np.concatenate([s, [nv, 3]]).astype(np.uint32)
                d = np.concatenate([d, [1, nv + 5]]).astype(np.uint32)
            if k == 4:
                s = np.concatenate([s, np.zeros(900, dtype=np.uint32)])
                d = np.concatenate([d, hub[:900]])
            if k == 5:
                s, d = np.concatenate([s, segs[1][0]]), np.concatenate([d, segs[1][1]])
            segs.append((s.astype(np.uint32), d.astype(np.uint32)))
        segs.append((np.zeros(0, dtype=np.uint32), np.zeros(0, dtype=np.uint32)))
        off = np.zeros(len(segs) + 1, dtype=np.int64)
        off[1:] = np.cumsum([a.size for a, _ in segs])
        src = np.concatenate([a for a, _ in segs])
        dst = np.concatenate([b for _, b in segs])
        cnt = torch.zeros(2 * len(segs), dtype=torch.int64, device="cuda")
        gv.gv_delete_edges_segmented(p.g.handle, dev_u32(src), dev_u32(dst), torch.from_numpy(off).cuda(),
                                     len(segs), cnt)
        got = cnt.cpu().numpy().reshape(-1, 2)
        exp = np.array([p.o.delete_edges(a, b) for a, b in segs])
        np.testing.assert_array_equal(got, exp)
        assert exp[:, 0].sum() > 0 and exp[2, 1] == 2
        p.check()
    finally:
        p.close()


def test_segmented_insert_pool_exhaustion_is_a_noop():
    # a merged insert that does not fit the pool changes nothing and reports
    # {0, 0} for every request; the exhaustion is latched for gv_sync
    import torch
    import paper_2306_08252_gb300 as gv
    from gpu_util import Pair
    nv, C = 2000, 8
    p = Pair(nv, C=C, pool_bytes=600 * (4 * C + 12))
    try:
        bs, bd = W.uniform_pairs(81, 0, 300, nv)  # ~290 sources: about half of the ~600 blocks
        p.bulk(bs, bd)
        p.check()
        segs = [W.uniform_pairs(81, 1 + k, 3000, nv) for k in range(3)]
        off = np.zeros(4, dtype=np.int64)
        off[1:] = np.cumsum([a.size for a, _ in segs])
        cnt = torch.full((6,), 7, dtype=torch.int64, device="cuda")
        gv.gv_insert_edges_segmented(p.g.handle, dev_u32(np.concatenate([a for a, _ in segs])),
                                     dev_u32(np.concatenate([b for _, b in segs])), torch.from_numpy(off).cuda(),
                                     3, cnt)
        assert cnt.cpu().tolist() == [0] * 6
        assert gv.gv_sync(p.g.handle) == gv.GV_ERR_OUT_OF_MEMORY
        p.check()  # unchanged: still equal to the oracle, which saw only the bulk build
    finally:
        p.close()


def test_native_loop_refuses_an_insert_that_cannot_fit():
    # the native loop's admission: a run whose worst-case block demand does
    # not fit the free blocks (after draining and reading the pool again)
    # fails with GV_ERR_OUT_OF_MEMORY and {0, 0}; the other requests run as
    # if it had not been sent
    import paper_2306_08252_gb300 as gv
    from paper_2306_08252_gb300 import serve
    nv, C = 2000, 8
    g = gv.Graph(nv, block_capacity=C, pool_bytes=600 * (4 * C + 12))
    o = oracle.OracleGraph(nv)
    try:
        bs, bd = W.uniform_pairs(91, 0, 300, nv)
        g.bulk_build(dev_u32(bs), dev_u32(bd))
        o.bulk_build(bs, bd)
        small = W.uniform_pairs(91, 1, 50, nv)
        huge = W.uniform_pairs(91, 2, 3000, nv)
        rs = [serve.Request("insert", *small), serve.Request("query", bs[:100], bd[:100]),
              serve.Request("insert", *huge), serve.Request("delete", bs[:50], bd[:50])]
        serve.serve_native(g, rs, slots=2, merge_pairs=4000, max_reqs=8, realtime=False)
        assert [r.status for r in rs] == [gv.GV_OK, gv.GV_OK, gv.GV_ERR_OUT_OF_MEMORY, gv.GV_OK]
        assert rs[0].result == o.insert_edges(*small)
        np.testing.assert_array_equal(rs[1].result, o.query_edges(bs[:100], bd[:100]))
        assert rs[2].result == (0, 0)
        assert rs[3].result == o.delete_edges(bs[:50], bd[:50])
        assert g.sync() == 0 and g.validate() == 0
        off, nb = g.export_csr()
        ooff, onb = o.export_csr()
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(canon(off, nb), onb)
    finally:
        g.close()
        o.close()

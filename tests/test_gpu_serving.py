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


@pytest.mark.parametrize("realtime", [False, True])
def test_served_results_equal_alone(realtime):
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
        server = serve.Server(served_graph, C, slots=3, merge_pairs=20_000, max_reqs=64)
        rs = [serve.Request(k, a, b, t) for (k, a, b), t in zip(reqs, arrivals)]
        server.run(rs, realtime=realtime)
        assert server.merged_requests == len(rs)
        assert server.runs < len(rs)  # some requests were merged
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

"""The source-sharded graph on the GPU: one rank (NCCL, world size 1) whose
shard is a library graph behind GpuShard, against the oracle.  With one
rank the routing is the identity; what runs is the adapter over the
library's segmented insert and delete, its queries, vertex deletes and
inserts, and the collectives on device tensors.  (Every run here has one
GPU; the routing between ranks is covered by the two-rank CPU test.)"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _main(port, out):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    import paper_2306_08252_gb300 as gv
    from paper_2306_08252_gb300.shard import GpuShard, ShardedGraph

    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        nv = 4096
        g = gv.Graph(nv, block_capacity=8, pool_bytes=64 << 20)
        sg = ShardedGraph(GpuShard(g))
        o = oracle.OracleGraph(nv)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()
        bs, bd = W.rmat_pairs(61, 0, 60000, 12)
        assert sg.insert_edges(t(bs), t(bd)) == o.insert_edges(bs, bd)
        qs, qd = W.rmat_queries(61, 12, 5000, bs, bd, 0)
        np.testing.assert_array_equal(sg.query_edges(t(qs), t(qd)).cpu().numpy(), o.query_edges(qs, qd))
        ds = np.concatenate([bs[:9000], qs[2500:]])
        dd = np.concatenate([bd[:9000], qd[2500:]])
        assert sg.delete_edges(t(ds), t(dd)) == o.delete_edges(ds, dd)
        vd = np.array([0, 1, 77, 4095], dtype=np.uint32)
        sg.delete_vertices(t(vd))
        o.delete_vertices(vd)
        ids = sg.insert_vertices(5)
        np.testing.assert_array_equal(ids, o.insert_vertices(5))
        s2, d2 = W.rmat_pairs(61, 1, 20000, 12)
        s2[:100] = np.arange(nv, nv + 5, dtype=np.uint32).repeat(20)
        assert sg.insert_edges(t(s2), t(d2)) == o.insert_edges(s2, d2)
        np.testing.assert_array_equal(sg.degrees(), o.degrees())
        off, nb = sg.export_csr()
        ooff, onb = o.export_csr()
        np.testing.assert_array_equal(off, ooff)
        seg = np.repeat(np.arange(off.size - 1), np.diff(off.astype(np.int64)))
        np.testing.assert_array_equal(nb[np.lexsort((nb, seg))], onb)
        assert g.sync() == 0 and g.validate() == 0
        g.close()
        o.close()
        out.put("ok")
    except Exception as e:
        out.put(repr(e))
        raise
    finally:
        dist.destroy_process_group()


def test_sharded_graph_one_gpu_matches_oracle():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_main, args=(port, q))
    p.start()
    res = q.get(timeout=300)
    p.join(timeout=60)
    assert res == "ok", res
    assert p.exitcode == 0

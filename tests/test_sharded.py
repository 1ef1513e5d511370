"""The source-sharded graph (paper_2306_08252_gb300.shard) as two gloo ranks
on the CPU.

Each rank's shard is the CPU oracle behind the shard interface; every rank
issues its own batches; the sharded results must equal those of one oracle
that applies the ranks' batches one after another in rank order: each rank's
{inserted, rejected} and {deleted, rejected} counts and query answers, the
degrees and the whole CSR, through vertex deletes and inserts.
"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class OracleShard:
    """The shard interface of paper_2306_08252_gb300.shard over the CPU
    oracle (segments applied one after another)."""

    def __init__(self, nv):
        import torch
        import oracle
        self.torch = torch
        self.o = oracle.OracleGraph(nv)
        self.device = torch.device("cpu")

    @property
    def num_vertices(self):
        return self.o.num_vertices

    def _u32(self, t):
        return t.numpy().view(np.uint32)

    def _segmented(self, fn, src, dst, offsets):
        s, d = self._u32(src), self._u32(dst)
        off = offsets.numpy()
        res = [fn(s[off[i]:off[i + 1]], d[off[i]:off[i + 1]]) for i in range(off.size - 1)]
        return self.torch.tensor(res, dtype=self.torch.int64).view(-1, 2)

    def insert_segmented(self, src, dst, offsets):
        return self._segmented(self.o.insert_edges, src, dst, offsets)

    def delete_segmented(self, src, dst, offsets):
        return self._segmented(self.o.delete_edges, src, dst, offsets)

    def query(self, src, dst):
        return self.torch.from_numpy(self.o.query_edges(self._u32(src), self._u32(dst)).astype(np.uint8))

    def insert_vertices(self, k):
        if k:
            self.o.insert_vertices(k)

    def delete_vertices(self, ids):
        if ids.numel():
            self.o.delete_vertices(self._u32(ids))

    def degrees(self):
        return self.o.degrees()

    def export_csr(self):
        return self.o.export_csr()


def _pairs(seed, r, n, nv, invalid=0.02):
    rng = np.random.default_rng(seed * 100 + r)
    s = rng.integers(0, nv, n).astype(np.uint32)
    d = rng.integers(0, nv, n).astype(np.uint32)
    bad = rng.random(n) < invalid
    s[bad] = nv + rng.integers(0, 50, int(bad.sum())).astype(np.uint32)  # out of range: rejected
    return s, d


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2306_08252_gb300.shard import ShardedGraph

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        nv = 600
        sg = ShardedGraph(OracleShard(nv))
        ref = oracle.OracleGraph(nv)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32))

        def each_rank(fn_ref, batches):
            """The reference applies every rank's batch in rank order; returns
            this rank's reference result."""
            mine = None
            for r in range(world):
                res = fn_ref(*batches[r])
                if r == rank:
                    mine = res
            return mine

        # inserts (with repeats and invalid ids), queries, deletes that overlap
        # between ranks, vertex deletes and inserts, more inserts and queries
        ins = [_pairs(1, r, 4000 + 700 * r, nv) for r in range(world)]
        got = sg.insert_edges(t(ins[rank][0]), t(ins[rank][1]))
        assert got == each_rank(ref.insert_edges, ins), (got,)
        qry = [_pairs(2, r, 3000, nv) for r in range(world)]
        for r in range(world):  # half of each query batch names stored pairs
            qry[r][0][:1500], qry[r][1][:1500] = ins[(r + 1) % world][0][:1500], ins[(r + 1) % world][1][:1500]
        ans = sg.query_edges(t(qry[rank][0]), t(qry[rank][1])).numpy()
        np.testing.assert_array_equal(ans, ref.query_edges(*qry[rank]))
        dels = []
        for r in range(world):
            a = np.concatenate([ins[0][0][r::3], ins[1][0][:500], _pairs(3, r, 300, nv)[0]])
            b = np.concatenate([ins[0][1][r::3], ins[1][1][:500], _pairs(3, r, 300, nv)[1]])
            dels.append((a, b))
        got = sg.delete_edges(t(dels[rank][0]), t(dels[rank][1]))
        assert got == each_rank(ref.delete_edges, dels), (got,)
        vd = [np.array([5 + r, 17, 200 + 3 * r], dtype=np.uint32) for r in range(world)]
        sg.delete_vertices(t(vd[rank]))
        ref.delete_vertices(np.unique(np.concatenate(vd)))
        ks = [3 + 2 * r for r in range(world)]
        ids = sg.insert_vertices(ks[rank])
        ref_ids = ref.insert_vertices(sum(ks))
        np.testing.assert_array_equal(ids, ref_ids[sum(ks[:rank]):sum(ks[:rank + 1])])
        nv2 = nv + sum(ks)
        ins2 = [_pairs(4, r, 2500, nv2) for r in range(world)]
        got = sg.insert_edges(t(ins2[rank][0]), t(ins2[rank][1]))
        assert got == each_rank(ref.insert_edges, ins2), (got,)
        ans = sg.query_edges(t(qry[rank][0]), t(qry[rank][1])).numpy()
        np.testing.assert_array_equal(ans, ref.query_edges(*qry[rank]))
        # empty batches are collective calls too
        assert sg.insert_edges(t(np.zeros(0, np.uint32)), t(np.zeros(0, np.uint32))) == (0, 0)
        np.testing.assert_array_equal(sg.degrees(), ref.degrees())
        off, nb = sg.export_csr()
        roff, rnb = ref.export_csr()
        np.testing.assert_array_equal(off, roff)
        seg = np.repeat(np.arange(off.size - 1), np.diff(off.astype(np.int64)))
        np.testing.assert_array_equal(nb[np.lexsort((nb, seg))], rnb)
        out.put((rank, "ok"))
    except Exception as e:  # reported to the test process
        out.put((rank, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_graph_two_ranks_match_one_oracle():
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: "ok", 1: "ok"}, res
    assert all(p.exitcode == 0 for p in procs)

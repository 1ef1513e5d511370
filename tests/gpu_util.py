"""Shared helpers of the GPU parity tests (not a test module)."""
import numpy as np

import oracle


def dev_u32(a):
    import torch
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()


def canon(off, nb):
    """Sort each adjacency (storage order within a vertex is unspecified)."""
    off = np.asarray(off, dtype=np.int64)
    nb = np.asarray(nb)
    seg = np.repeat(np.arange(off.size - 1), np.diff(off))
    order = np.lexsort((nb, seg))
    return nb[order]


class Pair:
    """A GPU graph and the oracle driven in lockstep, compared after each call."""

    def __init__(self, nv, C=16, pool_bytes=64 << 20, flags=0):
        import paper_2306_08252_gb300 as gv
        import torch
        self.torch = torch
        self.g = gv.Graph(nv, block_capacity=C, pool_bytes=pool_bytes, flags=flags)
        self.o = oracle.OracleGraph(nv, flags)
        self.counts = torch.zeros(2, dtype=torch.int64, device="cuda")

    def close(self):
        self.g.close()
        self.o.close()

    def _counts(self):
        return tuple(int(x) for x in self.counts.cpu().tolist())

    def bulk(self, s, d):
        self.g.bulk_build(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.bulk_build(s, d)
        assert self._counts() == exp, (self._counts(), exp)

    def insert(self, s, d):
        self.g.insert_edges(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.insert_edges(s, d)
        assert self._counts() == exp, (self._counts(), exp)

    def delete(self, s, d):
        self.g.delete_edges(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.delete_edges(s, d)
        assert self._counts() == exp, (self._counts(), exp)

    def query(self, s, d):
        out = self.torch.zeros(len(s), dtype=self.torch.uint8, device="cuda")
        self.g.query_edges(dev_u32(s), dev_u32(d), out)
        np.testing.assert_array_equal(out.cpu().numpy(), self.o.query_edges(s, d))

    def vdel(self, ids):
        self.g.delete_vertices(dev_u32(ids))
        self.o.delete_vertices(ids)

    def vins(self, k):
        ids = self.torch.zeros(max(k, 1), dtype=self.torch.int32, device="cuda")
        self.g.insert_vertices(k, ids if k else None)
        exp = self.o.insert_vertices(k)
        if k:
            np.testing.assert_array_equal(ids[:k].cpu().numpy().view(np.uint32), exp)

    def check(self, full=True, validate=True):
        assert self.g.sync() == 0
        st = self.g.stats()
        assert st["num_vertices"] == self.o.num_vertices
        assert st["num_edges"] == self.o.num_edges
        deg, alive = self.g.degrees()
        np.testing.assert_array_equal(deg, self.o.degrees())
        np.testing.assert_array_equal(alive, self.o.alive())
        if full:
            off, nb = self.g.export_csr()
            ooff, onb = self.o.export_csr()
            np.testing.assert_array_equal(off, ooff)
            np.testing.assert_array_equal(canon(off, nb), onb)
        if validate:
            assert self.g.validate() == 0
        # structural closed form: blocks = sum ceil(deg / C)
        C = st["block_capacity"]
        if C:
            d = self.o.degrees().astype(np.int64)
            assert st["pool_blocks_used"] == int(((d + C - 1) // C).sum())
        return st

    def check_sampled(self, vids):
        vids = np.asarray(vids, dtype=np.uint32)
        off, nb = self.g.neighbors(vids)
        ooff, onb = self.o.neighbors(vids)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(canon(off, nb), onb)

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


def blocks_owned(deg, hub, C, rs):
    """Blocks the adjacencies own: ceil(deg / C) for a plain vertex, whole
    runs of 2^rs blocks for a hub (a vertex in runs)."""
    d = np.asarray(deg, dtype=np.int64)
    nb = (d + C - 1) // C
    if rs:
        R = 1 << rs
        h = np.zeros(d.size, dtype=bool)
        h[:min(d.size, hub.size)] = hub[:d.size]
        nb = np.where(h, (nb + R - 1) // R * R, nb)
    return int(nb.sum())


class Pair:
    """A GPU graph and the oracle driven in lockstep, compared after each call.

    With hub runs (hub_shift > 0) the pair also tracks which vertices hold
    their blocks in runs, by the library's rule: a vertex with no entries
    whose call gives it at least hub_degree entries becomes a hub; a vertex
    that loses all its entries stops being one."""

    def __init__(self, nv, C=16, pool_bytes=64 << 20, flags=0, hub_shift=0, hub_degree=0, hub_percent=0):
        import paper_2306_08252_gb300 as gv
        import torch
        self.torch = torch
        self.g = gv.Graph(nv, block_capacity=C, pool_bytes=pool_bytes, flags=flags, hub_shift=hub_shift,
                          hub_degree=hub_degree, hub_percent=hub_percent)
        self.o = oracle.OracleGraph(nv, flags)
        self.counts = torch.zeros(2, dtype=torch.int64, device="cuda")
        self.rs = hub_shift
        self.C = C
        self.hub_degree = hub_degree
        self.hub = np.zeros(max(nv, 1), dtype=bool)

    def _hub_update(self, before):
        """Class model after a call that changed degrees from `before`."""
        if not self.rs:
            return
        after = self.o.degrees().astype(np.int64)
        if self.hub.size < after.size:
            self.hub = np.concatenate([self.hub, np.zeros(after.size - self.hub.size, dtype=bool)])
        b = np.zeros(after.size, dtype=np.int64)
        b[:before.size] = before
        if not self.C:
            self.C = self.g.stats()["block_capacity"]  # fixed by the first batch
        T = self.hub_degree or (self.C << self.rs)
        self.hub[:after.size] |= (b == 0) & (after - b >= T)
        self.hub[:after.size] &= after > 0

    def close(self):
        self.g.close()
        self.o.close()

    def _counts(self):
        return tuple(int(x) for x in self.counts.cpu().tolist())

    def bulk(self, s, d):
        before = self.o.degrees().astype(np.int64)
        self.g.bulk_build(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.bulk_build(s, d)
        assert self._counts() == exp, (self._counts(), exp)
        self._hub_update(before)

    def insert(self, s, d):
        before = self.o.degrees().astype(np.int64)
        self.g.insert_edges(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.insert_edges(s, d)
        assert self._counts() == exp, (self._counts(), exp)
        self._hub_update(before)

    def delete(self, s, d):
        before = self.o.degrees().astype(np.int64)
        self.g.delete_edges(dev_u32(s), dev_u32(d), self.counts)
        exp = self.o.delete_edges(s, d)
        assert self._counts() == exp, (self._counts(), exp)
        self._hub_update(before)

    def query(self, s, d):
        out = self.torch.zeros(len(s), dtype=self.torch.uint8, device="cuda")
        self.g.query_edges(dev_u32(s), dev_u32(d), out)
        np.testing.assert_array_equal(out.cpu().numpy(), self.o.query_edges(s, d))

    def reblock(self, C2):
        """Edge-block resize; with hub runs every vertex is re-decided: a hub
        iff its degree reaches the threshold at the new C."""
        c = self.g.reblock(C2)
        self.C = c
        if self.rs:
            d = self.o.degrees().astype(np.int64)
            T = self.hub_degree or (c << self.rs)
            self.hub = np.zeros(max(d.size, self.hub.size), dtype=bool)
            self.hub[:d.size] = (d > 0) & (d >= T)
        return c

    def vdel(self, ids):
        before = self.o.degrees().astype(np.int64)
        self.g.delete_vertices(dev_u32(ids))
        self.o.delete_vertices(ids)
        self._hub_update(before)

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
        # structural closed form: blocks = sum ceil(deg / C), hubs in whole runs
        C = st["block_capacity"]
        if C:
            assert st["pool_blocks_used"] == blocks_owned(self.o.degrees(), self.hub, C, self.rs)
        return st

    def check_sampled(self, vids):
        vids = np.asarray(vids, dtype=np.uint32)
        off, nb = self.g.neighbors(vids)
        ooff, onb = self.o.neighbors(vids)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(canon(off, nb), onb)

"""A graph split by source vertex over the ranks of a torch.distributed group.

The paper's structure keeps one adjacency per source vertex ("Vertex
dictionary and adjacency list structure"), so a graph splits by source:
rank r owns the sources u with u % world == r and holds them in its shard
(one graph of the library on its own GPU, over the whole id range; only
owned sources get entries).  Ids are dense and power-law graphs put their
hubs on low ids, so the modulo spreads the hubs over the ranks.

Every call is collective: each rank passes its own batch (possibly empty)
and gets the results for its own pairs.
* Insert, delete, query: one all-to-all routes every pair to the owner of
  its source; the owner applies the pairs as one segmented call whose
  segments are the origin ranks in rank order; a second all-to-all returns
  each origin its per-pair answers (queries) or its {done, rejected} counts.
  The result is that of applying the ranks' batches one after another in
  rank order: inserts commute, and a segmented delete credits each removed
  entry to the first segment (lowest rank) naming its pair.
* Vertex delete: the deleted ids are all-gathered and every shard deletes
  all of them (each removes its own entries pointing at them, and every
  shard must reject new pairs naming them).
* Vertex insert: every shard appends the total count; rank r gets the ids
  after those of the lower ranks.

The shard object is any adapter with the methods of `GpuShard` below (the
tests use one over the CPU oracle with the gloo backend).
"""
from __future__ import annotations

import numpy as np


def _dist():
    import torch.distributed as dist
    return dist


class GpuShard:
    """Adapter of one library graph (paper_2306_08252_gb300.Graph) for
    ShardedGraph: segmented calls on device arrays."""

    def __init__(self, graph):
        import torch
        from . import graphvine as gv
        self.torch, self.gv, self.g = torch, gv, graph
        self.device = torch.device("cuda", torch.cuda.current_device())

    @property
    def num_vertices(self):
        return int(self.g.stats()["num_vertices"])

    def _segmented(self, fn, src, dst, offsets):
        torch = self.torch
        nseg = offsets.numel() - 1
        cnt = torch.zeros(2 * nseg, dtype=torch.int64, device=self.device)
        fn(self.g.handle, src, dst, offsets.to(self.device), nseg, cnt, torch.cuda.current_stream().cuda_stream)
        return cnt.view(nseg, 2)

    def insert_segmented(self, src, dst, offsets):
        return self._segmented(self.gv.gv_insert_edges_segmented, src, dst, offsets)

    def delete_segmented(self, src, dst, offsets):
        return self._segmented(self.gv.gv_delete_edges_segmented, src, dst, offsets)

    def query(self, src, dst):
        out = self.torch.zeros(max(src.numel(), 1), dtype=self.torch.uint8, device=self.device)
        if src.numel():
            self.g.query_edges(src, dst, out)
        return out[:src.numel()]

    def insert_vertices(self, k):
        if k:
            self.g.insert_vertices(k)

    def delete_vertices(self, ids):
        if ids.numel():
            self.g.delete_vertices(ids)

    def degrees(self):
        deg, _ = self.g.degrees()
        return np.asarray(deg, dtype=np.uint32)

    def export_csr(self):
        return self.g.export_csr()


class ShardedGraph:
    """Collective view of the shards of one graph (see the module text)."""

    def __init__(self, shard, group=None):
        dist = _dist()
        self.shard = shard
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.device = shard.device

    # ------------------------------------------------------------- routing
    def owner(self, src):
        """Owning rank of each source id (int32 storage of uint32 ids)."""
        import torch
        return (src.to(torch.int64) & 0xFFFFFFFF) % self.world

    def _exchange(self, send, send_counts):
        """All-to-all of `send` (grouped by destination rank, send_counts[r]
        entries for rank r); returns (received, recv_counts), the received
        entries grouped by origin rank in rank order."""
        import torch
        dist = _dist()
        sc = torch.as_tensor(send_counts, dtype=torch.int64, device=self.device)
        rc = torch.empty_like(sc)
        dist.all_to_all_single(rc, sc, group=self.group)
        rcl = [int(x) for x in rc.tolist()]
        recv = torch.empty(sum(rcl), dtype=send.dtype, device=self.device)
        dist.all_to_all_single(recv, send, rcl, [int(x) for x in send_counts], group=self.group)
        return recv, rcl

    def _route(self, src, dst):
        """Pairs to their owners: (order of this rank's pairs by owner, send
        counts, received sources, received destinations, receive counts)."""
        import torch
        own = self.owner(src)
        order = torch.sort(own, stable=True).indices
        counts = torch.bincount(own, minlength=self.world).tolist()
        rs, rcl = self._exchange(src[order].contiguous(), counts)
        rd, _ = self._exchange(dst[order].contiguous(), counts)
        return order, counts, rs, rd, rcl

    def _update(self, src, dst, segmented):
        """Insert or delete: this rank's {done, rejected} counts."""
        import torch
        order, counts, rs, rd, rcl = self._route(src, dst)
        offs = torch.zeros(self.world + 1, dtype=torch.int64)
        offs[1:] = torch.cumsum(torch.as_tensor(rcl, dtype=torch.int64), 0)
        res = segmented(rs, rd, offs)                        # [world, 2]: counts per origin rank
        back, _ = self._exchange(res.reshape(-1).contiguous(), [2] * self.world)
        back = back.view(self.world, 2).sum(0)               # over the owners of this rank's pairs
        return int(back[0]), int(back[1])

    # ----------------------------------------------------------------- calls
    def insert_edges(self, src, dst):
        return self._update(src, dst, self.shard.insert_segmented)

    def delete_edges(self, src, dst):
        return self._update(src, dst, self.shard.delete_segmented)

    def query_edges(self, src, dst):
        """Answers (uint8, 1 = stored) for this rank's pairs, in their order."""
        import torch
        order, counts, rs, rd, rcl = self._route(src, dst)
        ans = self.shard.query(rs, rd)
        back, _ = self._exchange(ans.contiguous(), rcl)      # answers return along the reverse route
        out = torch.empty_like(back)
        out[order] = back
        return out

    def insert_vertices(self, k):
        """Appends k vertices for this rank (every rank may ask for its own
        count); returns the new ids, after those of the lower ranks."""
        import torch
        dist = _dist()
        ks = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        dist.all_gather(ks, torch.tensor([int(k)], dtype=torch.int64, device=self.device), group=self.group)
        ks = [int(x.item()) for x in ks]
        base = self.shard.num_vertices
        self.shard.insert_vertices(sum(ks))
        first = base + sum(ks[:self.rank])
        return np.arange(first, first + int(k), dtype=np.uint32)

    def delete_vertices(self, ids):
        """Deletes the union of every rank's ids on every shard."""
        import torch
        dist = _dist()
        n = torch.tensor([int(ids.numel())], dtype=torch.int64, device=self.device)
        ns = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        dist.all_gather(ns, n, group=self.group)
        ns = [int(x.item()) for x in ns]
        m = max(ns) if ns else 0
        if m == 0:
            return
        pad = torch.zeros(m, dtype=ids.dtype, device=self.device)
        pad[:ids.numel()] = ids
        parts = [torch.empty(m, dtype=ids.dtype, device=self.device) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        every = torch.cat([p[:c] for p, c in zip(parts, ns)])
        self.shard.delete_vertices(every)

    def degrees(self):
        """Out-degree of every vertex (each shard holds its owned sources)."""
        import torch
        dist = _dist()
        d = torch.as_tensor(self.shard.degrees().astype(np.int64), device=self.device)
        dist.all_reduce(d, group=self.group)
        return d.cpu().numpy().astype(np.uint32)

    def export_csr(self):
        """The whole graph as CSR (every rank gets it): vertex u's entries
        from its owner's shard."""
        dist = _dist()
        off, nb = self.shard.export_csr()
        parts = [None] * self.world
        dist.all_gather_object(parts, (np.asarray(off, np.uint64), np.asarray(nb, np.uint32)), group=self.group)
        nv = parts[0][0].size - 1
        deg = np.zeros(nv, dtype=np.int64)
        start = np.zeros(nv, dtype=np.int64)  # position of u's entries in the concatenated shards
        base = 0
        for r, (o, b) in enumerate(parts):
            o = o.astype(np.int64)
            deg[r::self.world] = np.diff(o)[r::self.world]
            start[r::self.world] = base + o[:-1][r::self.world]
            base += b.size
        out_off = np.zeros(nv + 1, dtype=np.uint64)
        out_off[1:] = np.cumsum(deg)
        every = np.concatenate([b for _, b in parts]) if parts else np.zeros(0, np.uint32)
        total = int(out_off[-1])
        idx = np.repeat(start - out_off[:-1].astype(np.int64), deg) + np.arange(total, dtype=np.int64)
        return out_off, every[idx].astype(np.uint32)

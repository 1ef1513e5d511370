"""GPU path vs the CPU oracle, bit-exact, after every call (integer results).

Inputs come from the seeded generators in `workloads`; the oracle and the
GPU library see the same arrays.  Sizes span many work items, multi-item
hub adjacencies and ragged tails; the full-size RMAT workload is checked on
every degree, every query bit and sampled neighbour lists.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import Pair, canon, dev_u32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("radix", [False, True])
def test_tiny_uniform_config_every_batch(radix):
    import paper_2306_08252_gb300 as gv
    cfg = W.tiny_uniform()
    p = Pair(cfg["nv"], C=cfg["block_capacity"], pool_bytes=32 << 20, flags=gv.GV_RADIX_GROUPING if radix else 0)
    try:
        p.bulk(*cfg["bulk"])
        p.check()
        for op in cfg["ops"]:
            if op.kind == "insert":
                p.insert(op.src, op.dst)
            else:
                p.delete(op.src, op.dst)
            p.check()
    finally:
        p.close()


def test_rule_capacity_above_512():
    """The paper's C rule on a first batch whose mean non-zero degree is past
    512: both sides take the largest block (512 slots); then a second batch,
    a delete spanning several blocks per source and the full CSR."""
    import oracle
    nv = 256
    rng = np.random.default_rng(5)
    srcs = np.repeat(np.arange(0, nv, 4, dtype=np.uint32), 700)  # 64 sources, 700 entries each
    dsts = rng.integers(0, nv, srcs.size).astype(np.uint32)
    p = Pair(nv, C=0, pool_bytes=32 << 20)
    try:
        p.bulk(srcs, dsts)
        st = p.check()
        rule = oracle.block_capacity_rule(np.bincount(srcs, minlength=nv))
        assert rule == 512
        assert st["block_capacity"] == rule
        s2 = rng.integers(0, nv, 5000).astype(np.uint32)
        d2 = rng.integers(0, nv, 5000).astype(np.uint32)
        p.insert(s2, d2)
        p.check()
        p.delete(np.concatenate([srcs[::3], s2[:100]]), np.concatenate([dsts[::3], d2[:100]]))
        p.check()
        p.query(srcs[::5], dsts[::5])
    finally:
        p.close()


@pytest.mark.parametrize("C", [4, 8, 16, 20, 64, 0])
def test_rmat_skewed_batches(C):
    scale, nv = 12, 1 << 12
    bs, bd = W.rmat_pairs(21, 0, 65536, scale)
    p = Pair(nv, C=C, pool_bytes=64 << 20)
    try:
        p.bulk(bs, bd)
        st = p.check()
        if C == 0:
            import oracle
            assert st["block_capacity"] == oracle.block_capacity_rule(np.bincount(bs, minlength=nv))
        for r, b in enumerate([1, 37, 5000, 20000]):
            s, d = W.rmat_pairs(21, 100 + r, b, scale)
            p.insert(s, d)
            p.check()
            qs, qd = W.rmat_queries(21, scale, 4000, s, d, r)
            p.query(qs, qd)
            # delete the batch, some base edges and some absent pairs
            es = bs[r * 1000:(r + 1) * 1000]
            ed = bd[r * 1000:(r + 1) * 1000]
            as_, ad = W.absent_pairs(21, 300 + r, 500, nv, W.keys(np.concatenate([bs, s]), np.concatenate([bd, d])))
            p.delete(np.concatenate([s, es, as_]), np.concatenate([d, ed, ad]))
            p.check()
            p.query(qs, qd)
    finally:
        p.close()


def test_hub_deletes_across_many_items():
    # one vertex with a long adjacency (hundreds of work items), deleted in
    # scattered pieces, including every copy of duplicated pairs
    nv = 3000
    rng = np.random.default_rng(5)
    hub_d = rng.integers(0, nv, 200_000).astype(np.uint32)
    hub_s = np.zeros_like(hub_d)
    other_s = rng.integers(1, nv, 50_000).astype(np.uint32)
    other_d = rng.integers(0, nv, 50_000).astype(np.uint32)
    p = Pair(nv, C=16, pool_bytes=64 << 20)
    try:
        p.bulk(np.concatenate([hub_s, other_s]), np.concatenate([hub_d, other_d]))
        p.check()
        for frac in (0.01, 0.3, 0.9):
            k = int(nv * frac)
            dd = rng.choice(nv, size=k, replace=False).astype(np.uint32)
            p.delete(np.zeros(k, dtype=np.uint32), dd)
            p.check()
            p.insert(np.zeros(777, dtype=np.uint32), rng.integers(0, nv, 777).astype(np.uint32))
            p.check()
        # delete everything of the hub
        p.delete(np.zeros(nv, dtype=np.uint32), np.arange(nv, dtype=np.uint32))
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_hub_batch_lists_past_one_shared_slice(weighted):
    """Sources with more batch entries than one shared-memory slice of the
    block-wide membership tier (several slices per group of work items), a
    single-item source with more than 256 batch entries (compacted in place
    by that tier), queries with repeats; plain and weighted graphs."""
    import paper_2306_08252_gb300 as gv
    nv = 20000
    rng = np.random.default_rng(11)
    hub_d = rng.integers(0, nv, 300_000).astype(np.uint32)
    small_d = rng.integers(0, nv, 400).astype(np.uint32)  # source 7: one work item at C = 16
    other_s = rng.integers(8, nv, 60_000).astype(np.uint32)
    other_d = rng.integers(0, nv, 60_000).astype(np.uint32)
    bs = np.concatenate([np.zeros(hub_d.size, np.uint32), np.full(400, 7, np.uint32), other_s])
    bd = np.concatenate([hub_d, small_d, other_d])
    p = Pair(nv, C=16, pool_bytes=96 << 20, flags=(gv.GV_WEIGHTED if weighted else 0) | gv.GV_RADIX_GROUPING)
    try:
        p.bulk(bs, bd)
        p.check()
        # queries: 12,000 on the hub (present and absent, repeated), 300 on source 7
        qd = np.concatenate([hub_d[:6000], rng.integers(0, nv, 6000).astype(np.uint32), small_d[:150],
                             rng.integers(0, nv, 150).astype(np.uint32)])
        qs = np.concatenate([np.zeros(12000, np.uint32), np.full(300, 7, np.uint32)])
        p.query(qs, qd)
        # deletes: 11,000 distinct destinations on the hub (three slices), 300
        # on source 7 (half present), plus scattered other pairs
        dh = rng.choice(nv, size=11000, replace=False).astype(np.uint32)
        d7 = np.concatenate([small_d[:150], rng.integers(0, nv, 150).astype(np.uint32)])
        ds = np.concatenate([np.zeros(dh.size, np.uint32), np.full(300, 7, np.uint32), other_s[:5000]])
        dd = np.concatenate([dh, d7, other_d[:5000]])
        p.delete(ds, dd)
        p.check()
        p.query(qs, qd)
        p.insert(np.zeros(5000, np.uint32), rng.integers(0, nv, 5000).astype(np.uint32))
        p.delete(np.zeros(dh.size, np.uint32), dh)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("C", [4, 16, 0])
def test_rmat_batches_radix_grouping(C):
    """Large batches through the radix-partition grouping (GV_RADIX_GROUPING)
    give the oracle's results, like the per-pair atomic grouping."""
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    bs, bd = W.rmat_pairs(22, 0, 65536, scale)
    p = Pair(nv, C=C, pool_bytes=64 << 20, flags=gv.GV_RADIX_GROUPING)
    try:
        p.bulk(bs, bd)
        p.check()
        for r, b in enumerate([5000, 20000]):
            s, d = W.rmat_pairs(22, 100 + r, b, scale)
            p.insert(s, d)
            p.check()
            qs, qd = W.rmat_queries(22, scale, 4000, s, d, r)
            p.query(qs, qd)
            p.delete(np.concatenate([s, bs[:1000]]), np.concatenate([d, bd[:1000]]))
            p.check()
    finally:
        p.close()


def test_queries_with_invalid_and_dead_ids():
    nv = 2000
    bs, bd = W.uniform_pairs(9, 0, 30000, nv)
    p = Pair(nv, C=8)
    try:
        p.bulk(bs, bd)
        p.vdel(np.array([5, 6, 7], dtype=np.uint32))
        qs = np.concatenate([bs[:3000], np.array([5, 1, nv, nv + 7, 0xFFFFFFFE], dtype=np.uint32)])
        qd = np.concatenate([bd[:3000], np.array([1, 6, 1, 0, 3], dtype=np.uint32)])
        p.query(qs, qd)
        p.check()
    finally:
        p.close()


def test_vertex_insert_and_delete():
    nv = 5000
    bs, bd = W.uniform_pairs(11, 0, 40000, nv)
    # a few heavy vertices so that incoming-edge removal spans multi-item adjacencies
    hs = np.repeat(np.arange(4, dtype=np.uint32), 3000)
    hd = W.uniform_u32(11, 1, hs.size, 0, nv)
    p = Pair(nv, C=16)
    try:
        p.bulk(np.concatenate([bs, hs]), np.concatenate([bd, hd]))
        p.check()
        ids = W.shuffled(11, 2, np.arange(nv, dtype=np.uint32))[:300]
        ids = np.concatenate([ids, ids[:10], np.array([nv + 3, 0xFFFFFFFF], dtype=np.uint32)])
        p.vdel(ids)
        p.check()
        p.vdel(ids[:50])  # already dead: no-op
        p.check()
        p.vins(4000)  # crosses the dictionary capacity (8192 -> 16384)
        p.check()
        new = np.arange(nv, nv + 4000, dtype=np.uint32)
        s = np.repeat(new, 8)
        d = W.uniform_u32(11, 3, s.size, 0, nv + 4000)
        p.insert(s, d)  # some endpoints are dead: rejected
        p.check()
        p.vdel(np.concatenate([new[:100], np.arange(4, dtype=np.uint32)]))
        p.check()
        p.insert(bs[:5000], bd[:5000])
        p.check()
    finally:
        p.close()


def test_empty_degenerate_and_duplicates():
    nv = 64
    p = Pair(nv, C=4, pool_bytes=1 << 20)
    e = np.zeros(0, dtype=np.uint32)
    try:
        p.insert(e, e)
        p.delete(e, e)
        p.query(e, e)
        p.check()
        # all-invalid batches
        bad = np.array([64, 65, 1000], dtype=np.uint32)
        p.insert(bad, np.array([0, 1, 2], dtype=np.uint32))
        p.delete(bad, np.array([0, 1, 2], dtype=np.uint32))
        p.check()
        # self loops and duplicates (multiset)
        s = np.array([1, 1, 1, 2, 2, 3] * 5, dtype=np.uint32)
        d = np.array([1, 1, 2, 2, 3, 3] * 5, dtype=np.uint32)
        p.insert(s, d)
        p.check()
        p.delete(np.array([1, 1], dtype=np.uint32), np.array([1, 1], dtype=np.uint32))
        p.check()
        # delete absent pairs: no-op
        p.delete(np.array([5, 6], dtype=np.uint32), np.array([7, 8], dtype=np.uint32))
        p.check()
        # delete every edge, then rebuild: pool accounting returns to zero
        s2, d2 = W.uniform_pairs(3, 0, 3000, nv)
        p.insert(s2, d2)
        p.check()
        p.delete(np.repeat(np.arange(nv, dtype=np.uint32), nv), np.tile(np.arange(nv, dtype=np.uint32), nv))
        st = p.check()
        assert st["num_edges"] == 0 and st["pool_blocks_used"] == 0
        p.insert(s2, d2)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("big", [5000, 1500])  # the general path and the one-CTA small-batch path
def test_pool_exhaustion_is_a_noop(big):
    import paper_2306_08252_gb300 as gv
    nv = 256
    # pool of ~200 blocks of C=4
    p = Pair(nv, C=4, pool_bytes=200 * (16 + 12) + 1024)
    try:
        s, d = W.uniform_pairs(4, 0, 300, nv)
        p.insert(s, d)
        p.check()
        before = p.g.export_csr()
        s2, d2 = W.uniform_pairs(4, 1, big, nv)
        p.g.insert_edges(dev_u32(s2), dev_u32(d2), p.counts)
        assert p.g.__class__  # call returns; error is latched on the device
        code = gv.gv_sync(p.g.handle)
        assert code == gv.GV_ERR_OUT_OF_MEMORY
        assert tuple(p.counts.cpu().tolist()) == (0, 0)
        after = p.g.export_csr()
        np.testing.assert_array_equal(before[0], after[0])
        np.testing.assert_array_equal(canon(*before), canon(*after))
        p.check()  # status cleared; still equal to the oracle (which skipped the batch)
        p.insert(s[:50], d[:50])
        p.check()
    finally:
        p.close()


def test_host_pointer_inputs_match_device_inputs():
    import torch
    import paper_2306_08252_gb300 as gv
    nv = 4096
    bs, bd = W.rmat_pairs(12, 0, 50000, 12)
    a = gv.Graph(nv, block_capacity=16, pool_bytes=32 << 20)
    b = gv.Graph(nv, block_capacity=16, pool_bytes=32 << 20)
    try:
        ca = np.zeros(2, dtype=np.uint64)
        a.bulk_build(bs, bd, ca)              # numpy (pageable host) arrays
        b.bulk_build(dev_u32(bs), dev_u32(bd))
        assert tuple(ca) == (50000, 0)
        pin_s = torch.from_numpy(bs[:9000].view(np.int32)).pin_memory()
        pin_d = torch.from_numpy(bd[:9000].view(np.int32)).pin_memory()
        a.delete_edges(pin_s, pin_d, ca)      # pinned host arrays
        b.delete_edges(dev_u32(bs[:9000]), dev_u32(bd[:9000]))
        out_h = np.zeros(20000, dtype=np.uint8)
        a.query_edges(bs[:20000], bd[:20000], out_h)
        out_d = torch.zeros(20000, dtype=torch.uint8, device="cuda")
        b.query_edges(dev_u32(bs[:20000]), dev_u32(bd[:20000]), out_d)
        np.testing.assert_array_equal(out_h, out_d.cpu().numpy())
        np.testing.assert_array_equal(canon(*a.export_csr()), canon(*b.export_csr()))
    finally:
        a.close()
        b.close()


def test_neighbors_subset_and_capacity_error():
    import paper_2306_08252_gb300 as gv
    nv = 3000
    bs, bd = W.rmat_pairs(13, 0, 40000, 12, limit=nv)
    p = Pair(nv, C=12)
    try:
        p.bulk(bs, bd)
        vids = np.array([0, 1, 2, 2999, 3000, 0xFFFFFFF0, 17, 0], dtype=np.uint32)
        p.check_sampled(vids)
        off = np.zeros(vids.size + 1, dtype=np.uint64)
        small = np.zeros(3, dtype=np.uint32)
        code, total = gv.gv_neighbors(p.g.handle, vids, off, small, small.size)
        assert code == gv.GV_ERR_INVALID_ARG and total == int(p.o.neighbors(vids)[0][-1])
    finally:
        p.close()


def test_er_mixed_scaled():
    cfg = W.er_mixed(seed=3, nv=1 << 16, base_edges=1 << 18, rounds=2, batch=20000, vdel=2048,
                     vins=2048, vins_edges=8)
    p = Pair(cfg["nv"], C=4, pool_bytes=64 << 20)
    try:
        p.bulk(*cfg["bulk"])
        p.check()
        for op in cfg["ops"]:
            if op.kind == "insert":
                p.insert(op.src, op.dst)
            elif op.kind == "delete":
                p.delete(op.src, op.dst)
            elif op.kind == "vdel":
                p.vdel(op.ids)
            else:
                p.vins(op.k)
            p.check()
    finally:
        p.close()


@pytest.mark.parametrize("radix", [False, True])
def test_rmat_full_size_sampled(radix):
    """RMAT 2^20 vertices, 16M edges, the 10M insert / 1M query / 10M delete
    step in the benchmark's launch configuration (and through the radix-
    partition grouping); every degree and query bit, sampled neighbour lists
    (top hubs and random vertices)."""
    import paper_2306_08252_gb300 as gv
    scale = 20
    bs, bd = W.rmat_graph(2, scale, 1 << 24)
    p = Pair(1 << scale, C=16, pool_bytes=1 << 30, flags=gv.GV_RADIX_GROUPING if radix else 0)
    try:
        p.bulk(bs, bd)
        p.check(full=False)
        s, d = W.rmat_update(2, scale, 10_000_000, 0)
        p.insert(s, d)
        p.check(full=False)
        qs, qd = W.rmat_queries(2, scale, 1_000_000, s, d, 0)
        p.query(qs, qd)
        p.delete(s, d)
        p.check(full=False)
        deg = p.o.degrees()
        hubs = np.argsort(deg)[-64:].astype(np.uint32)
        rnd = W.uniform_u32(2, 77, 4000, 0, 1 << scale)
        p.check_sampled(np.concatenate([hubs, rnd]))
        # a second step from the steady state
        p.insert(s, d)
        p.delete(s, d)
        p.check(full=False)
        p.check_sampled(np.concatenate([hubs, rnd]))
    finally:
        p.close()


@pytest.mark.parametrize("C", [4, 16, 0])
def test_set_semantics_inserts(C):
    # GV_DEDUP: a pair is added only when it is not stored and not already
    # added by the same batch; duplicates within a batch, against the graph,
    # hub sources with many work items, invalid ids and deletes in between
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    rng = np.random.default_rng(31)
    bs, bd = W.rmat_pairs(23, 0, 60000, scale)
    # repeat a slice of the bulk batch inside the batch itself
    bs = np.concatenate([bs, bs[:5000]])
    bd = np.concatenate([bd, bd[:5000]])
    p = Pair(nv, C=C, pool_bytes=64 << 20, flags=gv.GV_DEDUP)
    try:
        p.bulk(bs, bd)
        p.check()
        for r, b in enumerate([1, 50, 3000, 40000]):
            s, d = W.rmat_pairs(23, 10 + r, b, scale)
            # a third of the batch repeats stored edges, some pairs twice
            k = b // 3
            pick = rng.integers(0, bs.size, k)
            s = np.concatenate([s, bs[pick], s[: b // 4]])
            d = np.concatenate([d, bd[pick], d[: b // 4]])
            if r == 2:
                s = np.concatenate([s, np.array([nv, 5, 0xFFFFFFFF], dtype=np.uint32)])
                d = np.concatenate([d, np.array([1, nv + 3, 2], dtype=np.uint32)])
            perm = rng.permutation(s.size)
            p.insert(s[perm], d[perm])
            p.check()
            # the same batch again adds nothing
            p.insert(s, d)
            p.check()
            es, ed = bs[r * 2000:(r + 1) * 2000], bd[r * 2000:(r + 1) * 2000]
            p.delete(es, ed)
            p.check()
        # one hub source: a long adjacency, a batch that mixes stored and new
        hub_d = rng.integers(0, nv, 30000).astype(np.uint32)
        p.insert(np.zeros(hub_d.size, dtype=np.uint32), hub_d)
        p.check()
        hub_d2 = rng.integers(0, nv, 30000).astype(np.uint32)
        p.insert(np.zeros(hub_d2.size, dtype=np.uint32), hub_d2)
        p.check()
        p.insert(np.zeros(0, dtype=np.uint32), np.zeros(0, dtype=np.uint32))
        p.check()
    finally:
        p.close()


def test_pool_growth_policy():
    # GV_GROW: a pool of ~2K blocks grows by 25% steps ahead of inserts that
    # would take it past 80%; block ids survive the move (parity and the
    # structural self-check after every call), deletes return blocks to the
    # grown queue
    import paper_2306_08252_gb300 as gv
    scale, nv = 12, 1 << 12
    C = 8
    per_block = 4 * C + 12
    p = Pair(nv, C=C, pool_bytes=2048 * per_block + 4096, flags=gv.GV_GROW)
    try:
        st0 = p.g.stats()
        bs, bd = W.rmat_pairs(29, 0, 4000, scale)
        p.bulk(bs, bd)
        p.check()
        sizes = []
        for r, b in enumerate([3000, 20000, 70000, 5, 150000]):
            s, d = W.rmat_pairs(29, 1 + r, b, scale)
            p.insert(s, d)
            st = p.check()
            assert p.g.sync() == 0  # no exhaustion latched
            assert 5 * st["pool_blocks_used"] <= 4 * st["pool_blocks"]
            sizes.append(st["pool_blocks"])
            if r % 2:
                p.delete(s[: b // 2], d[: b // 2])
                p.check()
        assert sizes[-1] > st0["pool_blocks"] * 10
        assert all(b2 >= b1 for b1, b2 in zip(sizes, sizes[1:]))
    finally:
        p.close()


def test_pool_growth_rejects_caller_owned_pool():
    import torch
    import paper_2306_08252_gb300 as gv
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(gv.GraphVineError):
        gv.Graph(1024, block_capacity=16, pool_bytes=buf.numel(), pool_mem=buf, flags=gv.GV_GROW)


@pytest.mark.parametrize("pinned", [True, False])
def test_large_host_batches_staged_in_pieces(pinned):
    # host arrays of >= 2^20 pairs are staged in pieces, each counted as it
    # lands: results equal the oracle's, for inserts, queries and deletes
    # (pinned and pageable host memory)
    import torch
    scale, nv = 16, 1 << 16
    bs, bd = W.rmat_pairs(91, 0, 200_000, scale)
    s, d = W.rmat_pairs(91, 1, (1 << 20) + 12345, scale)
    p = Pair(nv, C=8, pool_bytes=256 << 20)
    try:
        p.bulk(bs, bd)
        host = (lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()) if pinned \
            else (lambda a: np.ascontiguousarray(a, dtype=np.uint32))
        hs, hd = host(s), host(d)
        cnt = np.zeros(2, dtype=np.uint64)
        p.g.insert_edges(hs, hd, cnt)
        assert tuple(int(x) for x in cnt) == p.o.insert_edges(s, d)
        p.check(full=False)
        out = np.zeros(s.size, dtype=np.uint8)
        p.g.query_edges(hs, hd, out)
        np.testing.assert_array_equal(out, p.o.query_edges(s, d))
        ks = np.concatenate([s[: s.size // 2 + 7], bs[:10]])
        kd = np.concatenate([d[: d.size // 2 + 7], bd[:10]])
        p.g.delete_edges(host(ks), host(kd), cnt)
        assert tuple(int(x) for x in cnt) == p.o.delete_edges(ks, kd)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_host_batches_in_flight_stream_order(weighted):
    # host-array calls issued back to back without a synchronisation: their
    # copies run on the library's copy stream into rotating staging sets
    # while earlier calls compute; page-locked outputs land in stream order.
    # Seven calls cycle through the sets twice (a set is refilled only after
    # the call that read it); one pinned input pair is reused by an insert
    # and a later delete; large batches take the piecewise path.
    import torch
    import paper_2306_08252_gb300 as gv
    scale, nv = 14, 1 << 14
    flags = gv.GV_WEIGHTED if weighted else 0
    p = Pair(nv, C=8, pool_bytes=256 << 20, flags=flags)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    try:
        bs, bd = W.rmat_pairs(77, 0, 100_000, scale)
        p.bulk(bs, bd)
        a_s, a_d = W.rmat_pairs(77, 1, (1 << 20) + 999, scale)     # piecewise staging
        b_s, b_d = W.rmat_pairs(77, 2, 30_000, scale)
        q_s = np.concatenate([a_s[:50_000], b_s[:10_000]])
        q_d = np.concatenate([a_d[:50_000], b_d[:10_000]])
        rng = np.random.default_rng(77)
        a_w = rng.integers(0, 1 << 32, a_s.size, dtype=np.uint64).astype(np.uint32)
        ha_s, ha_d, hb_s, hb_d = pin(a_s), pin(a_d), pin(b_s), pin(b_d)
        hq_s, hq_d, ha_w = pin(q_s), pin(q_d), pin(a_w)
        cnts = [torch.zeros(2, dtype=torch.int64).pin_memory() for _ in range(5)]
        outs = [torch.zeros(q_s.size, dtype=torch.uint8).pin_memory() for _ in range(2)]
        g = p.g
        if weighted:
            g.insert_edges_weighted(ha_s, ha_d, ha_w, cnts[0])
        else:
            g.insert_edges(ha_s, ha_d, cnts[0])
        g.query_edges(hq_s, hq_d, outs[0])
        g.insert_edges(hb_s, hb_d, cnts[1])
        g.delete_edges(ha_s, ha_d, cnts[2])                          # reuses the first call's pinned input
        g.query_edges(hq_s, hq_d, outs[1])
        g.delete_edges(hb_s[:7_000], hb_d[:7_000], cnts[3])
        g.insert_edges(ha_s[:5_000], ha_d[:5_000], cnts[4])
        torch.cuda.synchronize()
        o = p.o
        exp0 = o.insert_edges_weighted(a_s, a_d, a_w) if weighted else o.insert_edges(a_s, a_d)
        expq0 = o.query_edges(q_s, q_d)
        exp1 = o.insert_edges(b_s, b_d)
        exp2 = o.delete_edges(a_s, a_d)
        expq1 = o.query_edges(q_s, q_d)
        exp3 = o.delete_edges(b_s[:7_000], b_d[:7_000])
        exp4 = o.insert_edges(a_s[:5_000], a_d[:5_000])
        got = [tuple(int(x) for x in c.tolist()) for c in cnts]
        assert got == [exp0, exp1, exp2, exp3, exp4]
        np.testing.assert_array_equal(outs[0].numpy(), expq0)
        np.testing.assert_array_equal(outs[1].numpy(), expq1)
        p.check()
        if weighted:
            vids = np.arange(nv, dtype=np.uint32)
            off, nb, wt = g.neighbors_weighted(vids)
            ooff, onb, owt = o.neighbors_weighted(vids)
            np.testing.assert_array_equal(off, ooff)
            seg = np.repeat(np.arange(nv), np.diff(off.astype(np.int64)))
            order = np.lexsort((wt, nb, seg))
            np.testing.assert_array_equal(nb[order], onb)
            np.testing.assert_array_equal(wt[order], owt)
    finally:
        p.close()



@pytest.mark.parametrize("C", [4, 12, 64])
def test_small_insert_path_matches_general_path(C):
    # batches of at most 2,048 pairs take the one-CTA insert; sizes around
    # that bound, skewed sources (one source with more pairs than a block
    # and a new tree), invalid and dead ids, weighted and plain
    import paper_2306_08252_gb300 as gv
    rng = np.random.default_rng(40 + C)
    nv = 3000
    for flags in (0, gv.GV_WEIGHTED):
        p = Pair(nv, C=C, pool_bytes=64 << 20, flags=flags)
        try:
            bs, bd = W.rmat_pairs(40 + C, 0, 20000, 11)
            p.bulk(bs, bd)
            p.vdel(np.array([3, 7, 2999], dtype=np.uint32))
            for n in (1, 2, 31, 700, 2047, 2048, 2049, 4000):
                s = rng.integers(0, nv + 3, n).astype(np.uint32)
                d = rng.integers(0, nv + 3, n).astype(np.uint32)
                s[: n // 3] = 1                      # a hub of this batch
                s[n // 3: n // 3 + n // 10] = 2500  # a source with few or no blocks yet
                if flags:
                    import torch
                    w = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
                    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
                    p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
                    assert tuple(int(x) for x in cnt.cpu().tolist()) == p.o.insert_edges_weighted(s, d, w)
                else:
                    p.insert(s, d)
                p.check()
            if flags:
                vids = np.arange(nv, dtype=np.uint32)
                off, nb, wt = p.g.neighbors_weighted(vids)
                ooff, onb, owt = p.o.neighbors_weighted(vids)
                np.testing.assert_array_equal(off, ooff)
                seg = np.repeat(np.arange(nv), np.diff(off.astype(np.int64)))
                order = np.lexsort((wt, nb, seg))
                np.testing.assert_array_equal(nb[order], onb)
                np.testing.assert_array_equal(wt[order], owt)
        finally:
            p.close()

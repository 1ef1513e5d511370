"""Random operation sequences on the GPU against the oracle, checked after
every call: edge inserts (multiset and set semantics, weighted), deletes,
segmented deletes, queries, vertex inserts and deletes, pool growth, BFS,
shortest paths, edge-block resizes, for several block capacities and graph
sizes.  Seeded; every case is reproducible."""
import numpy as np
import pytest

from gpu_util import Pair, blocks_owned, dev_u32

pytestmark = pytest.mark.gpu


def _pairs(rng, n, nv, hub_frac=0.3):
    s = rng.integers(0, nv, n).astype(np.uint32)
    hub = rng.random(n) < hub_frac
    s[hub] = rng.integers(0, max(1, nv // 50), hub.sum()).astype(np.uint32)  # skewed sources
    d = rng.integers(0, nv, n).astype(np.uint32)
    bad = rng.random(n) < 0.01
    s[bad] = nv + rng.integers(0, 5, bad.sum()).astype(np.uint32)  # a few out-of-range ids
    return s, d


# flags: 1 set semantics, 2 pool growth, 4 weighted, 8 radix-partition
# grouping; 16 (this test's own bit) hub runs with a random run size and
# threshold
@pytest.mark.parametrize("seed,C,flags", [(1, 4, 0), (2, 8, 0), (3, 16, 1), (4, 12, 2), (5, 32, 3), (6, 0, 0),
                                          (7, 8, 4), (8, 20, 6), (9, 16, 8), (10, 4, 12), (11, 0, 10),
                                          (12, 4, 16), (13, 16, 20), (14, 0, 17), (15, 8, 16), (16, 8, 18)])
def test_random_operation_sequences(seed, C, flags):
    import torch
    import paper_2306_08252_gb300 as gv
    rng = np.random.default_rng(1000 + seed)
    nv = int(rng.integers(300, 3000))
    hubs = bool(flags & 16)
    flags &= 15
    pool = (8 << 20) if flags & gv.GV_GROW else (64 << 20)
    hub_kw = dict(hub_shift=int(rng.integers(3, 7)), hub_degree=int(rng.choice([0, 1, 20, 100]))) if hubs else {}
    p = Pair(nv, C=C, pool_bytes=pool, flags=flags, **hub_kw)
    try:
        bs, bd = _pairs(rng, int(rng.integers(1, 20000)), nv)
        p.bulk(bs, bd)
        p.check()
        stored_s, stored_d = bs, bd
        for step in range(25):
            op = rng.choice(["insert", "delete", "query", "segdel", "vdel", "vins", "bfs", "sssp", "reblock"],
                            p=[0.28, 0.22, 0.13, 0.09, 0.06, 0.06, 0.05, 0.05, 0.06])
            n_now = p.o.num_vertices
            if op == "insert" and flags & gv.GV_WEIGHTED and rng.random() < 0.6:
                s, d = _pairs(rng, int(rng.integers(0, 15000)), n_now)
                w = rng.integers(0, 1 << 32, s.size, dtype=np.uint64).astype(np.uint32)
                cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
                before = p.o.degrees().astype(np.int64)
                p.g.insert_edges_weighted(dev_u32(s), dev_u32(d), dev_u32(w), cnt)
                assert tuple(int(x) for x in cnt.cpu().tolist()) == p.o.insert_edges_weighted(s, d, w)
                p._hub_update(before)
                stored_s, stored_d = np.concatenate([stored_s, s]), np.concatenate([stored_d, d])
            elif op == "insert":
                s, d = _pairs(rng, int(rng.integers(0, 15000)), n_now)
                if s.size and rng.random() < 0.5:  # repeat stored pairs
                    k = rng.integers(0, stored_s.size, s.size // 3)
                    s[:k.size], d[:k.size] = stored_s[k], stored_d[k]
                p.insert(s, d)
                stored_s, stored_d = np.concatenate([stored_s, s]), np.concatenate([stored_d, d])
            elif op == "delete":
                k = rng.integers(0, stored_s.size, int(rng.integers(0, 8000)))
                s, d = _pairs(rng, k.size // 4, n_now)
                p.delete(np.concatenate([stored_s[k], s]), np.concatenate([stored_d[k], d]))
            elif op == "query":
                k = rng.integers(0, stored_s.size, 3000)
                s, d = _pairs(rng, 3000, n_now)
                p.query(np.concatenate([stored_s[k], s]), np.concatenate([stored_d[k], d]))
            elif op == "segdel":
                segs = []
                for _ in range(int(rng.integers(1, 6))):
                    k = rng.integers(0, stored_s.size, int(rng.integers(0, 3000)))
                    segs.append((stored_s[k], stored_d[k]))
                off = np.zeros(len(segs) + 1, dtype=np.int64)
                off[1:] = np.cumsum([a.size for a, _ in segs])
                cnt = torch.zeros(2 * len(segs), dtype=torch.int64, device="cuda")
                before = p.o.degrees().astype(np.int64)
                gv.gv_delete_edges_segmented(p.g.handle, dev_u32(np.concatenate([a for a, _ in segs])),
                                             dev_u32(np.concatenate([b for _, b in segs])),
                                             torch.from_numpy(off).cuda(), len(segs), cnt)
                exp = [p.o.delete_edges(a, b) for a, b in segs]
                np.testing.assert_array_equal(cnt.cpu().numpy().reshape(-1, 2), np.array(exp))
                p._hub_update(before)
            elif op == "vdel":
                ids = rng.choice(n_now, int(rng.integers(1, 20)), replace=False).astype(np.uint32)
                p.vdel(ids)
            elif op == "vins":
                p.vins(int(rng.integers(0, 40)))
            elif op == "bfs":
                src = int(rng.integers(0, n_now))
                dist, lv = p.g.bfs(src)
                odist, olv = p.o.bfs(src)
                np.testing.assert_array_equal(dist[:n_now], odist)
                assert lv == olv
            elif op == "sssp":
                src = int(rng.integers(0, n_now))
                dist, _ = p.g.sssp(src)
                odist, _ = p.o.sssp(src, bool(flags & gv.GV_WEIGHTED))
                np.testing.assert_array_equal(dist[:n_now], odist)
            elif op == "reblock":
                before = p.g.stats()["block_capacity"]
                want = int(rng.choice([0, gv.GV_REBLOCK_MIN_FOOTPRINT, 4, 8, 12, 16, 24, 32, 64, 128]))
                try:
                    got = p.reblock(want)  # with hub runs: every vertex re-decided by degree
                except gv.GraphVineError as e:
                    # only a resize that does not fit the pool may fail; nothing changes
                    assert e.code == gv.GV_ERR_OUT_OF_MEMORY
                    got = before
                assert p.g.stats()["block_capacity"] == got
                assert p.g.stats()["pool_blocks_used"] == blocks_owned(p.o.degrees(), p.hub, got, p.rs)
            p.check()
    finally:
        p.close()

"""Pins of the oracle's weighted entries: a pure-Python multiset model of
(destination, weight) pairs per source, random operation sequences with
invalid and dead ids; payloads travel with their entries through deletes,
vertex deletes and compaction; unweighted inserts store payload 0."""
import collections

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("seed", range(10))
def test_weighted_matches_multiset_model(seed):
    rng = np.random.default_rng(500 + seed)
    nv = int(rng.integers(2, 40))
    o = oracle.OracleGraph(nv)
    model = collections.defaultdict(collections.Counter)
    alive = [True] * nv
    for _ in range(40):
        op = rng.choice(["ins", "insw", "del", "vdel", "vins"], p=[0.2, 0.35, 0.3, 0.08, 0.07])
        n = len(alive)
        if op in ("ins", "insw"):
            k = int(rng.integers(0, 30))
            s = rng.integers(0, n + 2, k).astype(np.uint32)
            d = rng.integers(0, n + 2, k).astype(np.uint32)
            w = rng.integers(0, 4, k).astype(np.uint32) if op == "insw" else np.zeros(k, dtype=np.uint32)
            got = o.insert_edges_weighted(s, d, w) if op == "insw" else o.insert_edges(s, d)
            ins = rej = 0
            for a, b, c in zip(s.tolist(), d.tolist(), w.tolist()):
                if a < n and b < n and alive[a] and alive[b]:
                    model[a][(b, c)] += 1
                    ins += 1
                else:
                    rej += 1
            assert got == (ins, rej)
        elif op == "del":
            k = int(rng.integers(0, 20))
            s = rng.integers(0, n + 2, k).astype(np.uint32)
            d = rng.integers(0, n + 2, k).astype(np.uint32)
            got = o.delete_edges(s, d)
            dset = collections.defaultdict(set)
            rej = 0
            for a, b in zip(s.tolist(), d.tolist()):
                if a < n and b < n and alive[a] and alive[b]:
                    dset[a].add(b)
                else:
                    rej += 1
            removed = 0
            for a, bs in dset.items():
                for key in list(model[a]):
                    if key[0] in bs:
                        removed += model[a].pop(key)
            assert got == (removed, rej)
        elif op == "vdel":
            ids = rng.choice(n, int(rng.integers(1, 3)), replace=False).astype(np.uint32)
            o.delete_vertices(ids)
            gone = {int(x) for x in ids if alive[int(x)]}
            for x in gone:
                alive[x] = False
                model[x].clear()
            for a in list(model):
                for key in list(model[a]):
                    if key[0] in gone:
                        del model[a][key]
        else:
            k = int(rng.integers(0, 3))
            o.insert_vertices(k)
            alive.extend([True] * k)
        vids = np.arange(len(alive), dtype=np.uint32)
        off, nb, wt = o.neighbors_weighted(vids)
        for u in range(len(alive)):
            exp = sorted(model[u].elements()) if alive[u] else []
            got = list(zip(nb[off[u]:off[u + 1]].tolist(), wt[off[u]:off[u + 1]].tolist()))
            assert got == exp, (u, got, exp)
        assert o.num_edges == sum(sum(model[u].values()) for u in range(len(alive)) if alive[u])
    o.close()

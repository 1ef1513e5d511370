"""Pins of the CPU oracle against things other than itself.

* A pure-Python brute force over a |V| x |V| count matrix (multiset) or 0/1
  matrix (set semantics) on tiny graphs, over many random operation sequences
  that mix inserts, deletes, queries, vertex inserts and vertex deletes with
  out-of-range and dead ids.  The matrix is the plain definition of the
  multigraph the paper's structure stores; every output is compared.
* Invariants the paper's semantics fix: degree sum equals the edge count,
  query agrees with neighbour membership, insert-then-delete leaves none of
  the batch, deleting absent pairs changes nothing, a vertex delete leaves no
  incident edge, results do not depend on batch order or on splitting a
  batch in two, set-semantics inserts are idempotent.
* The paper's worked examples (tests/golden/paper_examples.json) and closed
  forms for the structural sizing rules.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


class BruteGraph:
    """Count-matrix model of a directed multigraph (definition, no cleverness)."""

    def __init__(self, nv, dedup=False):
        self.nv = nv
        self.dedup = dedup
        self.alive = [True] * nv
        self.M = {}  # (u, v) -> multiplicity

    def _valid(self, u, v):
        return u < self.nv and v < self.nv and self.alive[u] and self.alive[v]

    def insert(self, src, dst):
        ins = rej = 0
        for u, v in zip(src, dst):
            if not self._valid(u, v):
                rej += 1
                continue
            if self.dedup and self.M.get((u, v), 0) > 0:
                continue
            self.M[(u, v)] = self.M.get((u, v), 0) + 1
            ins += 1
        return ins, rej

    def delete(self, src, dst):
        rej = 0
        targets = set()
        for u, v in zip(src, dst):
            if not self._valid(u, v):
                rej += 1
                continue
            targets.add((u, v))
        dele = 0
        for key in targets:
            dele += self.M.pop(key, 0)
        return dele, rej

    def query(self, src, dst):
        return [1 if self._valid(u, v) and self.M.get((u, v), 0) > 0 else 0 for u, v in zip(src, dst)]

    def add_vertices(self, k):
        ids = list(range(self.nv, self.nv + k))
        self.nv += k
        self.alive += [True] * k
        return ids

    def del_vertices(self, ids):
        gone = {s for s in ids if s < self.nv and self.alive[s]}
        for s in gone:
            self.alive[s] = False
        for key in list(self.M):
            if key[0] in gone or key[1] in gone:
                del self.M[key]
        return len(gone)

    def csr(self):
        off = [0]
        nb = []
        for u in range(self.nv):
            row = sorted((v, c) for (uu, v), c in self.M.items() if uu == u)
            for v, c in row:
                nb += [v] * c
            off.append(len(nb))
        return np.array(off, dtype=np.uint64), np.array(nb, dtype=np.uint32)

    def degrees(self):
        d = [0] * self.nv
        for (u, _), c in self.M.items():
            d[u] += c
        return np.array(d, dtype=np.uint32)


def _compare(o, b):
    assert o.num_vertices == b.nv
    assert o.num_edges == sum(b.M.values())
    np.testing.assert_array_equal(o.degrees(), b.degrees())
    np.testing.assert_array_equal(o.alive(), np.array(b.alive, dtype=np.uint8))
    off, nb = o.export_csr()
    boff, bnb = b.csr()
    np.testing.assert_array_equal(off, boff)
    np.testing.assert_array_equal(nb, bnb)


def _random_pairs(rng, n, hi):
    return [rng.randrange(hi) for _ in range(n)], [rng.randrange(hi) for _ in range(n)]


@pytest.mark.parametrize("dedup", [False, True])
@pytest.mark.parametrize("seed", range(40))
def test_oracle_matches_bruteforce_matrix(seed, dedup):
    rng = random.Random(seed * 7919 + dedup)
    nv = rng.randrange(1, 40)
    o = oracle.OracleGraph(nv, oracle.DEDUP if dedup else 0)
    b = BruteGraph(nv, dedup)
    for step in range(30):
        op = rng.random()
        hi = o.num_vertices + 3  # a few out-of-range ids
        if op < 0.35:
            s, d = _random_pairs(rng, rng.randrange(0, 60), hi)
            assert o.insert_edges(s, d) == b.insert(s, d)
        elif op < 0.6:
            s, d = _random_pairs(rng, rng.randrange(0, 40), hi)
            # bias toward pairs that exist
            keys = list(b.M)
            for _ in range(rng.randrange(0, 10)):
                if keys:
                    u, v = rng.choice(keys)
                    s.append(u)
                    d.append(v)
            assert o.delete_edges(s, d) == b.delete(s, d)
        elif op < 0.8:
            s, d = _random_pairs(rng, rng.randrange(0, 50), hi)
            keys = list(b.M)
            for _ in range(5):
                if keys:
                    u, v = rng.choice(keys)
                    s.append(u)
                    d.append(v)
            np.testing.assert_array_equal(o.query_edges(s, d), np.array(b.query(s, d), dtype=np.uint8))
        elif op < 0.9:
            k = rng.randrange(0, 5)
            ids = o.insert_vertices(k)
            assert list(ids) == b.add_vertices(k)
        else:
            ids = [rng.randrange(hi) for _ in range(rng.randrange(0, 4))]
            ids += ids[:1]  # a repeated id
            assert o.delete_vertices(ids) == b.del_vertices(ids)
        _compare(o, b)
        if step % 5 == 0:
            vids = [rng.randrange(hi) for _ in range(rng.randrange(0, 10))]
            off, nb = o.neighbors(vids)
            boff, bnb = b.csr()
            exp = []
            expoff = [0]
            for u in vids:
                if u < b.nv and b.alive[u]:
                    exp += list(bnb[boff[u]:boff[u + 1]])
                expoff.append(len(exp))
            np.testing.assert_array_equal(off, np.array(expoff, dtype=np.uint64))
            np.testing.assert_array_equal(nb, np.array(exp, dtype=np.uint32))


def _state(o):
    off, nb = o.export_csr()
    return off.copy(), nb.copy(), o.degrees().copy(), o.alive().copy()


def _assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.fixture
def base_graph():
    rng = np.random.default_rng(5)
    nv = 200
    s = rng.integers(0, nv, 3000).astype(np.uint32)
    d = rng.integers(0, nv, 3000).astype(np.uint32)
    return nv, s, d


def test_invariant_degree_sum_and_query_membership(base_graph):
    nv, s, d = base_graph
    o = oracle.OracleGraph(nv)
    o.bulk_build(s, d)
    assert int(o.degrees().sum()) == o.num_edges == 3000
    off, nb = o.export_csr()
    qs = np.repeat(np.arange(nv, dtype=np.uint32), 7)
    qd = np.tile(np.arange(0, 200, 29, dtype=np.uint32), nv)
    q = o.query_edges(qs, qd)
    for i in range(qs.size):
        u, v = qs[i], qd[i]
        assert q[i] == (v in set(nb[off[u]:off[u + 1]].tolist()))


def test_invariant_insert_then_delete_removes_batch(base_graph):
    nv, s, d = base_graph
    o = oracle.OracleGraph(nv)
    o.bulk_build(s, d)
    rng = np.random.default_rng(9)
    bs = rng.integers(0, nv, 500).astype(np.uint32)
    bd = rng.integers(0, nv, 500).astype(np.uint32)
    o.insert_edges(bs, bd)
    o.delete_edges(bs, bd)
    assert not o.query_edges(bs, bd).any()


def test_invariant_delete_absent_is_noop(base_graph):
    nv, s, d = base_graph
    o = oracle.OracleGraph(nv)
    o.bulk_build(s, d)
    before = _state(o)
    present = set(zip(s.tolist(), d.tolist()))
    absent = [(u, v) for u in range(nv) for v in range(0, nv, 13) if (u, v) not in present][:400]
    deleted, rejected = o.delete_edges([a for a, _ in absent], [b for _, b in absent])
    assert deleted == 0 and rejected == 0
    _assert_same(before, _state(o))


def test_invariant_vertex_delete_removes_incident_edges(base_graph):
    nv, s, d = base_graph
    o = oracle.OracleGraph(nv)
    o.bulk_build(s, d)
    gone = np.array([3, 17, 150, 17], dtype=np.uint32)
    assert o.delete_vertices(gone) == 3
    off, nb = o.export_csr()
    for g in (3, 17, 150):
        assert off[g + 1] == off[g]
        assert not np.isin(nb, [g]).any()
    assert int(o.degrees().sum()) == o.num_edges
    # edges touching a dead vertex are rejected afterwards
    ins, rej = o.insert_edges([3, 4], [4, 150])
    assert (ins, rej) == (0, 2)


def test_invariant_batch_permutation_and_split(base_graph):
    nv, s, d = base_graph
    rng = np.random.default_rng(11)
    perm = rng.permutation(s.size)
    a = oracle.OracleGraph(nv)
    a.insert_edges(s, d)
    b = oracle.OracleGraph(nv)
    b.insert_edges(s[perm], d[perm])
    c = oracle.OracleGraph(nv)
    c.insert_edges(s[:1000], d[:1000])
    c.insert_edges(s[1000:], d[1000:])
    _assert_same(_state(a), _state(b))
    _assert_same(_state(a), _state(c))
    ds, dd = s[::3], d[::3]
    a.delete_edges(ds, dd)
    b.delete_edges(ds[::-1], dd[::-1])
    c.delete_edges(ds[:200], dd[:200])
    c.delete_edges(ds[200:], dd[200:])
    _assert_same(_state(a), _state(b))
    _assert_same(_state(a), _state(c))


def test_invariant_dedup_idempotent(base_graph):
    nv, s, d = base_graph
    a = oracle.OracleGraph(nv, oracle.DEDUP)
    a.insert_edges(s, d)
    st = _state(a)
    ins, _ = a.insert_edges(s, d)
    assert ins == 0
    _assert_same(st, _state(a))
    assert a.num_edges == len(set(zip(s.tolist(), d.tolist())))


def test_multiset_keeps_duplicates_and_delete_removes_all_copies():
    o = oracle.OracleGraph(4)
    assert o.insert_edges([1, 1, 1, 2], [2, 2, 3, 0]) == (4, 0)
    np.testing.assert_array_equal(o.neighbors([1])[1], [2, 2, 3])
    # one batch entry removes both stored copies; a repeated entry is idempotent
    assert o.delete_edges([1, 1], [2, 2]) == (2, 0)
    np.testing.assert_array_equal(o.neighbors([1])[1], [3])


def test_self_loops_are_edges():
    o = oracle.OracleGraph(3)
    assert o.insert_edges([1], [1]) == (1, 0)
    assert o.query_edges([1], [1])[0] == 1


def test_empty_batches():
    o = oracle.OracleGraph(5)
    assert o.insert_edges([], []) == (0, 0)
    assert o.delete_edges([], []) == (0, 0)
    assert o.query_edges([], []).size == 0
    assert o.num_edges == 0


# ------------------------------------------------------- structural rules

def test_golden_dictionary_capacity():
    g = json.load(open(GOLDEN))["dictionary_capacity"]
    assert oracle.dictionary_capacity(g["n"]) == g["capacity"]
    # closed form: the power of two at or above n
    for n in [1, 2, 3, 4, 5, 511, 512, 513, 1 << 20, (1 << 20) + 1]:
        c = oracle.dictionary_capacity(n)
        assert c >= n and c & (c - 1) == 0 and (c == 1 or c // 2 < n)


def test_golden_cbt_path():
    g = json.load(open(GOLDEN))["cbt_path"]
    assert oracle.cbt_path(g["k"]) == g["path"]


def test_cbt_path_walks_reach_heap_index():
    # Following the bit string from the root (heap index 1): left child 2i,
    # right child 2i+1.  Every index must be reached, root has empty path.
    assert oracle.cbt_path(1) == ""
    for k in range(1, 3000):
        i = 1
        for ch in oracle.cbt_path(k):
            i = 2 * i + (1 if ch == "1" else 0)
        assert i == k


def test_golden_pop_ranges():
    g = json.load(open(GOLDEN))["pop_ranges"]
    b, e = oracle.pop_ranges(g["need"])
    incl = np.cumsum(g["need"])
    np.testing.assert_array_equal(incl, g["inclusive_prefix"])
    # thread 1 reads the prefix vector at indices 0 and 1
    r0, r1 = g["thread1_reads"]
    assert (b[1], e[1]) == (incl[r0], incl[r1]) == tuple(g["thread1_pops"])
    assert b[0] == 0 and e[0] == incl[0]
    rng = np.random.default_rng(3)
    need = rng.integers(0, 9, 300)
    b, e = oracle.pop_ranges(need)
    # ranges tile [0, total) without overlap and have the requested lengths
    np.testing.assert_array_equal(e - b, need)
    np.testing.assert_array_equal(b[1:], e[:-1])
    assert b[0] == 0 and e[-1] == need.sum()


def test_block_demand_closed_form():
    for C in (4, 8, 16, 20, 64):
        for deg in range(0, 3 * C + 2):
            for cnt in range(0, 3 * C + 2):
                # brute force: fill slots deg..deg+cnt-1 block by block
                blocks_before = -(-deg // C)
                blocks_after = -(-(deg + cnt) // C)
                assert oracle.insert_block_demand(deg, cnt, C) == blocks_after - blocks_before
                assert oracle.blocks_for_degree(deg, C) == blocks_before


def test_block_capacity_rule():
    # average degree of the vertices with non-zero degree (zero-degree ones excluded)
    deg = [0, 0, 10, 20, 30, 0]
    assert oracle.block_capacity_rule(deg) == 20
    assert oracle.block_capacity_rule([0, 0, 0]) == 4
    assert oracle.block_capacity_rule([1, 1, 2]) == 4      # at least 4
    assert oracle.block_capacity_rule([17, 18]) == 20      # ceil(17.5) = 18 -> multiple of 4
    # the upper end: a mean non-zero degree past 512 gives the largest block
    assert oracle.block_capacity_rule([508]) == 508
    assert oracle.block_capacity_rule([509]) == 512        # 509 -> 512 by the rounding
    assert oracle.block_capacity_rule([513]) == 512        # 516 by the rounding, then the cap
    assert oracle.block_capacity_rule([2000, 3000, 0]) == 512
    assert oracle.block_capacity_rule([1] * 10 + [100000]) == 512  # ceil(100010 / 11) = 9092


def test_min_footprint_capacity():
    # closed forms: equal degrees that are a multiple of 4 (<= 512) are met
    # exactly by C = that degree (no empty slot, one block each)
    for d in (4, 8, 36, 200, 512):
        assert oracle.min_footprint_capacity([d] * 7) == d
        assert oracle.min_footprint_capacity([d] * 7, weighted=True) == d
    assert oracle.min_footprint_capacity([0, 0]) == 4  # nothing stored: every C ties
    # degree 1 everywhere: C = 4 (one block of the smallest size each)
    assert oracle.min_footprint_capacity([1] * 50) == 4
    # brute force over the candidates, written out with numpy
    rng = np.random.default_rng(7)
    for trial in range(40):
        nv = int(rng.integers(1, 60))
        deg = rng.zipf(1.6, nv).clip(0, 5000) * rng.integers(0, 2, nv)
        for weighted in (False, True):
            C = np.arange(4, 513, 4)
            blocks = (-(-deg[None, :].astype(np.int64) // C[:, None])).sum(axis=1)
            cost = blocks * (4 * C * (2 if weighted else 1) + 12)
            exp = int(C[np.flatnonzero(cost == cost.min())[0]])
            assert oracle.min_footprint_capacity(deg, weighted) == exp

"""The parallel CPU baseline gives the oracle's results.

Random operation sequences (inserts with repeats, invalid and dead ids,
deletes with absent pairs and repeats, queries, vertex deletes) applied to
two oracle graphs, one through the sequential oracle and one through the
OpenMP baseline with 1, 3 and 8 threads; counts, query bits and the
canonical CSR must be equal after every call.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("flags", [0, oracle.DEDUP])
def test_parallel_baseline_matches_oracle(threads, flags):
    rng = np.random.default_rng(1000 + threads + 10 * flags)
    nv = 3000
    a, b = oracle.OracleGraph(nv, flags), oracle.OracleGraph(nv, flags)
    try:
        bs, bd = W.rmat_pairs(5, 0, 30000, 12)
        bs, bd = bs % nv, bd % nv
        assert a.insert_edges(bs, bd) == b.par_insert_edges(bs, bd, threads)
        for step in range(8):
            k = int(rng.integers(0, 20000))
            s = rng.integers(0, nv + 5, k).astype(np.uint32)
            d = rng.integers(0, nv + 5, k).astype(np.uint32)
            s[: k // 3] = bs[: k // 3]  # some repeats of stored pairs
            d[: k // 3] = bd[: k // 3]
            assert a.insert_edges(s, d) == b.par_insert_edges(s, d, threads)
            q = rng.integers(0, 30000, 5000)
            np.testing.assert_array_equal(a.query_edges(bs[q], bd[q]), b.par_query_edges(bs[q], bd[q], threads))
            m = int(rng.integers(0, 15000))
            ds = np.concatenate([s[:m // 2], rng.integers(0, nv + 5, m // 2).astype(np.uint32)])
            dd = np.concatenate([d[:m // 2], rng.integers(0, nv + 5, m // 2).astype(np.uint32)])
            assert a.delete_edges(ds, dd) == b.par_delete_edges(ds, dd, threads)
            if step % 3 == 2:
                ids = rng.choice(nv, 20, replace=False).astype(np.uint32)
                a.delete_vertices(ids)
                b.delete_vertices(ids)
            oa, na = a.export_csr()
            ob, nb = b.export_csr()
            np.testing.assert_array_equal(oa, ob)
            np.testing.assert_array_equal(na, nb)
            assert a.num_edges == b.num_edges
    finally:
        a.close()
        b.close()


def test_parallel_baseline_empty_and_tiny():
    o = oracle.OracleGraph(1)
    try:
        e = np.zeros(0, dtype=np.uint32)
        assert o.par_insert_edges(e, e, 4) == (0, 0)
        assert o.par_delete_edges(e, e, 4) == (0, 0)
        assert o.par_query_edges(e, e, 4).size == 0
        assert o.par_insert_edges([0, 0, 1], [0, 0, 0], 4) == (2, 1)
        np.testing.assert_array_equal(o.par_query_edges([0, 0, 1], [0, 1, 0], 4), [1, 0, 0])
        assert o.par_delete_edges([0], [0], 4) == (2, 0)
    finally:
        o.close()

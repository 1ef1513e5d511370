"""Host logic of the serving loop, on the CPU: how runs are formed from the
request queue (consecutive requests of one kind, in arrival order, up to the
merge capacity and request count), the worst-case block demand used for
admission, and the latency statistics."""
import collections
import types

import numpy as np
import pytest

from paper_2306_08252_gb300 import serve


def _req(kind, n, t=0.0):
    return serve.Request(kind, np.arange(n), np.arange(n), t)


def _fake(cap=100, max_reqs=4, C=16, nv=1000):
    return types.SimpleNamespace(cap=cap, max_reqs=max_reqs, C=C, nv=nv)


def test_runs_merge_consecutive_requests_of_one_kind():
    f = _fake()
    q = collections.deque([_req(serve.INSERT, 10), _req(serve.INSERT, 20), _req(serve.QUERY, 5),
                           _req(serve.INSERT, 7)])
    run = serve.Server._form_run(f, q)
    assert [len(r) for r in run] == [10, 20] and all(r.kind == serve.INSERT for r in run)
    run = serve.Server._form_run(f, q)
    assert [r.kind for r in run] == [serve.QUERY]
    run = serve.Server._form_run(f, q)
    assert [len(r) for r in run] == [7] and not q


def test_runs_respect_capacity_and_request_count():
    f = _fake(cap=50, max_reqs=3)
    q = collections.deque([_req(serve.DELETE, 20), _req(serve.DELETE, 20), _req(serve.DELETE, 20)])
    assert [len(r) for r in serve.Server._form_run(f, q)] == [20, 20]  # a third would pass 50 pairs
    assert [len(r) for r in serve.Server._form_run(f, q)] == [20]
    q = collections.deque([_req(serve.QUERY, 1) for _ in range(7)])
    assert len(serve.Server._form_run(f, q)) == 3 and len(q) == 4
    # arrival order is kept inside a run
    q = collections.deque([_req(serve.INSERT, 1, t) for t in (0.1, 0.2, 0.3)])
    assert [r.arrival for r in serve.Server._form_run(f, q)] == [0.1, 0.2, 0.3]


def test_oversized_request_is_refused():
    f = _fake(cap=10)
    with pytest.raises(ValueError):
        serve.Server._form_run(f, collections.deque([_req(serve.INSERT, 11)]))


def test_block_demand_is_an_upper_bound():
    # ceil(n / C) new blocks for the pairs plus one partly filled block per
    # source at most; brute force over how n pairs can spread over sources
    f = _fake(C=4, nv=6)
    rng = np.random.default_rng(3)
    for n in range(0, 40):
        bound = serve.Server._demand(f, n)
        assert bound == -(-n // 4) + min(n, 6)
        for _ in range(50):
            src = rng.integers(0, 6, n)
            deg = rng.integers(0, 9, 6)  # current degrees
            need = 0
            for u in range(6):
                k = int((src == u).sum())
                space = (-deg[u]) % 4
                need += -(-max(0, k - space) // 4)
            assert need <= bound


def test_latency_stats():
    reqs = [_req(serve.QUERY, 1, t) for t in range(10)]
    for i, r in enumerate(reqs):
        r.done = r.arrival + 0.001 * (i + 1)
    reqs[3].status = 2  # failed requests are left out
    st = serve.latency_stats(reqs, skip=2)
    lat = np.array([0.001 * (i + 1) for i in range(2, 10) if i != 3])
    assert st["p50_ms"] == pytest.approx(np.percentile(lat, 50) * 1e3)
    assert st["p99_ms"] == pytest.approx(np.percentile(lat, 99) * 1e3)
    assert st["max_ms"] == pytest.approx(10.0)


def test_native_loop_rejects_malformed_requests():
    # argument checks of gv_serve happen before anything runs (no GPU needed:
    # a NULL graph is refused first, then malformed requests)
    import ctypes
    import paper_2306_08252_gb300.graphvine as gvb
    lib = gvb.load()
    arr = (gvb.gv_serve_request * 1)()
    assert lib.gv_serve(None, arr, 1, None, None, None) == gvb.GV_ERR_INVALID_ARG
    assert lib.gv_serve(None, None, 0, None, None, None) == gvb.GV_ERR_INVALID_ARG

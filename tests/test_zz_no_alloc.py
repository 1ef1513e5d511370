"""gv_degree_offsets_noalloc: degree offsets without any allocation.

Some callers cannot allocate device memory when they need the offsets:
serving loops that must not stall on cudaFree's device-wide
synchronisation, processes whose device memory is all held by another
allocator, code under a fixed memory budget.  This entry point keeps its
scan scratch in a fixed device array instead.  Its result must equal the
offsets that the existing gv_neighbors entry point returns and the oracle's
degrees prefix-summed on the host, call after call (the scratch array is
shared and keeps the previous call's contents).

Kept in a file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _graph():
    """A GPU graph and the oracle after the same bulk build and vertex deletes."""
    import workloads as W
    from gpu_util import Pair
    nv = 5000
    s, d = W.rmat_pairs(31, 0, 60000, 13, limit=nv)
    p = Pair(nv, C=8, pool_bytes=32 << 20)
    p.bulk(s, d)
    p.vdel(np.array([3, 4, 4999], dtype=np.uint32))
    p.check(full=False)
    return p


def _oracle_offsets(o, vids):
    """offsets[i] = sum of the oracle's degrees of vids[0 .. i-1]; ids that
    are out of range or deleted count 0."""
    deg = o.degrees().astype(np.uint64) * o.alive().astype(np.uint64)
    v = vids.astype(np.int64)
    ok = v < deg.size
    per = np.zeros(vids.size, dtype=np.uint64)
    per[ok] = deg[v[ok]]
    return np.concatenate([[0], np.cumsum(per, dtype=np.uint64)]).astype(np.uint64)


def test_noalloc_offsets_match_gv_neighbors_on_consecutive_calls():
    import torch
    import paper_2306_08252_gb300 as gv
    from gpu_util import dev_u32
    p = _graph()
    g = p.g
    try:
        rng = np.random.default_rng(8)
        # several scan chunks, a ragged tail, repeated, invalid and deleted ids
        v1 = rng.integers(0, 5200, 70_001).astype(np.uint32)
        v1[:4] = [0, 3, 0xFFFFFFFF, 4999]
        # a shorter second call: stale chunk sums of the first call must not leak
        v2 = rng.integers(0, 5000, 1_500).astype(np.uint32)
        for vids in (v1, v2, v1):
            d_off = torch.full((vids.size + 1,), -1, dtype=torch.int64, device="cuda")
            code = gv.gv_degree_offsets_noalloc(g.handle, dev_u32(vids), d_off, torch.cuda.current_stream().cuda_stream)
            assert code == gv.GV_OK
            torch.cuda.synchronize()
            got = d_off.cpu().numpy().astype(np.uint64)
            ref, _ = g.neighbors(vids)  # existing entry point (gv_neighbors)
            np.testing.assert_array_equal(got, ref)
            np.testing.assert_array_equal(got, _oracle_offsets(p.o, vids))
    finally:
        p.close()


def test_noalloc_rejects_oversize_and_host_arrays():
    import torch
    import paper_2306_08252_gb300 as gv
    p = _graph()
    g = p.g
    try:
        lib = gv.load()
        d_vids = torch.zeros(4, dtype=torch.int32, device="cuda")
        d_off = torch.zeros(5, dtype=torch.int64, device="cuda")
        # beyond the stated maximum: rejected before any device work
        assert lib.gv_degree_offsets_noalloc(g.handle, d_vids.data_ptr(), (1 << 26) + 1, d_off.data_ptr(),
                                             None) == gv.GV_ERR_INVALID_ARG
        h_off = np.zeros(5, dtype=np.uint64)
        assert lib.gv_degree_offsets_noalloc(g.handle, d_vids.data_ptr(), 4, h_off.ctypes.data,
                                             None) == gv.GV_ERR_INVALID_ARG
        assert lib.gv_degree_offsets_noalloc(None, d_vids.data_ptr(), 4, d_off.data_ptr(), None) == gv.GV_ERR_INVALID_ARG
        # empty list: offsets[0] = 0
        d_off.fill_(7)
        assert lib.gv_degree_offsets_noalloc(g.handle, d_vids.data_ptr(), 0, d_off.data_ptr(), None) == gv.GV_OK
        torch.cuda.synchronize()
        assert int(d_off[0].item()) == 0
    finally:
        p.close()

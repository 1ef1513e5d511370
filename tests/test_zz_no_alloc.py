"""gv_degree_offsets_noalloc: degree offsets without any allocation.

Some callers cannot allocate device memory when they need the offsets: code
running during CUDA-graph stream capture, serving loops that must not stall
on cudaFree's device-wide synchronisation, processes whose device memory is
owned by another allocator.  This entry point keeps its scan scratch in a
fixed device array instead.  Its result must equal the offsets that the
existing gv_neighbors entry point returns, call after call (the scratch
array is shared and keeps the previous call's contents).

Kept in a file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _graph():
    import paper_2306_08252_gb300 as gv
    import workloads as W
    from gpu_util import dev_u32
    nv = 5000
    s, d = W.rmat_pairs(31, 0, 60000, 13, limit=nv)
    g = gv.Graph(nv, block_capacity=8, pool_bytes=32 << 20)
    g.bulk_build(dev_u32(s), dev_u32(d))
    g.delete_vertices(dev_u32(np.array([3, 4, 4999], dtype=np.uint32)))
    g.sync()
    return g


def test_noalloc_offsets_match_gv_neighbors_on_consecutive_calls():
    import torch
    import paper_2306_08252_gb300 as gv
    from gpu_util import dev_u32
    g = _graph()
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
            ref, _ = g.neighbors(vids)  # existing entry point (gv_neighbors)
            np.testing.assert_array_equal(d_off.cpu().numpy().astype(np.uint64), ref)
    finally:
        g.close()


def test_noalloc_rejects_oversize_and_host_arrays():
    import torch
    import paper_2306_08252_gb300 as gv
    g = _graph()
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
        g.close()

"""Host arithmetic of the benchmark, on the CPU: the algorithmic-byte model
(per operation and per kernel, with the split between the two mark tiers)
against hand-computed values on a small graph state."""
import types

import numpy as np

import bench


def _fake_graph(deg):
    return types.SimpleNamespace(degrees=lambda: (np.asarray(deg, dtype=np.uint32), None))


def test_byte_model_closed_forms():
    C = bench.BLOCK
    deg = np.zeros(64, dtype=np.int64)
    deg[1] = 10          # tiny: <= 8 blocks, <= 128 entries
    deg[2] = 200         # warp tier (more than 128 entries)
    deg[3] = 5           # tiny for deletes, but 20 batch entries: warp tier
    src = np.array([1] * 3 + [2] * 4 + [3] * 20 + [70, 5], dtype=np.uint32)  # 70 is out of range
    dst = np.array([7] * (src.size - 2) + [1, 99], dtype=np.uint32)          # 99 out of range
    qs = np.array([1, 2, 2, 9, 80], dtype=np.uint32)
    qd = np.array([3, 3, 4, 5, 6], dtype=np.uint32)
    m = bench.byte_model(_fake_graph(deg), (src, dst), (qs, qd), inserted=27, deleted=27, newblocks=3)
    valid = (src < 64) & (dst < 64)
    us = np.unique(src[valid])                  # 1, 2, 3 (5's pair has dst 99)
    assert list(us) == [1, 2, 3]
    assert m["insert"] == 12 * 27 + 32 * 3 + 12 * 3
    assert m["query"] == 9 * 5 + 4 * (10 + 200 + 0)  # distinct queried sources 1, 2, 9
    assert m["delete"] == 8 * src.size + 4 * (10 + 200 + 5) + 32 * 3 + 4 * 3
    k = m["kernels"]
    # delete tiers: source 1 tiny (10 entries, 3 batch entries); 2 and 3 in the warp tier
    assert k["delete.mark_tiny"] == 4 * 10 + 4 * 3
    assert k["delete.mark"] == 4 * (200 + 5) + 4 * (4 + 20)
    # the two tiers cover every stored entry and batch entry of the touched sources
    assert k["delete.mark"] + k["delete.mark_tiny"] == 4 * (10 + 200 + 5) + 4 * 27
    # query tiers (tiny: <= 4 blocks, <= 64 entries): 1 tiny, 2 warp, 9 has no entries
    assert k["query.mark_tiny"] == 4 * 10 + 4 * 1
    assert k["query.mark"] == 4 * 200 + 4 * 2
    assert k["insert.count"] == 12 * src.size and k["insert.scatter"] == 16 * 27
    assert k["delete.scatter"] == 16 * src.size and k["query.scatter"] == 16 * qs.size
    assert k["insert.touched"] == 4 * 64  # the counter array of the dictionary's capacity
    # grouped path: pairs read once by the partition, one entry per placed pair
    assert k["insert.partition"] == 8 * src.size and k["query.partition"] == 8 * qs.size
    assert k["insert.slots"] == 4 * 27 and k["delete.group"] == 4 * int(valid.sum())
    assert k["query.group"] == 4 * int(((qs < 64) & (qd < 64)).sum())
    assert k["delete.mark_cta"] == 0 and k["query.mark_cta"] == 0  # no source past 256 batch entries
    assert m["step"] == m["insert"] + m["query"] + m["delete"]
    assert C == 16


def test_byte_model_block_wide_tier():
    deg = np.zeros(32, dtype=np.int64)
    deg[4] = 1000
    deg[5] = 600
    src = np.array([4] * 300 + [5] * 100, dtype=np.uint32)
    dst = np.arange(400, dtype=np.uint32) % 32
    m = bench.byte_model(_fake_graph(deg), (src, dst), (src[:10], dst[:10]), inserted=400, deleted=400,
                         newblocks=0, radix=True)
    k = m["kernels"]
    assert k["delete.mark_cta"] == 4 * 1000 + 4 * 300   # source 4: 300 batch entries
    assert k["delete.mark"] == 4 * 600 + 4 * 100        # source 5: 100
    assert k["delete.mark_tiny"] == 0
    # the default path has no block-wide tier: the warp tier takes both
    k = bench.byte_model(_fake_graph(deg), (src, dst), (src[:10], dst[:10]), inserted=400, deleted=400,
                         newblocks=0)["kernels"]
    assert k["delete.mark_cta"] == 0
    assert k["delete.mark"] == 4 * (1000 + 600) + 4 * 400


def test_whole_job_rate_and_config():
    assert bench.whole_job_rate(10, 4, 2.0) == 10 * 4 / 2e-3
    cfg = bench.config_dict(types.SimpleNamespace(batch=bench.BATCH, queries=bench.QUERIES, gpus=1), 1)
    assert "workload" in cfg and str(bench.BATCH) in cfg["workload"]

"""Graph sets (many member graphs in one structure) vs one oracle per member.

Every member's canonical CSR, its per-member counts and the structure's
self-check are compared after each set call; the set must also equal the
same members built as separate graphs, and a CUDA-graph capture of a set
insert + delete must replay to the same states.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import canon, dev_u32

pytestmark = pytest.mark.gpu


def _dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _members(graphs=16, seed=41):
    m = W.batched_rmat(seed=seed, graphs=graphs, xlo=5.0, xhi=11.0, smax=1e4)
    # a few rejected pairs in some members' batches (ids out of the member's range)
    for i in (1, 5, 9):
        if i < len(m):
            s, d = m[i]["insert"]
            m[i]["insert"] = (np.concatenate([s, [m[i]["nv"], 0]]).astype(np.uint32),
                              np.concatenate([d, [0, m[i]["nv"] + 3]]).astype(np.uint32))
    return m


def _check_members(gs, orcs):
    for i, o in enumerate(orcs):
        off, nb = gs.member_csr(i)
        ooff, onb = o.export_csr()
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(canon(off, nb), onb)
    assert gs.validate() == 0


def _apply(gs, orcs, members, key, op):
    import torch
    s, d, off = W.concat_member_batches(members, key)
    counts = torch.zeros(2 * len(members), dtype=torch.int64, device="cuda")
    if op == "insert":
        gs.insert_edges(dev_u32(s), dev_u32(d), _dev_u64(off), counts)
        exp = [o.insert_edges(*m[key]) for o, m in zip(orcs, members)]
    else:
        gs.delete_edges(dev_u32(s), dev_u32(d), _dev_u64(off), counts)
        exp = [o.delete_edges(*m[key]) for o, m in zip(orcs, members)]
    got = counts.cpu().numpy().reshape(-1, 2)
    np.testing.assert_array_equal(got, np.array(exp, dtype=np.int64))


def test_set_matches_member_oracles():
    import torch
    import paper_2306_08252_gb300 as gv
    members = _members()
    gs = gv.GraphSet([m["nv"] for m in members], block_capacity=8, pool_bytes=64 << 20)
    orcs = [oracle.OracleGraph(m["nv"]) for m in members]
    try:
        _apply(gs, orcs, members, "bulk", "insert")
        _check_members(gs, orcs)
        _apply(gs, orcs, members, "insert", "insert")
        _check_members(gs, orcs)
        # queries: each member's insert batch plus random pairs
        qm = [{"q": (np.concatenate([m["insert"][0], W.uniform_pairs(5, i, 50, m["nv"])[0]]).astype(np.uint32),
                     np.concatenate([m["insert"][1], W.uniform_pairs(5, i, 50, m["nv"])[1]]).astype(np.uint32))}
              for i, m in enumerate(members)]
        s, d, off = W.concat_member_batches(qm, "q")
        out = torch.zeros(s.size, dtype=torch.uint8, device="cuda")
        counts = torch.zeros(2 * len(members), dtype=torch.int64, device="cuda")
        gs.query_edges(dev_u32(s), dev_u32(d), _dev_u64(off), counts, out)
        exp = np.concatenate([o.query_edges(*q["q"]) for o, q in zip(orcs, qm)])
        np.testing.assert_array_equal(out.cpu().numpy(), exp)
        _apply(gs, orcs, members, "delete", "delete")
        _check_members(gs, orcs)
        _apply(gs, orcs, members, "insert", "delete")  # delete the inserted batches
        _check_members(gs, orcs)
        st = gs.stats()
        assert st["num_edges"] == sum(o.num_edges for o in orcs)
    finally:
        gs.close()


def test_set_equals_separate_graphs():
    import paper_2306_08252_gb300 as gv
    members = _members(graphs=6, seed=43)
    gs = gv.GraphSet([m["nv"] for m in members], block_capacity=8, pool_bytes=32 << 20)
    orcs = [oracle.OracleGraph(m["nv"]) for m in members]
    plain = [gv.Graph(m["nv"], block_capacity=8, pool_bytes=8 << 20) for m in members]
    try:
        for key, op in (("bulk", "insert"), ("insert", "insert"), ("delete", "delete")):
            _apply(gs, orcs, members, key, op)
            for g, m in zip(plain, members):
                (g.insert_edges if op == "insert" else g.delete_edges)(dev_u32(m[key][0]), dev_u32(m[key][1]))
        for i, g in enumerate(plain):
            off, nb = gs.member_csr(i)
            poff, pnb = g.export_csr()
            np.testing.assert_array_equal(off, poff)
            np.testing.assert_array_equal(canon(off, nb), canon(poff, pnb))
    finally:
        gs.close()
        for g in plain:
            g.close()


def test_set_cuda_graph_capture_replays():
    import torch
    import paper_2306_08252_gb300 as gv
    members = _members(graphs=12, seed=47)
    gs = gv.GraphSet([m["nv"] for m in members], block_capacity=8, pool_bytes=64 << 20)
    orcs = [oracle.OracleGraph(m["nv"]) for m in members]
    try:
        _apply(gs, orcs, members, "bulk", "insert")
        si, di, oi = W.concat_member_batches(members, "insert")
        sd, dd, od = W.concat_member_batches(members, "delete")
        a = [dev_u32(si), dev_u32(di), _dev_u64(oi)]
        b = [dev_u32(sd), dev_u32(dd), _dev_u64(od)]
        ci = torch.zeros(2 * len(members), dtype=torch.int64, device="cuda")
        cd = torch.zeros(2 * len(members), dtype=torch.int64, device="cuda")
        gs.reserve(max(si.size, sd.size))
        # warm the scratch once outside capture
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            gs.insert_edges(*a, ci)
            gs.delete_edges(*b, cd)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        for o, m in zip(orcs, members):
            o.insert_edges(*m["insert"])
            o.delete_edges(*m["delete"])
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="relaxed"):
            gs.insert_edges(*a, ci)
            gs.delete_edges(*b, cd)
        for _ in range(2):
            graph.replay()
            torch.cuda.synchronize()
            exp_i = [o.insert_edges(*m["insert"]) for o, m in zip(orcs, members)]
            exp_d = [o.delete_edges(*m["delete"]) for o, m in zip(orcs, members)]
            np.testing.assert_array_equal(ci.cpu().numpy().reshape(-1, 2), np.array(exp_i))
            np.testing.assert_array_equal(cd.cpu().numpy().reshape(-1, 2), np.array(exp_d))
            _check_members(gs, orcs)
    finally:
        gs.close()

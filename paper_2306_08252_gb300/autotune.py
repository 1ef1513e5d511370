"""Autotuner for graph sets.

Picks, for a workload of many member graphs, the edge-block capacity C, the
number of blocks one warp handles per work item in deletes (the threads per
adjacency) and the batch size above which grouping switches from per-tile
aggregation to one atomic per pair plus a vertex pass.  The search is a
coordinate descent over small candidate lists, timed with CUDA events on a
stratified sample of the members (insert batch + delete batch, then an
untimed restore), and the choice is cached in a JSON file keyed by the
workload's shape and the device name.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

CANDIDATES = {
    "block_capacity": [4, 8, 16, 32],
    "item_blocks": [32, 16, 8],
    "dense_shift": [3, 1, 6],
}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "graphvine", "autotune.json")


def _signature(members, device_name):
    nv = sum(m["nv"] for m in members)
    e = sum(m["bulk"][0].size for m in members)
    ni = sum(m["insert"][0].size for m in members)
    nd = sum(m["delete"][0].size for m in members)
    key = f"{len(members)}:{nv}:{e}:{ni}:{nd}:{device_name}"
    return hashlib.sha256(key.encode()).hexdigest()[:24], key


def concat_member_batches(members, key):
    """One batch kind over members: (src, dst, offsets[G+1])."""
    parts = [m[key] for m in members]
    off = np.zeros(len(parts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([p[0].size for p in parts])
    src = np.concatenate([np.asarray(p[0], dtype=np.uint32) for p in parts])
    dst = np.concatenate([np.asarray(p[1], dtype=np.uint32) for p in parts])
    return src, dst, off


def sample_members(members, k):
    """Every (G/k)-th member in size order: keeps the spread of sizes."""
    if len(members) <= k:
        return list(members)
    order = sorted(range(len(members)), key=lambda i: members[i]["nv"])
    pick = [order[int(j * len(order) / k)] for j in range(k)]
    return [members[i] for i in pick]


def _time_config(members, cfg, reps):
    import torch

    from . import graphvine as gv

    def dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()

    bs, bd, bo = concat_member_batches(members, "bulk")
    is_, id_, io = concat_member_batches(members, "insert")
    ds, dd, do = concat_member_batches(members, "delete")
    C = cfg["block_capacity"]
    blocks = (bs.size + 2 * is_.size) // C + sum(m["nv"] for m in members) + 4096
    gs = gv.GraphSet([m["nv"] for m in members], block_capacity=C, pool_bytes=int(blocks * (4 * C + 12) * 1.5),
                     item_blocks=cfg["item_blocks"], dense_shift=cfg["dense_shift"])
    try:
        cnt = torch.zeros(2 * len(members), dtype=torch.int64, device="cuda")
        gs.insert_edges(dev(bs, np.int32), dev(bd, np.int32), dev(bo, np.int64), cnt)
        gs.reserve(max(bs.size, is_.size, ds.size))
        a = (dev(is_, np.int32), dev(id_, np.int32), dev(io, np.int64))
        b = (dev(ds, np.int32), dev(dd, np.int32), dev(do, np.int64))
        times = []
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gs.insert_edges(*a, cnt)
            gs.delete_edges(*b, cnt)
            e1.record()
            gs.delete_edges(*a, cnt)  # restore (untimed)
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        gs.sync()
        return float(np.median(times))
    finally:
        gs.close()


def tune_set(members, sample=32, reps=3, cache=DEFAULT_CACHE, refresh=False, log=None):
    """Best {block_capacity, item_blocks, dense_shift} for this workload."""
    import torch

    name = torch.cuda.get_device_name()
    sig, key = _signature(members, name)
    db = {}
    if cache and os.path.exists(cache):
        try:
            db = json.load(open(cache))
        except Exception:
            db = {}
    if not refresh and sig in db:
        return dict(db[sig]["config"], cached=True)
    sub = sample_members(members, sample)
    best = {"block_capacity": 8, "item_blocks": 32, "dense_shift": 3}
    best_t = _time_config(sub, best, reps)
    trials = [(dict(best), best_t)]
    for knob in ("block_capacity", "item_blocks", "dense_shift"):
        for v in CANDIDATES[knob]:
            if v == best[knob]:
                continue
            cand = dict(best, **{knob: v})
            if cand["item_blocks"] > min(32, 512 // cand["block_capacity"]):
                continue
            t = _time_config(sub, cand, reps)
            trials.append((dict(cand), t))
            if log:
                log(f"autotune {cand} {t:.3f} ms")
            if t < best_t:
                best, best_t = cand, t
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        db[sig] = {"key": key, "config": best, "ms": best_t,
                   "trials": [{"config": c, "ms": t} for c, t in trials]}
        tmp = cache + f".tmp{os.getpid()}"
        json.dump(db, open(tmp, "w"), indent=1)
        os.replace(tmp, cache)
    return dict(best, cached=False, ms=best_t, trials=len(trials))

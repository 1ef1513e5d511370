"""Benchmark: batched edge updates on a power-law graph, one JSON line.

Workload (the paper's batched-update experiment, Tables 3 and 4, on a
synthetic stand-in for its co-paper graphs): RMAT graph with 2^20 vertices
and 16,777,216 edges (a, b, c, d = .57, .19, .19, .05), edge-block capacity
C = 16, bulk built once; one step = insert a 10,000,000-edge RMAT batch,
answer 1,000,000 edge-existence queries (half present), delete the same
10,000,000 edges.  metric = edge updates (inserted + deleted entries) per
second.  Inputs live in HBM before the timed region; L2 is flushed before
every timed step.

`--impl reference` times the CPU oracle (the plain definition the GPU
results are checked against) on a bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge updates/s (batch insert+delete)"
UNIT = "edges/s"
SCALE = 20
BASE_EDGES = 1 << 24
BATCH = 10_000_000
QUERIES = 1_000_000
C = 16
BLOCK = C
POOL_BYTES = 2 << 30
SEED = 2
HUB_SHIFT = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--queries", type=int, default=QUERIES)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay of the step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the short batched-form record")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving record")
    ap.add_argument("--requests", type=int, default=10_000)
    ap.add_argument("--serve-loop", default="native", choices=["native", "python"],
                    help="the serving loop: native (gv_serve, the C ABI) or the Python one (serve.Server)")
    ap.add_argument("--serve-scale", type=int, default=24)
    ap.add_argument("--workload", default="rmat", choices=["rmat", "batched", "serving", "rows"],
                    help="rmat: the single-graph step (default); batched: many member graphs, "
                         "one captured launch sequence vs one launch sequence per graph")
    ap.add_argument("--graphs", type=int, default=256)
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="RMAT scale of the graph (16 * 2^scale base edges); the default is the "
                         "measured workload, smaller scales are for profiling captures")
    ap.add_argument("--grouping", default="atomic", choices=["atomic", "radix"],
                    help="grouping of large batches: one atomic per pair (default) or the radix partition")
    ap.add_argument("--hub-shift", type=int, default=HUB_SHIFT,
                    help="the hub-runs record: runs of 2^s blocks for vertices whose first allocation takes "
                         "at least C * 2^s entries (0 skips the record)")
    return ap.parse_args()


def workload(batch, queries):
    import workloads as W
    bs, bd = W.rmat_graph(SEED, SCALE, BASE_EDGES)
    s, d = W.rmat_update(SEED, SCALE, batch, 0)
    qs, qd = W.rmat_queries(SEED, SCALE, queries, s, d, 0)
    return (bs, bd), (s, d), (qs, qd)


def config_dict(args, n):
    return {
        "workload": f"RMAT scale {SCALE} ({1 << SCALE} vertices, {BASE_EDGES} edges, a,b,c,d=.57,.19,.19,.05), "
                    f"C={C}; step = insert {args.batch} + query {args.queries} + delete the {args.batch}",
        "vertices": 1 << SCALE,
        "base_edges": BASE_EDGES,
        "batch": args.batch,
        "queries": args.queries,
        "block_capacity": C,
        "l2": "flushed before every timed step (256 MiB write)",
        "parallelism": f"replicas{n}" if n > 1 else "single",
    }


# ------------------------------------------------------------ CPU baseline

def oracle_sample_rate(base, upd, qry, budget_s=12.0, warmup=1):
    """The oracle (single thread, as it stands) on whole steps of the
    workload: insert the full batch, answer every query, delete the batch,
    on the full bulk-built graph; `warmup` untimed steps first (the first
    delete also removes the base graph's copies of batch pairs), then steps
    until `budget_s` of timed work (at least one)."""
    import oracle
    o = oracle.OracleGraph(1 << SCALE)
    o.bulk_build(*base)

    def ostep():
        ins, _ = o.insert_edges(*upd)
        o.query_edges(*qry)
        dele, _ = o.delete_edges(*upd)
        return ins + dele

    for _ in range(warmup):
        ostep()
    done = 0
    t_total = 0.0
    steps = 0
    while t_total < budget_s or steps == 0:
        t0 = time.perf_counter()
        done += ostep()
        t_total += time.perf_counter() - t0
        steps += 1
    o.close()
    return done / t_total, steps, t_total


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm
    implementer/part codes), with the machine architecture."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model Name", "Hardware"):
            for line in info.splitlines():
                if line.split(":")[0].strip() == key:
                    name = line.split(":", 1)[1].strip()
                    break
            if name:
                break
        if not name:
            kv = {}
            for line in info.splitlines():
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv.setdefault(k.strip(), v.strip())
            if "CPU implementer" in kv:
                name = f"implementer {kv['CPU implementer']} part {kv.get('CPU part', '?')}"
    except OSError:
        pass
    return f"{name or 'unknown'} ({platform.machine()})"


def parallel_cpu_rate(base, upd, qry, threads, budget_s=10.0, max_steps=3):
    """The oracle's sorted-vector algorithm run over `threads` host cores
    (OpenMP over source buckets) on the whole step: insert the full batch,
    answer every query, delete the batch; whole steps until `budget_s`."""
    import oracle
    o = oracle.OracleGraph(1 << SCALE)
    o.par_insert_edges(*base, threads)
    done, t_total, steps = 0, 0.0, 0
    while (t_total < budget_s and steps < max_steps) or steps == 0:
        t0 = time.perf_counter()
        ins, _ = o.par_insert_edges(upd[0], upd[1], threads)
        o.par_query_edges(qry[0], qry[1], threads)
        dele, _ = o.par_delete_edges(upd[0], upd[1], threads)
        t_total += time.perf_counter() - t0
        done += ins + dele
        steps += 1
    o.close()
    return done / t_total, steps, t_total


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------- byte model

def max_over_ranks(values, world, device="cpu"):
    """Per-figure maximum over the ranks of the job (one all_reduce of a
    float64 vector on `device`); the values themselves at world size 1."""
    values = [float(v) for v in values]
    if world <= 1:
        return values
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processed `units_per_rank` units and
    the job took `ms` (the slowest rank's time)."""
    return world * units_per_rank / (ms / 1e3)


def byte_model(g, batch, qry, inserted, deleted, newblocks, radix=False):
    """Algorithmic bytes.

    Per operation (the minimum the method must move): insert 12 B/edge +
    32 B/touched source + 12 B/new block; query 9 B/query + 4 B per stored
    entry of each distinct queried source; delete 8 B/edge + 4 B per stored
    entry of each touched source + 32 B per touched source + 4 B per freed
    block (entries moved by compaction are not counted: a lower bound).

    Per kernel (its compulsory traffic): the partition passes read the pairs
    once (8 B/pair; the partitioned copy is grouping scratch); the grouping
    by vertex writes one 4-byte batch-list entry per pair (deletes, queries;
    for inserts the grouped destination); the insert's slot pass writes one
    4-byte entry per inserted pair; mark kernels (thread-per-source, warp and
    block-wide tiers) read every stored entry of the sources they own and
    their batch entries (4 B each).  The per-pair atomic grouping (the
    default) has its counting passes at 12 B/pair and scatters at 16 B/pair."""
    s, d = batch
    deg, _ = g.degrees()  # state after the insert = state the query and delete see
    nv = deg.size
    C = BLOCK
    ok = (s < nv) & (d < nv)
    us = np.unique(s[ok])
    qs = np.unique(qry[0][qry[0] < nv])
    deg64 = deg.astype(np.int64)
    ins_b = 12 * inserted + 32 * us.size + 12 * newblocks
    qry_b = 9 * qry[0].size + 4 * int(deg64[qs].sum())
    del_b = 8 * s.size + 4 * int(deg64[us].sum()) + 32 * us.size + 4 * newblocks

    def tiers(src_ids, tiny_deg, tiny_nb):
        # thread-per-source tier: <= tiny_nb blocks, <= min(tiny_deg, tiny_nb*C)
        # entries, <= 16 batch entries (deletes 128 / 8, queries 64 / 4); the
        # others: the warp tier, or on the radix path the block-wide tier for
        # 257..4096 batch entries
        m = np.bincount(src_ids, minlength=nv)
        touched = m > 0
        nb = (deg64 + C - 1) // C
        tiny = touched & (deg64 > 0) & (deg64 <= min(tiny_deg, tiny_nb * C)) & (nb <= tiny_nb) & (m <= 16)
        big = touched & (deg64 > 0) & ~tiny
        # the block-wide tier exists only on the radix-partition path; the
        # default path's warp tier takes every source that is not tiny
        cta = big & (m > 256) & (m <= 4096) if radix else np.zeros_like(big)
        warp = big & ~cta
        f = lambda sel: 4 * int(deg64[sel].sum()) + 4 * int(m[sel].sum())
        return f(warp), f(cta), f(tiny)

    dmark, dcta, dtiny = tiers(s[ok], 128, 8)
    qok = (qry[0] < nv) & (qry[1] < nv)
    qmark, qcta, qtiny = tiers(qry[0][qok], 64, 4)
    scan = 4 * (1 << int(np.ceil(np.log2(max(nv, 1)))))
    nq = int(qok.sum())
    kernels = {
        "insert.partition": 8 * s.size, "insert.group": 4 * inserted, "insert.slots": 4 * inserted,
        "delete.partition": 8 * s.size, "delete.group": 4 * int(ok.sum()),
        "delete.mark": dmark, "delete.mark_cta": dcta, "delete.mark_tiny": dtiny,
        "query.partition": 8 * qry[0].size, "query.group": 4 * nq,
        "query.mark": qmark, "query.mark_cta": qcta, "query.mark_tiny": qtiny,
        # per-pair atomic grouping (the default)
        "insert.count": 12 * s.size, "insert.touched": scan, "insert.scatter": 16 * inserted,
        "delete.count": 12 * s.size, "delete.touched": scan, "delete.scatter": 16 * s.size,
        "query.count": 12 * qry[0].size, "query.touched": scan, "query.scatter": 16 * qry[0].size,
    }
    return {"insert": ins_b, "query": qry_b, "delete": del_b, "step": ins_b + qry_b + del_b,
            "touched_sources": int(us.size), "kernels": kernels}


# host-only sources that define and launch no kernel (the native serving
# loop): they do not change what a kernel reads or writes
HOST_ONLY = {"gv_serve.cu"}


def source_hash():
    """Hash of the sources the step's kernels come from (every file of
    csrc/ but the host-only ones); ncu figures taken on other sources are
    not used."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_08252_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f not in HOST_ONLY:
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_phase):
    """Per-launch DRAM bytes of the phase's kernel from the committed ncu
    summary, or None if absent or taken on different kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        data = json.load(open(p))
    except Exception:
        return None
    ent = data.get(kernel_phase)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_2306_08252_gb300 as gv

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gv.load()
    base, upd, qry = workload(args.batch, args.queries)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    d_bs, d_bd = t(base[0]), t(base[1])
    d_s, d_d = t(upd[0]), t(upd[1])
    d_qs, d_qd = t(qry[0]), t(qry[1])
    d_out = torch.zeros(args.queries, dtype=torch.uint8, device=dev)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    g = gv.Graph(1 << SCALE, block_capacity=C, pool_bytes=POOL_BYTES,
                 flags=gv.GV_RADIX_GROUPING if args.grouping == "radix" else 0)
    g.reserve(max(args.batch, BASE_EDGES))
    g.bulk_build(d_bs, d_bs.new_empty(0) if False else d_bd, counts[:2])
    g.sync()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        g.insert_edges(d_s, d_d, counts[:2])
        g.query_edges(d_qs, d_qd, d_out)
        g.delete_edges(d_s, d_d, counts[2:])

    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else args.warmup):
        step()
    torch.cuda.synchronize()
    assert g.sync() == 0

    # byte model from the steady state (after an insert)
    st0 = g.stats()
    g.insert_edges(d_s, d_d, counts[:2])
    torch.cuda.synchronize()
    st1 = g.stats()
    inserted = int(counts[0].item())
    newblocks = st1["pool_blocks_used"] - st0["pool_blocks_used"]
    g.delete_edges(d_s, d_d, counts[2:])
    torch.cuda.synchronize()
    deleted = int(counts[2].item())
    # degrees as the query/delete of a step see them: re-insert, measure, delete
    g.insert_edges(d_s, d_d, counts[:2])
    model = byte_model(g, upd, qry, inserted, deleted, newblocks, radix=args.grouping == "radix")
    g.delete_edges(d_s, d_d, counts[2:])
    torch.cuda.synchronize()

    # ---------------- timed region (device time, CUDA events on the stream
    # around each step; none inside a step, so consecutive kernels keep their
    # programmatic dependent launches)
    sampler = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    upd_done = args.steps * (inserted + deleted)
    if world > 1:
        dist.barrier()
    assert g.sync() == 0

    # ---------------- per-kernel device time: the same K steps again with the
    # library's per-phase CUDA events recorded around every kernel (the
    # roofline's kernel durations and the launch count come from here; the
    # events between kernels cost the step a little)
    g.profile_read()
    g.profile(True)
    torch.cuda.synchronize()
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        pev[i][0].record(stream)
        step()
        pev[i][1].record(stream)
    torch.cuda.synchronize()
    g.profile(False)
    phases = g.profile_read()
    profiled_ms = float(sum(a.elapsed_time(b) for a, b in pev))
    assert g.sync() == 0
    gpu_launches = int(sum(c for _, c in phases.values()))

    # ---------------- the same step replayed from a CUDA graph (captured once):
    # same calls, same work; the library's launch sequence without host
    # launch latency between kernels
    graph = None
    if not args.no_graph:
        ref_counts = counts.clone()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, capture_error_mode="relaxed"):
            step()
        cg.replay()
        torch.cuda.synchronize()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            gev[i][0].record(stream)
            cg.replay()
            gev[i][1].record(stream)
        torch.cuda.synchronize()
        assert torch.equal(counts, ref_counts) and g.sync() == 0
        g_ms = float(sum(a.elapsed_time(b) for a, b in gev))
        g_ms = max_over_ranks([g_ms], world, dev)[0]
        graph = {"value": whole_job_rate(upd_done, world, g_ms), "unit": UNIT, "ms_per_step": g_ms / args.steps,
                 "timer": "CUDA events around each replay of the captured step"}
        del cg

    # ---------------- the compaction-heavy delete: the first delete of the
    # batch on a freshly built graph (bulk build + the insert) also removes
    # the base graph's copies of batch pairs, spread through the adjacencies,
    # so compaction moves many entries (the steady-state step deletes only
    # the entries its own insert appended, at the adjacency tails)
    heavy_ms, heavy_phases, heavy_deleted = [], {}, 0
    for r in range(3):
        g2 = gv.Graph(1 << SCALE, block_capacity=C, pool_bytes=POOL_BYTES,
                      flags=gv.GV_RADIX_GROUPING if args.grouping == "radix" else 0)
        g2.reserve(max(args.batch, BASE_EDGES))
        g2.bulk_build(d_bs, d_bd)
        g2.insert_edges(d_s, d_d)
        if r == 2:
            g2.profile_read()
            g2.profile(True)
        flush.fill_(r & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g2.delete_edges(d_s, d_d, counts[2:])
        e1.record(stream)
        torch.cuda.synchronize()
        heavy_deleted = int(counts[2].item())
        if r == 2:
            g2.profile(False)
            heavy_phases = {k: v[0] for k, v in g2.profile_read().items() if v[1] and k.startswith("delete.")}
        else:
            heavy_ms.append(e0.elapsed_time(e1))
        assert g2.sync() == 0
        g2.close()
    heavy = {"ms": statistics.median(heavy_ms), "deleted": heavy_deleted,
             "value": heavy_deleted / (statistics.median(heavy_ms) / 1e3), "unit": UNIT,
             "phases_ms": heavy_phases,
             "workload": f"delete the {args.batch}-edge batch once, right after the bulk build and its insert "
                         "(every stored copy of a batch pair goes, base-graph copies included)",
             "timer": "CUDA events around the call; median of 2, phases from a third with per-kernel events"}

    # ---------------- end to end: host (pinned) inputs and outputs, through the C ABI
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
        h_s, h_d, h_qs, h_qd = pin(upd[0]), pin(upd[1]), pin(qry[0]), pin(qry[1])
        h_out = torch.zeros(args.queries, dtype=torch.uint8).pin_memory()
        h_counts = torch.zeros(4, dtype=torch.int64).pin_memory()

        def step_host():
            g.insert_edges(h_s, h_d, h_counts[:2])
            g.query_edges(h_qs, h_qd, h_out)
            g.delete_edges(h_s, h_d, h_counts[2:])

        step_host()
        torch.cuda.synchronize()
        e_ms = 0.0
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e_ms += (time.perf_counter() - t0) * 1e3
        assert g.sync() == 0
        h2d = 2 * 4 * args.batch * 2 + 2 * 4 * args.queries
        d2h = args.queries + 32
        e2e = {"value": args.steps * (inserted + deleted) / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e_ms / args.steps, "timer": "host wall clock from the first call of the step to the device synchronisation after its last"}

    # the slowest rank's times; every rank processed the same units
    mx = max_over_ranks([total_ms] + ([e2e["ms_per_step"]] if e2e else []), world, dev)
    total_ms = mx[0]
    if e2e:
        e2e["ms_per_step"] = mx[1]
        e2e["value"] = whole_job_rate(args.steps * (inserted + deleted), world, mx[1] * args.steps)

    value = whole_job_rate(upd_done, world, total_ms)
    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # dominant kernel phase = largest device time in the timed region among
    # the kernels on the call stream (the thread-per-source mark tier runs on
    # the library's second stream beside the warp tier: its event span
    # includes the time it shares the GPU with that kernel)
    concurrent = ("delete.mark_tiny", "query.mark_tiny")
    dom = max((k for k in phases if phases[k][1] > 0 and k in model["kernels"] and k not in concurrent),
              key=lambda k: phases[k][0])
    dom_ms = phases[dom][0] / phases[dom][1]
    dom_bytes = model["kernels"][dom]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = ncu_traffic(dom)
    step_gbs = model["step"] / (total_ms / args.steps / 1e3) / 1e9
    res = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (seeded RMAT generator; stands in for the paper's DIMACS co-paper graphs)",
        "config": config_dict(args, world),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": pk_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": dom_bytes, "launch_ms": dom_ms},
        "step_roofline": {"algorithmic_bytes": model["step"], "achieved_gbs": step_gbs, "frac_of_measured": step_gbs / hbm,
                          "frac_of_8000": step_gbs / 8000.0},
        "concurrent_phases": list(concurrent),
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items() if v[1]},
        "profiled_ms_per_step": profiled_ms / args.steps,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "e2e": e2e,
        "graph_replay": graph,
        "counts_per_step": {"inserted": inserted, "deleted": deleted},
        "latency": {"p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
                    "max_ms": float(max(step_ms)), "samples": len(step_ms),
                    "of": "one step (the 10M insert, 1M queries, 10M delete), device time per step"},
        "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "delete_compaction_heavy": heavy,
    }
    g.close()
    return res, (base, upd, qry)


def hub_record(args, dev, base, upd, qry, plain):
    """The same step on a graph whose hubs hold their blocks in runs of
    2^s blocks (a per-vertex block size): steps timed as in the main
    record, the per-kernel phases of a second pass, and the compaction-heavy
    delete; counts must equal the plain graph's."""
    import torch
    import paper_2306_08252_gb300 as gv
    rs = args.hub_shift
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    d_bs, d_bd = t(base[0]), t(base[1])
    d_s, d_d = t(upd[0]), t(upd[1])
    d_qs, d_qd = t(qry[0]), t(qry[1])
    d_out = torch.zeros(args.queries, dtype=torch.uint8, device=dev)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def make():
        g = gv.Graph(1 << SCALE, block_capacity=C, pool_bytes=POOL_BYTES, hub_shift=rs)
        g.reserve(max(args.batch, BASE_EDGES))
        g.bulk_build(d_bs, d_bd)
        return g

    g = make()
    st = g.stats()
    deg, _ = g.degrees()
    d64 = deg.astype(np.int64)
    hub = d64 >= (C << rs)  # every vertex's first allocation was the bulk build
    owned_plain = int(((d64 + C - 1) // C).sum())

    def step():
        g.insert_edges(d_s, d_d, counts[:2])
        g.query_edges(d_qs, d_qd, d_out)
        g.delete_edges(d_s, d_d, counts[2:])

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    assert g.sync() == 0
    assert (int(counts[0]), int(counts[2])) == (plain["inserted"], plain["deleted"])
    steps = max(args.steps // 2, 5)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    g.profile_read()
    g.profile(True)
    for i in range(steps):
        flush.fill_(i & 0xFF)
        step()
    torch.cuda.synchronize()
    g.profile(False)
    phases = {k: v[0] / steps for k, v in g.profile_read().items() if v[1]}
    assert g.sync() == 0 and g.validate() == 0
    g.close()
    heavy = []
    for r in range(3):
        g2 = make()
        g2.insert_edges(d_s, d_d)
        flush.fill_(r & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g2.delete_edges(d_s, d_d, counts[2:])
        e1.record(stream)
        torch.cuda.synchronize()
        heavy.append(e0.elapsed_time(e1))
        assert int(counts[2]) == plain["heavy_deleted"] and g2.sync() == 0
        g2.close()
    step_ms = statistics.median(ms)
    hv = statistics.median(heavy)
    keys = ("delete.mark", "delete.mark_tiny", "delete.move", "query.mark", "insert.link", "insert.scatter")
    return {"hub_shift": rs, "hub_degree": C << rs, "run_blocks": 1 << rs,
            "hub_vertices": int(hub.sum()), "hub_entries_share": float(d64[hub].sum() / max(d64.sum(), 1)),
            "max_tree_height_plain": int(np.ceil(np.log2(max(1, (d64.max() + C - 1) // C)))) + 1,
            "max_tree_height_runs": int(np.ceil(np.log2(max(1, -(-((d64.max() + C - 1) // C) // (1 << rs)))))) + 1,
            "pool_blocks_used_after_build": st["pool_blocks_used"], "blocks_plain_layout": owned_plain,
            "ms_per_step": step_ms, "value": (plain["inserted"] + plain["deleted"]) / (step_ms / 1e3), "unit": UNIT,
            "vs_plain_ms_per_step": plain["p50_ms"], "steps": steps,
            "phases_ms_per_step": {k: phases[k] for k in keys if k in phases},
            "plain_phases_ms_per_step": {k: plain["phases"][k] for k in keys if k in plain["phases"]},
            "delete_compaction_heavy_ms": hv, "plain_delete_compaction_heavy_ms": plain["heavy_ms"],
            "counts_match_plain": True,
            "timer": "CUDA events around each step (median), L2 flushed before each; phases from a second pass"}


def run_batched(args):
    print(json.dumps(batched_record(args.graphs, args.steps, args.warmup, tune=True)), flush=True)
    return 0


# configuration of the short batched record in the default line (the
# autotuner's usual pick for this workload; --workload batched tunes)
BATCHED_FIXED = {"block_capacity": 16, "item_blocks": 16, "dense_shift": 3}


def batched_record(graphs, steps, warmup, tune=True):
    """Many independent RMAT graphs (member sizes log-uniform in 2^10..2^18,
    average degree 8, batches log-uniform in 1..1M): one graph set whose
    insert + delete for all members is captured in one CUDA graph, against
    one graph object per member driven call by call.  A step is every
    member's insert batch then its delete batch; an untimed delete of the
    insert batches restores the state between steps."""
    import torch
    import workloads as W
    import paper_2306_08252_gb300 as gv
    from paper_2306_08252_gb300 import autotune

    torch.cuda.set_device(0)
    members = W.batched_rmat(seed=4, graphs=graphs)
    if tune:
        tuned = autotune.tune_set(members, log=lambda m: print(m, file=sys.stderr))
    else:
        tuned = dict(BATCHED_FIXED, cached=False)
    C, IBk, DS = tuned["block_capacity"], tuned["item_blocks"], tuned["dense_shift"]
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()
    bs, bd, bo = autotune.concat_member_batches(members, "bulk")
    is_, id_, io = autotune.concat_member_batches(members, "insert")
    ds, dd, do = autotune.concat_member_batches(members, "delete")
    updates = int(is_.size + ds.size)
    G = len(members)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # ---- batched: one set, captured
    blocks = (bs.size + 2 * is_.size) // C + sum(m["nv"] for m in members) + 4096
    gs = gv.GraphSet([m["nv"] for m in members], block_capacity=C, pool_bytes=int(blocks * (4 * C + 12) * 1.5),
                     item_blocks=IBk, dense_shift=DS)
    cnt = torch.zeros(2 * G, dtype=torch.int64, device="cuda")
    gs.insert_edges(dev(bs, np.int32), dev(bd, np.int32), dev(bo, np.int64), cnt)
    gs.reserve(max(bs.size, is_.size, ds.size))
    a = (dev(is_, np.int32), dev(id_, np.int32), dev(io, np.int64))
    b = (dev(ds, np.int32), dev(dd, np.int32), dev(do, np.int64))
    ci = torch.zeros(2 * G, dtype=torch.int64, device="cuda")
    cd = torch.zeros(2 * G, dtype=torch.int64, device="cuda")
    cr = torch.zeros(2 * G, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gs.insert_edges(*a, ci)
        gs.delete_edges(*b, cd)
        gs.delete_edges(*a, cr)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    step_g, rest_g = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(step_g, capture_error_mode="relaxed"):
        gs.insert_edges(*a, ci)
        gs.delete_edges(*b, cd)
    with torch.cuda.graph(rest_g, capture_error_mode="relaxed"):
        gs.delete_edges(*a, cr)
    for _ in range(max(warmup, 1)):
        step_g.replay()
        rest_g.replay()
    torch.cuda.synchronize()
    t_b = 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step_g.replay()
        e1.record()
        rest_g.replay()
        torch.cuda.synchronize()
        t_b += e0.elapsed_time(e1)
    assert gs.sync() == 0
    batched_counts = (ci.cpu().numpy().reshape(-1, 2), cd.cpu().numpy().reshape(-1, 2))
    gs.close()
    del step_g, rest_g
    # ---- plain: one graph per member, one launch sequence per call
    plain = []
    for m in members:
        nb_ = (m["bulk"][0].size + 2 * m["insert"][0].size) // C + m["nv"] + 64
        g = gv.Graph(m["nv"], block_capacity=C, pool_bytes=int(nb_ * (4 * C + 12) * 1.5) + (1 << 16),
                     item_blocks=IBk, dense_shift=DS)
        g.bulk_build(dev(m["bulk"][0], np.int32), dev(m["bulk"][1], np.int32))
        plain.append((g, dev(m["insert"][0], np.int32), dev(m["insert"][1], np.int32),
                      dev(m["delete"][0], np.int32), dev(m["delete"][1], np.int32)))
    pc = torch.zeros(2 * G, dtype=torch.int64, device="cuda")
    pd = torch.zeros(2 * G, dtype=torch.int64, device="cuda")

    def plain_step(restore):
        for i, (g, s_, d_, s2, d2) in enumerate(plain):
            if restore:
                g.delete_edges(s_, d_)
            else:
                g.insert_edges(s_, d_, pc[2 * i:2 * i + 2])
                g.delete_edges(s2, d2, pd[2 * i:2 * i + 2])

    for _ in range(max(warmup, 1)):
        plain_step(False)
        plain_step(True)
    torch.cuda.synchronize()
    t_p = 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plain_step(False)
        e1.record()
        torch.cuda.synchronize()
        plain_step(True)
        torch.cuda.synchronize()
        t_p += e0.elapsed_time(e1)
    same = (np.array_equal(pc.cpu().numpy().reshape(-1, 2), batched_counts[0]) and
            np.array_equal(pd.cpu().numpy().reshape(-1, 2), batched_counts[1]))
    for g, *_ in plain:
        g.close()
    vb = steps * updates / (t_b / 1e3)
    vp = steps * updates / (t_p / 1e3)
    res = {"metric": "edge updates/s (batched form: all members in one captured launch sequence)",
           "value": vb, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
           "ms_per_step": t_b / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u32", "data": "synthetic (seeded RMAT members)",
           "config": {"workload": f"{G} RMAT graphs, vertices log-uniform 2^10..2^18, average degree 8, "
                                  f"insert + delete batches log-uniform 1..1M per member",
                      "members": G, "vertices": int(sum(m["nv"] for m in members)), "base_edges": int(bs.size),
                      "updates_per_step": updates, "tuned": {k: tuned[k] for k in ("block_capacity", "item_blocks",
                                                                                      "dense_shift")},
                      "l2": "flushed before every timed step"},
           "plain": {"value": vp, "ms_per_step": t_p / steps,
                     "form": "one graph object per member, insert + delete call per member"},
           "speedup_vs_plain": vb / vp, "counts_match_plain": bool(same),
           "tuned_here": bool(tune and not tuned.get("cached", False))}
    return res


def run_serving(args):
    print(json.dumps(serving_record(args.serve_scale, args.requests, (0.5, 0.7, 0.9),
                                    native=args.serve_loop == "native")), flush=True)
    return 0


def serving_record(scale, requests, loads, native=True):
    """Serving: RMAT 2^24 vertices / 2^28 edges resident on the device;
    requests of mixed kind (40% insert, 40% delete of base edges, 20% query),
    sizes log-uniform in 1..1M, Poisson arrivals at 50%, 70% and 90% of the
    measured saturated capacity (a second stream of the same size and
    mix, every request present at time 0); the first 10% of each stream is
    warm-up.
    Latency = completion observed by the loop - arrival."""
    import torch
    import workloads as W
    import paper_2306_08252_gb300 as gv
    from paper_2306_08252_gb300 import serve

    torch.cuda.set_device(0)
    C = 16
    edges = 1 << (scale + 4)
    t_gen = time.perf_counter()
    bs, bd = W.rmat_pairs(5, 0, edges, scale)
    reqs, gaps = W.serving_requests(5, bs, bd, scale, requests)
    cap_reqs, _ = W.serving_requests(6, bs, bd, scale, requests)
    t_gen = time.perf_counter() - t_gen
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    d_bs, d_bd = dev(bs), dev(bd)
    blocks = edges // C * 2 + (1 << scale) + (1 << 22)
    state = {}

    def fresh():
        """Every measurement starts from the same bulk-built graph (a stream
        of 10,000 requests inserts ~3e8 pairs on top of the base)."""
        if "g" in state:
            state["g"].close()
        g = gv.Graph(1 << scale, block_capacity=C, pool_bytes=int(blocks * (4 * C + 12)), flags=gv.GV_GROW)
        g.bulk_build(d_bs, d_bd)
        assert g.sync() == 0
        state["g"] = g
        return g

    def serve_all(g, rs, realtime):
        """The native loop (gv_serve) or the Python one; (runs, merged)."""
        if native:
            st = serve.serve_native(g, rs, slots=4, merge_pairs=2_000_000, max_reqs=1024, realtime=realtime)
            return st["runs"], st["merged_requests"]
        server = serve.Server(g, C, slots=4, merge_pairs=2_000_000, max_reqs=1024)
        server.run(rs, realtime=realtime)
        return server.runs, server.merged_requests

    # saturated capacity (all requests present at time 0)
    g = fresh()
    crs = [serve.Request(k, a, b, 0.0) for k, a, b in cap_reqs]
    cbuf = serve.pin_requests(crs)  # requests arrive in pinned host memory (registered receive buffers)
    t0 = time.perf_counter()
    serve_all(g, crs, False)
    cap = len(crs) / (time.perf_counter() - t0)
    del crs, cbuf
    levels = []
    for load in loads:
        g = fresh()
        rate = load * cap
        arrivals = np.cumsum(gaps) / rate
        rs = [serve.Request(k, a, b, t) for (k, a, b), t in zip(reqs, arrivals)]
        lbuf = serve.pin_requests(rs)  # freed with the level's requests
        runs, merged = serve_all(g, rs, True)
        skip = len(rs) // 10
        meas = [r for r in rs[skip:] if r.status == gv.GV_OK]
        upd = sum(len(r) for r in meas if r.kind in (serve.INSERT, serve.DELETE))
        span = max(r.done for r in meas) - min(r.arrival for r in meas)
        lat = serve.latency_stats(rs, skip=skip)
        worst = max(meas, key=lambda r: r.done - r.arrival)
        levels.append({"load": load, "rate_req_per_s": rate, "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"],
                       "mean_ms": lat["mean_ms"], "max_ms": lat["max_ms"],
                       "worst": {"arrival_s": worst.arrival - rs[0].arrival, "kind": worst.kind,
                                 "pairs": len(worst)},
                       "updates_per_s": upd / span, "requests": len(rs),
                       "warmup_requests": skip, "runs": runs,
                       "requests_per_run": merged / max(runs, 1),
                       "failed": sum(1 for r in rs if r.status != gv.GV_OK)})
    g = state["g"]
    assert g.sync() == 0
    st = g.stats()
    g.close()
    res = {"metric": "serving: p50/p99 latency and edge updates/s under Poisson load",
           "value": levels[-1]["updates_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic (seeded RMAT graph and request stream)",
           "config": {"workload": f"RMAT scale {scale} ({1 << scale} vertices, {edges} edges), C={C}; "
                                  f"{requests} requests, 40/40/20 insert/delete/query, sizes log-uniform 1..1M",
                      "slots": 4, "merge_pairs": 2_000_000, "generation_s": t_gen,
                      "requests_in": "pinned host memory, uploaded straight from each request",
                      "loop": "native (gv_serve)" if native else "python (serve.Server)"},
           "capacity_req_per_s": cap, "levels": levels, "final_edges": st["num_edges"],
           "final_pool_bytes": st["pool_bytes"]}
    return res


# ------------------------------------------------------- per-row sweep

def run_rows(args):
    """Each step of the path timed on its own with its algorithmic bytes:
    create, bulk build, insert and delete at batch sizes 1K..10M, queries,
    neighbours (RMAT 2^20 / 16M), vertex insert and delete (uniform 2^22 /
    16M).  Device time by CUDA events on the call stream, median of the
    repeats, L2 flushed before each timed call; restores are untimed."""
    import torch
    import paper_2306_08252_gb300 as gv
    import workloads as W

    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    reps = max(args.steps, 10)  # median of at least 10 repeats after a warm-up call
    rows = []

    def timed(fn, pre=None, post=None, n=reps):
        ms = []
        for i in range(n + 1):
            if pre:
                pre()
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i:
                ms.append(e0.elapsed_time(e1))
            if post:
                post()
        return float(statistics.median(ms))

    def row(name, what, units, unit_name, ms, nbytes, **extra):
        gbs = nbytes / (ms / 1e3) / 1e9
        r = {"row": name, "what": what, "units": units, "ms": ms, "rate": units / (ms / 1e3),
             "rate_unit": unit_name + "/s", "algorithmic_bytes": int(nbytes), "achieved_gbs": gbs,
             "frac_of_measured_hbm": gbs / hbm}
        r.update(extra)
        rows.append(r)
        print(json.dumps(r), file=sys.stderr, flush=True)

    nv = 1 << SCALE
    (bs, bd), (us, ud), (qs, qd) = workload(BATCH, QUERIES)
    d_bs, d_bd = t(bs), t(bd)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")

    # a1: create (pool + dictionary); host wall clock, allocation included
    ct = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES)
        g.sync()
        ct.append((time.perf_counter() - t0) * 1e3)
        st = g.stats()
        g.close()
    P = st["pool_blocks"]
    row("a1", "create: dictionary, sentinels, pool and edge queue", nv, "vertices", float(statistics.median(ct)),
        17 * st["vertex_capacity"] + 4 * P, timer="host wall clock (allocation included)")

    # a5: bulk build of the 16M-edge graph
    holder = {}

    def mk():
        if "g" in holder:
            holder["g"].close()
        holder["g"] = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES)
        holder["g"].reserve(max(BATCH, BASE_EDGES))
        torch.cuda.synchronize()

    ms = timed(lambda: holder["g"].bulk_build(d_bs, d_bd, cnt), pre=mk)
    row("a5", "bulk build", bs.size, "edges", ms, 12 * bs.size + 16 * nv)

    # f4 (memory footprint, the paper's Table 5): device memory of the
    # structure after the bulk build, and after one insert batch of 100K / 1M
    # / 10M pairs on top of it (fresh graph each): the library's own
    # allocations, the part of the pool in use, and the drop of free device
    # memory reported by the driver (which includes the whole pool
    # reservation)
    fp = []
    batches = {B: (t(us[:B]), t(ud[:B])) for B in (100_000, 1_000_000, 10_000_000)}
    for B in (0, 100_000, 1_000_000, 10_000_000):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        gf = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES)
        gf.bulk_build(d_bs, d_bd, cnt)
        if B:
            gf.insert_edges(batches[B][0], batches[B][1], cnt)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        st = gf.stats()
        used = st["pool_blocks_used"] * (4 * C + 12)
        fp.append({"batch": B or "bulk only", "entries": st["num_edges"], "pool_blocks_used": st["pool_blocks_used"],
                   "pool_in_use_bytes": used, "bytes_per_entry": used / max(st["num_edges"], 1),
                   "library_device_bytes": st["device_bytes"], "pool_reserved_bytes": st["pool_bytes"],
                   "driver_free_drop_bytes": free0 - free1})
        gf.close()
    del batches
    rows.append({"row": "f4-footprint", "what": "device memory after bulk build (+ one insert batch), C=16, "
                 "2 GiB pool", "footprint": fp})
    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    g = holder["g"]
    deg0, _ = g.degrees()
    deg0 = deg0.astype(np.int64)

    # a2-a4 / a6: insert and delete sweeps
    for B in (1_000, 10_000, 100_000, 1_000_000, 10_000_000):
        s, d = t(us[:B]), t(ud[:B])
        srcs = np.unique(us[:B])
        st0 = g.stats()
        ms_i = timed(lambda: g.insert_edges(s, d, cnt), post=lambda: g.delete_edges(s, d, cnt))
        g.insert_edges(s, d, cnt)
        torch.cuda.synchronize()
        st1 = g.stats()
        newb = st1["pool_blocks_used"] - st0["pool_blocks_used"]
        deg1, _ = g.degrees()
        g.delete_edges(s, d, cnt)
        ms_d = timed(lambda: g.delete_edges(s, d, cnt), pre=lambda: g.insert_edges(s, d, cnt))
        row("a2-a4", f"insert batch of {B}", B, "edges", ms_i, 12 * B + 32 * srcs.size + 12 * newb)
        row("a6", f"delete batch of {B}", B, "edges", ms_d,
            8 * B + 4 * int(deg1.astype(np.int64)[srcs].sum()) + 32 * srcs.size + 4 * newb)

    # small batches replayed from CUDA graphs: the same insert and delete
    # calls captured once (scratch sized before the capture), so the launch
    # sequence runs without host launch gaps
    g.reserve(max(BATCH, BASE_EDGES))
    for B in (1_000, 10_000):
        s, d = t(us[:B]), t(ud[:B])
        srcs = np.unique(us[:B])
        ci = torch.zeros(2, dtype=torch.int64, device="cuda")
        cd = torch.zeros(2, dtype=torch.int64, device="cuda")
        g.insert_edges(s, d, ci)
        g.delete_edges(s, d, cd)
        torch.cuda.synchronize()
        exp_i, exp_d = tuple(ci.tolist()), tuple(cd.tolist())
        gi, gdl = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gi, capture_error_mode="relaxed"):
            g.insert_edges(s, d, ci)
        with torch.cuda.graph(gdl, capture_error_mode="relaxed"):
            g.delete_edges(s, d, cd)
        ci.zero_()
        cd.zero_()
        ms_i = timed(gi.replay, post=gdl.replay)
        ms_d = timed(gdl.replay, pre=gi.replay)
        torch.cuda.synchronize()
        assert tuple(ci.tolist()) == exp_i and tuple(cd.tolist()) == exp_d and g.sync() == 0
        row("a2-a4 graph", f"insert batch of {B}, replayed from a CUDA graph", B, "edges", ms_i,
            12 * B + 32 * srcs.size)
        row("a6 graph", f"delete batch of {B}, replayed from a CUDA graph", B, "edges", ms_d,
            8 * B + 4 * int(deg0[srcs].sum() + B) + 32 * srcs.size)
        del gi, gdl

    # a7: 1M queries (half present) on the base graph
    d_qs, d_qd = t(qs), t(qd)
    out = torch.zeros(qs.size, dtype=torch.uint8, device="cuda")
    qsrc = np.unique(qs[qs < nv])
    ms = timed(lambda: g.query_edges(d_qs, d_qd, out))
    row("a7", f"edge-existence queries ({qs.size})", qs.size, "queries", ms, 9 * qs.size + 4 * int(deg0[qsrc].sum()))

    # a8: neighbours of every vertex (CSR of the whole graph)
    vids = torch.arange(nv, dtype=torch.int32, device="cuda")
    offs = torch.zeros(nv + 1, dtype=torch.int64, device="cuda")
    E = int(deg0.sum())
    nbrs = torch.zeros(E, dtype=torch.int32, device="cuda")
    ms = timed(lambda: gv.gv_neighbors(g.handle, vids, offs, nbrs, E, stream.cuda_stream))
    row("a8", f"neighbours of all {nv} vertices", E, "entries", ms, 8 * E + 4 * nv + 16 * nv + 8 * (nv + 1))

    # next rows: BFS from the largest hub, PageRank (10 iterations)
    dist = torch.zeros(nv, dtype=torch.int32, device="cuda")
    src = int(np.argmax(deg0))
    ms = timed(lambda: gv.gv_bfs(g.handle, src, dist, stream.cuda_stream))
    reached = dist.cpu().numpy().view(np.uint32) != 0xFFFFFFFF
    trav = int(deg0[reached].sum())
    row("f2-bfs", f"BFS from vertex {src} ({int(reached.sum())} reached)", trav, "traversed edges", ms,
        8 * trav + 16 * int(reached.sum()) + 4 * nv, timer="CUDA events (one host read per four levels)")
    rank = torch.zeros(nv, dtype=torch.float64, device="cuda")
    iters = 10
    ms = timed(lambda: gv.gv_pagerank(g.handle, iters, 0.85, rank, stream.cuda_stream))
    row("f2-pagerank", f"PageRank, {iters} iterations", iters * E, "edge visits", ms,
        iters * (4 * E + 8 * E + 48 * nv))
    g.close()

    # f2 (shortest paths): the base graph with a 32-bit length per entry,
    # lengths spread over [0, 1000) by a multiplicative hash of the position
    gs = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES, flags=gv.GV_WEIGHTED)
    gs.reserve(BASE_EDGES)
    d_bw = t((np.arange(bs.size, dtype=np.uint64) * 2654435761 % 1000).astype(np.uint32))
    gs.insert_edges_weighted(d_bs, d_bd, d_bw, cnt)
    sdist = torch.zeros(nv, dtype=torch.int64, device="cuda")
    rounds = []
    ms = timed(lambda: rounds.append(gv.gv_sssp(gs.handle, src, sdist, stream.cuda_stream)))
    sreached = sdist.cpu().numpy().view(np.uint64) != np.uint64(0xFFFFFFFFFFFFFFFF)
    strav = int(deg0[sreached].sum())
    row("f2-sssp", f"shortest paths from vertex {src}, lengths in [0, 1000) ({int(sreached.sum())} reached, "
        f"{rounds[-1]} relaxation rounds)", strav, "traversed edges", ms,
        16 * strav + 16 * int(sreached.sum()) + 12 * nv, timer="CUDA events (one host read per four rounds)")
    gs.close()

    # f3 (dynamic edge-block size): re-block the base graph from C to the
    # paper's rule over its degrees (and back, untimed, before each repeat)
    gr = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES)
    gr.bulk_build(d_bs, d_bd, cnt)
    torch.cuda.synchronize()
    used_c = gr.stats()["pool_blocks_used"]
    c_rule = gr.reblock(0)
    used_r = gr.stats()["pool_blocks_used"]
    ms = timed(lambda: gr.reblock(c_rule), pre=lambda: gr.reblock(C))
    E0 = int(deg0.sum())
    P_r = gr.stats()["pool_blocks"]
    c_min = gr.reblock(gv.GV_REBLOCK_MIN_FOOTPRINT)
    used_m = gr.stats()["pool_blocks_used"]
    row("f3-reblock", f"re-block {E0} entries from C={C} to C={c_rule} (the block-size rule over current degrees)",
        E0, "entries", ms, 8 * E0 + 32 * nv + 8 * used_r + 4 * P_r,
        timer="CUDA events (the call synchronises twice: degree totals, slot total)",
        footprint={"entries": E0, "bytes_per_block": "4C slots + 12 links and queue",
                   "at_C": {"C": C, "blocks": used_c, "bytes": used_c * (4 * C + 12)},
                   "at_rule": {"C": c_rule, "blocks": used_r, "bytes": used_r * (4 * c_rule + 12)},
                   "at_min_footprint": {"C": c_min, "blocks": used_m, "bytes": used_m * (4 * c_min + 12)}})
    gr.close()

    # f1: set-semantics insert of the 10M batch (half of it already stored)
    # on a GV_DEDUP graph: membership pass over the stored blocks + insert
    gd = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES, flags=gv.GV_DEDUP)
    gd.reserve(max(BATCH, BASE_EDGES))
    gd.bulk_build(d_bs, d_bd, cnt)
    half = BATCH // 2
    d_h, d_hd = t(us[:half]), t(ud[:half])
    d_s, d_d = t(us), t(ud)
    gd.insert_edges(d_h, d_hd, cnt)  # the first half is stored before every timed call
    torch.cuda.synchronize()
    degd, _ = gd.degrees()
    srcs = np.unique(us)
    ms = timed(lambda: gd.insert_edges(d_s, d_d, cnt), post=lambda: (gd.delete_edges(d_s, d_d, cnt),
                                                                     gd.insert_edges(d_h, d_hd, cnt)))
    gd.insert_edges(d_s, d_d, cnt)
    added = int(cnt[0].item())
    row("f1-dedup", f"set-semantics insert of {BATCH} pairs ({added} new)", BATCH, "edges", ms,
        12 * BATCH + 4 * int(degd.astype(np.int64)[srcs].sum()) + 32 * srcs.size)
    gd.close()

    # f3 (weighted entries): insert the 10M batch with payloads and delete it
    # again on a GV_WEIGHTED graph (payloads move with every compaction)
    gw = gv.Graph(nv, block_capacity=C, pool_bytes=POOL_BYTES, flags=gv.GV_WEIGHTED)
    gw.reserve(max(BATCH, BASE_EDGES))
    gw.bulk_build(d_bs, d_bd, cnt)
    d_w = t(np.arange(BATCH, dtype=np.uint32))
    ms_i = timed(lambda: gw.insert_edges_weighted(d_s, d_d, d_w, cnt), post=lambda: gw.delete_edges(d_s, d_d, cnt))
    gw.insert_edges_weighted(d_s, d_d, d_w, cnt)
    torch.cuda.synchronize()
    degw, _ = gw.degrees()
    gw.delete_edges(d_s, d_d, cnt)
    ms_d = timed(lambda: gw.delete_edges(d_s, d_d, cnt), pre=lambda: gw.insert_edges_weighted(d_s, d_d, d_w, cnt))
    srcs = np.unique(us)
    row("f3-weighted-insert", f"weighted insert of {BATCH} pairs", BATCH, "edges", ms_i, 16 * BATCH + 32 * srcs.size)
    row("f3-weighted-delete", f"delete of the {BATCH} weighted pairs", BATCH, "edges", ms_d,
        8 * BATCH + 8 * int(degw.astype(np.int64)[srcs].sum()) + 32 * srcs.size)
    gw.close()

    # f4: bulk build into a pool of 1/8 of the blocks it needs, grown by
    # GV_GROW in 25% steps (allocation and copies inside the timed call)
    need_blocks = int(((np.bincount(bs, minlength=nv) + C - 1) // C).sum())
    small = (need_blocks // 8) * (4 * C + 12)
    holder3 = {}

    def mk3():
        if "g" in holder3:
            holder3["g"].close()
        holder3["g"] = gv.Graph(nv, block_capacity=C, pool_bytes=small, flags=gv.GV_GROW)
        holder3["g"].reserve(BASE_EDGES)
        torch.cuda.synchronize()

    ms = timed(lambda: holder3["g"].bulk_build(d_bs, d_bd, cnt), pre=mk3)
    grown = holder3["g"].stats()
    row("f4-grow", f"bulk build with pool growth ({small >> 20} MiB -> {grown['pool_bytes'] >> 20} MiB)",
        bs.size, "edges", ms, 12 * bs.size + 16 * nv, pool_bytes_final=grown["pool_bytes"],
        device_bytes=grown["device_bytes"], timer="CUDA events (growth allocations and copies included)")
    holder3["g"].close()

    # a9 / a10 on the uniform 2^22 graph, and its mixed round (1M uniform
    # inserts, then 1M deletes: half stored pairs, half absent ones)
    er = W.er_mixed(3, rounds=1)
    nv2 = er["nv"]
    es, ed = er["bulk"]
    vdel = next(op for op in er["ops"] if op.kind == "vdel").ids
    ins_op = er["ops"][0]
    del_op = er["ops"][1]
    d_es, d_ed = t(es), t(ed)
    d_ids = t(vdel)
    holder2 = {}

    ge = gv.Graph(nv2, block_capacity=4, pool_bytes=1 << 30)
    ge.reserve(max(es.size, 1 << 20))
    ge.bulk_build(d_es, d_ed, cnt)
    d_is, d_id = t(ins_op.src), t(ins_op.dst)
    d_ds, d_dd = t(del_op.src), t(del_op.dst)
    srcs = np.unique(ins_op.src)
    ms = timed(lambda: ge.insert_edges(d_is, d_id, cnt), post=lambda: ge.delete_edges(d_is, d_id, cnt))
    row("a2-a4 ER", f"uniform insert of {ins_op.src.size} pairs (2^22 vertices, 16.7M edges, C=4)",
        ins_op.src.size, "edges", ms, 12 * ins_op.src.size + 32 * srcs.size + 12 * ins_op.src.size // 4)
    ge.close()
    dsrc = np.unique(del_op.src)
    deg_er = np.bincount(es, minlength=nv2).astype(np.int64)
    holder_e = {}

    def mk_e():  # every timed delete starts from the bulk-built graph
        if "g" in holder_e:
            holder_e["g"].close()
        holder_e["g"] = gv.Graph(nv2, block_capacity=4, pool_bytes=1 << 30)
        holder_e["g"].reserve(max(es.size, 1 << 20))
        holder_e["g"].bulk_build(d_es, d_ed, cnt)
        torch.cuda.synchronize()

    ms = timed(lambda: holder_e["g"].delete_edges(d_ds, d_dd, cnt), pre=mk_e)
    holder_e["g"].close()
    row("a6 ER", f"mixed delete of {del_op.src.size} pairs (half stored, half absent)", del_op.src.size, "edges",
        ms, 8 * del_op.src.size + 4 * int(deg_er[dsrc].sum()) + 32 * dsrc.size)

    spare = t(np.setdiff1d(np.arange(nv2 - 64, nv2, dtype=np.uint32), vdel)[:1])

    def mk2(warm=True):
        if "g" in holder2:
            holder2["g"].close()
        holder2["g"] = gv.Graph(nv2, block_capacity=4, pool_bytes=1 << 30)
        holder2["g"].bulk_build(d_es, d_ed, cnt)
        if warm:
            # sizes the per-call scratch (a pass over every live vertex) outside the timed call
            holder2["g"].delete_vertices(spare)
        torch.cuda.synchronize()

    ms = timed(lambda: holder2["g"].delete_vertices(d_ids), pre=mk2)
    E2 = int(es.size)
    row("a10", f"delete {vdel.size} vertices (outgoing and incoming edges)", vdel.size, "vertices", ms,
        4 * E2 + 16 * vdel.size + 16 * nv2 // 8)
    k = 65_536
    newids = torch.zeros(k, dtype=torch.int32, device="cuda")
    ms = timed(lambda: holder2["g"].insert_vertices(k, newids), pre=lambda: mk2(False))
    row("a9", f"insert {k} vertices (dictionary doubling from 2^22)", k, "vertices", ms,
        2 * 17 * nv2 + 17 * k + 4 * k, timer="CUDA events (the dictionary's new allocation included)")
    holder2["g"].close()

    res = {"metric": "per-step device time and algorithmic bytes of each step of the path",
           "value": None, "unit": None, "n_gpus": 1, "steps": reps, "warmup": 1, "higher_is_better": True,
           "dtype": "u32", "data": "synthetic (seeded RMAT and uniform graphs)",
           "config": {"workload": f"RMAT scale {SCALE} / {BASE_EDGES} edges, C={C}; uniform 2^22 / 16777216 "
                                  "edges, C=4 for vertex operations", "l2": "flushed before every timed call"},
           "peak_gbs": hbm, "peak_kind": pk_kind, "rows": rows}
    print(json.dumps(res), flush=True)
    return 0


def main():
    global SCALE, BASE_EDGES
    args = parse()
    if args.scale != SCALE:
        SCALE, BASE_EDGES = args.scale, 16 << args.scale
    if args.workload == "rows":
        return run_rows(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        base, upd, qry = workload(args.batch, args.queries)
        import oracle
        o = oracle.OracleGraph(1 << SCALE)
        o.bulk_build(*base)

        # every step is the whole step of the GPU arm's config: insert the
        # full batch, answer every query, delete the batch
        def ostep():
            a, _ = o.insert_edges(*upd)
            o.query_edges(*qry)
            b, _ = o.delete_edges(*upd)
            return a + b

        for _ in range(args.warmup):
            ostep()
        t0 = time.perf_counter()
        done = 0
        for _ in range(args.steps):
            done += ostep()
        dt = time.perf_counter() - t0
        v = done / dt
        o.close()
        a = argparse.Namespace(**vars(args))
        res = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
               "data": "synthetic", "config": config_dict(a, world),
               "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{args.steps} whole steps after {args.warmup} untimed ones: insert the "
                                          f"{args.batch}-edge batch, {args.queries} queries, delete the batch, "
                                          f"on the full bulk-built graph"},
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(res), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res, (base, upd, qry) = run_ours(args, rank, world, local_rank)
    if world == 1 and args.hub_shift:
        plain = {"inserted": res["counts_per_step"]["inserted"], "deleted": res["counts_per_step"]["deleted"],
                 "p50_ms": res["p50_ms"], "phases": res["phases_ms_per_step"],
                 "heavy_ms": res["delete_compaction_heavy"]["ms"],
                 "heavy_deleted": res["delete_compaction_heavy"]["deleted"]}
        res["hub_runs"] = hub_record(args, torch.device("cuda", local_rank), base, upd, qry, plain)
    if world == 1 and not args.no_batched:
        # the batched form, short: the 256-member workload, 3 steps, the
        # autotuner's usual configuration (no tuning pass)
        b = batched_record(256, 3, 1, tune=False)
        res["batched"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "config",
                                            "plain", "speedup_vs_plain", "counts_match_plain")}
        res["batched_speedup_vs_plain"] = b["speedup_vs_plain"]
    if world == 1 and not args.no_serving:
        # the serving loop, short: RMAT scale 20 resident, 4,000 requests
        # (the p99 then rests on 40 of them), Poisson arrivals at 70% of the
        # measured capacity
        sv = serving_record(20, 4000, (0.7,))
        lv = sv["levels"][0]
        res["serving"] = {"metric": sv["metric"], "config": sv["config"], "capacity_req_per_s": sv["capacity_req_per_s"],
                          "load": lv["load"], "p50_ms": lv["p50_ms"], "p99_ms": lv["p99_ms"], "max_ms": lv["max_ms"],
                          "updates_per_s": lv["updates_per_s"], "requests_per_run": lv["requests_per_run"],
                          "failed": lv["failed"],
                          "note": "short form of --workload serving (RMAT scale 24, three load levels)"}
        res["serving_p99_ms"] = lv["p99_ms"]
    if rank == 0 and not args.no_cpu_baseline:
        v, steps, secs = oracle_sample_rate(base, upd, qry)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{steps} whole steps after one untimed step: insert the {args.batch}-edge "
                                         f"batch, {args.queries} queries, delete the batch, on the full bulk-built "
                                         f"graph ({secs:.1f} s timed)"}
        cores = host_cores()
        v, steps, secs = parallel_cpu_rate(base, upd, qry, cores)
        res["cpu_parallel"] = {"value": v, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
                               "kind": "the oracle's sorted-vector algorithm, OpenMP over source buckets",
                               "sample": f"{steps} full steps (insert the 10M batch, 1M queries, delete the batch) "
                                         f"on the full bulk-built graph ({secs:.1f} s)"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

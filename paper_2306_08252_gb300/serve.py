"""Continuous-batching request loop over one device-resident graph.

Requests (insert / delete / query batches of (src, dst) pairs) arrive over
time.  The loop admits every request that has arrived while earlier work is
still on the GPU, and forms "runs" from the head of the queue in arrival
order:

* consecutive insert requests merge into one segmented insert (the library
  returns per-request {inserted, rejected}; multiset inserts commute, so each
  request's result is the one it would get alone, in order);
* consecutive query requests merge into one query batch (each request gets
  its slice of the answers; no update separates them);
* consecutive delete requests merge into one segmented delete (the library
  removes the union of their pairs, which is what the requests do one after
  another, and credits each removed entry to the first request that names
  its pair, which is what that request alone would have removed).

Up to `slots` runs are in flight, each with its own pinned host and device
buffers, on three streams ordered by events: the host-to-device copy of its
pairs on an upload stream (straight from each request's own memory when the
request lives in pinned host memory -- `pin_requests` -- else packed into
the run's pinned buffer first), the library call on the compute stream (after
the copy's event), the device-to-host copy of its results on a download
stream (after the call's event), then the run's completion event.  So one
run's upload and another's download overlap the kernels of the run between
them.  The calls themselves stay in arrival order on one stream: every call
on a graph uses the graph's shared per-call device scratch, and update runs
change the graph the next run reads.  An insert run is admitted
only if its worst-case block demand (ceil(B / C) + B new blocks for B pairs)
fits the free blocks of the pool as last known; otherwise the loop drains
the in-flight runs, refreshes the pool counters and tries again.  A run that
still does not fit fails with an out-of-memory result, unless the graph was
created with GV_GROW: then it is launched and the library grows the pool
before inserting.

Latency of a request = completion (its run's event observed by the loop)
minus its arrival time.
"""
from __future__ import annotations

import collections
import gc
import time

import numpy as np

from . import graphvine as gv

INSERT, DELETE, QUERY = "insert", "delete", "query"


class Request:
    __slots__ = ("kind", "src", "dst", "arrival", "result", "done", "status", "t_src", "t_dst")

    def __init__(self, kind, src, dst, arrival=0.0):
        self.kind = kind
        self.src = np.ascontiguousarray(src, dtype=np.uint32)
        self.dst = np.ascontiguousarray(dst, dtype=np.uint32)
        self.arrival = float(arrival)
        self.result = None
        self.done = None
        self.status = gv.GV_OK
        self.t_src = self.t_dst = None  # pinned int32 views (pin_requests)

    def __len__(self):
        return int(self.src.size)


def pin_requests(reqs):
    """Moves the pairs of `reqs` into one pinned host buffer (as a server
    that receives requests into registered buffers has them), so that the
    loop uploads each request straight from its own memory with no packing
    copy on the host.  Returns the buffer (keep it alive while the requests
    are served)."""
    import torch
    total = sum(len(r) for r in reqs)
    buf = torch.empty(max(2 * total, 1), dtype=torch.int32).pin_memory()
    view = buf.numpy()
    a = 0
    for r in reqs:
        n = len(r)
        view[a:a + n] = r.src.view(np.int32)
        view[a + n:a + 2 * n] = r.dst.view(np.int32)
        r.t_src, r.t_dst = buf[a:a + n], buf[a + n:a + 2 * n]
        r.src, r.dst = view[a:a + n].view(np.uint32), view[a + n:a + 2 * n].view(np.uint32)
        a += 2 * n
    return buf


class _Slot:
    def __init__(self, cap, max_reqs, torch):
        self.d_src = torch.empty(cap, dtype=torch.int32, device="cuda")
        self.d_dst = torch.empty(cap, dtype=torch.int32, device="cuda")
        self.d_off = torch.empty(max_reqs + 1, dtype=torch.int64, device="cuda")
        self.d_cnt = torch.empty(2 * max_reqs, dtype=torch.int64, device="cuda")
        self.d_out = torch.empty(cap, dtype=torch.uint8, device="cuda")
        self.h_src = torch.empty(cap, dtype=torch.int32).pin_memory()
        self.h_dst = torch.empty(cap, dtype=torch.int32).pin_memory()
        self.h_off = torch.empty(max_reqs + 1, dtype=torch.int64).pin_memory()
        self.h_cnt = torch.empty(2 * max_reqs, dtype=torch.int64).pin_memory()
        self.h_out = torch.empty(cap, dtype=torch.uint8).pin_memory()
        self.copied = torch.cuda.Event()    # pairs on the device (upload stream)
        self.computed = torch.cuda.Event()  # the library call done (compute stream)
        self.event = torch.cuda.Event()     # results on the host (download stream)
        self.reqs = []
        self.kind = None
        self.n = 0
        self.blocks = 0


class Server:
    """Continuous batching over `graph` (a paper_2306_08252_gb300.Graph)."""

    def __init__(self, graph, block_capacity, slots=4, merge_pairs=2_000_000, max_reqs=1024):
        import torch
        self.torch = torch
        self.g = graph
        self.C = int(block_capacity)
        self.cap = int(merge_pairs)
        self.max_reqs = int(max_reqs)
        self.stream = torch.cuda.Stream()
        self.up = torch.cuda.Stream()
        self.down = torch.cuda.Stream()
        self.slots = [_Slot(self.cap, self.max_reqs, torch) for _ in range(slots)]
        self.free_slots = collections.deque(self.slots)
        self.inflight = collections.deque()
        graph.reserve(self.cap)
        st = graph.stats()
        self.grow = bool(st["flags"] & gv.GV_GROW)
        self.nv = st["num_vertices"]
        self.free_blocks = st["pool_blocks_free"]
        self.reserved_blocks = 0
        self.runs = 0
        self.merged_requests = 0
        self.completed = 0

    # ------------------------------------------------------------ dispatch
    def _demand(self, n):
        return -(-n // self.C) + min(n, self.nv)

    def _form_run(self, queue):
        head = queue[0]
        if len(head) > self.cap:
            raise ValueError(f"request of {len(head)} pairs exceeds the merge capacity {self.cap}")
        run, n = [], 0
        while queue and queue[0].kind == head.kind and len(run) < self.max_reqs and n + len(queue[0]) <= self.cap:
            r = queue.popleft()
            run.append(r)
            n += len(r)
        return run

    def _launch(self, slot, run):
        torch = self.torch
        slot.reqs = run
        slot.kind = run[0].kind
        offs = np.zeros(len(run) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([len(r) for r in run])
        n = int(offs[-1])
        slot.n = n
        pinned = all(r.t_src is not None for r in run)
        if not pinned:
            hs = slot.h_src.numpy()
            hd = slot.h_dst.numpy()
            for r, a in zip(run, offs[:-1]):
                hs[a:a + len(r)] = r.src.view(np.int32)
                hd[a:a + len(r)] = r.dst.view(np.int32)
        slot.h_off.numpy()[:len(run) + 1] = offs
        k = len(run)
        with torch.cuda.stream(self.up):
            if n and pinned:
                for r, a in zip(run, offs[:-1]):
                    if len(r):
                        slot.d_src[a:a + len(r)].copy_(r.t_src, non_blocking=True)
                        slot.d_dst[a:a + len(r)].copy_(r.t_dst, non_blocking=True)
            elif n:
                slot.d_src[:n].copy_(slot.h_src[:n], non_blocking=True)
                slot.d_dst[:n].copy_(slot.h_dst[:n], non_blocking=True)
            if slot.kind != QUERY:
                slot.d_off[:k + 1].copy_(slot.h_off[:k + 1], non_blocking=True)
            slot.copied.record(self.up)
        self.stream.wait_event(slot.copied)
        s = self.stream.cuda_stream
        if slot.kind == INSERT:
            gv.gv_insert_edges_segmented(self.g.handle, slot.d_src[:n], slot.d_dst[:n],
                                         slot.d_off[:k + 1], k, slot.d_cnt, s)
        elif slot.kind == DELETE:
            gv.gv_delete_edges_segmented(self.g.handle, slot.d_src[:n], slot.d_dst[:n],
                                         slot.d_off[:k + 1], k, slot.d_cnt, s)
        else:
            gv.gv_query_edges(self.g.handle, slot.d_src[:n], slot.d_dst[:n], slot.d_out[:max(n, 1)], s)
        slot.computed.record(self.stream)
        self.down.wait_event(slot.computed)
        with torch.cuda.stream(self.down):
            if slot.kind != QUERY:
                slot.h_cnt[:2 * k].copy_(slot.d_cnt[:2 * k], non_blocking=True)
            elif n:
                slot.h_out[:n].copy_(slot.d_out[:n], non_blocking=True)
            slot.event.record(self.down)
        self.inflight.append(slot)
        self.runs += 1
        self.merged_requests += len(run)

    def _finish(self, slot, now):
        run = slot.reqs
        self.completed += len(run)
        if slot.kind in (INSERT, DELETE):
            cnt = slot.h_cnt.numpy()[:2 * len(run)].reshape(-1, 2)
            for r, c in zip(run, cnt):
                r.result = (int(c[0]), int(c[1]))
            if slot.kind == INSERT:
                self.reserved_blocks -= slot.blocks
                self.free_blocks -= slot.blocks  # conservative until the next refresh
        else:
            out = slot.h_out.numpy()[:slot.n]
            a = 0
            for r in run:
                r.result = out[a:a + len(r)].copy()
                a += len(r)
        for r in run:
            r.done = now
        slot.reqs = []
        self.free_slots.append(slot)

    def _refresh_pool(self):
        self.stream.synchronize()
        self.down.synchronize()
        st = self.g.stats()
        self.free_blocks = st["pool_blocks_free"]
        self.reserved_blocks = 0

    # ----------------------------------------------------------------- run
    def run(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival, seconds from the start).
        realtime=False treats every request as arrived at time 0 (saturated
        capacity measurement)."""
        reqs = list(requests)
        # no cyclic garbage collection while serving: a full collection over
        # the request objects stalls the loop for tens of milliseconds
        gc_was_on = gc.isenabled()
        gc.disable()
        try:
            return self._run(reqs, realtime)
        finally:
            if gc_was_on:
                gc.enable()

    def _run(self, reqs, realtime):
        q = collections.deque()
        i = 0
        t0 = time.perf_counter()
        target = self.completed + len(reqs)
        while self.completed < target:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                reqs[i].arrival = reqs[i].arrival if realtime else 0.0
                q.append(reqs[i])
                i += 1
            progressed = False
            while self.inflight and self.inflight[0].event.query():
                self._finish(self.inflight.popleft(), time.perf_counter() - t0)
                progressed = True
            while q and self.free_slots:
                run = self._form_run(q)
                if run[0].kind == INSERT:
                    need = self._demand(sum(len(r) for r in run))
                    if need > self.free_blocks - self.reserved_blocks:
                        while self.inflight:
                            self.inflight[0].event.synchronize()
                            self._finish(self.inflight.popleft(), time.perf_counter() - t0)
                        self._refresh_pool()
                        if need > self.free_blocks and not self.grow:
                            for r in run:
                                r.status = gv.GV_ERR_OUT_OF_MEMORY
                                r.done = time.perf_counter() - t0
                            self.completed += len(run)
                            progressed = True
                            continue
                    slot = self.free_slots.popleft()
                    slot.blocks = need
                    self.reserved_blocks += need
                else:
                    slot = self.free_slots.popleft()
                    slot.blocks = 0
                self._launch(slot, run)
                progressed = True
            if not progressed:
                if i < len(reqs) and not self.inflight and not q and realtime:
                    wait = reqs[i].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.0005))
        self.stream.synchronize()
        self.down.synchronize()
        return reqs


def latency_stats(reqs, skip=0):
    lat = np.array([r.done - r.arrival for r in reqs[skip:] if r.status == gv.GV_OK])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}


def serve_native(graph, requests, slots=4, merge_pairs=2_000_000, max_reqs=1024, realtime=True):
    """The same loop in native code (gv_serve): the C ABI runs admission,
    run forming, the three streams and the completion polling; this wrapper
    only builds the request array and copies the results back into the
    Request objects (result, done, status).  `done` and `arrival` share the
    loop's clock (seconds after the call started); with realtime=False every
    arrival counts as 0.  Returns {"runs", "merged_requests"}."""
    import ctypes
    reqs = list(requests)
    arr = (gv.gv_serve_request * max(len(reqs), 1))()
    answers = []
    code = {INSERT: 0, DELETE: 1, QUERY: 2}
    for i, r in enumerate(reqs):
        q = arr[i]
        q.kind = code[r.kind]
        q.n = len(r)
        q.src = r.src.ctypes.data if len(r) else None
        q.dst = r.dst.ctypes.data if len(r) else None
        if r.kind == QUERY:
            a = np.zeros(max(len(r), 1), dtype=np.uint8)
            answers.append(a)
            q.answers = a.ctypes.data
        else:
            answers.append(None)
        if not realtime:
            r.arrival = 0.0
        q.arrival = r.arrival
    cfg = gv.gv_serve_config(slots, max_reqs, merge_pairs, 1 if realtime else 0, 0)
    stats = (ctypes.c_uint64 * 2)()
    gv.check(gv.load().gv_serve(graph.handle, arr, len(reqs), ctypes.byref(cfg), stats, graph._s()), "gv_serve")
    for i, r in enumerate(reqs):
        q = arr[i]
        r.status = int(q.status)
        r.done = float(q.done)
        if r.kind == QUERY:
            r.result = answers[i][:len(r)]
        else:
            r.result = (int(q.counts[0]), int(q.counts[1]))
    return {"runs": int(stats[0]), "merged_requests": int(stats[1])}


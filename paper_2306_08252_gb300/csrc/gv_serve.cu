// gv_serve.cu -- the continuous-batching request loop, native (gv_serve).
//
// Host code only: the loop drives the library's own batch calls.  Requests
// (insert, delete or query batches of (src, dst) pairs, each with an
// arrival time) are admitted once they have arrived; runs are formed from
// the head of the queue in arrival order, each of consecutive requests of
// one kind (at most max_reqs requests and merge_pairs pairs):
//   * inserts merge into one segmented insert (per-request {inserted,
//     rejected}; multiset inserts commute, so each request gets what it would
//     get alone, in order);
//   * deletes merge into one segmented delete (the union of their pairs goes,
//     each removed entry credited to the first request naming its pair: what
//     the requests remove one after another);
//   * queries merge into one query batch (no update separates them).
// Up to `slots` runs are in flight, each with its own device buffers, on
// three streams ordered by events: the upload of its pairs on a stream of the
// loop's own (straight from each request's memory when that is pinned host
// memory, else packed into the slot's pinned staging first), the library call
// on the caller's stream, and the download of its results on a second stream
// of the loop's own, after which the run's completion event fires.
// Calls stay in arrival order on the caller's stream (every call on a
// graph shares the graph's per-call scratch, and updates change what the
// next run reads).  An insert run is admitted only while its worst-case block
// demand fits the free blocks as last read; otherwise the loop drains the
// runs in flight, reads the pool again and retries once; a run that still
// does not fit fails with GV_ERR_OUT_OF_MEMORY unless the graph grows its
// pool (GV_GROW).
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "graphvine.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
    uint32_t *d_src = nullptr, *d_dst = nullptr;
    uint64_t *d_off = nullptr, *d_cnt = nullptr;
    uint8_t *d_out = nullptr;
    uint32_t *h_src = nullptr, *h_dst = nullptr;  // pinned staging of pageable requests
    uint64_t *h_off = nullptr, *h_cnt = nullptr;
    uint8_t *h_out = nullptr;
    cudaEvent_t copied = nullptr, computed = nullptr, done = nullptr;
    std::vector<uint64_t> reqs;  // request indices of the run in flight
    uint32_t kind = 0;
    uint64_t n = 0, blocks = 0;
};

bool pinned_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

void free_slot(Slot &s) {
    cudaFree(s.d_src);
    cudaFree(s.d_dst);
    cudaFree(s.d_off);
    cudaFree(s.d_cnt);
    cudaFree(s.d_out);
    cudaFreeHost(s.h_src);
    cudaFreeHost(s.h_dst);
    cudaFreeHost(s.h_off);
    cudaFreeHost(s.h_cnt);
    cudaFreeHost(s.h_out);
    if (s.copied) cudaEventDestroy(s.copied);
    if (s.computed) cudaEventDestroy(s.computed);
    if (s.done) cudaEventDestroy(s.done);
    s = Slot{};
}

bool alloc_slot(Slot &s, uint64_t cap, uint32_t max_reqs) {
    bool ok = cudaMalloc(&s.d_src, cap * 4) == cudaSuccess && cudaMalloc(&s.d_dst, cap * 4) == cudaSuccess &&
              cudaMalloc(&s.d_off, (max_reqs + 1) * 8ull) == cudaSuccess &&
              cudaMalloc(&s.d_cnt, 2ull * max_reqs * 8) == cudaSuccess && cudaMalloc(&s.d_out, cap) == cudaSuccess &&
              cudaMallocHost(&s.h_src, cap * 4) == cudaSuccess && cudaMallocHost(&s.h_dst, cap * 4) == cudaSuccess &&
              cudaMallocHost(&s.h_off, (max_reqs + 1) * 8ull) == cudaSuccess &&
              cudaMallocHost(&s.h_cnt, 2ull * max_reqs * 8) == cudaSuccess &&
              cudaMallocHost(&s.h_out, cap) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
}

struct Loop {
    gv_graph *g;
    gv_serve_request *r;
    uint64_t nr;
    gv_serve_config cfg;
    std::vector<uint8_t> pinned;      // per request: pairs in pinned host memory
    std::vector<uint8_t> pinned_ans;  // per query: answer buffer in pinned host memory
    std::vector<Slot> slots;
    std::deque<uint32_t> free_slots, inflight;
    std::deque<uint64_t> queue;
    cudaStream_t comp = nullptr, up = nullptr, down = nullptr;
    Clock::time_point t0;
    uint64_t C = 0, nv = 0, rs = 0, free_blocks = 0, reserved = 0;
    bool grow = false;
    uint64_t completed = 0, runs = 0, merged = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    gv_status refresh_pool() {
        if (cudaStreamSynchronize(comp) != cudaSuccess || cudaStreamSynchronize(down) != cudaSuccess)
            return GV_ERR_CUDA;
        gv_stats_t st;
        const gv_status e = gv_stats(g, &st);
        if (e != GV_OK) return e;
        free_blocks = st.pool_blocks_free;
        reserved = 0;
        return GV_OK;
    }

    // worst-case blocks of an insert of n pairs: ceil(n / C) + one partial
    // block per touched source (a whole run of 2^rs blocks with hub runs)
    uint64_t demand(uint64_t n) const { return (n + C - 1) / C + (std::min<uint64_t>(n, nv) << rs); }

    void form_run(std::vector<uint64_t> &run) {
        const uint32_t kind = r[queue.front()].kind;
        uint64_t n = 0;
        while (!queue.empty() && r[queue.front()].kind == kind && run.size() < cfg.max_reqs &&
               n + r[queue.front()].n <= cfg.merge_pairs) {
            n += r[queue.front()].n;
            run.push_back(queue.front());
            queue.pop_front();
        }
    }

    gv_status launch(uint32_t si, std::vector<uint64_t> &run) {
        Slot &s = slots[si];
        s.reqs.swap(run);
        s.kind = r[s.reqs[0]].kind;
        const uint32_t k = (uint32_t)s.reqs.size();
        uint64_t a = 0;
        s.h_off[0] = 0;
        for (uint32_t i = 0; i < k; ++i) {
            a += r[s.reqs[i]].n;
            s.h_off[i + 1] = a;
        }
        s.n = a;
        // uploads: each pinned request straight from its memory, the others
        // packed into the slot's pinned staging first
        for (uint32_t i = 0; i < k; ++i) {
            const gv_serve_request &q = r[s.reqs[i]];
            const uint64_t o = s.h_off[i];
            if (!q.n) continue;
            if (pinned[s.reqs[i]]) {
                if (cudaMemcpyAsync(s.d_src + o, q.src, q.n * 4, cudaMemcpyHostToDevice, up) != cudaSuccess ||
                    cudaMemcpyAsync(s.d_dst + o, q.dst, q.n * 4, cudaMemcpyHostToDevice, up) != cudaSuccess)
                    return GV_ERR_CUDA;
            } else {
                std::memcpy(s.h_src + o, q.src, q.n * 4);
                std::memcpy(s.h_dst + o, q.dst, q.n * 4);
                if (cudaMemcpyAsync(s.d_src + o, s.h_src + o, q.n * 4, cudaMemcpyHostToDevice, up) != cudaSuccess ||
                    cudaMemcpyAsync(s.d_dst + o, s.h_dst + o, q.n * 4, cudaMemcpyHostToDevice, up) != cudaSuccess)
                    return GV_ERR_CUDA;
            }
        }
        if (s.kind != GV_SERVE_QUERY &&
            cudaMemcpyAsync(s.d_off, s.h_off, (k + 1) * 8ull, cudaMemcpyHostToDevice, up) != cudaSuccess)
            return GV_ERR_CUDA;
        if (cudaEventRecord(s.copied, up) != cudaSuccess || cudaStreamWaitEvent(comp, s.copied, 0) != cudaSuccess)
            return GV_ERR_CUDA;
        gv_status e = GV_OK;
        if (s.kind == GV_SERVE_INSERT)
            e = gv_insert_edges_segmented(g, s.d_src, s.d_dst, s.n, s.d_off, k, s.d_cnt, comp);
        else if (s.kind == GV_SERVE_DELETE)
            e = gv_delete_edges_segmented(g, s.d_src, s.d_dst, s.n, s.d_off, k, s.d_cnt, comp);
        else if (s.n)
            e = gv_query_edges(g, s.d_src, s.d_dst, s.n, s.d_out, comp);
        if (e != GV_OK) return e;
        if (cudaEventRecord(s.computed, comp) != cudaSuccess || cudaStreamWaitEvent(down, s.computed, 0) != cudaSuccess)
            return GV_ERR_CUDA;
        if (s.kind != GV_SERVE_QUERY) {
            if (cudaMemcpyAsync(s.h_cnt, s.d_cnt, 2ull * k * 8, cudaMemcpyDeviceToHost, down) != cudaSuccess)
                return GV_ERR_CUDA;
        } else {
            // answers straight into each request's buffer when it is pinned
            for (uint32_t i = 0; i < k; ++i) {
                const gv_serve_request &q = r[s.reqs[i]];
                if (!q.n) continue;
                uint8_t *dst = pinned_ans[s.reqs[i]] ? q.answers : s.h_out + s.h_off[i];
                if (cudaMemcpyAsync(dst, s.d_out + s.h_off[i], q.n, cudaMemcpyDeviceToHost, down) != cudaSuccess)
                    return GV_ERR_CUDA;
            }
        }
        if (cudaEventRecord(s.done, down) != cudaSuccess) return GV_ERR_CUDA;
        inflight.push_back(si);
        ++runs;
        merged += k;
        return GV_OK;
    }

    void finish(uint32_t si) {
        Slot &s = slots[si];
        const double t = now();
        for (uint32_t i = 0; i < s.reqs.size(); ++i) {
            gv_serve_request &q = r[s.reqs[i]];
            if (s.kind != GV_SERVE_QUERY) {
                q.counts[0] = s.h_cnt[2 * i];
                q.counts[1] = s.h_cnt[2 * i + 1];
            } else if (q.n && !pinned_ans[s.reqs[i]]) {
                std::memcpy(q.answers, s.h_out + s.h_off[i], q.n);
            }
            q.done = t;
            q.status = GV_OK;
        }
        if (s.kind == GV_SERVE_INSERT) {
            reserved -= s.blocks;
            free_blocks = free_blocks > s.blocks ? free_blocks - s.blocks : 0;  // conservative until a refresh
        }
        completed += s.reqs.size();
        s.reqs.clear();
        free_slots.push_back(si);
    }

    gv_status drain() {
        while (!inflight.empty()) {
            const uint32_t si = inflight.front();
            if (cudaEventSynchronize(slots[si].done) != cudaSuccess) return GV_ERR_CUDA;
            inflight.pop_front();
            finish(si);
        }
        return GV_OK;
    }

    gv_status run() {
        t0 = Clock::now();
        uint64_t i = 0;
        while (completed < nr) {
            const double t = now();
            while (i < nr && (!cfg.realtime || r[i].arrival <= t)) queue.push_back(i++);
            bool progressed = false;
            while (!inflight.empty()) {
                const cudaError_t q = cudaEventQuery(slots[inflight.front()].done);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) return GV_ERR_CUDA;
                const uint32_t si = inflight.front();
                inflight.pop_front();
                finish(si);
                progressed = true;
            }
            while (!queue.empty() && !free_slots.empty()) {
                if (r[queue.front()].n > cfg.merge_pairs) return GV_ERR_INVALID_ARG;
                std::vector<uint64_t> run;
                form_run(run);
                uint64_t need = 0;
                if (r[run[0]].kind == GV_SERVE_INSERT) {
                    uint64_t n = 0;
                    for (uint64_t x : run) n += r[x].n;
                    need = demand(n);
                    if (need + reserved > free_blocks) {
                        gv_status e = drain();
                        if (e == GV_OK) e = refresh_pool();
                        if (e != GV_OK) return e;
                        if (need > free_blocks && !grow) {
                            const double tf = now();
                            for (uint64_t x : run) {
                                r[x].status = GV_ERR_OUT_OF_MEMORY;
                                r[x].counts[0] = r[x].counts[1] = 0;
                                r[x].done = tf;
                            }
                            completed += run.size();
                            progressed = true;
                            continue;
                        }
                    }
                }
                const uint32_t si = free_slots.front();
                free_slots.pop_front();
                slots[si].blocks = need;
                reserved += need;
                const gv_status e = launch(si, run);
                if (e != GV_OK) return e;
                progressed = true;
            }
            if (!progressed && inflight.empty() && queue.empty() && i < nr && cfg.realtime) {
                // idle until the next arrival (at most half a millisecond a nap)
                const double wait = r[i].arrival - now();
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.0005)));
            }
        }
        if (cudaStreamSynchronize(comp) != cudaSuccess || cudaStreamSynchronize(down) != cudaSuccess)
            return GV_ERR_CUDA;
        return GV_OK;
    }
};

}  // namespace

extern "C" gv_status gv_serve(gv_graph *g, gv_serve_request *reqs, uint64_t n_reqs, const gv_serve_config *cfg,
                              uint64_t *h_stats, void *stream) {
    if (!g || (n_reqs && !reqs)) return GV_ERR_INVALID_ARG;
    gv_serve_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (!c.slots) c.slots = 4;
    if (!c.max_reqs) c.max_reqs = 1024;
    if (!c.merge_pairs) c.merge_pairs = 2000000;
    if (c.slots > 64 || c.max_reqs > 1024 || c.merge_pairs > (1ull << 32)) return GV_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < n_reqs; ++i) {
        const gv_serve_request &q = reqs[i];
        if (q.kind > GV_SERVE_QUERY || q.n > c.merge_pairs) return GV_ERR_INVALID_ARG;
        if (q.n && (!q.src || !q.dst || (q.kind == GV_SERVE_QUERY && !q.answers))) return GV_ERR_INVALID_ARG;
        if (i && c.realtime && q.arrival < reqs[i - 1].arrival) return GV_ERR_INVALID_ARG;
    }
    gv_stats_t st;
    gv_status e = gv_stats(g, &st);
    if (e != GV_OK) return e;
    e = gv_reserve(g, c.merge_pairs);
    if (e != GV_OK) return e;
    Loop L;
    L.g = g;
    L.r = reqs;
    L.nr = n_reqs;
    L.cfg = c;
    L.C = st.block_capacity ? st.block_capacity : 4;
    L.nv = st.num_vertices;
    L.rs = st.hub_shift;
    L.free_blocks = st.pool_blocks_free;
    L.grow = (st.flags & GV_GROW) != 0;
    L.pinned.resize(n_reqs);
    L.pinned_ans.resize(n_reqs);
    for (uint64_t i = 0; i < n_reqs; ++i) {
        L.pinned[i] = pinned_ptr(reqs[i].src) && pinned_ptr(reqs[i].dst);
        L.pinned_ans[i] = reqs[i].kind == GV_SERVE_QUERY && pinned_ptr(reqs[i].answers);
        reqs[i].status = GV_OK;
        reqs[i].done = -1.0;
    }
    L.slots.resize(c.slots);
    // the library calls run on the caller's stream (it stays the graph's
    // stream after the loop); uploads and downloads on two of the loop's own
    L.comp = static_cast<cudaStream_t>(stream);
    bool ok = cudaStreamCreateWithFlags(&L.up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&L.down, cudaStreamNonBlocking) == cudaSuccess;
    for (uint32_t s = 0; ok && s < c.slots; ++s) {
        ok = alloc_slot(L.slots[s], c.merge_pairs ? c.merge_pairs : 1, c.max_reqs);
        L.free_slots.push_back(s);
    }
    e = ok ? L.run() : GV_ERR_OUT_OF_MEMORY;
    if (e != GV_OK) {
        // leave nothing in flight on the library's graph or the slots
        cudaStreamSynchronize(L.comp);
        if (L.up) cudaStreamSynchronize(L.up);
        if (L.down) cudaStreamSynchronize(L.down);
        cudaGetLastError();
    }
    if (h_stats) {
        h_stats[0] = L.runs;
        h_stats[1] = L.merged;
    }
    for (auto &s : L.slots) free_slot(s);
    if (L.up) cudaStreamDestroy(L.up);
    if (L.down) cudaStreamDestroy(L.down);
    return e;
}

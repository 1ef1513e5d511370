// gv_capi.cu -- the extern "C" entry points declared in include/graphvine.h.
//
// Host code only: argument checks, device memory of the graph (dictionary,
// pool, scratch), staging of host arrays, and the launch sequence of each
// operation.  Every step of an operation runs in the kernels of
// gv_kernels.cu / gv_misc.cu; nothing here touches graph data on the host.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/graphvine.h"
#include "gv_launch.h"

using gv::Dev;
using gv::GraphView;
using gv::LaunchCfg;

namespace {

constexpr uint64_t kMaxBatch = 1ull << 29;  // pairs per call (32-bit ranks and arena offsets: 5n words)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Staging {
    DevBuf buf[6];
};

// One staging set for the host inputs of a batch call (sources,
// destinations, payloads) and the events that order it: one per piece
// landed, and one when the call that read it has finished with it.
constexpr int kInSets = 3;
constexpr int kPipePieces = 4;
struct InSet {
    DevBuf src, dst, wts;
    cudaEvent_t piece[kPipePieces] = {};
    cudaEvent_t free_ev = nullptr;
    bool used = false;
};

}  // namespace

struct gv_graph {
    int device = 0;
    int num_sms = 0;
    uint32_t C = 0, IB = 0, flags = 0;
    uint32_t item_blocks_cfg = 0, dense_shift = 3;
    uint32_t nv = 0, vcap = 0;
    unsigned long long P = 0;
    uint64_t pool_bytes_cfg = 0;
    void *pool_mem_cfg = nullptr;
    // pool (one allocation unless caller-owned)
    void *pool_alloc = nullptr;
    uint64_t pool_bytes = 0;
    uint32_t *data = nullptr, *links = nullptr, *queue = nullptr;
    uint32_t *wdata = nullptr;  // per-slot payloads (GV_WEIGHTED), parallel to data
    // dictionary and vertex scratch
    uint4 *sent = nullptr;
    uint8_t *alive = nullptr;
    uint32_t *vcnt = nullptr, *vtid = nullptr, *dead = nullptr;
    uint4 *vinfo = nullptr;
    // control block
    Dev *dev = nullptr;
    Dev *h_dev = nullptr;  // pinned mirror for stats
    // touched scratch
    unsigned long long tcap = 0;
    uint32_t *t_vid = nullptr, *t_tiny = nullptr;
    uint4 *t_a = nullptr, *t_b = nullptr;
    unsigned long long rcap = 0;
    uint32_t *prank = nullptr;
    unsigned long long dcap = 0;
    uint8_t *pflag = nullptr;      // set-semantics insert scratch
    uint32_t *dsrc2 = nullptr;
    unsigned long long *dtmp = nullptr;
    unsigned long long ocap = 0;
    uint32_t *t_owner = nullptr;
    uint32_t *t_rowner = nullptr;  // hub runs: run pop index -> touched index (ocap entries)
    // hub runs (per-vertex block size): log2 R (0 = off), the entry count of a
    // first allocation that makes a source a hub (0 = C << rs), the percent
    // of the pool in runs, the runs and the ring of free run heads
    uint32_t rs = 0, hub_deg_cfg = 0, hub_pct = 0;
    unsigned long long RP = 0;
    uint32_t *rqueue = nullptr;
    // items
    unsigned long long icap = 0;
    uint32_t ib_alloc = 0;  // blocks per item the work-item arrays were sized for
    uint2 *items = nullptr;
    uint32_t *it_mask = nullptr, *it_cnt = nullptr, *it_H = nullptr, *it_S = nullptr, *it_bid = nullptr;
    // arena
    unsigned long long acap = 0;
    uint32_t *arena = nullptr, *found = nullptr;
    unsigned long long qcap = 0;
    uint32_t *qpos = nullptr;
    // neighbour scan partials
    unsigned long long pcap = 0;
    unsigned long long *partials = nullptr;
    // validation
    uint32_t *owner_bits = nullptr;
    unsigned long long *vres = nullptr;
    unsigned long long *h_small = nullptr;  // pinned scratch (8 words)
    Staging stage;
    cudaStream_t last_stream = nullptr;
    uint64_t scratch_bytes = 0;
    uint64_t dict_bytes = 0;
    bool any_vertex_deleted = false;
    unsigned long long used_ub = 0;  // upper bound of blocks in use (pool growth policy)
    cudaStream_t side = nullptr;     // second stream: concurrent mark tiers, staging copies
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host input staging: kInSets rotating sets of device buffers filled on
    // the copy stream; a set's free event is recorded on the call stream
    // after the last kernel of the call that read it
    cudaStream_t copy = nullptr;
    InSet in_sets[kInSets];
    uint32_t in_round = 0;
    // analytics scratch: items, two frontiers, counters, PageRank vectors
    unsigned long long an_icap = 0, an_vcap = 0;
    uint2 *an_items = nullptr;
    uint32_t *an_cur = nullptr, *an_next = nullptr, *an_ctr = nullptr;
    uint32_t *an_stamp = nullptr;  // shortest paths: round in which a vertex last joined the frontier
    unsigned long long *rb_stats = nullptr;  // edge-block resize: degree totals / blocks per candidate C
    double *pr_c = nullptr, *pr_acc = nullptr, *pr_scal = nullptr;
    unsigned long long *pr_n = nullptr;
    // PageRank's incoming-edge CSR: per-vertex cursor, offsets, chunk sums,
    // source and destination of every entry
    unsigned long long pr_vcap = 0, pr_ecap = 0;
    uint32_t *pr_cursor = nullptr, *pr_src = nullptr, *pr_dst = nullptr;
    unsigned long long *pr_off = nullptr, *pr_part = nullptr;
    // grouped path of large batches: partitioned pairs, per-CTA bucket
    // counts, bucket totals and bases, chunk list, block-wide tier groups
    unsigned long long gp_ncap = 0, gp_acap = 0, gp_hcap = 0, gp_ccap = 0, gp_icap = 0, gp_rcap = 0, go_cap = 0;
    uint32_t *gp_src = nullptr, *gp_dst = nullptr, *gp_aux = nullptr, *gp_hist = nullptr;
    uint32_t *gp_btot = nullptr, *gp_bbase = nullptr, *gp_mbkt = nullptr, *gp_rows = nullptr;
    uint32_t *go_src = nullptr, *go_dst = nullptr, *go_aux = nullptr;
    uint4 *gp_chunks = nullptr;
    uint2 *grp_items = nullptr;
    // graph set: members' vertex ranges (set_G == 0 for a plain graph)
    uint32_t set_G = 0;
    uint32_t *set_vbase = nullptr;          // device, G+1
    std::vector<uint32_t> set_vbase_h;      // host copy
    unsigned long long scap = 0;
    uint32_t *set_src = nullptr, *set_dst = nullptr;  // remapped batch
    gv::Prof prof;
};

namespace {

#define GV_CK(expr)                                                  \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) {                                     \
            return _e == cudaErrorMemoryAllocation ? GV_ERR_OUT_OF_MEMORY : GV_ERR_CUDA; \
        }                                                            \
    } while (0)

#define GV_TRY(expr)                  \
    do {                              \
        gv_status _s = (expr);        \
        if (_s != GV_OK) return _s;   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
gv_status dalloc(T **p, size_t count, uint64_t *acct) {
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GV_ERR_OUT_OF_MEMORY;
    }
    *p = static_cast<T *>(q);
    if (acct) *acct += count * sizeof(T);
    return GV_OK;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

GraphView view(const gv_graph *g) {
    GraphView v{};  // every field not set below is zero (NULL)
    v.sent = g->sent;
    v.alive = g->alive;
    v.data = g->data;
    v.wdata = g->wdata;
    v.links = g->links;
    v.queue = g->queue;
    v.dev = g->dev;
    v.P = g->P;
    v.C = g->C;
    v.IB = g->IB;
    v.nv = g->nv;
    v.all_alive = g->any_vertex_deleted ? 0u : 1u;
    v.vmask = g->vcap ? g->vcap - 1 : 0;
    v.cmul = g->C ? ((1ull << 40) + g->C - 1) / g->C : 0ull;
    v.dense_shift = g->dense_shift;
    v.vcnt = g->vcnt;
    v.vinfo = g->vinfo;
    v.vtid = g->vtid;
    v.t_vid = g->t_vid;
    v.t_a = g->t_a;
    v.t_b = g->t_b;
    v.t_owner = g->t_owner;
    v.t_tiny = g->t_tiny;
    v.prank = g->prank;
    v.pflag = g->pflag;
    v.items = g->items;
    v.it_mask = g->it_mask;
    v.it_cnt = g->it_cnt;
    v.it_H = g->it_H;
    v.it_S = g->it_S;
    v.it_bid = g->it_bid;
    v.arena = g->arena;
    v.hbase = 0;
    v.found = g->found;
    v.qpos = g->qpos;
    v.dead = g->dead;
    v.max_items = g->icap;
    v.tiny_cap = g->tcap;
    v.arena_cap = g->acap;
    v.set_G = 0;
    v.set_vbase = nullptr;
    v.set_off = nullptr;
    v.set_counts = nullptr;
    if (g->RP) {
        v.rs = g->rs;
        v.hub_deg = g->hub_deg_cfg ? g->hub_deg_cfg : g->C << g->rs;
        v.RP = g->RP;
        v.rqueue = g->rqueue;
        v.t_rowner = g->t_rowner;
    }
    return v;
}

LaunchCfg lcfg(const gv_graph *g, cudaStream_t s) {
    LaunchCfg lc;
    lc.num_sms = g->num_sms;
    lc.stream = s;
    lc.prof = const_cast<gv::Prof *>(&g->prof);
    lc.side = g->side;
    lc.fork = g->ev_fork;
    lc.join = g->ev_join;
    return lc;
}

uint32_t next_pow2(uint64_t n) {
    uint64_t c = 1;
    while (c < n) c <<= 1;
    return (uint32_t)std::min<uint64_t>(c, 1ull << 31);
}

// Is p a host address (pageable or pinned) rather than device memory?
bool is_host_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

gv_status stage_buf(gv_graph *g, int slot, size_t bytes, void **out) {
    DevBuf &b = g->stage.buf[slot];
    if (b.bytes < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        size_t want = std::max(bytes, (size_t)4096);
        if (cudaMalloc(&b.p, want) != cudaSuccess) {
            cudaGetLastError();
            return GV_ERR_OUT_OF_MEMORY;
        }
        b.bytes = want;
    }
    *out = b.p;
    return GV_OK;
}

// Device view of an input array: itself, or a staged copy of a host array.
gv_status input_ptr(gv_graph *g, int slot, const void *p, size_t bytes, cudaStream_t s, const void **out) {
    if (!is_host_ptr(p) || bytes == 0) {
        *out = p;
        return GV_OK;
    }
    void *d = nullptr;
    GV_TRY(stage_buf(g, slot, bytes, &d));
    GV_CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
    *out = d;
    return GV_OK;
}

// Device target for an output array; *host is set when the caller's array
// is in host memory and must be copied back after the kernels.
gv_status output_ptr(gv_graph *g, int slot, void *p, size_t bytes, void **out, bool *host) {
    *host = is_host_ptr(p);
    if (!*host) {
        *out = p;
        return GV_OK;
    }
    return stage_buf(g, slot, bytes, out);
}

// ------------------------------------------------------------- capacities

gv_status ensure_vertex_capacity(gv_graph *g, uint32_t need, cudaStream_t s) {
    if (need <= g->vcap) return GV_OK;
    uint32_t cap = std::max<uint32_t>(g->vcap ? g->vcap : 1, 1);
    while (cap < need) cap *= 2;  // dictionary doubles ("Dynamic vertex updates")
    uint4 *sent = nullptr;
    uint8_t *alive = nullptr;
    uint32_t *vcnt = nullptr, *vtid = nullptr, *dead = nullptr;
    uint4 *vinfo = nullptr;
    uint64_t acct = 0;
    gv_status st;
    if ((st = dalloc(&sent, cap, &acct)) != GV_OK || (st = dalloc(&alive, cap, &acct)) != GV_OK ||
        (st = dalloc(&vcnt, cap, &acct)) != GV_OK || (st = dalloc(&vinfo, cap, &acct)) != GV_OK ||
        (st = dalloc(&vtid, cap, &acct)) != GV_OK || (st = dalloc(&dead, cap / 32 + 1, &acct)) != GV_OK) {
        dfree(sent); dfree(alive); dfree(vcnt); dfree(vinfo); dfree(vtid); dfree(dead);
        return st;
    }
    GV_CK(cudaMemsetAsync(vcnt, 0, (size_t)cap * 4, s));
    GV_CK(cudaMemsetAsync(dead, 0, (size_t)(cap / 32 + 1) * 4, s));
    GV_CK(cudaMemsetAsync(alive, 0, cap, s));
    if (g->vcap) {
        GV_CK(gv::launch_copy_dictionary(sent, alive, g->sent, g->alive, g->nv, lcfg(g, s)));
        GV_CK(cudaStreamSynchronize(s));
    }
    dfree(g->sent); dfree(g->alive); dfree(g->vcnt); dfree(g->vinfo); dfree(g->vtid); dfree(g->dead);
    g->sent = sent;
    g->alive = alive;
    g->vcnt = vcnt;
    g->vinfo = vinfo;
    g->vtid = vtid;
    g->dead = dead;
    g->vcap = cap;
    g->dict_bytes = acct;
    return GV_OK;
}

gv_status ensure_touched(gv_graph *g, unsigned long long need) {
    if (need <= g->tcap && g->tcap) return GV_OK;
    unsigned long long cap = std::max<unsigned long long>(need, std::max<unsigned long long>(2 * g->tcap, 1024));
    dfree(g->t_vid); dfree(g->t_a); dfree(g->t_b); dfree(g->t_tiny);
    g->tcap = 0;
    GV_TRY(dalloc(&g->t_tiny, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->t_vid, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->t_a, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->t_b, cap, &g->scratch_bytes));
    g->tcap = cap;
    return GV_OK;
}

gv_status ensure_owner(gv_graph *g, unsigned long long need) {
    if (need <= g->ocap && g->ocap) return GV_OK;
    unsigned long long cap = std::max<unsigned long long>(need, std::max<unsigned long long>(2 * g->ocap, 1024));
    dfree(g->t_owner);
    dfree(g->t_rowner);
    g->ocap = 0;
    GV_TRY(dalloc(&g->t_owner, cap, &g->scratch_bytes));
    // run pops of a call are bounded like its block pops (a run holds R >= 1 blocks)
    if (g->rs) GV_TRY(dalloc(&g->t_rowner, cap, &g->scratch_bytes));
    g->ocap = cap;
    return GV_OK;
}

gv_status ensure_items(gv_graph *g, unsigned long long need) {
    if (need <= g->icap && g->icap) return GV_OK;
    unsigned long long cap = std::max<unsigned long long>(need, std::max<unsigned long long>(2 * g->icap, 1024));
    dfree(g->items); dfree(g->it_mask); dfree(g->it_cnt); dfree(g->it_H); dfree(g->it_S); dfree(g->it_bid);
    g->icap = 0;
    GV_TRY(dalloc(&g->items, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->it_mask, cap * gv::MASK_WORDS, &g->scratch_bytes));
    GV_TRY(dalloc(&g->it_cnt, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->it_H, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->it_S, cap, &g->scratch_bytes));
    GV_TRY(dalloc(&g->it_bid, cap * (g->IB ? g->IB : 32), &g->scratch_bytes));
    g->ib_alloc = g->IB ? g->IB : 32;
    g->icap = cap;
    return GV_OK;
}

gv_status ensure_arena(gv_graph *g, unsigned long long words, bool query, unsigned long long nq) {
    if (words > g->acap || !g->acap) {
        unsigned long long cap = std::max<unsigned long long>(words, std::max<unsigned long long>(2 * g->acap, 4096));
        dfree(g->arena); dfree(g->found);
        g->acap = 0;
        GV_TRY(dalloc(&g->arena, cap, &g->scratch_bytes));
        GV_TRY(dalloc(&g->found, cap, &g->scratch_bytes));
        g->acap = cap;
    }
    if (query && (nq > g->qcap || !g->qcap)) {
        unsigned long long cap = std::max<unsigned long long>(nq, std::max<unsigned long long>(2 * g->qcap, 4096));
        dfree(g->qpos);
        g->qcap = 0;
        GV_TRY(dalloc(&g->qpos, cap, &g->scratch_bytes));
        g->qcap = cap;
    }
    return GV_OK;
}

// Items over all touched sources never exceed touched + pool blocks / IB.
unsigned long long item_bound(const gv_graph *g, unsigned long long touched) {
    return touched + (g->IB ? (g->P + g->IB - 1) / g->IB : 0) + 1;
}

// End of the laid-out pool arrays for P blocks of C slots: slots, payloads
// (weighted graphs), links and queue, each starting on a 256-byte boundary.
uint64_t layout_end(unsigned long long P, uint32_t C, bool weighted) {
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    uint64_t off = al(P * C * 4ull);
    if (weighted) off = al(off + P * C * 4ull);
    off = al(off + P * 8ull);
    return off + P * 4ull;
}

// The largest block count whose layout fits in `bytes` (every array must lie
// inside the allocation: the queue is written in full).
unsigned long long fit_blocks(uint64_t bytes, uint32_t C, bool weighted) {
    const uint64_t per_block = 4ull * C * (weighted ? 2 : 1) + 8 + 4;
    unsigned long long P = bytes / per_block;
    if (P > 0xFFFFFFFEull) P = 0xFFFFFFFEull;
    while (P > 0 && layout_end(P, C, weighted) > bytes) --P;
    return P;
}

// Points the graph's pool arrays into `base` for P blocks of C slots; false
// if that layout does not fit in `bytes`.
bool lay_out_pool(gv_graph *g, char *base, uint64_t bytes, uint32_t C, unsigned long long P) {
    const bool weighted = (g->flags & GV_WEIGHTED) != 0;
    if (layout_end(P, C, weighted) > bytes) return false;
    auto align = [](uint64_t x) { return (x + 255) & ~255ull; };
    uint64_t off = 0;
    g->data = reinterpret_cast<uint32_t *>(base + off);
    off = align(off + P * C * 4ull);
    g->wdata = nullptr;
    if (weighted) {
        g->wdata = reinterpret_cast<uint32_t *>(base + off);
        off = align(off + P * C * 4ull);
    }
    g->links = reinterpret_cast<uint32_t *>(base + off);
    off = align(off + P * 8ull);
    g->queue = reinterpret_cast<uint32_t *>(base + off);
    g->C = C;
    g->P = P;
    return true;
}

// Blocks per work item of the delete / query pipelines: up to 512 slots.
void set_item_blocks(gv_graph *g) {
    g->IB = std::min<uint32_t>(32, std::max<uint32_t>(1, 512 / g->C));
    if (g->item_blocks_cfg) g->IB = std::min<uint32_t>(g->IB, g->item_blocks_cfg);
}

// Pool: one allocation holding block storage, links and the edge queue.
gv_status setup_pool(gv_graph *g, uint32_t C, cudaStream_t s) {
    if (C < 4 || C > 512 || (C % 4) != 0) return GV_ERR_INVALID_ARG;
    g->C = C;
    set_item_blocks(g);
    uint64_t bytes = g->pool_bytes_cfg;
    if (bytes == 0) {
        size_t fr = 0, tot = 0;
        GV_CK(cudaMemGetInfo(&fr, &tot));
        bytes = fr / 2;  // "Edge Queue": at least half of the GPU memory
    }
    const bool weighted = (g->flags & GV_WEIGHTED) != 0;
    unsigned long long P = fit_blocks(bytes, C, weighted);
    // with hub runs a root word carries RUN_BIT: block ids stay below 2^31 - 1
    if (g->rs && P > 0x7FFFFFFEull) P = 0x7FFFFFFEull;
    if (P == 0) return GV_ERR_INVALID_ARG;
    const unsigned long long RP = g->rs ? (P * g->hub_pct / 100) >> g->rs : 0ull;
    if (g->rs && RP == 0) return GV_ERR_INVALID_ARG;  // the pool holds no run
    char *base = nullptr;
    if (g->pool_mem_cfg) {
        if (reinterpret_cast<uintptr_t>(g->pool_mem_cfg) % 16 != 0) return GV_ERR_INVALID_ARG;
        base = static_cast<char *>(g->pool_mem_cfg);
    } else {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return GV_ERR_OUT_OF_MEMORY;
        }
        g->pool_alloc = p;
        base = static_cast<char *>(p);
    }
    if (!lay_out_pool(g, base, bytes, C, P)) return GV_ERR_STATE;  // cannot happen: P was fitted
    g->pool_bytes = bytes;
    // Dev: the edge queue holds every block outside the run region [0, H);
    // the run queue the heads of the region's runs
    const unsigned long long H = RP << g->rs;
    GV_CK(gv::launch_init_queue(g->queue, P - H, lcfg(g, s), (uint32_t)H, 1u));
    g->h_small[4] = P - H;
    GV_CK(cudaMemcpyAsync(&g->dev->q_back, &g->h_small[4], 8, cudaMemcpyHostToDevice, s));
    if (RP) {
        GV_TRY(dalloc(&g->rqueue, RP, &g->scratch_bytes));
        GV_CK(gv::launch_init_queue(g->rqueue, RP, lcfg(g, s), 0u, 1u << g->rs));
        g->h_small[5] = RP;
        GV_CK(cudaMemcpyAsync(&g->dev->rq_back, &g->h_small[5], 8, cudaMemcpyHostToDevice, s));
        g->RP = RP;
    }
    GV_CK(cudaStreamSynchronize(s));
    GV_TRY(ensure_items(g, item_bound(g, 1024)));
    return GV_OK;
}

gv_status ensure_ranks(gv_graph *g, unsigned long long n) {
    if (n <= g->rcap && g->rcap) return GV_OK;
    unsigned long long cap = std::max<unsigned long long>(n, std::max<unsigned long long>(2 * g->rcap, 4096));
    dfree(g->prank);
    g->rcap = 0;
    GV_TRY(dalloc(&g->prank, cap, &g->scratch_bytes));
    g->rcap = cap;
    return GV_OK;
}

// Scratch for a pair batch of n (insert / delete / query).
gv_status ensure_batch(gv_graph *g, uint64_t n, int mode) {
    const unsigned long long touched = std::min<unsigned long long>(n, g->nv ? g->nv : 1);
    GV_TRY(ensure_touched(g, touched));
    GV_TRY(ensure_ranks(g, n));
    if (mode == gv::MODE_INSERT) {
        GV_TRY(ensure_owner(g, (g->C ? n / g->C : n) + touched + 1));
    } else {
        GV_TRY(ensure_items(g, item_bound(g, touched)));
        GV_TRY(ensure_arena(g, 5 * n + 128, mode == gv::MODE_QUERY, n));
    }
    return GV_OK;
}

// Does a plain batch call of n pairs take the grouped path?  Large batches
// (the dense threshold) on dictionaries of at most GP_BMAX * GP_WMAX
// vertices, when the graph asked for the radix-partition grouping.
bool use_grouped(const gv_graph *g, uint64_t n) {
    if (!(g->flags & GV_RADIX_GROUPING) || g->rs) return false;
    if (g->set_G || g->C == 0 || n == 0) return false;
    if ((unsigned long long)g->vcap > (unsigned long long)gv::GP_BMAX * gv::GP_WMAX) return false;
    return n >= ((unsigned long long)g->nv >> g->dense_shift);
}

template <typename T>
gv_status grow_buf(T **p, unsigned long long *cap, unsigned long long need, uint64_t *acct) {
    if (need <= *cap && *cap) return GV_OK;
    const unsigned long long c = std::max<unsigned long long>(need, std::max<unsigned long long>(2 * *cap, 1024));
    dfree(*p);
    *cap = 0;
    GV_TRY(dalloc(p, c, acct));
    *cap = c;
    return GV_OK;
}

// Scratch of a grouped call of n pairs (aux: a word per pair travels with
// it; out: the insert's grouped copy; items: block-wide tier groups).
gv_status ensure_group(gv_graph *g, uint64_t n, bool aux, bool out, unsigned long long items) {
    uint32_t ctas = 0;
    unsigned long long len = 0;
    gv::group_shape(n, g->num_sms, &ctas, &len);
    if (n > g->gp_ncap || !g->gp_ncap) {
        const unsigned long long c = std::max<unsigned long long>(n, std::max<unsigned long long>(2 * g->gp_ncap, 4096));
        dfree(g->gp_src);
        dfree(g->gp_dst);
        g->gp_ncap = 0;
        GV_TRY(dalloc(&g->gp_src, c, &g->scratch_bytes));
        GV_TRY(dalloc(&g->gp_dst, c, &g->scratch_bytes));
        g->gp_ncap = c;
    }
    if (aux) GV_TRY(grow_buf(&g->gp_aux, &g->gp_acap, n, &g->scratch_bytes));
    if (out && (n > g->go_cap || !g->go_cap)) {
        const unsigned long long c = std::max<unsigned long long>(n, std::max<unsigned long long>(2 * g->go_cap, 4096));
        dfree(g->go_src);
        dfree(g->go_dst);
        dfree(g->go_aux);
        g->go_cap = 0;
        GV_TRY(dalloc(&g->go_src, c, &g->scratch_bytes));
        GV_TRY(dalloc(&g->go_dst, c, &g->scratch_bytes));
        GV_TRY(dalloc(&g->go_aux, c, &g->scratch_bytes));
        g->go_cap = c;
    }
    GV_TRY(grow_buf(&g->gp_hist, &g->gp_hcap, (unsigned long long)ctas * gv::GP_BMAX, &g->scratch_bytes));
    GV_TRY(grow_buf(&g->gp_chunks, &g->gp_ccap, n / gv::GP_CHUNK + gv::GP_BMAX + 1, &g->scratch_bytes));
    // rows: one per chunk of a bucket of several chunks (at most 2n /
    // GP_CHUNK), W words each; sized for every batch of at most n pairs
    // (smaller batches have fewer buckets, so longer rows)
    unsigned long long rw = 0;
    for (unsigned long long m = n; m > 0; m /= 2) {
        const unsigned long long wm = 1ull << gv::group_bucket_shift(m, g->vcap);  // vertices per bucket
        rw = std::max<unsigned long long>(rw, (2 * (m / gv::GP_CHUNK) + 2) * wm);
    }
    GV_TRY(grow_buf(&g->gp_rows, &g->gp_rcap, rw, &g->scratch_bytes));
    if (!g->gp_btot) GV_TRY(dalloc(&g->gp_btot, gv::GP_BMAX, &g->scratch_bytes));
    if (!g->gp_bbase) GV_TRY(dalloc(&g->gp_bbase, gv::GP_BMAX, &g->scratch_bytes));
    if (!g->gp_mbkt) GV_TRY(dalloc(&g->gp_mbkt, gv::GP_BMAX, &g->scratch_bytes));
    if (items) GV_TRY(grow_buf(&g->grp_items, &g->gp_icap, items, &g->scratch_bytes));
    return GV_OK;
}

// The graph's view for a grouped call of n pairs.
GraphView grouped_view(const gv_graph *g, uint64_t n) {
    GraphView v = view(g);
    v.grouped = 1;
    v.gb_shift = gv::group_bucket_shift(n, g->vcap);
    v.gb_n = g->vcap >> v.gb_shift;
    gv::group_shape(n, g->num_sms, &v.gp_ctas, &v.gp_len);
    v.gp_src = g->gp_src;
    v.gp_dst = g->gp_dst;
    v.gp_aux = g->gp_aux;
    v.gp_hist = g->gp_hist;
    v.gp_btot = g->gp_btot;
    v.gp_bbase = g->gp_bbase;
    v.gp_chunks = g->gp_chunks;
    v.gp_mbkt = g->gp_mbkt;
    v.gp_rows = g->gp_rows;
    v.go_src = g->go_src;
    v.go_dst = g->go_dst;
    v.go_aux = g->go_aux;
    v.gcur = g->vtid;  // the touched-index array is free during a grouped call
    v.grp_items = g->grp_items;
    v.grp_cap = g->gp_icap;
    v.hbase = (uint32_t)((n + 63) / 64 * 64);  // deletes, queries: batch lists below, hash sets above
    return v;
}

gv_status check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return GV_ERR_CUDA;
    return GV_OK;
}

// C by the paper's rule from the counted first batch: average degree of the
// sources with at least one edge, rounded up to a multiple of 4 (>= 4).
uint32_t rule_capacity(unsigned long long valid, unsigned long long touched) {
    if (touched == 0 || valid == 0) return 4;
    unsigned long long avg = (valid + touched - 1) / touched;
    unsigned long long c = (avg + 3) / 4 * 4;
    if (c < 4) c = 4;
    if (c > 512) c = 512;
    return (uint32_t)c;
}

// Moves the pool into a larger allocation of P2 blocks: block storage and
// tree links are copied (block ids keep their meaning), the queue ring is
// rebuilt with the new ids behind the free ones.  qf/qb: queue counters read
// after the stream was synchronised.
gv_status grow_pool(gv_graph *g, unsigned long long P2, unsigned long long qf, unsigned long long qb,
                    cudaStream_t s) {
    auto align = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t C = g->C;
    const bool weighted = g->wdata != nullptr;
    const uint64_t off_w = align(P2 * C * 4ull);
    const uint64_t off_links = weighted ? align(off_w + P2 * C * 4ull) : off_w;
    const uint64_t off_queue = align(off_links + P2 * 8ull);
    const uint64_t bytes = off_queue + P2 * 4ull;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return GV_ERR_OUT_OF_MEMORY;
    }
    char *base = static_cast<char *>(p);
    uint32_t *data2 = reinterpret_cast<uint32_t *>(base);
    uint32_t *w2 = weighted ? reinterpret_cast<uint32_t *>(base + off_w) : nullptr;
    uint32_t *links2 = reinterpret_cast<uint32_t *>(base + off_links);
    uint32_t *queue2 = reinterpret_cast<uint32_t *>(base + off_queue);
    const unsigned long long nfree = qb - qf;
    GV_CK(cudaMemcpyAsync(data2, g->data, g->P * C * 4ull, cudaMemcpyDeviceToDevice, s));
    if (weighted) GV_CK(cudaMemcpyAsync(w2, g->wdata, g->P * C * 4ull, cudaMemcpyDeviceToDevice, s));
    GV_CK(cudaMemcpyAsync(links2, g->links, g->P * 8ull, cudaMemcpyDeviceToDevice, s));
    GV_CK(gv::launch_grow_queue(g->queue, g->P, qf, nfree, queue2, P2, lcfg(g, s)));
    g->h_small[2] = 0;
    g->h_small[3] = nfree + (P2 - g->P);
    GV_CK(cudaMemcpyAsync(&g->dev->q_front, &g->h_small[2], 8, cudaMemcpyHostToDevice, s));
    GV_CK(cudaMemcpyAsync(&g->dev->q_back, &g->h_small[3], 8, cudaMemcpyHostToDevice, s));
    GV_CK(cudaStreamSynchronize(s));
    cudaFree(g->pool_alloc);
    g->pool_alloc = p;
    g->data = data2;
    g->wdata = w2;
    g->links = links2;
    g->queue = queue2;
    g->P = P2;
    g->pool_bytes = bytes;
    return GV_OK;
}

// Pool growth ("Edge Queue": once 80% of the pool is in use it grows by
// 25%), checked on the host before an insert of n pairs.  The library keeps
// an upper bound of the blocks in use (exact after a read, plus the
// worst-case demand of every insert since, ceil(n / C) + min(n, |V|)); only
// when that bound passes 80% does it synchronise to read the exact count,
// then grows by 25% steps until the exact count plus this insert's
// worst-case demand fits under 80%.  A failed allocation keeps the old pool
// (the insert may then report pool exhaustion as usual).
gv_status maybe_grow(gv_graph *g, uint64_t n, cudaStream_t s) {
    if (!(g->flags & GV_GROW) || !g->C || n == 0) return GV_OK;
    const unsigned long long demand = (n + g->C - 1) / g->C + std::min<unsigned long long>(n, g->nv);
    // with hub runs the policy applies to the blocks outside the run
    // region, which has a fixed size: growth adds single blocks only
    const unsigned long long H = g->RP << g->rs;
    const unsigned long long pmax = g->rs ? 0x7FFFFFFEull : 0xFFFFFFFEull;
    if (5 * (g->used_ub + demand) <= 4 * (g->P - H)) {
        g->used_ub += demand;
        return GV_OK;
    }
    GV_CK(cudaMemcpyAsync(&g->h_small[0], &g->dev->q_front, 8, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaMemcpyAsync(&g->h_small[1], &g->dev->q_back, 8, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    const unsigned long long qf = g->h_small[0], qb = g->h_small[1];
    const unsigned long long used = g->P - H - (qb - qf);
    unsigned long long P2 = g->P;
    while (5 * (used + demand) > 4 * (P2 - H) && P2 < pmax) P2 = std::min<unsigned long long>(P2 + (P2 + 3) / 4, pmax);
    if (P2 > g->P) {
        const gv_status st = grow_pool(g, P2, qf, qb, s);
        if (st != GV_OK && st != GV_ERR_OUT_OF_MEMORY) return st;
    }
    g->used_ub = used + demand;
    return GV_OK;
}

// Host-array batches are staged into the next of kInSets rotating sets of
// device buffers on the graph's copy stream, so that a call's copies can run
// while the kernels of earlier calls still read their own sets; the call
// stream waits for the copies, and a set is refilled only after the call
// that read it recorded its free event.  Batches of at least kPipeMin pairs
// are copied in kPipePieces pieces and each piece is counted on the call
// stream as soon as it has landed: the counting pass overlaps the copies of
// the later pieces (counting is order-independent: ranks come from atomics).
constexpr uint64_t kPipeMin = 1ull << 20;

gv_status set_buf(DevBuf &b, size_t bytes, void **out) {
    if (b.bytes < bytes) {
        if (b.p) cudaFree(b.p);  // synchronises the device: no copy or kernel still uses it
        b.p = nullptr;
        b.bytes = 0;
        const size_t want = std::max(bytes, (size_t)4096);
        if (cudaMalloc(&b.p, want) != cudaSuccess) {
            cudaGetLastError();
            return GV_ERR_OUT_OF_MEMORY;
        }
        b.bytes = want;
    }
    *out = b.p;
    return GV_OK;
}

// Device views of a batch's inputs (host arrays staged, device arrays as
// they are); with `count`, also the counting pass of `mode`.  *set_out = the
// staging set used (-1: none); the caller records its free event on `s`
// after the call's last launch.
gv_status stage_batch(gv_graph *g, const GraphView &v, int mode, const uint32_t *src, const uint32_t *dst,
                      const uint32_t *wts, uint64_t n, cudaStream_t s, bool count, const void **dsrc,
                      const void **ddst, const void **dwts, int *set_out) {
    *set_out = -1;
    *dsrc = src;
    *ddst = dst;
    if (dwts) *dwts = wts;
    const bool hs = is_host_ptr(src), hd = is_host_ptr(dst), hw = wts && is_host_ptr(wts);
    const bool grp = v.grouped != 0;
    // counting of pairs [lo, hi) as soon as they are on the device, and the
    // rest of the grouping once all of them are
    auto count_range = [&](const uint32_t *cs, const uint32_t *cd, uint64_t lo, uint64_t hi) {
        return grp ? gv::launch_group_hist(mode, v, cs, cd, n, lo, hi, lcfg(g, s))
                   : gv::launch_count_range(mode, v, cs, cd, n, lo, hi, lcfg(g, s));
    };
    auto count_finish = [&](const uint32_t *cs, const uint32_t *cd, const uint32_t *cw) {
        return grp ? gv::launch_group_finish(mode, v, cs, cd, cw, n, lcfg(g, s))
                   : gv::launch_count_finish(mode, v, n, lcfg(g, s));
    };
    if (!hs && !hd && !hw) {
        if (count) {
            GV_CK(count_range(src, dst, 0, n));
            GV_CK(count_finish(src, dst, wts));
        }
        return GV_OK;
    }
    const int k = (int)(g->in_round++ % kInSets);
    InSet &set = g->in_sets[k];
    void *bs = nullptr, *bd = nullptr, *bw = nullptr;
    if (hs) GV_TRY(set_buf(set.src, n * 4, &bs));
    if (hd) GV_TRY(set_buf(set.dst, n * 4, &bd));
    if (hw) GV_TRY(set_buf(set.wts, n * 4, &bw));
    const bool async = g->copy && set.free_ev;  // a set with free_ev has all its events
    cudaStream_t cs = async ? g->copy : s;
    if (async && set.used) GV_CK(cudaStreamWaitEvent(cs, set.free_ev, 0));
    const uint32_t *ss = hs ? static_cast<const uint32_t *>(bs) : src;
    const uint32_t *sd = hd ? static_cast<const uint32_t *>(bd) : dst;
    const uint32_t *sw = hw ? static_cast<const uint32_t *>(bw) : wts;
    const int pieces = (count && n >= kPipeMin && g->C != 0) ? kPipePieces : 1;
    for (int p = 0; p < pieces; ++p) {
        uint64_t lo = n * p / pieces, hi = n * (p + 1) / pieces;
        if (grp) {
            // piece boundaries on whole partition-CTA ranges
            lo = std::min<uint64_t>(n, lo / v.gp_len * v.gp_len);
            hi = p + 1 == pieces ? n : std::min<uint64_t>(n, hi / v.gp_len * v.gp_len);
        }
        if (hi > lo) {
            if (hs) GV_CK(cudaMemcpyAsync(static_cast<uint32_t *>(bs) + lo, src + lo, (hi - lo) * 4,
                                          cudaMemcpyHostToDevice, cs));
            if (hd) GV_CK(cudaMemcpyAsync(static_cast<uint32_t *>(bd) + lo, dst + lo, (hi - lo) * 4,
                                          cudaMemcpyHostToDevice, cs));
            if (hw) GV_CK(cudaMemcpyAsync(static_cast<uint32_t *>(bw) + lo, wts + lo, (hi - lo) * 4,
                                          cudaMemcpyHostToDevice, cs));
        }
        if (async) {
            GV_CK(cudaEventRecord(set.piece[p], cs));
            GV_CK(cudaStreamWaitEvent(s, set.piece[p], 0));
        }
        if (count && pieces > 1) GV_CK(count_range(ss, sd, lo, hi));
    }
    if (count) {
        if (pieces == 1) GV_CK(count_range(ss, sd, 0, n));
        GV_CK(count_finish(ss, sd, sw));
    }
    set.used = true;
    // free once the kernels launched so far are done; the caller records it
    // again after its last launch (an error return in between still leaves
    // the set guarded by this record)
    if (async) GV_CK(cudaEventRecord(set.free_ev, s));
    *set_out = k;
    *dsrc = ss;
    *ddst = sd;
    if (dwts) *dwts = sw;
    return GV_OK;
}

// The staging set of a call is free once the call stream reaches this point.
gv_status release_set(gv_graph *g, int set, cudaStream_t s) {
    if (set >= 0 && g->in_sets[set].free_ev) GV_CK(cudaEventRecord(g->in_sets[set].free_ev, s));
    return GV_OK;
}

gv_status insert_impl(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                      uint64_t *counts, cudaStream_t s, const uint32_t *wts = nullptr) {
    if (!g) return GV_ERR_INVALID_ARG;
    if (n > kMaxBatch) return GV_ERR_INVALID_ARG;
    if (n > 0 && (!src || !dst)) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    g->last_stream = s;
    const void *dsrc = src, *ddst = dst, *dwts = wts;
    // the plain insert of a laid-out graph stages host inputs on the copy
    // stream (stage_batch); the first batch and set semantics copy them here
    const bool plain = g->C != 0 && !(g->flags & GV_DEDUP) && n > 0;
    if (!plain) {
        GV_TRY(input_ptr(g, 0, src, n * 4, s, &dsrc));
        GV_TRY(input_ptr(g, 1, dst, n * 4, s, &ddst));
        if (wts) GV_TRY(input_ptr(g, 3, wts, n * 4, s, &dwts));
    }
    void *dcounts = counts;
    bool host_counts = false;
    if (counts) GV_TRY(output_ptr(g, 2, counts, 16, &dcounts, &host_counts));
    const unsigned long long touched = std::min<unsigned long long>(n, g->nv ? g->nv : 1);
    GV_TRY(ensure_touched(g, touched));
    GV_TRY(ensure_ranks(g, n));
    GV_TRY(maybe_grow(g, n, s));
    if (g->C == 0) {
        // First batch fixes C (paper rule), then the pool can be laid out.
        GraphView v = view(g);
        GV_CK(gv::launch_count(gv::MODE_INSERT, v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, lcfg(g, s)));
        GV_CK(cudaMemcpyAsync(g->h_small, &g->dev->call_b, 8, cudaMemcpyDeviceToHost, s));
        unsigned int nt = 0;
        GV_CK(cudaMemcpyAsync(&g->h_small[1], &g->dev->n_touched, 4, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        nt = (unsigned int)(g->h_small[1] & 0xFFFFFFFFull);
        const unsigned long long valid = n - g->h_small[0];
        GV_TRY(setup_pool(g, rule_capacity(valid, nt), s));
        GV_TRY(ensure_batch(g, n, gv::MODE_INSERT));
        if (!(g->flags & GV_DEDUP)) GV_TRY(maybe_grow(g, n, s));  // set semantics: checked by the call below
        GraphView v2 = view(g);
        if (g->flags & GV_DEDUP) {
            // the counting pass above only fixed C: clear it and run the
            // set-semantics insert from the start
            GV_CK(gv::launch_finalize_count_only(v2, lcfg(g, s)));
            if (host_counts) {
                GV_TRY(insert_impl(g, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, counts, s));
                return check_launch();
            }
            return insert_impl(g, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, counts, s);
        }
        GV_CK(gv::launch_insert_tail(v2, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, g->tcap,
                                     (unsigned long long *)dcounts, lcfg(g, s), (const uint32_t *)dwts));
    } else if ((g->flags & GV_DEDUP) && n > 0) {
        // set semantics: membership pass over the batch, mask of the pairs
        // that add a new value, then the plain insert of the masked batch
        GV_TRY(ensure_batch(g, n, gv::MODE_INSERT));
        GV_TRY(ensure_batch(g, n, gv::MODE_QUERY));
        if (n > kMaxBatch / 2) return GV_ERR_INVALID_ARG;  // 8n arena words stay below 2^32
        GV_TRY(ensure_arena(g, 8 * n + 128, true, n));       // one hash set per source
        if (n > g->dcap || !g->dcap) {
            dfree(g->pflag);
            dfree(g->dsrc2);
            g->dcap = 0;
            const unsigned long long cap = std::max<unsigned long long>(n, 2 * g->dcap);
            GV_TRY(dalloc(&g->pflag, cap, &g->scratch_bytes));
            GV_TRY(dalloc(&g->dsrc2, cap, &g->scratch_bytes));
            g->dcap = cap;
        }
        if (!g->dtmp) GV_TRY(dalloc(&g->dtmp, 4, &g->scratch_bytes));
        GV_CK(cudaMemsetAsync(g->dtmp, 0, 32, s));
        GraphView v = view(g);
        GV_CK(gv::launch_count(gv::MODE_DELETE, v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, lcfg(g, s)));
        GV_CK(gv::launch_dedup_insert_prepare(v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, g->tcap,
                                              g->dsrc2, g->dtmp, lcfg(g, s)));
        GV_CK(gv::launch_count(gv::MODE_INSERT, v, g->dsrc2, (const uint32_t *)ddst, n, lcfg(g, s)));
        GV_CK(gv::launch_insert_tail(v, g->dsrc2, (const uint32_t *)ddst, n, g->tcap, g->dtmp + 2, lcfg(g, s)));
        GV_CK(gv::launch_dedup_counts(g->dev, g->dtmp, n, (unsigned long long *)dcounts, lcfg(g, s)));
    } else {
        GV_TRY(ensure_batch(g, n, gv::MODE_INSERT));
        if (n == 0) {
            if (counts) GV_CK(cudaMemsetAsync(dcounts, 0, 16, s));
        } else {
            int set = -1;
            // (hub runs: the one-CTA path takes single blocks only)
            const bool small = n <= gv::small_insert_max() && !g->rs;
            const bool grp = !small && use_grouped(g, n);
            if (grp) GV_TRY(ensure_group(g, n, g->wdata != nullptr, true, 0));
            const GraphView v = grp ? grouped_view(g, n) : view(g);
            GV_TRY(stage_batch(g, v, gv::MODE_INSERT, src, dst, wts, n, s, !small, &dsrc, &ddst, &dwts, &set));
            if (small)
                GV_CK(gv::launch_insert_small(v, (const uint32_t *)dsrc, (const uint32_t *)ddst,
                                              (const uint32_t *)dwts, n, (unsigned long long *)dcounts, lcfg(g, s)));
            else
                GV_CK(gv::launch_insert_tail(v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, g->tcap,
                                             (unsigned long long *)dcounts, lcfg(g, s), (const uint32_t *)dwts));
            GV_TRY(release_set(g, set, s));
        }
    }
    // host counts land in stream order (a pageable target completes here)
    if (host_counts) GV_CK(cudaMemcpyAsync(counts, dcounts, 16, cudaMemcpyDeviceToHost, s));
    return check_launch();
}

gv_status member_impl(gv_graph *g, int mode, const uint32_t *src, const uint32_t *dst, uint64_t n,
                      uint64_t *counts, uint8_t *qout, cudaStream_t s) {
    if (!g) return GV_ERR_INVALID_ARG;
    if (n > kMaxBatch) return GV_ERR_INVALID_ARG;
    if (n > 0 && (!src || !dst)) return GV_ERR_INVALID_ARG;
    if (mode == gv::MODE_QUERY && n > 0 && !qout) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    g->last_stream = s;
    void *dcounts = counts;
    bool host_counts = false;
    if (counts) GV_TRY(output_ptr(g, 2, counts, 16, &dcounts, &host_counts));
    if (n == 0 || g->C == 0) {
        // Empty batch, or no edge stored yet (C is fixed by the first edge
        // batch): nothing can match.  Deletes still count rejected pairs.
        if (mode == gv::MODE_QUERY) {
            if (n) {
                void *dq = qout;
                bool hq = false;
                GV_TRY(output_ptr(g, 3, qout, n, &dq, &hq));
                GV_CK(cudaMemsetAsync(dq, 0, n, s));
                if (hq) {
                    GV_CK(cudaMemcpyAsync(qout, dq, n, cudaMemcpyDeviceToHost, s));
                    GV_CK(cudaStreamSynchronize(s));
                }
            }
            return check_launch();
        }
        if (counts) {
            GV_CK(cudaMemsetAsync(dcounts, 0, 16, s));
            if (n) {
                const void *dsrc = src, *ddst = dst;
                GV_TRY(input_ptr(g, 0, src, n * 4, s, &dsrc));
                GV_TRY(input_ptr(g, 1, dst, n * 4, s, &ddst));
                GV_CK(gv::launch_count_rejects(view(g), (const uint32_t *)dsrc, (const uint32_t *)ddst, n,
                                               (unsigned long long *)dcounts + 1, lcfg(g, s)));
            }
            if (host_counts) {
                GV_CK(cudaMemcpyAsync(counts, dcounts, 16, cudaMemcpyDeviceToHost, s));
                GV_CK(cudaStreamSynchronize(s));
            }
        }
        return check_launch();
    }
    const void *dsrc = src, *ddst = dst;
    void *dq = qout;
    bool hq = false;
    if (mode == gv::MODE_QUERY) GV_TRY(output_ptr(g, 3, qout, n, &dq, &hq));
    GV_TRY(ensure_batch(g, n, mode));
    const bool grp = use_grouped(g, n);
    if (grp) {
        const unsigned long long touched = std::min<unsigned long long>(n, g->nv ? g->nv : 1);
        GV_TRY(ensure_group(g, n, mode == gv::MODE_QUERY, false, item_bound(g, touched)));
    }
    const GraphView v = grp ? grouped_view(g, n) : view(g);
    // small batches: grouping, plan and placement in one kernel of one CTA
    const bool small = !grp && n <= gv::small_member_max();
    int set = -1;
    GV_TRY(stage_batch(g, v, mode, src, dst, nullptr, n, s, !small, &dsrc, &ddst, nullptr, &set));
    if (small)
        GV_CK(gv::launch_member_small(mode, v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, g->tcap,
                                      (unsigned long long *)dcounts, (uint8_t *)dq, lcfg(g, s)));
    else
        GV_CK(gv::launch_member_tail(mode, v, (const uint32_t *)dsrc, (const uint32_t *)ddst, n, g->tcap,
                                     (unsigned long long *)dcounts, (uint8_t *)dq, lcfg(g, s)));
    GV_TRY(release_set(g, set, s));
    // host outputs land in stream order (a pageable target completes here)
    if (host_counts) GV_CK(cudaMemcpyAsync(counts, dcounts, 16, cudaMemcpyDeviceToHost, s));
    if (hq) GV_CK(cudaMemcpyAsync(qout, dq, n, cudaMemcpyDeviceToHost, s));
    return check_launch();
}

gv_status neighbors_impl(gv_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets, uint32_t *nbrs,
                         uint64_t cap, uint64_t *total, cudaStream_t s, bool all, uint32_t *wts = nullptr) {
    if (!g || !total || !offsets) return GV_ERR_INVALID_ARG;
    if (n > 0 && !all && !vids) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    g->last_stream = s;
    const void *dv = vids;
    if (all) {
        void *d = nullptr;
        GV_TRY(stage_buf(g, 0, (size_t)n * 4 + 4, &d));
        GV_CK(gv::launch_iota((uint32_t *)d, 0, n, lcfg(g, s)));
        dv = d;
    } else {
        GV_TRY(input_ptr(g, 0, vids, (size_t)n * 4, s, &dv));
    }
    void *doff = offsets;
    bool hoff = false;
    GV_TRY(output_ptr(g, 1, offsets, ((size_t)n + 1) * 8, &doff, &hoff));
    const unsigned long long nchunks = ((unsigned long long)n + 1023) / 1024;
    if (nchunks + 1 > g->pcap) {
        dfree(g->partials);
        g->pcap = 0;
        GV_TRY(dalloc(&g->partials, nchunks + 1, &g->scratch_bytes));
        g->pcap = nchunks + 1;
    }
    GraphView v = view(g);
    GV_CK(gv::launch_neighbor_offsets(v, (const uint32_t *)dv, n, (unsigned long long *)doff, g->partials, lcfg(g, s)));
    GV_CK(cudaMemcpyAsync(g->h_small, (unsigned long long *)doff + n, 8, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    *total = g->h_small[0];
    if (hoff) {
        GV_CK(cudaMemcpyAsync(offsets, doff, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
    }
    if (*total > cap) return GV_ERR_INVALID_ARG;
    if (*total == 0 || g->C == 0) return check_launch();
    if (!nbrs) return GV_ERR_INVALID_ARG;
    void *dn = nbrs, *dw = wts;
    bool hn = false, hw = false;
    GV_TRY(output_ptr(g, 2, nbrs, (size_t)*total * 4, &dn, &hn));
    if (wts) GV_TRY(output_ptr(g, 4, wts, (size_t)*total * 4, &dw, &hw));
    GV_TRY(ensure_touched(g, n));
    GV_TRY(ensure_items(g, item_bound(g, n)));
    v = view(g);
    GV_CK(gv::launch_neighbor_copy(v, (const uint32_t *)dv, n, (const unsigned long long *)doff, (uint32_t *)dn,
                                   lcfg(g, s), (uint32_t *)dw));
    if (hn) GV_CK(cudaMemcpyAsync(nbrs, dn, (size_t)*total * 4, cudaMemcpyDeviceToHost, s));
    if (hw) GV_CK(cudaMemcpyAsync(wts, dw, (size_t)*total * 4, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    return check_launch();
}

}  // namespace

// ====================================================================== ABI

extern "C" {

const char *gv_status_string(gv_status s) {
    switch (s) {
    case GV_OK: return "GV_OK";
    case GV_ERR_INVALID_ARG: return "GV_ERR_INVALID_ARG";
    case GV_ERR_OUT_OF_MEMORY: return "GV_ERR_OUT_OF_MEMORY";
    case GV_ERR_CUDA: return "GV_ERR_CUDA";
    case GV_ERR_TIMEOUT: return "GV_ERR_TIMEOUT";
    case GV_ERR_STATE: return "GV_ERR_STATE";
    }
    return "GV_ERR_UNKNOWN";
}

gv_status gv_create(const gv_config *cfg, uint32_t num_vertices, void *stream, gv_graph **out) {
    if (!out) return GV_ERR_INVALID_ARG;
    *out = nullptr;
    gv_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.block_capacity != 0 && (c.block_capacity < 4 || c.block_capacity > 512 || c.block_capacity % 4))
        return GV_ERR_INVALID_ARG;
    if (c.flags & ~(GV_DEDUP | GV_GROW | GV_WEIGHTED | GV_RADIX_GROUPING)) return GV_ERR_INVALID_ARG;
    // which of several repeated (u, v) a set-semantics batch keeps is not
    // defined, so their payloads would be: the two flags exclude each other
    if ((c.flags & GV_DEDUP) && (c.flags & GV_WEIGHTED)) return GV_ERR_INVALID_ARG;
    if ((c.flags & GV_GROW) && c.pool_mem) return GV_ERR_INVALID_ARG;  // a caller-owned pool cannot grow
    if (c.pool_mem && c.pool_bytes == 0) return GV_ERR_INVALID_ARG;
    if (num_vertices > 0x7FFFFFFFu) return GV_ERR_INVALID_ARG;
    // hub runs: R = 2^s with TINY_NB <= R (a small run adjacency lies in one
    // run) and s <= 8; excluded with the radix grouping
    if (c.hub_shift != 0 && (c.hub_shift < 3 || c.hub_shift > 8)) return GV_ERR_INVALID_ARG;
    if (c.hub_shift && (c.flags & GV_RADIX_GROUPING)) return GV_ERR_INVALID_ARG;
    if (c.hub_percent > 90) return GV_ERR_INVALID_ARG;
    gv_graph *g = new (std::nothrow) gv_graph();
    if (!g) return GV_ERR_OUT_OF_MEMORY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return GV_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (g->num_sms <= 0) g->num_sms = 1;
    // without them the two mark tiers simply run one after the other
    if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (g->side) cudaStreamDestroy(g->side);
        if (g->ev_fork) cudaEventDestroy(g->ev_fork);
        g->side = nullptr;
        g->ev_fork = g->ev_join = nullptr;
    }
    // copy stream and staging events; without them host inputs are copied
    // on the call stream
    if (cudaStreamCreateWithFlags(&g->copy, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g->copy = nullptr;
    }
    for (auto &set : g->in_sets) {
        bool ok = g->copy && cudaEventCreateWithFlags(&set.free_ev, cudaEventDisableTiming) == cudaSuccess;
        for (auto &e : set.piece) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (set.free_ev) cudaEventDestroy(set.free_ev);
            for (auto &e : set.piece) {
                if (e) cudaEventDestroy(e);
                e = nullptr;
            }
            set.free_ev = nullptr;  // this set copies on the call stream
        }
    }
    g->flags = c.flags;
    g->rs = c.hub_shift;
    g->hub_deg_cfg = c.hub_degree;
    g->hub_pct = c.hub_percent ? c.hub_percent : 50;
    g->item_blocks_cfg = c.item_blocks;
    if (c.dense_shift) g->dense_shift = std::min<uint32_t>(c.dense_shift, 31);
    g->pool_bytes_cfg = c.pool_bytes;
    g->pool_mem_cfg = c.pool_mem;
    g->last_stream = s;
    gv_status st = GV_OK;
    do {
        if ((st = dalloc(&g->dev, 1, &g->scratch_bytes)) != GV_OK) break;
        if (cudaMemsetAsync(g->dev, 0, sizeof(Dev), s) != cudaSuccess) { st = GV_ERR_CUDA; break; }
        void *hp = nullptr;
        if (cudaMallocHost(&hp, 64) != cudaSuccess) { st = GV_ERR_OUT_OF_MEMORY; break; }
        g->h_small = static_cast<unsigned long long *>(hp);
        if (cudaMallocHost(&hp, sizeof(Dev)) != cudaSuccess) { st = GV_ERR_OUT_OF_MEMORY; break; }
        g->h_dev = static_cast<Dev *>(hp);
        uint32_t want = std::max<uint32_t>(num_vertices, c.vertex_capacity);
        want = next_pow2(std::max<uint32_t>(want, 1));  // "closest power of 2" at or above
        if ((st = ensure_vertex_capacity(g, want, s)) != GV_OK) break;
        g->nv = num_vertices;
        GraphView v = view(g);
        if (gv::launch_init_vertices(v, 0, num_vertices, lcfg(g, s)) != cudaSuccess) { st = GV_ERR_CUDA; break; }
        if (c.block_capacity) {
            if ((st = setup_pool(g, c.block_capacity, s)) != GV_OK) break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) { st = GV_ERR_CUDA; break; }
    } while (0);
    if (st != GV_OK) {
        cudaGetLastError();
        gv_destroy(g);
        return st;
    }
    *out = g;
    return GV_OK;
}

gv_status gv_destroy(gv_graph *g) {
    if (!g) return GV_OK;
    {
        DeviceGuard dg(g->device);
        cudaStreamSynchronize(g->last_stream);
        cudaGetLastError();
        if (g->pool_alloc) cudaFree(g->pool_alloc);
        dfree(g->sent); dfree(g->alive); dfree(g->vcnt); dfree(g->vinfo); dfree(g->vtid); dfree(g->dead);
        dfree(g->dev);
        dfree(g->t_vid); dfree(g->t_a); dfree(g->t_b); dfree(g->t_owner); dfree(g->t_rowner); dfree(g->rqueue); dfree(g->t_tiny); dfree(g->prank);
        dfree(g->items); dfree(g->it_mask); dfree(g->it_cnt); dfree(g->it_H); dfree(g->it_S); dfree(g->it_bid);
        dfree(g->arena); dfree(g->found); dfree(g->qpos); dfree(g->partials);
        dfree(g->owner_bits); dfree(g->vres);
        dfree(g->set_vbase); dfree(g->set_src); dfree(g->set_dst);
        dfree(g->pflag); dfree(g->dsrc2); dfree(g->dtmp);
        dfree(g->an_items); dfree(g->an_cur); dfree(g->an_next); dfree(g->an_ctr); dfree(g->an_stamp); dfree(g->rb_stats);
        dfree(g->pr_c); dfree(g->pr_acc); dfree(g->pr_scal); dfree(g->pr_n);
        dfree(g->pr_cursor); dfree(g->pr_src); dfree(g->pr_dst); dfree(g->pr_off); dfree(g->pr_part);
        dfree(g->gp_src); dfree(g->gp_dst); dfree(g->gp_aux); dfree(g->gp_hist);
        dfree(g->gp_btot); dfree(g->gp_bbase); dfree(g->gp_chunks); dfree(g->grp_items);
        dfree(g->gp_mbkt); dfree(g->gp_rows); dfree(g->go_src); dfree(g->go_dst); dfree(g->go_aux);
        for (auto &b : g->stage.buf) dfree(b.p);
        for (auto &r : g->prof.recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : g->prof.pool) cudaEventDestroy(e);
        if (g->h_small) cudaFreeHost(g->h_small);
        if (g->h_dev) cudaFreeHost(g->h_dev);
        if (g->side) {
            cudaStreamSynchronize(g->side);
            cudaStreamDestroy(g->side);
        }
        if (g->ev_fork) cudaEventDestroy(g->ev_fork);
        if (g->ev_join) cudaEventDestroy(g->ev_join);
        if (g->copy) {
            cudaStreamSynchronize(g->copy);
            cudaStreamDestroy(g->copy);
        }
        for (auto &set : g->in_sets) {
            dfree(set.src.p);
            dfree(set.dst.p);
            dfree(set.wts.p);
            if (set.free_ev) cudaEventDestroy(set.free_ev);
            for (auto e : set.piece)
                if (e) cudaEventDestroy(e);
        }
        cudaGetLastError();
    }
    delete g;
    return GV_OK;
}

gv_status gv_bulk_build(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, uint64_t *d_counts,
                        void *stream) {
    return insert_impl(g, src, dst, n, d_counts, static_cast<cudaStream_t>(stream));
}

gv_status gv_insert_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, uint64_t *d_counts,
                          void *stream) {
    return insert_impl(g, src, dst, n, d_counts, static_cast<cudaStream_t>(stream));
}

gv_status gv_delete_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, uint64_t *d_counts,
                          void *stream) {
    return member_impl(g, gv::MODE_DELETE, src, dst, n, d_counts, nullptr, static_cast<cudaStream_t>(stream));
}

gv_status gv_query_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *out,
                         void *stream) {
    return member_impl(g, gv::MODE_QUERY, src, dst, n, nullptr, out, static_cast<cudaStream_t>(stream));
}

gv_status gv_neighbors(gv_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets, uint32_t *nbrs,
                       uint64_t nbr_capacity, uint64_t *total, void *stream) {
    return neighbors_impl(g, vids, n, offsets, nbrs, nbr_capacity, total, static_cast<cudaStream_t>(stream), false);
}

gv_status gv_export_csr(gv_graph *g, uint64_t *offsets, uint32_t *nbrs, uint64_t nbr_capacity, uint64_t *total,
                        void *stream) {
    if (!g) return GV_ERR_INVALID_ARG;
    return neighbors_impl(g, nullptr, g->nv, offsets, nbrs, nbr_capacity, total, static_cast<cudaStream_t>(stream),
                          true);
}

gv_status gv_degrees(gv_graph *g, uint32_t *deg, uint8_t *alive, void *stream) {
    if (!g || (!deg && g->nv)) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    if (g->nv == 0) return GV_OK;
    void *dd = deg, *da = alive;
    bool hd = false, ha = false;
    GV_TRY(output_ptr(g, 0, deg, (size_t)g->nv * 4, &dd, &hd));
    if (alive) GV_TRY(output_ptr(g, 1, alive, g->nv, &da, &ha));
    GV_CK(gv::launch_degrees(view(g), (uint32_t *)dd, (uint8_t *)da, lcfg(g, s)));
    if (hd) GV_CK(cudaMemcpyAsync(deg, dd, (size_t)g->nv * 4, cudaMemcpyDeviceToHost, s));
    if (ha) GV_CK(cudaMemcpyAsync(alive, da, g->nv, cudaMemcpyDeviceToHost, s));
    if (hd || ha) GV_CK(cudaStreamSynchronize(s));
    return check_launch();
}

gv_status gv_insert_vertices(gv_graph *g, uint32_t k, uint32_t *new_ids, void *stream) {
    if (!g) return GV_ERR_INVALID_ARG;
    if ((uint64_t)g->nv + k > 0x7FFFFFFFull) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    if (k == 0) return GV_OK;
    const uint32_t first = g->nv;
    GV_TRY(ensure_vertex_capacity(g, first + k, s));
    GV_CK(gv::launch_init_vertices(view(g), first, first + k, lcfg(g, s)));
    g->nv = first + k;
    if (new_ids) {
        void *d = new_ids;
        bool h = false;
        GV_TRY(output_ptr(g, 4, new_ids, (size_t)k * 4, &d, &h));
        GV_CK(gv::launch_iota((uint32_t *)d, first, k, lcfg(g, s)));
        if (h) {
            GV_CK(cudaMemcpyAsync(new_ids, d, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
            GV_CK(cudaStreamSynchronize(s));
        }
    }
    return check_launch();
}

gv_status gv_delete_vertices(gv_graph *g, const uint32_t *ids, uint32_t k, void *stream) {
    if (!g) return GV_ERR_INVALID_ARG;
    if (k > 0 && !ids) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    if (k == 0) return GV_OK;
    const void *di = ids;
    GV_TRY(input_ptr(g, 0, ids, (size_t)k * 4, s, &di));
    GV_TRY(ensure_touched(g, std::max<unsigned long long>(g->nv, 1)));
    if (g->C == 0) {
        // No pool yet, hence no edges: only the alive flags change.  Reuse
        // the delete kernels with an empty pool view (no items are formed).
        GV_TRY(ensure_items(g, 1024));
    } else {
        GV_TRY(ensure_items(g, item_bound(g, g->nv)));
    }
    GraphView v = view(g);
    if (v.C == 0) {
        v.C = 4;
        v.IB = 32;
        v.cmul = (1ull << 40) / 4;
    }
    g->any_vertex_deleted = true;
    v.all_alive = 0;
    GV_CK(gv::launch_vertex_delete(v, (const uint32_t *)di, k, lcfg(g, s)));
    return check_launch();
}

gv_status gv_reserve(gv_graph *g, uint64_t max_batch) {
    if (!g || max_batch > kMaxBatch) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    GV_TRY(ensure_touched(g, std::min<unsigned long long>(max_batch, g->nv ? g->nv : 1)));
    GV_TRY(ensure_owner(g, (g->C ? max_batch / g->C : max_batch) + std::min<unsigned long long>(max_batch, g->nv) + 1));
    if (g->C) GV_TRY(ensure_items(g, item_bound(g, std::min<unsigned long long>(max_batch, g->nv ? g->nv : 1))));
    if ((g->flags & GV_RADIX_GROUPING) && !g->set_G && max_batch > 0)
        GV_TRY(ensure_group(g, max_batch, true, true,
                            g->C ? item_bound(g, std::min<unsigned long long>(max_batch, g->nv ? g->nv : 1)) : 0));
    GV_TRY(ensure_arena(g, 5 * max_batch + 128, true, max_batch));
    GV_TRY(ensure_ranks(g, max_batch));
    if (g->set_G && (max_batch > g->scap || !g->scap)) {
        dfree(g->set_src);
        dfree(g->set_dst);
        g->scap = 0;
        GV_TRY(dalloc(&g->set_src, std::max<uint64_t>(max_batch, 1), &g->scratch_bytes));
        GV_TRY(dalloc(&g->set_dst, std::max<uint64_t>(max_batch, 1), &g->scratch_bytes));
        g->scap = std::max<uint64_t>(max_batch, 1);
    }
    for (int slot = 0; slot < 4; ++slot) {
        void *d = nullptr;
        GV_TRY(stage_buf(g, slot, max_batch * 4 + 64, &d));
    }
    return GV_OK;
}

gv_status gv_reblock(gv_graph *g, uint32_t block_capacity, uint32_t *h_block_capacity, void *stream) {
    if (!g) return GV_ERR_INVALID_ARG;
    if (block_capacity && block_capacity != GV_REBLOCK_MIN_FOOTPRINT &&
        (block_capacity < 4 || block_capacity > 512 || block_capacity % 4))
        return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g->C == 0) return GV_ERR_STATE;  // nothing laid out yet: the first edge batch fixes C
    // a latched device error is reported first; nothing changes
    GV_CK(cudaStreamSynchronize(g->last_stream));
    g->last_stream = s;
    GV_CK(cudaMemcpyAsync(&g->h_small[0], &g->dev->status, 4, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    const unsigned int st0 = (unsigned int)(g->h_small[0] & 0xFFFFFFFFull);
    if (st0) return static_cast<gv_status>(st0);
    const uint32_t n = g->nv;
    const bool weighted = (g->flags & GV_WEIGHTED) != 0;

    // 1. the new C: given, the paper's rule over the current degrees, or the
    // size of least pool footprint (blocks at every candidate size counted
    // on the device, bytes compared here; the smallest C wins ties)
    if (!g->rb_stats) GV_TRY(dalloc(&g->rb_stats, 128, &g->scratch_bytes));
    uint32_t C2 = block_capacity;
    if (block_capacity == GV_REBLOCK_MIN_FOOTPRINT) {
        std::vector<unsigned long long> blocks(128);
        GV_CK(gv::launch_footprint_blocks(view(g), g->rb_stats, lcfg(g, s)));
        GV_CK(cudaMemcpyAsync(blocks.data(), g->rb_stats, 128 * 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        unsigned long long best = ~0ull;
        for (uint32_t i = 0; i < 128; ++i) {
            const uint32_t c = 4 * (i + 1);
            const unsigned long long bytes = blocks[i] * (4ull * c * (weighted ? 2 : 1) + 12);
            if (bytes < best) {
                best = bytes;
                C2 = c;
            }
        }
    } else if (block_capacity == 0) {
        GV_CK(gv::launch_degree_stats(view(g), g->rb_stats, lcfg(g, s)));
        GV_CK(cudaMemcpyAsync(&g->h_small[0], g->rb_stats, 16, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        C2 = rule_capacity(g->h_small[0], g->h_small[1]);
    }
    unsigned long long P2 = fit_blocks(g->pool_bytes, C2, weighted);
    // hub runs: the run region is laid out again for C2 (the same share of
    // the pool), and every vertex of degree >= T2 (the hub threshold at C2)
    // becomes a hub, every other vertex a plain one
    const bool hubs = g->rs != 0;
    if (hubs && P2 > 0x7FFFFFFEull) P2 = 0x7FFFFFFEull;
    const unsigned long long RP2 = hubs ? (P2 * g->hub_pct / 100) >> g->rs : 0ull;
    const unsigned long long H2 = RP2 << g->rs;
    const uint32_t T2 = hubs ? (g->hub_deg_cfg ? g->hub_deg_cfg : C2 << g->rs) : 0xFFFFFFFFu;
    if (hubs && RP2 == 0) return GV_ERR_OUT_OF_MEMORY;

    // 2. slot offsets of the new layout (each vertex's degree rounded up to
    // whole blocks of C2): the run of u starts at block slots[u] / C2.  With
    // hub runs the scratch holds the hubs' runs (whole runs of 2^s blocks)
    // first, then the plain vertices'.
    // Scratch is the graph's own, kept between calls: the vertex list and
    // the run offsets in staging buffers, the new slots (and payloads) in the
    // membership arena and its parallel array (per-call scratch of deletes
    // and queries).
    unsigned long long *slots = nullptr;
    uint32_t *nd = nullptr, *nw = nullptr;
    void *dv = nullptr;
    GV_TRY(stage_buf(g, 0, (size_t)n * 4 + 4, &dv));
    GV_CK(gv::launch_iota((uint32_t *)dv, 0, n, lcfg(g, s)));
    const unsigned long long nchunks = ((unsigned long long)n + 1023) / 1024;
    if (nchunks + 1 > g->pcap) {
        dfree(g->partials);
        g->pcap = 0;
        GV_TRY(dalloc(&g->partials, nchunks + 1, &g->scratch_bytes));
        g->pcap = nchunks + 1;
    }
    void *ds = nullptr;
    GV_TRY(stage_buf(g, 1, ((size_t)n + 1) * 8, &ds));
    slots = static_cast<unsigned long long *>(ds);
    unsigned long long T = 0, hub_total = 0;  // slots of the new layout, of its hubs' runs
    if (!hubs) {
        GV_CK(gv::launch_neighbor_offsets(view(g), (const uint32_t *)dv, n, slots, g->partials, lcfg(g, s), C2));
        GV_CK(cudaMemcpyAsync(&g->h_small[0], slots + n, 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        T = g->h_small[0];
    } else {
        void *dh = nullptr;
        GV_TRY(stage_buf(g, 2, ((size_t)n + 1) * 8, &dh));
        unsigned long long *hslots = static_cast<unsigned long long *>(dh);
        GV_CK(gv::launch_reblock_offsets(view(g), (const uint32_t *)dv, n, hslots, g->partials, lcfg(g, s), C2, true,
                                         T2, g->rs));
        GV_CK(cudaMemcpyAsync(&g->h_small[0], hslots + n, 8, cudaMemcpyDeviceToHost, s));
        GV_CK(gv::launch_reblock_offsets(view(g), (const uint32_t *)dv, n, slots, g->partials, lcfg(g, s), C2, false,
                                         T2, g->rs));
        GV_CK(cudaMemcpyAsync(&g->h_small[1], slots + n, 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        hub_total = g->h_small[0];
        T = hub_total + g->h_small[1];
        GV_CK(gv::launch_reblock_merge(view(g), slots, hslots, T2, hub_total, lcfg(g, s)));
    }
    const unsigned long long nb2 = T / C2;
    const unsigned long long hb2 = hub_total / C2;  // blocks in runs
    // the entries must fit the pool at this block size (with hub runs: the
    // plain blocks outside the run region, the hubs' runs inside it)
    if (nb2 > P2 || nb2 > 0xFFFFFFFEull) return GV_ERR_OUT_OF_MEMORY;
    if (hubs && (nb2 - hb2 > P2 - H2 || hb2 > H2)) return GV_ERR_OUT_OF_MEMORY;

    // 3. every entry (and payload) copied to its place in the new layout,
    // read through the old trees
    GV_TRY(ensure_arena(g, std::max<unsigned long long>(T, 4), false, 0));
    GV_TRY(ensure_touched(g, n));
    GV_TRY(ensure_items(g, item_bound(g, n)));
    nd = g->arena;
    nw = weighted ? g->found : nullptr;
    // the unused tail slots of each run's last block hold NIL
    GV_CK(cudaMemsetAsync(nd, 0xFF, T * 4ull, s));
    if (n) GV_CK(gv::launch_neighbor_copy(view(g), (const uint32_t *)dv, n, slots, nd, lcfg(g, s), nw));
    GV_CK(cudaStreamSynchronize(s));

    // 4. the same pool memory laid out for C2: slots back in place, trees
    // and sentinels over the runs, the queue holding the blocks past them
    uint32_t *rq2 = nullptr;  // the run queue at the new size, allocated before the pool changes
    if (hubs && RP2 > g->RP) GV_TRY(dalloc(&rq2, RP2, &g->scratch_bytes));
    char *base = reinterpret_cast<char *>(g->data);
    if (!lay_out_pool(g, base, g->pool_bytes, C2, P2)) return GV_ERR_STATE;  // cannot happen: P2 was fitted
    set_item_blocks(g);
    if (rq2) {
        dfree(g->rqueue);
        g->rqueue = rq2;
    }
    if (hubs) g->RP = RP2;
    const GraphView v = view(g);
    bool ok = true;
    // hubs' runs at block 0 (the run region), the plain vertices' from block H2
    const unsigned long long hs = hb2 * C2, ps = T - hs, pdst = H2 * C2;
    if (hs) ok = ok && cudaMemcpyAsync(g->data, nd, hs * 4ull, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    if (ps) ok = ok && cudaMemcpyAsync(g->data + pdst, nd + hs, ps * 4ull, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    if (hs && weighted) ok = ok && cudaMemcpyAsync(g->wdata, nw, hs * 4ull, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    if (ps && weighted)
        ok = ok && cudaMemcpyAsync(g->wdata + pdst, nw + hs, ps * 4ull, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    // long runs are listed in the touched-vertex scratch (n entries), counted in rb_stats[0]
    ok = ok && gv::launch_reblock_place(v, slots, g->t_vid, g->rb_stats, lcfg(g, s), T2, pdst - hs) == cudaSuccess;
    // the edge queue: the blocks past the plain runs (outside the run
    // region); the run queue: the runs past the hubs'
    ok = ok && gv::launch_init_queue(g->queue, P2 - H2, lcfg(g, s), (uint32_t)H2, 1u) == cudaSuccess;
    g->h_small[2] = nb2 - hb2;
    g->h_small[3] = P2 - H2;
    ok = ok && cudaMemcpyAsync(&g->dev->q_front, &g->h_small[2], 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&g->dev->q_back, &g->h_small[3], 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (hubs) {
        ok = ok && gv::launch_init_queue(g->rqueue, RP2, lcfg(g, s), 0u, 1u << g->rs) == cudaSuccess;
        g->h_small[4] = hb2 >> g->rs;
        g->h_small[5] = RP2;
        ok = ok && cudaMemcpyAsync(&g->dev->rq_front, &g->h_small[4], 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(&g->dev->rq_back, &g->h_small[5], 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) return GV_ERR_CUDA;
    g->used_ub = nb2;
    // work-item scratch is sized by the blocks per item, which follow C
    if (g->IB > g->ib_alloc) g->icap = 0;  // forces a new allocation
    GV_TRY(ensure_items(g, item_bound(g, 1024)));
    if (h_block_capacity) *h_block_capacity = C2;
    return check_launch();
}

gv_status gv_sync(gv_graph *g) {
    if (!g) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    GV_CK(cudaStreamSynchronize(g->last_stream));
    unsigned int st = 0;
    GV_CK(cudaMemcpy(&st, &g->dev->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st) GV_CK(cudaMemset(&g->dev->status, 0, sizeof(st)));
    return static_cast<gv_status>(st);
}

gv_status gv_stats(gv_graph *g, gv_stats_t *out) {
    if (!g || !out) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    GV_CK(cudaStreamSynchronize(g->last_stream));
    GV_CK(cudaMemcpy(g->h_dev, g->dev, sizeof(Dev), cudaMemcpyDeviceToHost));
    const Dev &d = *g->h_dev;
    std::memset(out, 0, sizeof(*out));
    out->num_vertices = g->nv;
    out->vertex_capacity = g->vcap;
    out->block_capacity = g->C;
    out->flags = g->flags;
    out->num_edges = d.num_edges;
    out->pool_blocks = g->P;
    out->pool_blocks_free = d.q_back - d.q_front + ((d.rq_back - d.rq_front) << g->rs);
    out->pool_blocks_used = g->P - out->pool_blocks_free;
    out->hub_shift = g->rs;
    out->pool_runs = g->RP;
    out->pool_runs_free = d.rq_back - d.rq_front;
    out->pool_bytes = g->pool_bytes;
    uint64_t stage_bytes = 0;
    for (auto &b : g->stage.buf) stage_bytes += b.bytes;
    out->device_bytes = (g->pool_alloc ? g->pool_bytes : 0) + g->dict_bytes + g->scratch_bytes + stage_bytes;
    out->total_inserted = d.tot_ins;
    out->total_deleted = d.tot_del;
    out->total_rejected = d.tot_rej;
    out->device_status = d.status;
    if (d.status) GV_CK(cudaMemset(&g->dev->status, 0, sizeof(unsigned int)));
    return static_cast<gv_status>(d.status);
}

gv_status gv_validate(gv_graph *g, uint64_t *violations, void *stream) {
    if (!g || !violations) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    const unsigned long long words = g->P / 32 + 1;
    dfree(g->owner_bits);
    GV_TRY(dalloc(&g->owner_bits, words, nullptr));
    if (!g->vres) GV_TRY(dalloc(&g->vres, 4, nullptr));
    GV_CK(cudaMemsetAsync(g->owner_bits, 0, words * 4, s));
    GV_CK(cudaMemsetAsync(g->vres, 0, 32, s));
    GraphView v = view(g);
    GV_CK(gv::launch_validate(v, g->owner_bits, g->vres, lcfg(g, s)));
    unsigned long long r[4];
    GV_CK(cudaMemcpyAsync(r, g->vres, 32, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaMemcpyAsync(g->h_dev, g->dev, sizeof(Dev), cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    uint64_t viol = r[0];
    if (r[1] != g->h_dev->num_edges) ++viol;         // degree sum = edge count
    if (g->C && r[2] + r[3] != g->P) ++viol;          // owned + queued = pool
    *violations = viol;
    dfree(g->owner_bits);
    return check_launch();
}

// ----------------------------------------------------------------------------
// Allocation-free degree offsets (gv_degree_offsets_noalloc).
//
// The chunk sums of the prefix scan live in a fixed device array instead of
// library-allocated memory, so the call performs no allocation at all.  Every
// GPU that loads this library holds the array (512 KiB) until the process
// exits.  In host code `g_noalloc_partials` is only a host-side stand-in for
// the symbol: its device address is taken by cudaGetSymbolAddress, with the
// device current, on the first call made on that device, and taken again
// only if the device's context has been replaced since (cudaDeviceReset
// destroys the context and the module with it, so an address cached from the
// old context would point at freed memory).

}  // extern "C"

namespace {
constexpr uint32_t kNoAllocMaxVertices = 1u << 26;  // ids per call
constexpr uint32_t kNoAllocChunks = (kNoAllocMaxVertices + gv::SCAN_CHUNK - 1) / gv::SCAN_CHUNK;
// launch_neighbor_offsets writes one chunk sum per SCAN_CHUNK ids plus the
// total: the array must hold that many for the largest call accepted
static_assert((unsigned long long)kNoAllocChunks * gv::SCAN_CHUNK >= kNoAllocMaxVertices,
              "scratch array too small for the largest call");
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};
CUcontext g_noalloc_ctx[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned long long g_noalloc_partials[kNoAllocChunks + 1];

namespace {
// The driver's current context of the calling thread, through the runtime's
// driver entry point (no link against the driver library); nullptr if the
// entry point is unavailable.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<Fn>(p);
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of the scratch array on `dev` (which must be current).
gv_status noalloc_scratch(int dev, unsigned long long **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const CUcontext ctx = current_context();
    // without a context handle to compare, look the address up on every call
    if (!g_noalloc_addr[dev] || ctx == nullptr || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();  // this call's own error (no error was pending at entry)
            g_noalloc_addr[dev] = nullptr;
            return GV_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned long long *>(g_noalloc_addr[dev]);
    return GV_OK;
}
}  // namespace

extern "C" {

gv_status gv_degree_offsets_noalloc(gv_graph *g, const uint32_t *d_vids, uint32_t n, uint64_t *d_offsets,
                                    void *stream) {
    if (!g || !d_offsets || (n > 0 && !d_vids)) return GV_ERR_INVALID_ARG;
    if (n > kNoAllocMaxVertices) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    // an error the caller's own work left pending is reported, not cleared
    if (cudaPeekAtLastError() != cudaSuccess) return GV_ERR_CUDA;
    // Host arrays would need staging buffers, i.e. an allocation.
    if (is_host_ptr(d_offsets) || (n > 0 && is_host_ptr(d_vids))) return GV_ERR_INVALID_ARG;
    unsigned long long *scratch = nullptr;
    GV_TRY(noalloc_scratch(g->device, &scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    gv::LaunchCfg lc;  // no profiler: event creation is avoided as well
    lc.num_sms = g->num_sms;
    lc.stream = s;
    lc.prof = nullptr;
    GV_CK(gv::launch_neighbor_offsets(view(g), d_vids, n, reinterpret_cast<unsigned long long *>(d_offsets),
                                      scratch, lc));
    return check_launch();
}

// ---------------------------------------------------------------- graph sets

}  // extern "C"

namespace {

gv_status set_batch(gv_graph *g, int mode, const uint32_t *src, const uint32_t *dst, uint64_t n,
                    const uint64_t *d_offsets, uint64_t *d_counts, uint8_t *out, cudaStream_t s) {
    if (!g || g->set_G == 0) return GV_ERR_INVALID_ARG;
    if (n > kMaxBatch || !d_offsets || !d_counts || (n > 0 && (!src || !dst))) return GV_ERR_INVALID_ARG;
    if (mode == gv::MODE_QUERY && n > 0 && !out) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    // device arrays only: host staging would allocate and synchronise
    if (is_host_ptr(d_offsets) || is_host_ptr(d_counts) || (n > 0 && (is_host_ptr(src) || is_host_ptr(dst))) ||
        (out && is_host_ptr(out)))
        return GV_ERR_INVALID_ARG;
    g->last_stream = s;
    GV_CK(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 2 * g->set_G, s));
    if (n == 0) return check_launch();
    if (n > g->scap || !g->scap) {
        unsigned long long cap = std::max<unsigned long long>(n, 2 * g->scap);
        dfree(g->set_src);
        dfree(g->set_dst);
        g->scap = 0;
        GV_TRY(dalloc(&g->set_src, cap, &g->scratch_bytes));
        GV_TRY(dalloc(&g->set_dst, cap, &g->scratch_bytes));
        g->scap = cap;
    }
    GraphView v = view(g);
    v.set_G = g->set_G;
    v.set_vbase = g->set_vbase;
    v.set_off = reinterpret_cast<const unsigned long long *>(d_offsets);
    v.set_counts = reinterpret_cast<unsigned long long *>(d_counts);
    GV_CK(gv::launch_set_remap(v, src, dst, n, g->set_src, g->set_dst, lcfg(g, s)));
    if (mode == gv::MODE_INSERT) {
        if (g->C == 0) return GV_ERR_STATE;  // sets are created with a fixed C
        GV_TRY(ensure_batch(g, n, gv::MODE_INSERT));
        GraphView w = view(g);
        GV_CK(gv::launch_count(gv::MODE_INSERT, w, g->set_src, g->set_dst, n, lcfg(g, s)));
        GV_CK(gv::launch_insert_tail(w, g->set_src, g->set_dst, n, g->tcap, nullptr, lcfg(g, s)));
        GV_CK(gv::launch_set_insert_counts(v, lcfg(g, s)));
    } else {
        GV_TRY(ensure_batch(g, n, mode));
        GraphView w = view(g);
        w.set_G = v.set_G;
        w.set_vbase = v.set_vbase;
        w.set_off = v.set_off;
        w.set_counts = v.set_counts;
        GV_CK(gv::launch_count(mode, w, g->set_src, g->set_dst, n, lcfg(g, s)));
        GV_CK(gv::launch_member_tail(mode, w, g->set_src, g->set_dst, n, g->tcap, nullptr, out, lcfg(g, s)));
    }
    return check_launch();
}

}  // namespace

extern "C" {

gv_status gv_insert_edges_segmented(gv_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    const uint64_t *d_offsets, uint32_t nseg, uint64_t *d_counts, void *stream) {
    if (!g || g->set_G || nseg == 0 || nseg > gv::SET_MAX_G || !d_offsets || !d_counts) return GV_ERR_INVALID_ARG;
    if (n > kMaxBatch || (n > 0 && (!d_src || !d_dst))) return GV_ERR_INVALID_ARG;
    if (g->flags & GV_DEDUP) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (is_host_ptr(d_offsets) || is_host_ptr(d_counts) || (n > 0 && (is_host_ptr(d_src) || is_host_ptr(d_dst))))
        return GV_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    GV_CK(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 2 * nseg, s));
    if (n == 0) return check_launch();
    if (g->C == 0) return GV_ERR_STATE;  // the first edge batch fixes C: use gv_bulk_build
    GraphView v = view(g);
    v.set_G = nseg;
    v.set_off = reinterpret_cast<const unsigned long long *>(d_offsets);
    v.set_counts = reinterpret_cast<unsigned long long *>(d_counts);
    GV_CK(gv::launch_segment_counts(v, d_src, d_dst, n, lcfg(g, s)));
    GV_CK(gv::launch_set_insert_counts(v, lcfg(g, s)));
    if (!g->dtmp) GV_TRY(dalloc(&g->dtmp, 4, &g->scratch_bytes));
    GV_TRY(insert_impl(g, d_src, d_dst, n, reinterpret_cast<uint64_t *>(g->dtmp), s));
    // an insert that ran out of pool blocks is a no-op: every segment {0, 0}
    GV_CK(gv::launch_segment_noop_check(v, g->dtmp, n, lcfg(g, s)));
    return check_launch();
}

gv_status gv_insert_edges_weighted(gv_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                                   uint64_t n, uint64_t *d_counts, void *stream) {
    if (!g || (n > 0 && !w)) return GV_ERR_INVALID_ARG;
    if (!(g->flags & GV_WEIGHTED) || g->set_G) return GV_ERR_INVALID_ARG;
    return insert_impl(g, src, dst, n, d_counts, static_cast<cudaStream_t>(stream), w);
}

gv_status gv_neighbors_weighted(gv_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets, uint32_t *nbrs,
                                uint32_t *weights, uint64_t nbr_capacity, uint64_t *total, void *stream) {
    if (!g || !(g->flags & GV_WEIGHTED)) return GV_ERR_INVALID_ARG;
    return neighbors_impl(g, vids, n, offsets, nbrs, nbr_capacity, total, static_cast<cudaStream_t>(stream), false,
                          weights);
}

gv_status gv_delete_edges_segmented(gv_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    const uint64_t *d_offsets, uint32_t nseg, uint64_t *d_counts, void *stream) {
    if (!g || g->set_G || nseg == 0 || nseg > gv::SET_MAX_G || !d_offsets || !d_counts) return GV_ERR_INVALID_ARG;
    if (n > kMaxBatch || (n > 0 && (!d_src || !d_dst))) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (is_host_ptr(d_offsets) || is_host_ptr(d_counts) || (n > 0 && (is_host_ptr(d_src) || is_host_ptr(d_dst))))
        return GV_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    GV_CK(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 2 * nseg, s));
    if (n == 0) return check_launch();
    GraphView v = view(g);
    v.set_G = nseg;
    v.set_off = reinterpret_cast<const unsigned long long *>(d_offsets);
    v.set_counts = reinterpret_cast<unsigned long long *>(d_counts);
    GV_CK(gv::launch_segment_counts(v, d_src, d_dst, n, lcfg(g, s)));  // rejected pairs per segment
    if (g->C == 0) return check_launch();                               // nothing stored: nothing to delete
    GV_TRY(ensure_batch(g, n, gv::MODE_DELETE));
    GraphView w = view(g);
    w.set_G = nseg;
    w.set_off = v.set_off;
    w.set_counts = v.set_counts;
    w.seg_own = g->found;  // owner segment per arena word (the delete leaves `found` unused)
    GV_CK(gv::launch_count(gv::MODE_DELETE, w, d_src, d_dst, n, lcfg(g, s)));
    GV_CK(gv::launch_member_tail(gv::MODE_DELETE, w, d_src, d_dst, n, g->tcap, nullptr, nullptr, lcfg(g, s)));
    return check_launch();
}

gv_status gv_set_create(const gv_config *cfg, uint32_t num_graphs, const uint32_t *num_vertices, void *stream,
                        gv_graph **out) {
    if (!out || num_graphs == 0 || num_graphs > gv::SET_MAX_G || !num_vertices) return GV_ERR_INVALID_ARG;
    if (!cfg || cfg->block_capacity == 0 || (cfg->flags & GV_DEDUP)) return GV_ERR_INVALID_ARG;
    if (cfg->hub_shift) return GV_ERR_INVALID_ARG;  // hub runs: plain graphs only
    std::vector<uint32_t> base(num_graphs + 1, 0);
    uint64_t tot = 0;
    for (uint32_t i = 0; i < num_graphs; ++i) {
        base[i] = (uint32_t)tot;
        tot += num_vertices[i];
        if (tot > 0x7FFFFFFFull) return GV_ERR_INVALID_ARG;
    }
    base[num_graphs] = (uint32_t)tot;
    gv_graph *g = nullptr;
    GV_TRY(gv_create(cfg, (uint32_t)tot, stream, &g));
    DeviceGuard dg(g->device);
    gv_status st = dalloc(&g->set_vbase, num_graphs + 1, &g->scratch_bytes);
    if (st == GV_OK &&
        cudaMemcpy(g->set_vbase, base.data(), sizeof(uint32_t) * (num_graphs + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        st = GV_ERR_CUDA;
    if (st != GV_OK) {
        gv_destroy(g);
        return st;
    }
    g->set_G = num_graphs;
    g->set_vbase_h = base;
    *out = g;
    return GV_OK;
}

gv_status gv_set_insert_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              const uint64_t *d_offsets, uint64_t *d_counts, void *stream) {
    return set_batch(set, gv::MODE_INSERT, d_src, d_dst, n, d_offsets, d_counts, nullptr,
                     static_cast<cudaStream_t>(stream));
}

gv_status gv_set_delete_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              const uint64_t *d_offsets, uint64_t *d_counts, void *stream) {
    return set_batch(set, gv::MODE_DELETE, d_src, d_dst, n, d_offsets, d_counts, nullptr,
                     static_cast<cudaStream_t>(stream));
}

gv_status gv_set_query_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                             const uint64_t *d_offsets, uint64_t *d_counts, uint8_t *d_out, void *stream) {
    return set_batch(set, gv::MODE_QUERY, d_src, d_dst, n, d_offsets, d_counts, d_out,
                     static_cast<cudaStream_t>(stream));
}

gv_status gv_set_member_neighbors(gv_graph *set, uint32_t member, uint64_t *offsets, uint32_t *nbrs,
                                  uint64_t nbr_capacity, uint64_t *total, void *stream) {
    if (!set || set->set_G == 0 || member >= set->set_G) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(set->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t first = set->set_vbase_h[member];
    const uint32_t cnt = set->set_vbase_h[member + 1] - first;
    void *d = nullptr;
    GV_TRY(stage_buf(set, 5, (size_t)cnt * 4 + 4, &d));
    GV_CK(gv::launch_iota((uint32_t *)d, first, cnt, lcfg(set, s)));
    return neighbors_impl(set, (const uint32_t *)d, cnt, offsets, nbrs, nbr_capacity, total, s, false);
}

// --------------------------------------------------------------- analytics

namespace {

// Blocks per analytics work item: up to 512 entries, at most 32 blocks.
uint32_t analytics_item_blocks(const gv_graph *g) {
    return g->C ? std::min<uint32_t>(32, std::max<uint32_t>(1, 512 / g->C)) : 32;
}

gv_status ensure_analytics(gv_graph *g, bool pagerank, bool sssp = false) {
    const uint32_t aib = analytics_item_blocks(g);
    const unsigned long long items = (unsigned long long)g->nv + (g->P + aib - 1) / aib + 1;
    if (items > g->an_icap || !g->an_icap) {
        dfree(g->an_items);
        g->an_icap = 0;
        GV_TRY(dalloc(&g->an_items, items, &g->scratch_bytes));
        g->an_icap = items;
    }
    const unsigned long long nv = std::max<unsigned long long>(g->nv, 1);
    if (nv > g->an_vcap || !g->an_vcap) {
        dfree(g->an_cur); dfree(g->an_next); dfree(g->pr_c); dfree(g->pr_acc); dfree(g->an_stamp);
        g->an_vcap = 0;
        GV_TRY(dalloc(&g->an_cur, nv, &g->scratch_bytes));
        GV_TRY(dalloc(&g->an_next, nv, &g->scratch_bytes));
        g->an_vcap = nv;
    }
    if (!g->an_ctr) GV_TRY(dalloc(&g->an_ctr, 4, &g->scratch_bytes));
    if (sssp && !g->an_stamp) GV_TRY(dalloc(&g->an_stamp, g->an_vcap, &g->scratch_bytes));
    if (pagerank) {
        if (!g->pr_c) GV_TRY(dalloc(&g->pr_c, g->an_vcap, &g->scratch_bytes));
        if (!g->pr_acc) GV_TRY(dalloc(&g->pr_acc, g->an_vcap, &g->scratch_bytes));
        if (!g->pr_scal) GV_TRY(dalloc(&g->pr_scal, 2, &g->scratch_bytes));
        if (!g->pr_n) GV_TRY(dalloc(&g->pr_n, 1, &g->scratch_bytes));
    }
    return GV_OK;
}

}  // namespace

gv_status gv_bfs(gv_graph *g, uint32_t source, uint32_t *dist, uint32_t *h_levels, void *stream) {
    if (!g || !dist || source >= g->nv) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    GV_TRY(ensure_analytics(g, false));
    void *dd = dist;
    bool hd = false;
    GV_TRY(output_ptr(g, 0, dist, (size_t)g->nv * 4, &dd, &hd));
    const GraphView v = view(g);
    const uint32_t aib = analytics_item_blocks(g);
    GV_CK(gv::launch_bfs_seed(v, source, (uint32_t *)dd, g->an_cur, g->an_ctr, lcfg(g, s)));
    uint32_t *cur = g->an_cur, *nxt = g->an_next;
    // Levels go out in groups of kGroup between two reads of the frontier
    // size (levels past the last one find an empty frontier and do nothing),
    // so a search of L levels synchronises about L / kGroup times.
    constexpr uint32_t kGroup = 4;
    for (uint32_t level = 0; level <= g->nv;) {
        for (uint32_t k = 0; k < kGroup; ++k, ++level) {
            GV_CK(gv::launch_bfs_level(v, aib, cur, nxt, g->an_items, g->an_ctr, (uint32_t *)dd, level, lcfg(g, s)));
            std::swap(cur, nxt);
        }
        GV_CK(cudaMemcpyAsync(g->h_small, g->an_ctr, 16, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        if ((uint32_t)(g->h_small[0] & 0xFFFFFFFFull) == 0) break;  // frontier empty
    }
    const uint32_t levels = (uint32_t)(g->h_small[1] >> 32);  // ctr[3]
    if (hd) {
        GV_CK(cudaMemcpyAsync(dist, dd, (size_t)g->nv * 4, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
    }
    if (h_levels) *h_levels = levels;
    return check_launch();
}

gv_status gv_sssp(gv_graph *g, uint32_t source, uint64_t *dist, uint32_t *h_rounds, void *stream) {
    if (!g || !dist || source >= g->nv) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    GV_TRY(ensure_analytics(g, false, true));
    void *dd = dist;
    bool hd = false;
    GV_TRY(output_ptr(g, 0, dist, (size_t)g->nv * 8, &dd, &hd));
    const GraphView v = view(g);
    const uint32_t aib = analytics_item_blocks(g);
    unsigned long long *ddist = static_cast<unsigned long long *>(dd);
    GV_CK(gv::launch_sssp_seed(v, source, ddist, g->an_stamp, g->an_cur, g->an_ctr, lcfg(g, s)));
    uint32_t *cur = g->an_cur, *nxt = g->an_next;
    // rounds go out in groups between two reads of the frontier size, as
    // the BFS levels do; with non-negative lengths round nv finds an empty
    // frontier
    constexpr uint32_t kGroup = 4;
    for (uint32_t round = 0; round <= g->nv;) {
        for (uint32_t k = 0; k < kGroup; ++k, ++round) {
            GV_CK(gv::launch_sssp_round(v, aib, cur, nxt, g->an_items, g->an_ctr, ddist, g->an_stamp, round,
                                        lcfg(g, s)));
            std::swap(cur, nxt);
        }
        GV_CK(cudaMemcpyAsync(g->h_small, g->an_ctr, 16, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
        if ((uint32_t)(g->h_small[0] & 0xFFFFFFFFull) == 0) break;  // frontier empty
    }
    const uint32_t rounds = (uint32_t)(g->h_small[1] >> 32);  // ctr[3]
    if (hd) {
        GV_CK(cudaMemcpyAsync(dist, dd, (size_t)g->nv * 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
    }
    if (h_rounds) *h_rounds = rounds;
    return check_launch();
}

gv_status gv_pagerank(gv_graph *g, uint32_t iterations, double damping, double *rank, void *stream) {
    if (!g || (!rank && g->nv) || !(damping >= 0.0 && damping <= 1.0)) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    if (g->nv == 0) return GV_OK;
    GV_TRY(ensure_analytics(g, true));
    // incoming-edge CSR scratch: sized by the vertex count and by the stored
    // entries (read once from the device)
    GV_CK(cudaMemcpyAsync(g->h_small, &g->dev->num_edges, 8, cudaMemcpyDeviceToHost, s));
    GV_CK(cudaStreamSynchronize(s));
    const unsigned long long E = std::max<unsigned long long>(g->h_small[0], 1);
    if (g->nv > g->pr_vcap || !g->pr_vcap) {
        dfree(g->pr_cursor); dfree(g->pr_off); dfree(g->pr_part);
        g->pr_vcap = 0;
        const unsigned long long cap = std::max<unsigned long long>(g->nv, 1024);
        GV_TRY(dalloc(&g->pr_cursor, cap, &g->scratch_bytes));
        GV_TRY(dalloc(&g->pr_off, cap + 1, &g->scratch_bytes));
        GV_TRY(dalloc(&g->pr_part, cap / 1024 + 2, &g->scratch_bytes));
        g->pr_vcap = cap;
    }
    if (E > g->pr_ecap || !g->pr_ecap) {
        dfree(g->pr_src); dfree(g->pr_dst);
        g->pr_ecap = 0;
        GV_TRY(dalloc(&g->pr_src, E, &g->scratch_bytes));
        GV_TRY(dalloc(&g->pr_dst, E, &g->scratch_bytes));
        g->pr_ecap = E;
    }
    void *dr = rank;
    bool hr = false;
    GV_TRY(output_ptr(g, 0, rank, (size_t)g->nv * 8, &dr, &hr));
    GV_CK(gv::launch_pagerank(view(g), analytics_item_blocks(g), iterations, damping, (double *)dr, g->pr_c,
                              g->pr_acc, g->pr_scal, g->pr_n, g->an_items, g->an_ctr + 1, g->pr_cursor, g->pr_off,
                              g->pr_part, g->pr_src, g->pr_dst, g->pr_ecap, lcfg(g, s)));
    if (hr) {
        GV_CK(cudaMemcpyAsync(rank, dr, (size_t)g->nv * 8, cudaMemcpyDeviceToHost, s));
        GV_CK(cudaStreamSynchronize(s));
    }
    return check_launch();
}

static const char *kPhaseNames[gv::PH_COUNT] = {
    "insert.count",   "insert.touched", "insert.plan",     "insert.link",      "insert.scatter",
    "insert.finalize",
    "delete.count",   "delete.touched", "delete.plan",     "delete.arena",     "delete.scatter",
    "delete.mark",    "delete.mark_tiny", "delete.vscan",  "delete.move",      "delete.finalize",
    "query.count",    "query.touched",  "query.plan",      "query.arena",      "query.scatter",
    "query.mark",     "query.mark_tiny", "query.out",      "query.finalize",
    "vertex_delete",  "neighbors",      "other",          "analytics",      "insert.small",
    "insert.partition", "insert.group", "insert.slots",
    "delete.partition", "delete.group", "delete.mark_cta",
    "query.partition",  "query.group",  "query.mark_cta"};

uint32_t gv_profile_num_phases(void) { return gv::PH_COUNT; }

const char *gv_profile_phase_name(uint32_t phase) {
    return phase < gv::PH_COUNT ? kPhaseNames[phase] : nullptr;
}

gv_status gv_profile(gv_graph *g, int enable) {
    if (!g) return GV_ERR_INVALID_ARG;
    g->prof.on = enable != 0;
    return GV_OK;
}

gv_status gv_profile_read(gv_graph *g, double *ms, uint64_t *launches, uint32_t n) {
    if (!g) return GV_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    for (uint32_t i = 0; i < n; ++i) {
        if (ms) ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    gv_status st = GV_OK;
    for (auto &r : g->prof.recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) st = GV_ERR_CUDA;
        float t = 0.f;
        if (st == GV_OK && cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) st = GV_ERR_CUDA;
        if ((uint32_t)r.phase < n) {
            if (ms) ms[r.phase] += t;
            if (launches) launches[r.phase] += 1;
        }
        g->prof.pool.push_back(r.a);
        g->prof.pool.push_back(r.b);
    }
    g->prof.recs.clear();
    cudaGetLastError();
    return st;
}

}  // extern "C"

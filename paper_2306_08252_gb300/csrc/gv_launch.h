// gv_launch.h -- host-side launchers of the GraphVine kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "gv_internal.cuh"

namespace gv {

// Kernel phases timed by the optional per-graph profiler.
enum Phase : int {
    PH_INS_COUNT = 0, PH_INS_TOUCHED, PH_INS_PLAN, PH_INS_LINK, PH_INS_SCATTER, PH_INS_FINALIZE,
    PH_DEL_COUNT, PH_DEL_TOUCHED, PH_DEL_PLAN, PH_DEL_ARENA, PH_DEL_SCATTER, PH_DEL_MARK, PH_DEL_MARK_TINY,
    PH_DEL_VSCAN, PH_DEL_MOVE, PH_DEL_FINALIZE,
    PH_QRY_COUNT, PH_QRY_TOUCHED, PH_QRY_PLAN, PH_QRY_ARENA, PH_QRY_SCATTER, PH_QRY_MARK, PH_QRY_MARK_TINY,
    PH_QRY_OUT, PH_QRY_FINALIZE,
    PH_VDEL, PH_NEIGHBORS, PH_OTHER, PH_ANALYTICS, PH_INS_SMALL,
    // grouped path of large batches: radix partition by source, grouping of
    // each bucket by vertex, the insert's slot pass, the block-wide tier
    PH_INS_PART, PH_INS_GROUP, PH_INS_SLOTS,
    PH_DEL_PART, PH_DEL_GROUP, PH_DEL_MARK_CTA,
    PH_QRY_PART, PH_QRY_GROUP, PH_QRY_MARK_CTA,
    PH_COUNT
};

// CUDA events recorded around each kernel launch while profiling is on.
struct Prof {
    bool on = false;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

struct LaunchCfg {
    int num_sms;
    cudaStream_t stream;
    Prof *prof = nullptr;
    // optional second stream of the graph and a fork/join event pair: the
    // two mark tiers (warp items, thread-per-source) run concurrently
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Records a start event now and a stop event when the scope ends.
struct PhaseScope {
    const LaunchCfg &lc;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseScope(const LaunchCfg &l, int ph) : lc(l), phase(ph) {
        if (lc.prof && lc.prof->on) {
            a = lc.prof->get();
            cudaEventRecord(a, lc.stream);
        }
    }
    ~PhaseScope() {
        if (a) {
            cudaEvent_t b = lc.prof->get();
            cudaEventRecord(b, lc.stream);
            lc.prof->recs.push_back({phase, a, b});
        }
    }
};

// Group-by-source counting pass over a pair batch (all modes).


// Launch with programmatic stream serialization: the grid may be scheduled
// while the previous kernel on the stream drains (every kernel of this
// library starts with pdl_wait(), so none reads its predecessor's results
// early).  Errors are left for cudaGetLastError, as with <<<>>>.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Blocks for `work` units at `per_block` units per block, at least 1 and at
// most `cap` (grid-stride kernels cover the rest).
inline int grid_for(unsigned long long work, int per_block, int cap) {
    unsigned long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (unsigned long long)cap) g = cap;
    return (int)g;
}

cudaError_t launch_count_range(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n_total, unsigned long long lo, unsigned long long hi,
                               const LaunchCfg &lc);
cudaError_t launch_count_finish(int mode, const GraphView &g, unsigned long long n_total, const LaunchCfg &lc);
cudaError_t launch_count(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                         unsigned long long n, const LaunchCfg &lc);
// Rejected-pair count only (batches that cannot match any stored edge).
cudaError_t launch_count_rejects(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                 unsigned long long n, unsigned long long *rejected,
                                 const LaunchCfg &lc);
// Insert of at most small_insert_max() pairs in one kernel of one CTA
// (grouping included: no counting pass before it).
cudaError_t launch_insert_small(const GraphView &g, const uint32_t *src, const uint32_t *dst, const uint32_t *wts,
                                unsigned long long n, unsigned long long *counts, const LaunchCfg &lc);
uint32_t small_insert_max();
// Insert: plan (block demand, pop offsets), link (CBT), scatter (slots), finalize.
cudaError_t launch_insert_tail(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, const LaunchCfg &lc,
                               const uint32_t *wts = nullptr);  // per-pair payloads of a weighted graph
// Delete / query: plan, arena init, scatter into membership sets, mark,
// (delete) vscan + move, finalize; (query) result gather.
cudaError_t launch_member_tail(int mode, const GraphView &g, const uint32_t *src,
                               const uint32_t *dst, unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, uint8_t *qout, const LaunchCfg &lc);
// A plain delete or query of at most small_member_max() pairs with the
// counting pass, plan, arena initialisation and scatter in one kernel of one
// CTA (the batch not counted before), then the general path's mark and
// finalize kernels.
uint64_t small_member_max();
cudaError_t launch_member_small(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                unsigned long long n, unsigned long long tcap, unsigned long long *counts,
                                uint8_t *qout, const LaunchCfg &lc);
// Grouped path of large plain batches (gv_group.cu).  group_shape: the
// partition CTAs and their pair range for a batch of n.  launch_group_hist:
// per-bucket counts of the partition CTAs whose ranges lie in pairs [lo, hi)
// (lo a multiple of the range, hi one or n).  launch_group_finish: the rest
// of the grouping once every pair has landed (and, for deletes and queries,
// the batch lists of deletes and queries).  launch_group_place: the insert's
// slot pass over the grouped pairs (after the plan and the links).
void group_shape(unsigned long long n, int num_sms, uint32_t *ctas, unsigned long long *len);
// log2 of the vertices per bucket of the partition for n pairs, dictionary vcap.
uint32_t group_bucket_shift(unsigned long long n, uint32_t vcap);
cudaError_t launch_group_hist(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                              unsigned long long n, unsigned long long lo, unsigned long long hi,
                              const LaunchCfg &lc);
cudaError_t launch_group_finish(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                const uint32_t *wts, unsigned long long n, const LaunchCfg &lc);
cudaError_t launch_group_place(int mode, const GraphView &g, unsigned long long n, const LaunchCfg &lc);
cudaError_t launch_gp_plan_insert(const GraphView &g, int grid, const LaunchCfg &lc);
cudaError_t launch_gp_plan_member(int mode, const GraphView &g, int grid, const LaunchCfg &lc);
cudaError_t launch_mark_cta(int mode, const GraphView &g, unsigned long long nt, const LaunchCfg &lc);
// Grouped queries: the hits of the sources past CT_KEYS batch entries (found
// in their arena hash sets) copied back to their list entries.
cudaError_t launch_gp_hash_found(const GraphView &g, const LaunchCfg &lc);
// Vertex delete: mark dead, free own blocks, remove incoming edges, finalize.
cudaError_t launch_vertex_delete(const GraphView &g, const uint32_t *ids, uint32_t k,
                                 const LaunchCfg &lc);
// Vertices [from, to): alive, empty sentinel.
cudaError_t launch_init_vertices(const GraphView &g, uint32_t from, uint32_t to,
                                 const LaunchCfg &lc);
// Dictionary doubling copy.
cudaError_t launch_copy_dictionary(uint4 *dst_sent, uint8_t *dst_alive, const uint4 *src_sent,
                                   const uint8_t *src_alive, uint32_t n, const LaunchCfg &lc);
// Edge queue initialisation: queue[i] = i.
cudaError_t launch_init_queue(uint32_t *queue, unsigned long long n, const LaunchCfg &lc, uint32_t first = 0,
                              uint32_t step = 1);
// Neighbour lists: offsets (exclusive scan of degrees), then copy.
// offsets[i] = sum over vids[0 .. i-1] of the degree (rounded up to a
// multiple of round_to when that is non-zero); offsets[n] = the total.
cudaError_t launch_neighbor_offsets(const GraphView &g, const uint32_t *vids, uint32_t n,
                                    unsigned long long *offsets, unsigned long long *partials,
                                    const LaunchCfg &lc, uint32_t round_to = 0);
// Edge-block resize: res[0..1] = {entries, non-empty live vertices}; then the
// trees and sentinels over contiguous block runs starting at slots[u] / C.
cudaError_t launch_degree_stats(const GraphView &g, unsigned long long *res, const LaunchCfg &lc);
// res[i] = blocks the live vertices would hold at C = 4 (i + 1), i < 128.
cudaError_t launch_footprint_blocks(const GraphView &g, unsigned long long *res, const LaunchCfg &lc);
// big: scratch of one id per vertex (the runs longer than a thread writes
// alone), nbig: one counter
// T: degree from which a vertex is placed in runs (hub runs on), plain_shift:
// added to a plain vertex's slot offset to give its place in the pool
cudaError_t launch_reblock_place(const GraphView &g, const unsigned long long *slots, uint32_t *big,
                                 unsigned long long *nbig, const LaunchCfg &lc, uint32_t T = 0xFFFFFFFFu,
                                 unsigned long long plain_shift = 0ull);
cudaError_t launch_reblock_merge(const GraphView &g, unsigned long long *plain_off, const unsigned long long *hub_off,
                                 uint32_t T, unsigned long long hub_total, const LaunchCfg &lc);
// Slot offsets of the edge-block resize of a graph with hub runs: over the
// plain vertices (degree < T, rounded to round_to) or over the hubs (rounded
// to whole runs of round_to << rs slots); offsets[n] = total.
cudaError_t launch_reblock_offsets(const GraphView &g, const uint32_t *vids, uint32_t n, unsigned long long *offsets,
                                   unsigned long long *partials, const LaunchCfg &lc, uint32_t round_to, bool hubs,
                                   uint32_t T, uint32_t rs);
cudaError_t launch_neighbor_copy(const GraphView &g, const uint32_t *vids, uint32_t n,
                                 const unsigned long long *offsets, uint32_t *nbrs,
                                 const LaunchCfg &lc,
                                 uint32_t *wts = nullptr);
cudaError_t launch_degrees(const GraphView &g, uint32_t *deg, uint8_t *alive,
                           const LaunchCfg &lc);
cudaError_t launch_iota(uint32_t *out, uint32_t first, uint32_t k, const LaunchCfg &lc);
// Graph sets: member batches -> one global batch; per-member insert counts.
cudaError_t launch_set_remap(const GraphView &g, const uint32_t *src, const uint32_t *dst, unsigned long long n,
                             uint32_t *gsrc, uint32_t *gdst, const LaunchCfg &lc);
cudaError_t launch_set_insert_counts(const GraphView &g, const LaunchCfg &lc);
cudaError_t launch_segment_counts(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                  unsigned long long n, const LaunchCfg &lc);
// Set-semantics insert: membership pass, then the mask of pairs to insert.
cudaError_t launch_dedup_insert_prepare(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                        unsigned long long n, unsigned long long tcap, uint32_t *src2,
                                        unsigned long long *tmp, const LaunchCfg &lc);
cudaError_t launch_dedup_counts(Dev *dev, const unsigned long long *tmp, unsigned long long n,
                                unsigned long long *counts, const LaunchCfg &lc);
cudaError_t launch_grow_queue(const uint32_t *q, unsigned long long P, unsigned long long qf,
                              unsigned long long nfree, uint32_t *q2, unsigned long long P2, const LaunchCfg &lc);
// graph analytics (gv_analytics.cu)
cudaError_t launch_bfs_seed(const GraphView &g, uint32_t source, uint32_t *dist, uint32_t *cur, uint32_t *ctr,
                            const LaunchCfg &lc);
cudaError_t launch_bfs_level(const GraphView &g, uint32_t aib, const uint32_t *cur, uint32_t *next, uint2 *items,
                             uint32_t *ctr, uint32_t *dist, uint32_t level, const LaunchCfg &lc);
cudaError_t launch_sssp_seed(const GraphView &g, uint32_t source, unsigned long long *dist, uint32_t *stamp,
                             uint32_t *cur, uint32_t *ctr, const LaunchCfg &lc);
cudaError_t launch_sssp_round(const GraphView &g, uint32_t aib, const uint32_t *cur, uint32_t *next, uint2 *items,
                              uint32_t *ctr, unsigned long long *dist, uint32_t *stamp, uint32_t round,
                              const LaunchCfg &lc);
cudaError_t launch_pagerank(const GraphView &g, uint32_t aib, uint32_t iterations, double damping, double *r,
                            double *c, double *acc, double *scal, unsigned long long *N, uint2 *items,
                            uint32_t *nitems, uint32_t *cursor, unsigned long long *in_off,
                            unsigned long long *part, uint32_t *in_src, uint32_t *in_dst, unsigned long long ecap,
                            const LaunchCfg &lc);
cudaError_t launch_segment_noop_check(const GraphView &g, const unsigned long long *tot, unsigned long long n,
                                      const LaunchCfg &lc);
cudaError_t launch_finalize_count_only(const GraphView &g, const LaunchCfg &lc);
cudaError_t launch_validate(const GraphView &g, uint32_t *owner_bits,
                            unsigned long long *violations, const LaunchCfg &lc);

// Sizes shared with the host code (overridable at build time for tuning).
#ifndef GV_AGG_THREADS
#define GV_AGG_THREADS 256
#endif
#ifndef GV_AGG_EPT
#define GV_AGG_EPT 8
#endif
#ifndef GV_AGG_HBITS
#define GV_AGG_HBITS 12
#endif
#ifndef GV_PP
#define GV_PP 4
#endif
#ifndef GV_PP_MEMBER
#define GV_PP_MEMBER 1
#endif
#ifndef GV_CD_PER
#define GV_CD_PER 8
#endif
#ifndef GV_GRID_MULT
#define GV_GRID_MULT 16
#endif
constexpr int AGG_THREADS = GV_AGG_THREADS;
constexpr int AGG_EPT = GV_AGG_EPT;
constexpr int AGG_TILE = AGG_THREADS * AGG_EPT;  // pairs per tile
constexpr int AGG_HBITS = GV_AGG_HBITS;
constexpr int AGG_H = 1 << AGG_HBITS;            // shared hash slots per tile (>= 2 * tile)
constexpr int AGG_SPT = AGG_H / AGG_THREADS;     // hash slots per thread
constexpr int PP = GV_PP;                        // pairs per thread per step (streaming kernels)
// The membership scatter holds more per pair (a plan record, two half
// buckets): with one pair a thread more CTAs fit an SM, which hides its
// scattered accesses better than more pairs in flight per thread (on the
// 10M delete: 141 us at one pair, 166 at two, 200 at four).
constexpr int PP_MEMBER = GV_PP_MEMBER;
constexpr int CD_PER = GV_CD_PER;                // pairs per thread per step of the per-pair counting pass
constexpr int GRID_MULT = GV_GRID_MULT;          // CTAs per SM of grid-stride kernels
constexpr int MASK_WORDS = 16;                   // survivor bits per item (512 slots)
// Neighbour-offset scan: SCAN_T threads per CTA, SCAN_PER ids each; one
// chunk sum per SCAN_CHUNK ids (launch_neighbor_offsets' `partials` holds
// ceil(n / SCAN_CHUNK) + 1 of them).
constexpr int SCAN_T = 256;
constexpr int SCAN_PER = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_PER;
static_assert(AGG_H >= 2 * AGG_TILE, "aggregation table must be at most half full");
static_assert(AGG_SPT <= 32 && AGG_SPT % 2 == 0, "slots per thread");
static_assert(AGG_TILE <= (1 << (32 - AGG_HBITS)), "slot and rank must pack into 32 bits");

}  // namespace gv

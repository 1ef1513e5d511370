// Graph analytics over the stored structure: breadth-first search
// distances, single-source shortest paths and PageRank.  The paper names
// analytics on the dynamic structure (BFS, shortest paths) as future work
// ("Conclusion and future work"); the definitions are the textbook ones
// (level-synchronous BFS; Bellman-Ford shortest paths over a frontier of
// improved vertices; PageRank power iteration with damping, dangling mass
// spread over all live vertices, gathered over an incoming-edge CSR built
// once per call).
//
// All read adjacencies the way the delete and query pipelines do: work
// items of up to AIB blocks of one vertex, one warp per item, block ids by
// lane-parallel walks of the vertex's complete binary tree ("Dynamic edge
// inserts", bit-string rule), entries by 16-byte streaming loads.
#include "gv_internal.cuh"
#include "gv_launch.h"

namespace gv {

namespace {

// Calls f(e4, vm) -- f(e4, w4, vm) with WTS, w4 the entries' payloads --
// once per round of 32 quads of the item's stored entries (all lanes call
// it: f may use warp collectives); vm bit j = entry j of the lane's quad is a
// stored entry.  Returns false if a tree walk left the pool.
template <bool WTS = false, typename F>
__device__ __forceinline__ bool for_item_entries(const GraphView &g, uint32_t u, uint32_t c, uint32_t aib,
                                                 uint32_t *sb, F &&f) {
    const uint4 s = g.sent[u];
    const uint32_t deg = s.x, nb = s.y, root = s.z;
    const uint32_t kb = c * aib;
    if (kb >= nb) return true;
    const uint32_t nblk = min(aib, nb - kb);
    const uint32_t lane = lane_id();
    uint32_t bid = NIL;
    if (lane < nblk) bid = blk_at(g, root, kb + 1 + lane);
    if (__any_sync(FULL, lane < nblk && bid == NIL)) return false;
    sb[lane] = bid;
    __syncwarp();
    const uint32_t C = g.C;
    const uint32_t sbase = kb * C;
    const uint32_t nslots = min(nblk * C, deg - sbase);
    const uint32_t nquads = (nslots + 3) >> 2;
    for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
        const uint32_t q = q0 + lane;
        uint4 e4 = make_uint4(NIL, NIL, NIL, NIL);
        uint4 w4 = make_uint4(0, 0, 0, 0);
        uint32_t vm = 0;
        if (q < nquads) {
            const uint32_t x = q << 2;
            const uint32_t lb = divc(g.cmul, x);
            const size_t off = (size_t)sb[lb] * C + (x - lb * C);
            e4 = ld_stream4(reinterpret_cast<const uint4 *>(g.data + off));
            if constexpr (WTS) w4 = ld_stream4(reinterpret_cast<const uint4 *>(g.wdata + off));
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j)
                if (x + j < nslots) vm |= 1u << j;
        }
        if constexpr (WTS)
            f(e4, w4, vm);
        else
            f(e4, vm);
    }
    __syncwarp();
    return true;
}

}  // namespace

// Work items (vertex, chunk of aib blocks) for the live vertices of a list
// (`*nlist` entries, read on the device) or of all vertices (list == NULL).
__global__ void __launch_bounds__(256) k_an_items(GraphView g, const uint32_t *__restrict__ list,
                                                  const uint32_t *nlist, uint32_t aib, uint2 *items,
                                                  uint32_t *nitems) {
    pdl_wait();
    const uint32_t n = list ? *nlist : g.nv;
    __shared__ uint32_t s_base;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t u = NIL, ni = 0;
        if (i < n) {
            u = list ? list[i] : i;
            if (g.alive[u]) ni = (g.sent[u].y + aib - 1) / aib;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(ni, &tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(nitems, tot) : 0u;
        __syncthreads();
        for (uint32_t c = 0; c < ni; ++c) items[s_base + ex + c] = make_uint2(u, c);
        __syncthreads();
    }
}

// ------------------------------------------------------------------- BFS

// Source of the search: distance 0 and the first frontier, if alive.
__global__ void k_bfs_seed(GraphView g, uint32_t source, uint32_t *dist, uint32_t *cur, uint32_t *ctr) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool live = source < g.nv && g.alive[source];
        if (live) {
            dist[source] = 0;
            cur[0] = source;
        }
        ctr[0] = live ? 1u : 0u;  // frontier size
        ctr[1] = 0;               // items
        ctr[2] = 0;               // next frontier size
        ctr[3] = live ? 1u : 0u;  // levels reached so far
    }
}

// One level: every stored entry v of a frontier vertex with no distance yet
// is claimed by CAS (distance level + 1) and appended to the next frontier
// (warp-aggregated append).
__global__ void __launch_bounds__(256) k_bfs_expand(GraphView g, const uint2 *__restrict__ items,
                                                    const uint32_t *nitems, uint32_t aib, uint32_t *dist,
                                                    uint32_t level, uint32_t *next, uint32_t *nnext) {
    pdl_wait();
    __shared__ uint32_t s_bid[8][32];
    const uint32_t n = *nitems;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nv = g.nv;
    for (uint32_t it = warp; it < n; it += nwarps) {
        const uint2 itm = items[it];
        bool bad = false;
        const bool ok = for_item_entries(g, itm.x, itm.y, aib, s_bid[threadIdx.x >> 5], [&](uint4 e4, uint32_t vm) {
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
            uint32_t push = 0;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                if ((vm >> j) & 1u) {
                    const uint32_t v = e[j];
                    if (v >= nv) {
                        bad = true;
                    } else if (__ldcg(dist + v) == NIL && atomicCAS(dist + v, NIL, level + 1) == NIL) {
                        push |= 1u << j;
                    }
                }
            }
            uint32_t tot;
            const uint32_t ex = warp_excl_scan(__popc(push), &tot);
            uint32_t base = 0;
            if (lane == 0 && tot) base = atomicAdd(nnext, tot);
            base = __shfl_sync(FULL, base, 0);
            uint32_t w = base + ex;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j)
                if ((push >> j) & 1u) next[w++] = e[j];
        });
        if ((!ok || bad) && lane == 0) latch_status(g.dev, 5u /* GV_ERR_STATE */);
    }
}

// Next frontier becomes the current one: ctr = {frontier, items, next,
// levels}.  A level with an empty frontier changes nothing, so the host may
// launch several levels between two reads of the frontier size.
__global__ void k_bfs_advance(uint32_t *ctr, uint32_t level) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (ctr[2]) ctr[3] = level + 2;
        ctr[0] = ctr[2];
        ctr[1] = 0;
        ctr[2] = 0;
    }
}

cudaError_t launch_bfs_seed(const GraphView &g, uint32_t source, uint32_t *dist, uint32_t *cur, uint32_t *ctr,
                            const LaunchCfg &lc) {
    PhaseScope ps(lc, PH_ANALYTICS);
    if (g.nv) cudaMemsetAsync(dist, 0xFF, (size_t)g.nv * 4, lc.stream);
    k_bfs_seed<<<1, 32, 0, lc.stream>>>(g, source, dist, cur, ctr);
    return cudaGetLastError();
}

cudaError_t launch_bfs_level(const GraphView &g, uint32_t aib, const uint32_t *cur, uint32_t *next, uint2 *items,
                             uint32_t *ctr, uint32_t *dist, uint32_t level, const LaunchCfg &lc) {
    PhaseScope ps(lc, PH_ANALYTICS);
    const int grid = lc.num_sms * GRID_MULT;
    launch_pdl(k_an_items, grid, 256, 0, lc.stream, g, cur, ctr, aib, items, ctr + 1);
    launch_pdl(k_bfs_expand, grid, 256, 0, lc.stream, g, items, ctr + 1, aib, dist, level, next, ctr + 2);
    launch_pdl(k_bfs_advance, 1, 32, 0, lc.stream, ctr, level);
    return cudaGetLastError();
}

// ------------------------------------------------ single-source shortest paths

// Frontier Bellman-Ford with atomic minima: the frontier of round r holds
// the vertices whose distance fell in round r - 1; each of their stored
// entries (u, v) offers dist[u] + length to v (payload on a weighted graph,
// 1 otherwise), taken by a 64-bit atomicMin.  A vertex whose distance fell
// joins the next frontier once per round (stamp[v] = r + 1 by exchange).
// Distances are lengths of real paths and every fall is propagated, so the
// fixpoint is the shortest-path distance whatever the order of the minima;
// with non-negative lengths it is reached within nv rounds.

__global__ void k_sssp_seed(GraphView g, uint32_t source, unsigned long long *dist, uint32_t *cur, uint32_t *ctr) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool live = source < g.nv && g.alive[source];
        if (live) {
            dist[source] = 0ull;
            cur[0] = source;
        }
        ctr[0] = live ? 1u : 0u;  // frontier size
        ctr[1] = 0;               // items
        ctr[2] = 0;               // next frontier size
        ctr[3] = live ? 1u : 0u;  // rounds with a non-empty frontier
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(256) k_sssp_relax(GraphView g, const uint2 *__restrict__ items,
                                                    const uint32_t *nitems, uint32_t aib, unsigned long long *dist,
                                                    uint32_t *stamp, uint32_t round, uint32_t *next,
                                                    uint32_t *nnext) {
    pdl_wait();
    __shared__ uint32_t s_bid[8][32];
    const uint32_t n = *nitems;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nv = g.nv;
    for (uint32_t it = warp; it < n; it += nwarps) {
        const uint2 itm = items[it];
        const unsigned long long du = __ldcg(dist + itm.x);
        bool bad = false;
        auto relax = [&](uint4 e4, uint4 w4, uint32_t vm) {
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
            const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
            uint32_t push = 0;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                if ((vm >> j) & 1u) {
                    const uint32_t v = e[j];
                    const unsigned long long nd = du + (WEIGHTED ? (unsigned long long)w[j] : 1ull);
                    if (v >= nv) {
                        bad = true;
                    } else if (nd < __ldcg(dist + v) && nd < atomicMin(dist + v, nd) &&
                               atomicExch(stamp + v, round + 1) != round + 1) {
                        push |= 1u << j;
                    }
                }
            }
            uint32_t tot;
            const uint32_t ex = warp_excl_scan(__popc(push), &tot);
            uint32_t base = 0;
            if (lane == 0 && tot) base = atomicAdd(nnext, tot);
            base = __shfl_sync(FULL, base, 0);
            uint32_t o = base + ex;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j)
                if ((push >> j) & 1u) next[o++] = e[j];
        };
        bool ok;
        if constexpr (WEIGHTED)
            ok = for_item_entries<true>(g, itm.x, itm.y, aib, s_bid[threadIdx.x >> 5], relax);
        else
            ok = for_item_entries(g, itm.x, itm.y, aib, s_bid[threadIdx.x >> 5],
                                  [&](uint4 e4, uint32_t vm) { relax(e4, make_uint4(1, 1, 1, 1), vm); });
        if ((!ok || bad) && lane == 0) latch_status(g.dev, 5u /* GV_ERR_STATE */);
    }
}

cudaError_t launch_sssp_seed(const GraphView &g, uint32_t source, unsigned long long *dist, uint32_t *stamp,
                             uint32_t *cur, uint32_t *ctr, const LaunchCfg &lc) {
    PhaseScope ps(lc, PH_ANALYTICS);
    if (g.nv) {
        cudaMemsetAsync(dist, 0xFF, (size_t)g.nv * 8, lc.stream);
        cudaMemsetAsync(stamp, 0, (size_t)g.nv * 4, lc.stream);
    }
    k_sssp_seed<<<1, 32, 0, lc.stream>>>(g, source, dist, cur, ctr);
    return cudaGetLastError();
}

cudaError_t launch_sssp_round(const GraphView &g, uint32_t aib, const uint32_t *cur, uint32_t *next, uint2 *items,
                              uint32_t *ctr, unsigned long long *dist, uint32_t *stamp, uint32_t round,
                              const LaunchCfg &lc) {
    PhaseScope ps(lc, PH_ANALYTICS);
    const int grid = lc.num_sms * GRID_MULT;
    launch_pdl(k_an_items, grid, 256, 0, lc.stream, g, cur, ctr, aib, items, ctr + 1);
    if (g.wdata)
        launch_pdl(k_sssp_relax<true>, grid, 256, 0, lc.stream, g, items, ctr + 1, aib, dist, stamp, round, next, ctr + 2);
    else
        launch_pdl(k_sssp_relax<false>, grid, 256, 0, lc.stream, g, items, ctr + 1, aib, dist, stamp, round, next, ctr + 2);
    launch_pdl(k_bfs_advance, 1, 32, 0, lc.stream, ctr, round);
    return cudaGetLastError();
}

// -------------------------------------------------------------- PageRank

// N = live vertices (64-bit counter, zeroed by the caller).
__global__ void __launch_bounds__(256) k_pr_count(GraphView g, unsigned long long *N) {
    pdl_wait();
    unsigned long long k = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) k += g.alive[v];
    k = block_sum_u64(k);
    if (threadIdx.x == 0 && k) atomicAdd(N, k);
}

__global__ void __launch_bounds__(256) k_pr_start(GraphView g, double *r, const unsigned long long *N) {
    pdl_wait();
    const unsigned long long n = *N;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x)
        r[v] = (n && g.alive[v]) ? 1.0 / (double)n : 0.0;
}

// Per vertex: its share r(u) / deg(u) (0 for dead or dangling vertices),
// the accumulator cleared, and the dangling mass summed into *dang.
__global__ void __launch_bounds__(256) k_pr_contrib(GraphView g, const double *__restrict__ r, double *c,
                                                    double *acc, double *dang) {
    pdl_wait();
    __shared__ double s_p[8];
    double dm = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) {
        const uint32_t deg = g.sent[v].x;
        const bool live = g.alive[v];
        double share = 0.0;
        if (live && deg) share = r[v] / (double)deg;
        if (live && !deg) dm += r[v];
        c[v] = share;
        acc[v] = 0.0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) dm += __shfl_xor_sync(FULL, dm, d);
    if (lane_id() == 0) s_p[threadIdx.x >> 5] = dm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) t += s_p[w];
        if (t != 0.0) atomicAdd(dang, t);
    }
}

// Incoming-edge CSR of the stored graph, built once per PageRank call so
// that every iteration gathers (no atomic per entry): in-degrees by one
// atomic per stored entry, an exclusive scan into offsets, then each entry
// (u, v) placed in v's segment at an atomically claimed position.
__global__ void __launch_bounds__(256) k_pr_indeg(GraphView g, const uint2 *__restrict__ items,
                                                  const uint32_t *nitems, uint32_t aib, uint32_t *indeg) {
    pdl_wait();
    __shared__ uint32_t s_bid[8][32];
    const uint32_t n = *nitems;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nv = g.nv;
    for (uint32_t it = warp; it < n; it += nwarps) {
        const uint2 itm = items[it];
        bool bad = false;
        const bool ok = for_item_entries(g, itm.x, itm.y, aib, s_bid[threadIdx.x >> 5], [&](uint4 e4, uint32_t vm) {
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                if ((vm >> j) & 1u) {
                    if (e[j] < nv) atomicAdd(indeg + e[j], 1u);
                    else bad = true;
                }
            }
        });
        if ((!ok || bad) && lane == 0) latch_status(g.dev, 5u /* GV_ERR_STATE */);
    }
}

constexpr uint32_t PR_CHUNK = 1024;  // entries per scan chunk (256 threads x 4)

// Chunk sums of x[0..n).
__global__ void __launch_bounds__(256) k_pr_chunk_sums(const uint32_t *__restrict__ x, uint32_t n,
                                                       unsigned long long *part) {
    pdl_wait();
    const uint32_t base = blockIdx.x * PR_CHUNK;
    unsigned long long t = 0;
    for (uint32_t k = threadIdx.x; k < PR_CHUNK; k += blockDim.x)
        if (base + k < n) t += x[base + k];
    t = block_sum_u64(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Exclusive scan of the chunk sums in place; part[nchunks] = total.  One
// block; each thread scans a contiguous run of chunks.
__global__ void __launch_bounds__(1024) k_pr_scan_parts(unsigned long long *part, uint32_t nchunks) {
    pdl_wait();
    __shared__ unsigned long long s_run[1024];
    const uint32_t per = (nchunks + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per, hi = min(nchunks, lo + per);
    unsigned long long run = 0;
    for (uint32_t c = lo; c < hi; ++c) run += part[c];
    s_run[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {  // scan of the per-thread runs (1024 values)
        unsigned long long acc = 0;
        for (uint32_t i = 0; i < blockDim.x; ++i) {
            const unsigned long long v = s_run[i];
            s_run[i] = acc;
            acc += v;
        }
        part[nchunks] = acc;
    }
    __syncthreads();
    unsigned long long acc = s_run[threadIdx.x];
    for (uint32_t c = lo; c < hi; ++c) {
        const unsigned long long v = part[c];
        part[c] = acc;
        acc += v;
    }
}

// off[i] = exclusive prefix sum of x at i (i < n); off[n] = total.
__global__ void __launch_bounds__(256) k_pr_scan_apply(const uint32_t *__restrict__ x, uint32_t n,
                                                       const unsigned long long *__restrict__ part,
                                                       uint32_t nchunks, unsigned long long *off) {
    pdl_wait();
    const uint32_t base = blockIdx.x * PR_CHUNK;
    uint32_t v[4];
    uint32_t loc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t k = base + threadIdx.x * 4 + j;
        v[j] = k < n ? x[k] : 0u;
        loc += v[j];
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(loc, &tot);
    unsigned long long run = part[blockIdx.x] + ex;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t k = base + threadIdx.x * 4 + j;
        if (k < n) off[k] = run;
        run += v[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = part[nchunks];
}

__global__ void __launch_bounds__(256) k_pr_fill(GraphView g, const uint2 *__restrict__ items,
                                                 const uint32_t *nitems, uint32_t aib,
                                                 const unsigned long long *__restrict__ off, uint32_t *cursor,
                                                 uint32_t *in_src, uint32_t *in_dst, unsigned long long ecap) {
    pdl_wait();
    __shared__ uint32_t s_bid[8][32];
    const uint32_t n = *nitems;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nv = g.nv;
    for (uint32_t it = warp; it < n; it += nwarps) {
        const uint2 itm = items[it];
        const uint32_t u = itm.x;
        for_item_entries(g, u, itm.y, aib, s_bid[threadIdx.x >> 5], [&](uint4 e4, uint32_t vm) {
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                if (((vm >> j) & 1u) && e[j] < nv) {
                    const unsigned long long pos = off[e[j]] + atomicAdd(cursor + e[j], 1u);
                    if (pos < ecap) {  // the entry count read by the host bounds the arrays
                        in_src[pos] = u;
                        in_dst[pos] = e[j];
                    } else {
                        latch_status(g.dev, 5u /* GV_ERR_STATE */);
                    }
                }
            }
        });
    }
}

// acc(v) += sum of c(u) over v's incoming entries.  Entries are taken 32 at
// a time by a warp in CSR order, so equal destinations sit in consecutive
// lanes: a segmented sum by shuffles leaves each segment's total in its
// first lane, which adds it with one atomic (one or a few per warp round
// instead of one per entry).
__global__ void __launch_bounds__(256) k_pr_gather(const uint32_t *__restrict__ in_src,
                                                   const uint32_t *__restrict__ in_dst,
                                                   const unsigned long long *total, const double *__restrict__ c,
                                                   double *acc, unsigned long long ecap) {
    pdl_wait();
    const unsigned long long E = min(*total, ecap);
    const uint32_t lane = lane_id();
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long k0 = warp * 32; k0 < E; k0 += nwarps * 32) {
        const unsigned long long k = k0 + lane;
        uint32_t key = NIL;
        double s = 0.0;
        if (k < E) {
            key = ld_stream(in_dst + k);
            s = c[ld_stream(in_src + k)];
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double o = __shfl_down_sync(FULL, s, d);
            const uint32_t ok = __shfl_down_sync(FULL, key, d);
            if (lane + d < 32 && ok == key) s += o;
        }
        const uint32_t prev = __shfl_up_sync(FULL, key, 1);
        if (key != NIL && (lane == 0 || prev != key)) atomicAdd(acc + key, s);
    }
}

// r(v) = (1 - d)/N + d * (acc(v) + dangling/N) for live v, 0 otherwise; the
// other dangling slot is cleared for the next iteration.
__global__ void __launch_bounds__(256) k_pr_update(GraphView g, double *r, const double *__restrict__ acc,
                                                   double *dang, uint32_t slot, const unsigned long long *N,
                                                   double damping) {
    pdl_wait();
    const double n = (double)*N;
    const double dm = dang[slot];
    if (blockIdx.x == 0 && threadIdx.x == 0) dang[slot ^ 1u] = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x)
        r[v] = g.alive[v] ? (1.0 - damping) / n + damping * (acc[v] + dm / n) : 0.0;
}

cudaError_t launch_pagerank(const GraphView &g, uint32_t aib, uint32_t iterations, double damping, double *r,
                            double *c, double *acc, double *scal, unsigned long long *N, uint2 *items,
                            uint32_t *nitems, uint32_t *cursor, unsigned long long *in_off,
                            unsigned long long *part, uint32_t *in_src, uint32_t *in_dst, unsigned long long ecap,
                            const LaunchCfg &lc) {
    PhaseScope ps(lc, PH_ANALYTICS);
    const int grid = lc.num_sms * GRID_MULT;
    const int gnv = grid_for(g.nv ? g.nv : 1, 256, grid);
    const uint32_t nchunks = (g.nv + PR_CHUNK - 1) / PR_CHUNK;
    cudaMemsetAsync(N, 0, 8, lc.stream);
    cudaMemsetAsync(nitems, 0, 4, lc.stream);
    cudaMemsetAsync(scal, 0, 2 * sizeof(double), lc.stream);
    cudaMemsetAsync(cursor, 0, (size_t)g.nv * 4, lc.stream);
    // kernels right after a memset are ordinary launches
    k_pr_count<<<gnv, 256, 0, lc.stream>>>(g, N);
    launch_pdl(k_pr_start, gnv, 256, 0, lc.stream, g, r, N);
    launch_pdl(k_an_items, grid, 256, 0, lc.stream, g, nullptr, nullptr, aib, items, nitems);
    // incoming CSR: in-degrees -> offsets -> entries placed per destination
    launch_pdl(k_pr_indeg, grid, 256, 0, lc.stream, g, items, nitems, aib, cursor);
    launch_pdl(k_pr_chunk_sums, nchunks, 256, 0, lc.stream, cursor, g.nv, part);
    launch_pdl(k_pr_scan_parts, 1, 1024, 0, lc.stream, part, nchunks);
    launch_pdl(k_pr_scan_apply, nchunks, 256, 0, lc.stream, cursor, g.nv, part, nchunks, in_off);
    cudaMemsetAsync(cursor, 0, (size_t)g.nv * 4, lc.stream);
    k_pr_fill<<<grid, 256, 0, lc.stream>>>(g, items, nitems, aib, in_off, cursor, in_src, in_dst, ecap);
    for (uint32_t it = 0; it < iterations; ++it) {
        const uint32_t slot = it & 1u;
        launch_pdl(k_pr_contrib, gnv, 256, 0, lc.stream, g, r, c, acc, scal + slot);
        launch_pdl(k_pr_gather, grid, 256, 0, lc.stream, in_src, in_dst, in_off + g.nv, c, acc, ecap);
        launch_pdl(k_pr_update, gnv, 256, 0, lc.stream, g, r, acc, scal, slot, N, damping);
    }
    return cudaGetLastError();
}

}  // namespace gv

// gv_misc.cu -- initialisation, dictionary growth, neighbour lists, degrees
// and the structural self-check of the GraphVine library.
#include "gv_launch.h"

namespace gv {

// Sentinel attach ("Dynamic vertex updates": one thread per vertex attaches
// an empty edge sentinel).
__global__ void __launch_bounds__(256) k_init_vertices(GraphView g, uint32_t from, uint32_t to) {
    pdl_wait();
    for (uint32_t u = from + blockIdx.x * blockDim.x + threadIdx.x; u < to; u += gridDim.x * blockDim.x) {
        g.sent[u] = make_uint4(0, 0, NIL, NIL);
        g.alive[u] = 1;
    }
}

// Dictionary doubling: one kernel copies the old dictionary into the new one.
__global__ void __launch_bounds__(256) k_copy_dictionary(uint4 *dst_sent, uint8_t *dst_alive,
                                                         const uint4 *src_sent, const uint8_t *src_alive,
                                                         uint32_t n) {
    pdl_wait();
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        dst_sent[u] = src_sent[u];
        dst_alive[u] = src_alive[u];
    }
}

// Edge queue: every pool block id, in order ("Edge Queue").
// queue[i] = first + i * step for i < n (the free block ids of a fresh pool,
// or the heads of its runs).
__global__ void __launch_bounds__(256) k_init_queue(uint32_t *queue, unsigned long long n, uint32_t first,
                                                    uint32_t step) {
    pdl_wait();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        queue[i] = first + (uint32_t)i * step;
}

__global__ void __launch_bounds__(256) k_iota(uint32_t *out, uint32_t first, uint32_t k) {
    pdl_wait();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        out[i] = first + i;
}

__global__ void __launch_bounds__(256) k_degrees(GraphView g, uint32_t *deg, uint8_t *alive) {
    pdl_wait();
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.nv; u += gridDim.x * blockDim.x) {
        deg[u] = g.sent[u].x;
        if (alive) alive[u] = g.alive[u];
    }
}

// ------------------------------------------------------------- neighbours

// Degree of a requested vertex (0 for invalid or deleted ids), rounded up to
// a multiple of `round_to` when that is non-zero (slots of whole blocks).
__device__ __forceinline__ unsigned long long vid_degree(const GraphView &g, uint32_t u, uint32_t round_to) {
    const unsigned long long d = (u < g.nv && g.alive[u]) ? g.sent[u].x : 0u;
    return round_to ? (d + round_to - 1) / round_to * round_to : d;
}

// Slots a requested vertex takes in a layout: SEL 0 its degree rounded as
// above; for the edge-block resize of a graph with hub runs, SEL 1 the same
// for a plain vertex (degree below T) and 0 for a hub, SEL 2 a hub's degree
// rounded up to whole runs (round_to << rs slots) and 0 for a plain vertex.
template <int SEL>
__device__ __forceinline__ unsigned long long vid_size(const GraphView &g, uint32_t u, uint32_t round_to,
                                                       uint32_t T, uint32_t rs) {
    if (SEL == 0) return vid_degree(g, u, round_to);
    const unsigned long long d = vid_degree(g, u, 0);
    const bool hub = d > 0 && d >= T;
    if (SEL == 1 ? hub : !hub) return 0ull;
    const unsigned long long r = SEL == 2 ? (unsigned long long)round_to << rs : round_to;
    return (d + r - 1) / r * r;
}

// Per-chunk sums of the requested vertices' degrees.
template <int SEL>
__global__ void __launch_bounds__(SCAN_T) k_nbr_partials(GraphView g, const uint32_t *__restrict__ vids,
                                                         uint32_t n, uint32_t round_to, uint32_t T, uint32_t rs,
                                                         unsigned long long *partials) {
    pdl_wait();
    const uint32_t chunk = blockIdx.x;
    unsigned long long s = 0;
    for (int j = 0; j < SCAN_PER; ++j) {
        const uint32_t i = chunk * SCAN_CHUNK + j * SCAN_T + threadIdx.x;
        if (i < n) s += vid_size<SEL>(g, vids[i], round_to, T, rs);
    }
    s = block_sum_u64(s);
    if (threadIdx.x == 0) partials[chunk] = s;
}

// Exclusive scan of the chunk sums by one CTA.
__global__ void __launch_bounds__(1024) k_nbr_scan_partials(unsigned long long *partials, uint32_t nchunks) {
    pdl_wait();
    __shared__ unsigned long long s_carry;
    __shared__ unsigned long long s_w[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nchunks; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long v = i < nchunks ? partials[i] : 0ull;
        // inclusive warp scan
        unsigned long long incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, incl, d);
            if (lane_id() >= (uint32_t)d) incl += y;
        }
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long x = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0ull;
            unsigned long long xi = x;
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL, xi, d);
                if (lane_id() >= (uint32_t)d) xi += y;
            }
            s_w[threadIdx.x] = xi - x;
        }
        __syncthreads();
        const unsigned long long ex = s_carry + s_w[threadIdx.x >> 5] + incl - v;
        if (i < nchunks) partials[i] = ex;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = ex + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[nchunks] = s_carry;
}

// offsets[i] = chunk prefix + exclusive scan inside the chunk; offsets[n] = total.
template <int SEL>
__global__ void __launch_bounds__(SCAN_T) k_nbr_apply(GraphView g, const uint32_t *__restrict__ vids,
                                                      uint32_t n, uint32_t round_to, uint32_t T, uint32_t rs,
                                                      const unsigned long long *partials,
                                                      uint32_t nchunks, unsigned long long *offsets) {
    pdl_wait();
    const uint32_t chunk = blockIdx.x;
    // thread-local run over SCAN_PER consecutive elements
    unsigned long long v[SCAN_PER];
    unsigned long long s = 0;
    for (int j = 0; j < SCAN_PER; ++j) {
        const uint32_t i = chunk * SCAN_CHUNK + threadIdx.x * SCAN_PER + j;
        v[j] = i < n ? vid_size<SEL>(g, vids[i], round_to, T, rs) : 0ull;
        s += v[j];
    }
    __shared__ unsigned long long s_w[SCAN_T / 32];
    unsigned long long incl = s;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, incl, d);
        if (lane_id() >= (uint32_t)d) incl += y;
    }
    if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    unsigned long long wpre = 0;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) wpre += s_w[w];
    unsigned long long run = partials[chunk] + wpre + incl - s;
    for (int j = 0; j < SCAN_PER; ++j) {
        const uint32_t i = chunk * SCAN_CHUNK + threadIdx.x * SCAN_PER + j;
        if (i < n) offsets[i] = run;
        run += v[j];
    }
    if (chunk == nchunks - 1 && threadIdx.x == 0) offsets[n] = partials[nchunks];
}

// Items over the requested vertices' blocks (touched index = request index).
__global__ void __launch_bounds__(256) k_nbr_plan(GraphView g, const uint32_t *__restrict__ vids, uint32_t n) {
    pdl_wait();
    const uint32_t IB = g.IB;
    __shared__ uint32_t s_ai;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t ni = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (i < n) {
            const uint32_t u = vids[i];
            if (u < g.nv && g.alive[u]) {
                s = g.sent[u];
                ni = (s.y + IB - 1) / IB;
            }
        }
        uint32_t itot;
        const uint32_t iex = block_excl_scan(ni, &itot);
        if (threadIdx.x == 0) s_ai = itot ? atomicAdd(&g.dev->n_items, itot) : 0u;
        __syncthreads();
        if (i < n) {
            const uint32_t item0 = s_ai + iex;
            g.t_b[i] = make_uint4(s.x, s.y, s.z, ni);
            for (uint32_t c = 0; c < ni; ++c) g.items[item0 + c] = make_uint2(i, c);
        }
        __syncthreads();
    }
}

// One warp per item: copy the item's slots in heap (storage) order.
__global__ void __launch_bounds__(256) k_nbr_copy(GraphView g, const unsigned long long *__restrict__ offsets,
                                                  uint32_t *__restrict__ nbrs, uint32_t *__restrict__ wts) {
    pdl_wait();
    const uint32_t nitems = g.dev->n_items;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB;
    for (uint32_t it = warp; it < nitems; it += nwarps) {
        const uint2 itm = g.items[it];
        const uint4 b = g.t_b[itm.x];
        const uint32_t kb = itm.y * IB;
        const uint32_t nblk = min(IB, b.y - kb);
        uint32_t bid = NIL;
        if (lane < nblk) bid = blk_at(g, b.z, kb + 1 + lane);
        if (__any_sync(FULL, lane < nblk && bid == NIL)) {
            if (lane == 0) latch_status(g.dev, 5u /* GV_ERR_STATE */);
            continue;
        }
        const uint32_t sbase = kb * C;
        const uint32_t nslots = min(nblk * C, b.x - sbase);
        const uint32_t nquads = (nslots + 3) >> 2;
        uint32_t *out = nbrs + offsets[itm.x] + sbase;
        uint32_t *wout = wts ? wts + offsets[itm.x] + sbase : nullptr;
        for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
            const uint32_t q = q0 + lane;
            const uint32_t x = q << 2;
            const uint32_t lb = divc(g.cmul, x);
            const uint32_t myb = __shfl_sync(FULL, bid, lb & 31u);
            if (q < nquads) {
                const size_t qoff = (size_t)myb * C + (x - lb * C);
                const uint4 e4 = *reinterpret_cast<const uint4 *>(g.data + qoff);
                const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x + j < nslots) out[x + j] = e[j];
                if (wout) {
                    // payloads of a weighted graph (0 for an unweighted one)
                    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
                    if (g.wdata) w4 = *reinterpret_cast<const uint4 *>(g.wdata + qoff);
                    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x + j < nslots) wout[x + j] = w[j];
                }
            }
        }
    }
}

__global__ void k_clear_items(GraphView g) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) g.dev->n_items = 0;
}

// ------------------------------------------------------ edge-block resize

// res[0] += stored entries of live vertices, res[1] += live vertices with at
// least one entry (the paper's block-size rule, "Initialization").
__global__ void __launch_bounds__(256) k_degree_stats(GraphView g, unsigned long long *res) {
    pdl_wait();
    unsigned long long e = 0, nz = 0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.nv; u += gridDim.x * blockDim.x) {
        const uint32_t d = g.alive[u] ? g.sent[u].x : 0u;
        e += d;
        nz += d ? 1u : 0u;
    }
    e = block_sum_u64(e);
    nz = block_sum_u64(nz);
    if (threadIdx.x == 0) {
        if (e) atomicAdd(&res[0], e);
        if (nz) atomicAdd(&res[1], nz);
    }
}

// res[i] += sum over live vertices of ceil(deg / C_i), C_i = 4 (i + 1), for
// the 128 block sizes 4 .. 512.  Each lane owns four sizes (i = lane,
// lane + 32, + 64, + 96) and walks the degrees of 32 vertices at a time
// (shuffled from the lane that loaded them); sums meet in shared memory and
// then in `res`, 128 atomics per CTA.
__global__ void __launch_bounds__(256) k_footprint_blocks(GraphView g, unsigned long long *res) {
    pdl_wait();
    __shared__ unsigned long long s_acc[128];
    for (uint32_t i = threadIdx.x; i < 128; i += blockDim.x) s_acc[i] = 0;
    __syncthreads();
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long acc[4] = {0, 0, 0, 0};
    unsigned long long mag[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        const unsigned long long c = 4u * (lane + 32u * k + 1u);
        mag[k] = ((1ull << 40) + c - 1) / c;
    }
    for (uint32_t base = warp * 32; base < g.nv; base += nwarps * 32) {
        const uint32_t u = base + lane;
        const uint32_t d = (u < g.nv && g.alive[u]) ? g.sent[u].x : 0u;
        for (uint32_t j = 0; j < 32; ++j) {
            const uint32_t dj = __shfl_sync(FULL, d, j);
            if (dj == 0) continue;
            // ceil(dj / c) = floor((dj - 1) / c) + 1 for dj > 0; the quotient
            // by multiply-shift (x * ceil(2^40 / c)) >> 40, exact for
            // x < 2^31 and c <= 512, else a division
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t x = dj - 1u;
                const uint32_t q = x < 0x80000000u ? (uint32_t)(((unsigned long long)x * mag[k]) >> 40)
                                                   : x / (4u * (lane + 32u * k + 1u));
                acc[k] += q + 1u;
            }
        }
    }
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
        if (acc[k]) atomicAdd(&s_acc[lane + 32u * k], acc[k]);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 128; i += blockDim.x)
        if (s_acc[i]) atomicAdd(&res[i], s_acc[i]);
}

cudaError_t launch_footprint_blocks(const GraphView &g, unsigned long long *res, const LaunchCfg &lc) {
    cudaMemsetAsync(res, 0, 128 * sizeof(unsigned long long), lc.stream);
    if (g.nv) k_footprint_blocks<<<grid_for(g.nv, 256, lc.num_sms * 4), 256, 0, lc.stream>>>(g, res);
    return cudaGetLastError();
}

// Rebuilt trees over a contiguous run of blocks per vertex: slots[u] = first
// slot of u's run (a multiple of C); the run's blocks are heap positions
// 1 .. nblocks in id order, so block k's children are the run's blocks 2k
// and 2k + 1 ("Dynamic edge inserts": heap-numbered complete binary tree);
// the entries were already copied to the run.  One thread per vertex writes
// the sentinel and the links of a run of up to PLACE_SMALL blocks; longer
// runs (the hubs of a skewed graph) are listed for k_reblock_big, which
// spreads each over a whole CTA.
constexpr uint32_t PLACE_SMALL = 32;

//
// With hub runs (g.rs != 0) a vertex of degree >= T is a hub: its run starts
// at slots[u] (R-aligned: hubs fill the run region from block 0 in whole
// runs) and its tree is one of run heads, the head of run k (1-based) being
// block base + (k - 1) * R; every other vertex's run starts at slots[u] +
// plain_shift (the scratch placed the hubs first, the pool puts the plain
// vertices past the run region).
__device__ __forceinline__ void place_links(const GraphView &g, uint32_t base, uint32_t n, uint32_t stride,
                                            uint32_t k) {
    const uint32_t b = base + (k - 1) * stride;
    g.links[2ull * b] = 2ull * k <= n ? base + (2 * k - 1) * stride : NIL;
    g.links[2ull * b + 1] = 2ull * k + 1 <= n ? base + 2 * k * stride : NIL;
}

__global__ void __launch_bounds__(256) k_reblock_place(GraphView g, const unsigned long long *__restrict__ slots,
                                                       uint32_t *big, unsigned long long *nbig, uint32_t T,
                                                       unsigned long long plain_shift) {
    pdl_wait();
    const uint32_t C = g.C;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.nv; u += gridDim.x * blockDim.x) {
        const uint32_t deg = g.alive[u] ? g.sent[u].x : 0u;
        const uint32_t nb = (deg + C - 1) / C;
        const bool hub = g.rs && deg > 0 && deg >= T;
        const uint32_t base = (uint32_t)((hub ? slots[u] : slots[u] + plain_shift) / C);
        const uint32_t stride = hub ? 1u << g.rs : 1u;          // heads of runs, or blocks
        const uint32_t n = hub ? (nb + stride - 1) >> g.rs : nb;  // tree nodes
        g.sent[u] = make_uint4(deg, nb, nb ? (hub ? base | RUN_BIT : base) : NIL, nb ? base + nb - 1 : NIL);
        if (n > PLACE_SMALL) {
            big[atomicAdd(nbig, 1ull)] = u;
            continue;
        }
        for (uint32_t k = 1; k <= n; ++k) place_links(g, base, n, stride, k);
    }
}

// Links of the long runs, one CTA per listed vertex.
__global__ void __launch_bounds__(256) k_reblock_big(GraphView g, const unsigned long long *__restrict__ slots,
                                                     const uint32_t *__restrict__ big,
                                                     const unsigned long long *nbig) {
    pdl_wait();
    const uint32_t n = (uint32_t)*nbig;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t u = big[i];
        const uint4 st = g.sent[u];  // written by k_reblock_place
        const bool hub = is_run(st.z);
        const uint32_t base = st.z & ~RUN_BIT;
        const uint32_t stride = hub ? 1u << g.rs : 1u;
        const uint32_t nodes = hub ? (st.y + stride - 1) >> g.rs : st.y;
        for (uint32_t k = 1 + threadIdx.x; k <= nodes; k += blockDim.x) place_links(g, base, nodes, stride, k);
    }
}

// Edge-block resize of a graph with hub runs: one scratch offset per vertex,
// the hubs' runs first (hub_off), the plain vertices' runs after them
// (hub_total + plain_off), written over plain_off.
__global__ void __launch_bounds__(256) k_reblock_merge(GraphView g, unsigned long long *plain_off,
                                                       const unsigned long long *__restrict__ hub_off, uint32_t T,
                                                       unsigned long long hub_total) {
    pdl_wait();
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.nv; u += gridDim.x * blockDim.x) {
        const uint32_t deg = g.alive[u] ? g.sent[u].x : 0u;
        plain_off[u] = (deg > 0 && deg >= T) ? hub_off[u] : hub_total + plain_off[u];
    }
}

cudaError_t launch_reblock_merge(const GraphView &g, unsigned long long *plain_off, const unsigned long long *hub_off,
                                 uint32_t T, unsigned long long hub_total, const LaunchCfg &lc) {
    if (g.nv) k_reblock_merge<<<grid_for(g.nv, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(g, plain_off, hub_off, T,
                                                                                            hub_total);
    return cudaGetLastError();
}

cudaError_t launch_degree_stats(const GraphView &g, unsigned long long *res, const LaunchCfg &lc) {
    cudaMemsetAsync(res, 0, 2 * sizeof(unsigned long long), lc.stream);
    if (g.nv) k_degree_stats<<<grid_for(g.nv, 256, lc.num_sms * 8), 256, 0, lc.stream>>>(g, res);
    return cudaGetLastError();
}

cudaError_t launch_reblock_place(const GraphView &g, const unsigned long long *slots, uint32_t *big,
                                 unsigned long long *nbig, const LaunchCfg &lc, uint32_t T,
                                 unsigned long long plain_shift) {
    cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), lc.stream);
    if (g.nv) {
        k_reblock_place<<<grid_for(g.nv, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(g, slots, big, nbig, T,
                                                                                      plain_shift);
        launch_pdl(k_reblock_big, lc.num_sms * 4, 256, 0, lc.stream, g, slots, big, nbig);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------- self-check

// res[0] violations, res[1] sum of degrees, res[2] owned blocks, res[3] queued blocks
__device__ __forceinline__ uint32_t cbt_walk_checked(const uint32_t *links, unsigned long long P,
                                                     uint32_t root, uint32_t k, bool &bad) {
    uint32_t b = root;
    if (b >= P) {
        bad = true;
        return NIL;
    }
    int top = 31 - __clz(k);
    for (int i = top - 1; i >= 0; --i) {
        b = links[2ull * b + ((k >> i) & 1u)];
        if (b >= P) {
            bad = true;
            return NIL;
        }
    }
    return b;
}

__global__ void __launch_bounds__(256) k_validate_vertices(GraphView g, uint32_t *owner,
                                                           unsigned long long *res) {
    pdl_wait();
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C;
    const uint32_t R = 1u << g.rs;
    const unsigned long long H = g.rs ? (g.RP << g.rs) : 0ull;  // run region [0, H)
    unsigned long long viol = 0, sdeg = 0, snb = 0;
    for (uint32_t u = warp; u < g.nv; u += nwarps) {
        const uint4 s = g.sent[u];
        const uint32_t deg = s.x, nb = s.y;
        const bool run = is_run(s.z);
        const uint32_t nr = run ? (nb + R - 1u) >> g.rs : 0u;
        if (lane == 0) {
            sdeg += deg;
            snb += run ? (unsigned long long)nr << g.rs : nb;  // blocks owned
            if (C == 0 ? (deg != 0 || nb != 0) : (nb != (deg + C - 1) / C)) ++viol;
            if (!g.alive[u] && (deg != 0 || nb != 0)) ++viol;
            if (nb == 0 && (s.z != NIL || s.w != NIL)) ++viol;
            if (run && g.rs == 0) ++viol;
        }
        if (run) {
            // tree of run heads: each head R-aligned inside the run region,
            // all R blocks of each run owned once, the last block in the last run
            const uint32_t head0 = s.z & ~RUN_BIT;
            for (uint32_t k = 1 + lane; k <= nr; k += 32) {
                bool bad = false;
                const uint32_t h = cbt_walk_checked(g.links, g.P, head0, k, bad);
                if (bad || h >= H || (h & (R - 1u))) {
                    ++viol;
                    continue;
                }
                for (uint32_t i = 0; i < R; ++i) {
                    const uint32_t b = h + i, bit = 1u << (b & 31u);
                    if (atomicOr(&owner[b >> 5], bit) & bit) ++viol;
                }
                if (k == nr && s.w != h + ((nb - 1u) & (R - 1u))) ++viol;
                if (2ull * k > nr && g.links[2ull * h] != NIL) ++viol;
                if (2ull * k + 1 > nr && g.links[2ull * h + 1] != NIL) ++viol;
            }
            continue;
        }
        for (uint32_t k = 1 + lane; k <= nb; k += 32) {
            bool bad = false;
            const uint32_t b = cbt_walk_checked(g.links, g.P, s.z, k, bad);
            if (bad || b < H) {  // a plain adjacency's blocks lie outside the run region
                ++viol;
                continue;
            }
            const uint32_t bit = 1u << (b & 31u);
            if (atomicOr(&owner[b >> 5], bit) & bit) ++viol;
            if (k == nb && b != s.w) ++viol;
            if (2ull * k > nb && g.links[2ull * b] != NIL) ++viol;
            if (2ull * k + 1 > nb && g.links[2ull * b + 1] != NIL) ++viol;
        }
    }
    viol = warp_sum_u64(viol);
    sdeg = warp_sum_u64(sdeg);
    snb = warp_sum_u64(snb);
    if (lane == 0) {
        if (viol) atomicAdd(&res[0], viol);
        if (sdeg) atomicAdd(&res[1], sdeg);
        if (snb) atomicAdd(&res[2], snb);
    }
}

__global__ void __launch_bounds__(256) k_validate_queue(GraphView g, uint32_t *owner,
                                                        unsigned long long *res) {
    pdl_wait();
    const unsigned long long qf = g.dev->q_front, qb = g.dev->q_back, P = g.P;
    if (P == 0) return;
    const unsigned long long H = g.rs ? (g.RP << g.rs) : 0ull;
    unsigned long long viol = 0, cnt = 0;
    for (unsigned long long p = qf + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < qb;
         p += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t b = g.queue[p % P];
        ++cnt;
        if (b >= P || b < H) {
            ++viol;
            continue;
        }
        const uint32_t bit = 1u << (b & 31u);
        if (atomicOr(&owner[b >> 5], bit) & bit) ++viol;
    }
    if (g.rs) {
        // free runs: R-aligned heads inside the run region, each covering R
        // blocks that nothing else owns
        const uint32_t R = 1u << g.rs;
        const unsigned long long rqf = g.dev->rq_front, rqb = g.dev->rq_back;
        for (unsigned long long p = rqf + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < rqb;
             p += (unsigned long long)gridDim.x * blockDim.x) {
            const uint32_t h = g.rqueue[p % g.RP];
            if (h >= H || (h & (R - 1u))) {
                ++viol;
                continue;
            }
            cnt += R;
            for (uint32_t i = 0; i < R; ++i) {
                const uint32_t b = h + i, bit = 1u << (b & 31u);
                if (atomicOr(&owner[b >> 5], bit) & bit) ++viol;
            }
        }
    }
    viol = warp_sum_u64(viol);
    cnt = warp_sum_u64(cnt);
    if (lane_id() == 0) {
        if (viol) atomicAdd(&res[0], viol);
        if (cnt) atomicAdd(&res[3], cnt);
    }
}

// ------------------------------------------------------------------ launch


cudaError_t launch_init_vertices(const GraphView &g, uint32_t from, uint32_t to, const LaunchCfg &lc) {
    if (to > from) k_init_vertices<<<grid_for(to - from, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(g, from, to);
    return cudaGetLastError();
}

cudaError_t launch_copy_dictionary(uint4 *dst_sent, uint8_t *dst_alive, const uint4 *src_sent,
                                   const uint8_t *src_alive, uint32_t n, const LaunchCfg &lc) {
    if (n) k_copy_dictionary<<<grid_for(n, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(dst_sent, dst_alive, src_sent, src_alive, n);
    return cudaGetLastError();
}

cudaError_t launch_init_queue(uint32_t *queue, unsigned long long n, const LaunchCfg &lc, uint32_t first,
                              uint32_t step) {
    if (n) k_init_queue<<<grid_for(n, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(queue, n, first, step);
    return cudaGetLastError();
}

// Edge queue of a grown pool: the free ids in ring order at positions
// 0 .. free-1, then the new ids P .. P2-1.
__global__ void k_grow_queue(const uint32_t *__restrict__ q, unsigned long long P, unsigned long long qf,
                             unsigned long long nfree, uint32_t *__restrict__ q2, unsigned long long P2) {
    pdl_wait();
    const unsigned long long tot = nfree + (P2 - P);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < tot;
         i += (unsigned long long)gridDim.x * blockDim.x)
        q2[i] = i < nfree ? q[(qf + i) % P] : (uint32_t)(P + (i - nfree));
}

cudaError_t launch_grow_queue(const uint32_t *q, unsigned long long P, unsigned long long qf,
                              unsigned long long nfree, uint32_t *q2, unsigned long long P2, const LaunchCfg &lc) {
    const unsigned long long tot = nfree + (P2 - P);
    if (tot) k_grow_queue<<<grid_for(tot, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(q, P, qf, nfree, q2, P2);
    return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t *out, uint32_t first, uint32_t k, const LaunchCfg &lc) {
    if (k) k_iota<<<grid_for(k, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(out, first, k);
    return cudaGetLastError();
}

cudaError_t launch_degrees(const GraphView &g, uint32_t *deg, uint8_t *alive, const LaunchCfg &lc) {
    if (g.nv) k_degrees<<<grid_for(g.nv, 256, lc.num_sms * 16), 256, 0, lc.stream>>>(g, deg, alive);
    return cudaGetLastError();
}

cudaError_t launch_neighbor_offsets(const GraphView &g, const uint32_t *vids, uint32_t n,
                                    unsigned long long *offsets, unsigned long long *partials,
                                    const LaunchCfg &lc, uint32_t round_to) {
    const uint32_t nchunks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nchunks == 0) {
        cudaError_t e = cudaMemsetAsync(offsets, 0, sizeof(unsigned long long), lc.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(partials, 0, sizeof(unsigned long long), lc.stream);
        return e;
    }
    PhaseScope ps(lc, PH_NEIGHBORS);
    k_nbr_partials<0><<<nchunks, SCAN_T, 0, lc.stream>>>(g, vids, n, round_to, 0u, 0u, partials);
    launch_pdl(k_nbr_scan_partials, 1, 1024, 0, lc.stream, partials, nchunks);
    launch_pdl(k_nbr_apply<0>, nchunks, SCAN_T, 0, lc.stream, g, vids, n, round_to, 0u, 0u, partials, nchunks,
               offsets);
    return cudaGetLastError();
}

cudaError_t launch_reblock_offsets(const GraphView &g, const uint32_t *vids, uint32_t n, unsigned long long *offsets,
                                   unsigned long long *partials, const LaunchCfg &lc, uint32_t round_to, bool hubs,
                                   uint32_t T, uint32_t rs) {
    const uint32_t nchunks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nchunks == 0) {
        cudaError_t e = cudaMemsetAsync(offsets, 0, sizeof(unsigned long long), lc.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(partials, 0, sizeof(unsigned long long), lc.stream);
        return e;
    }
    PhaseScope ps(lc, PH_OTHER);
    if (hubs) k_nbr_partials<2><<<nchunks, SCAN_T, 0, lc.stream>>>(g, vids, n, round_to, T, rs, partials);
    else k_nbr_partials<1><<<nchunks, SCAN_T, 0, lc.stream>>>(g, vids, n, round_to, T, rs, partials);
    launch_pdl(k_nbr_scan_partials, 1, 1024, 0, lc.stream, partials, nchunks);
    if (hubs)
        launch_pdl(k_nbr_apply<2>, nchunks, SCAN_T, 0, lc.stream, g, vids, n, round_to, T, rs, partials, nchunks,
                   offsets);
    else
        launch_pdl(k_nbr_apply<1>, nchunks, SCAN_T, 0, lc.stream, g, vids, n, round_to, T, rs, partials, nchunks,
                   offsets);
    return cudaGetLastError();
}

cudaError_t launch_neighbor_copy(const GraphView &g, const uint32_t *vids, uint32_t n,
                                 const unsigned long long *offsets, uint32_t *nbrs, const LaunchCfg &lc,
                                 uint32_t *wts) {
    if (n == 0) return cudaSuccess;
    PhaseScope ps(lc, PH_NEIGHBORS);
    k_nbr_plan<<<grid_for(n, 256, lc.num_sms * 8), 256, 0, lc.stream>>>(g, vids, n);
    launch_pdl(k_nbr_copy, lc.num_sms * 8, 256, 0, lc.stream, g, offsets, nbrs, wts);
    launch_pdl(k_clear_items, 1, 32, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_validate(const GraphView &g, uint32_t *owner_bits, unsigned long long *res,
                            const LaunchCfg &lc) {
    k_validate_vertices<<<lc.num_sms * 8, 256, 0, lc.stream>>>(g, owner_bits, res);
    launch_pdl(k_validate_queue, lc.num_sms * 8, 256, 0, lc.stream, g, owner_bits, res);
    return cudaGetLastError();
}

}  // namespace gv

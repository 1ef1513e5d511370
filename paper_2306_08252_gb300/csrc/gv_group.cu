// gv_group.cu -- grouping a large pair batch by source vertex, and the kernels
// of the insert, delete and query paths that consume the grouped batch.
//
// The paper builds each update batch as CSR on the host ("Initialization and
// batch updates": sources in order, each with its destinations).  Here large
// batches are grouped on the device by a two-level radix partition of the
// source id, with no global atomic per pair:
//   hist     each partition CTA owns a contiguous range of the batch and
//            counts its valid pairs per bucket (bucket = u >> gb_shift, the
//            high bits of the source) in shared memory: one row of counts per
//            CTA.  Invalid pairs (an endpoint out of range or deleted) are
//            counted as rejected and dropped.
//   colscan  per bucket, the exclusive prefix of the rows over the CTAs, and
//            the bucket's total.
//   bktscan  one CTA: bucket bases (exclusive scan of the totals) and the
//            chunk list (every bucket cut into chunks of at most GP_CHUNK).
//   scatter  each partition CTA writes its valid pairs at shared cursors
//            started from its prefixes: the pairs of a bucket are contiguous.
//   count    per chunk: pairs per vertex of the bucket in shared memory, then
//            one global atomic per (chunk, vertex) on the vertex's count.
//   vscan    per vertex: the start of its segment (bucket base + exclusive
//            prefix of the counts within the bucket) and the touched list.
//   place    per chunk: a counting sort by vertex in shared memory, one global
//            atomic per (chunk, vertex) that reserves the chunk's run inside
//            the vertex's segment, then the chunk written out run by run.
//            Deletes and queries write the destinations as the per-source
//            batch lists of the membership pipeline; inserts write them
//            straight into their adjacency slots (slot deg + rank, Algorithm 1)
//            after the plan and the links, so runs of one source land in
//            consecutive slots.
// Traffic per valid pair: 8 B read (hist), 8 B read + 8 B written (scatter),
// 4 B read (count), 8 B read (place) and 4 B written (a slot or a list entry).
#include "gv_launch.h"

namespace gv {

__device__ __forceinline__ bool gp_valid(const GraphView &g, uint32_t u, uint32_t v) {
    return u < g.nv && v < g.nv && (g.all_alive || (g.alive[u] && g.alive[v]));
}

// ------------------------------------------------------------- partition

constexpr int GP_UNROLL = 4;

// Per-bucket counts of partition CTAs [c0, c0 + gridDim.x) (pairs [c*L,
// min(n, (c+1)*L)) of CTA c).  A launch covers whole CTA ranges, so the
// batch may be counted piece by piece while later pieces are still copied.
template <int MODE>
__global__ void __launch_bounds__(GP_THREADS) k_gp_hist(GraphView g, const uint32_t *__restrict__ src,
                                                        const uint32_t *__restrict__ dst, unsigned long long n,
                                                        uint32_t c0) {
    pdl_wait();
    __shared__ uint32_t hist[GP_BMAX];
    const uint32_t nb = g.gb_n, sh = g.gb_shift;
    for (uint32_t b = threadIdx.x; b < nb; b += GP_THREADS) hist[b] = 0;
    __syncthreads();
    const uint32_t c = c0 + blockIdx.x;
    const unsigned long long beg = (unsigned long long)c * g.gp_len;
    const unsigned long long end = min(n, beg + g.gp_len);
    unsigned long long rej = 0;
    for (unsigned long long i0 = beg + threadIdx.x; i0 < end; i0 += GP_THREADS * GP_UNROLL) {
        uint32_t u[GP_UNROLL], v[GP_UNROLL];
#pragma unroll
        for (int j = 0; j < GP_UNROLL; ++j) {
            const unsigned long long i = i0 + (unsigned long long)j * GP_THREADS;
            u[j] = i < end ? ld_stream(src + i) : NIL;
            v[j] = i < end ? ld_stream(dst + i) : NIL;
        }
#pragma unroll
        for (int j = 0; j < GP_UNROLL; ++j) {
            const unsigned long long i = i0 + (unsigned long long)j * GP_THREADS;
            if (i < end) {
                if (gp_valid(g, u[j], v[j])) atomicAdd(&hist[u[j] >> sh], 1u);
                else ++rej;
            }
        }
    }
    __syncthreads();
    uint32_t *row = g.gp_hist + (size_t)c * nb;
    for (uint32_t b = threadIdx.x; b < nb; b += GP_THREADS) row[b] = hist[b];
    if (MODE != MODE_QUERY) {
        rej = warp_sum_u64(rej);
        if (lane_id() == 0 && rej) atomicAdd(&g.dev->call_b, rej);
    }
}

// Per bucket (32 per CTA, one per lane): the exclusive prefix of its counts
// over the partition CTAs, written over the counts; the total to gp_btot.
// The 8 warps of a CTA take consecutive slices of the rows.
__global__ void __launch_bounds__(256) k_gp_colscan(GraphView g) {
    pdl_wait();
    __shared__ uint32_t s_tot[8][32];
    const uint32_t nb = g.gb_n, G = g.gp_ctas;
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * 32 + lane;
    const bool ok = b < nb;
    const uint32_t r0 = (uint32_t)((unsigned long long)G * w / 8);
    const uint32_t r1 = (uint32_t)((unsigned long long)G * (w + 1) / 8);
    uint32_t sum = 0;
#pragma unroll 8
    for (uint32_t r = r0; r < r1; ++r)
        if (ok) sum += g.gp_hist[(size_t)r * nb + b];
    s_tot[w][lane] = sum;
    __syncthreads();
    uint32_t run = 0;
    for (uint32_t k = 0; k < w; ++k) run += s_tot[k][lane];
    for (uint32_t r = r0; r < r1; ++r) {
        if (ok) {
            const size_t at = (size_t)r * nb + b;
            const uint32_t x = g.gp_hist[at];
            g.gp_hist[at] = run;
            run += x;
        }
    }
    if (w == 7 && ok) g.gp_btot[b] = run;
}

// One CTA of 1024 threads, four buckets each: bucket bases and the chunk list.
__global__ void __launch_bounds__(1024) k_gp_bktscan(GraphView g) {
    pdl_wait();
    const uint32_t nb = g.gb_n;
    uint32_t tot[4], nch[4], st = 0, sc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t b = threadIdx.x * 4 + j;
        tot[j] = b < nb ? g.gp_btot[b] : 0u;
        nch[j] = (tot[j] + GP_CHUNK - 1) / GP_CHUNK;
        st += tot[j];
        sc += nch[j];
    }
    uint32_t all_t, all_c;
    uint32_t et = block_excl_scan(st, &all_t);
    uint32_t ec = block_excl_scan(sc, &all_c);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t b = threadIdx.x * 4 + j;
        if (b < nb) {
            g.gp_bbase[b] = et;
            for (uint32_t k = 0; k < nch[j]; ++k)
                g.gp_chunks[ec + k] = make_uint4(et + k * GP_CHUNK, min(GP_CHUNK, tot[j] - k * GP_CHUNK), b, 0u);
        }
        et += tot[j];
        ec += nch[j];
    }
    if (threadIdx.x == 0) g.dev->n_chunks = all_c;
}

// Valid pairs of each partition CTA to their buckets.  A query's original
// index (or an insert's payload) travels with its pair; an invalid query is
// answered 0 (no arena position).
template <int MODE, bool AUX>
__global__ void __launch_bounds__(GP_THREADS) k_gp_scatter(GraphView g, const uint32_t *__restrict__ src,
                                                           const uint32_t *__restrict__ dst,
                                                           const uint32_t *__restrict__ wts, unsigned long long n) {
    pdl_wait();
    __shared__ uint32_t cur[GP_BMAX];
    const uint32_t nb = g.gb_n, sh = g.gb_shift;
    const uint32_t c = blockIdx.x;
    const uint32_t *row = g.gp_hist + (size_t)c * nb;
    for (uint32_t b = threadIdx.x; b < nb; b += GP_THREADS) cur[b] = g.gp_bbase[b] + row[b];
    __syncthreads();
    const unsigned long long beg = (unsigned long long)c * g.gp_len;
    const unsigned long long end = min(n, beg + g.gp_len);
    for (unsigned long long i0 = beg + threadIdx.x; i0 < end; i0 += GP_THREADS * GP_UNROLL) {
        uint32_t u[GP_UNROLL], v[GP_UNROLL];
#pragma unroll
        for (int j = 0; j < GP_UNROLL; ++j) {
            const unsigned long long i = i0 + (unsigned long long)j * GP_THREADS;
            u[j] = i < end ? ld_stream(src + i) : NIL;
            v[j] = i < end ? ld_stream(dst + i) : NIL;
        }
#pragma unroll
        for (int j = 0; j < GP_UNROLL; ++j) {
            const unsigned long long i = i0 + (unsigned long long)j * GP_THREADS;
            if (i >= end) continue;
            if (gp_valid(g, u[j], v[j])) {
                const uint32_t pos = atomicAdd(&cur[u[j] >> sh], 1u);
                g.gp_src[pos] = u[j];
                g.gp_dst[pos] = v[j];
                if (AUX) g.gp_aux[pos] = MODE == MODE_QUERY ? (uint32_t)i : (wts ? ld_stream(wts + i) : 0u);
            } else if (MODE == MODE_QUERY) {
                g.qpos[i] = NIL;
            }
        }
    }
}

// -------------------------------------------------------- per-vertex counts

__global__ void __launch_bounds__(GP_THREADS) k_gp_count(GraphView g) {
    pdl_wait();
    __shared__ uint32_t hist[GP_WMAX];
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    const uint32_t nch = g.dev->n_chunks;
    for (uint32_t k = blockIdx.x; k < nch; k += gridDim.x) {
        const uint4 ck = g.gp_chunks[k];  // {start, length, bucket}
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS) hist[w] = 0;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < ck.y; j += GP_THREADS)
            atomicAdd(&hist[ld_stream(g.gp_src + ck.x + j) & (W - 1)], 1u);
        __syncthreads();
        const uint32_t vb = ck.z << sh;
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS)
            if (hist[w]) atomicAdd(&g.vcnt[vb + w], hist[w]);
        __syncthreads();
    }
}

// Per vertex: segment start = bucket base + exclusive prefix of the counts of
// the bucket's vertices before it (GP_VPC consecutive vertices per CTA, whole
// buckets since GP_VPC >= vertices per bucket); touched vertices are listed.
__global__ void __launch_bounds__(1024) k_gp_vscan(GraphView g) {
    pdl_wait();
    __shared__ uint32_t s_pre[GP_VPC];
    __shared__ uint32_t s_tb;
    const uint32_t ncap = g.vmask + 1;
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    for (uint32_t base = blockIdx.x * GP_VPC; base < ncap; base += gridDim.x * GP_VPC) {
        const uint32_t u0 = base + threadIdx.x * 4;
        uint32_t c[4] = {0u, 0u, 0u, 0u};
        if (u0 + 3 < ncap) {
            const uint4 x = *reinterpret_cast<const uint4 *>(g.vcnt + u0);
            c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (u0 + j < ncap) c[j] = g.vcnt[u0 + j];
        }
        uint32_t tot;
        uint32_t p = block_excl_scan(c[0] + c[1] + c[2] + c[3], &tot);
        uint32_t pj[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pj[j] = p;
            s_pre[threadIdx.x * 4 + j] = p;
            p += c[j];
        }
        uint32_t flags = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c[j]) flags |= 1u << j;
        uint32_t ntot;
        const uint32_t ex = block_excl_scan(__popc(flags), &ntot);  // its barriers also publish s_pre
        if (threadIdx.x == 0) s_tb = ntot ? atomicAdd(&g.dev->n_touched, ntot) : 0u;
        __syncthreads();
        uint32_t t = s_tb + ex;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((flags >> j) & 1u) {
                const uint32_t u = u0 + j;
                const uint32_t fb = (u & ~(W - 1)) - base;  // the bucket's first vertex, inside this range
                g.gcur[u] = g.gp_bbase[u >> sh] + pj[j] - s_pre[fb];
                g.t_vid[t++] = u;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- place

// Shared memory of k_gp_place for W vertices per bucket.
__host__ __device__ constexpr size_t gp_place_smem(uint32_t W) { return (size_t)(3 * W + 3 * GP_CHUNK) * 4; }

// Exclusive scan of cnt[0, W) into out[] by the whole CTA (GP_THREADS
// threads, W a power of two <= GP_WMAX); all threads call.
__device__ __forceinline__ void gp_scan_counts(const uint32_t *cnt, uint32_t *out, uint32_t W) {
    const uint32_t per = W > GP_THREADS ? W / GP_THREADS : 1u;
    const uint32_t first = threadIdx.x * per;
    uint32_t s = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (first + k < W) s += cnt[first + k];
    uint32_t tot;
    uint32_t e = block_excl_scan(s, &tot);
    for (uint32_t k = 0; k < per; ++k) {
        if (first + k < W) {
            out[first + k] = e;
            e += cnt[first + k];
        }
    }
}

template <int MODE, bool WEIGHTED>
__global__ void __launch_bounds__(GP_THREADS) k_gp_place(GraphView g) {
    pdl_wait();
    if (MODE == MODE_INSERT && g.dev->abort) return;
    extern __shared__ __align__(16) uint32_t gsm[];
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    uint32_t *hist = gsm;            // [W]
    uint32_t *loff = hist + W;       // [W] run start inside the chunk
    uint32_t *rbase = loff + W;      // [W] run start inside the vertex's segment
    uint32_t *sv = rbase + W;        // [GP_CHUNK] destinations in run order
    uint32_t *sw = sv + GP_CHUNK;    // [GP_CHUNK] vertex within the bucket
    uint32_t *sx = sw + GP_CHUNK;    // [GP_CHUNK] original index / payload
    constexpr bool AUX = MODE == MODE_QUERY || WEIGHTED;
    constexpr int PER = GP_CHUNK / GP_THREADS;
    const uint32_t nch = g.dev->n_chunks;
    const uint32_t C = g.C;
    const unsigned long long P = g.P;
    const unsigned long long qbase = MODE == MODE_INSERT ? qmod(g.dev->q_front, P) : 0ull;
    for (uint32_t k = blockIdx.x; k < nch; k += gridDim.x) {
        const uint4 ck = g.gp_chunks[k];
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS) hist[w] = 0;
        __syncthreads();
        uint32_t wv[PER], vv[PER], xv[PER], lr[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t j = threadIdx.x + e * GP_THREADS;
            if (j < ck.y) {
                wv[e] = ld_stream(g.gp_src + ck.x + j) & (W - 1);
                vv[e] = ld_stream(g.gp_dst + ck.x + j);
                xv[e] = AUX ? ld_stream(g.gp_aux + ck.x + j) : 0u;
            }
        }
#pragma unroll
        for (int e = 0; e < PER; ++e)
            if (threadIdx.x + e * GP_THREADS < ck.y) lr[e] = atomicAdd(&hist[wv[e]], 1u);
        __syncthreads();
        gp_scan_counts(hist, loff, W);
        const uint32_t vb = ck.z << sh;
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS)
            if (hist[w]) rbase[w] = atomicAdd(&g.gcur[vb + w], hist[w]);
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            if (threadIdx.x + e * GP_THREADS < ck.y) {
                const uint32_t p = loff[wv[e]] + lr[e];
                sv[p] = vv[e];
                sw[p] = wv[e];
                if (AUX) sx[p] = xv[e];
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < ck.y; j += GP_THREADS) {
            const uint32_t w = sw[j];
            const uint32_t pos = rbase[w] + (j - loff[w]);
            if (MODE == MODE_INSERT) {
                // slot deg + rank of the source (Algorithm 1): the free slots of
                // the last block first, then the blocks popped for it
                const uint4 vi = g.vinfo[vb + w];  // {deg, last block, queue offset, segment start}
                const uint32_t r = pos - vi.w;
                const uint32_t deg = vi.x;
                const uint32_t nb = divc(g.cmul, deg + C - 1);
                const uint32_t space = nb * C - deg;
                uint32_t blk, ln;
                if (r < space) {
                    blk = vi.y;
                    ln = deg - (nb - 1) * C + r;
                } else {
                    const uint32_t q = r - space;
                    const uint32_t jb = divc(g.cmul, q);
                    ln = q - jb * C;
                    blk = g.queue[ring(qbase, vi.z + jb, P)];
                }
                if (blk < P) {
                    const size_t slot = (size_t)blk * C + ln;
                    g.data[slot] = sv[j];
                    if (WEIGHTED) g.wdata[slot] = sx[j];
                } else {
                    latch_status(g.dev, 5u /* GV_ERR_STATE */);
                }
            } else {
                g.arena[pos] = sv[j];
                if (MODE == MODE_QUERY) {
                    g.found[pos] = 0u;
                    g.qpos[sx[j]] = pos;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ insert plan

// Per touched source: block demand, queue offsets by a block-wide prefix sum
// (Figure 3), the source's plan record {deg, last block, queue offset,
// segment start} for the placement.
__global__ void __launch_bounds__(256) k_gp_plan_insert(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t C = g.C;
    __shared__ unsigned long long s_base;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t need = 0, deg = 0, last = NIL, u = 0, seg = 0;
        if (t < nt) {
            u = g.t_vid[t];
            const uint32_t cnt = g.vcnt[u];
            seg = g.gcur[u];
            const uint4 s = g.sent[u];
            deg = s.x;
            last = s.w;
            const uint32_t space = s.y * C - deg;
            need = cnt > space ? divc(g.cmul, cnt - space + C - 1) : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(need, &tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(&g.dev->alloc_total, (unsigned long long)tot) : 0ull;
        __syncthreads();
        const unsigned long long off = s_base + ex;
        if (t < nt) {
            g.t_a[t] = make_uint4(deg, last, (uint32_t)off, need);
            g.vinfo[u] = make_uint4(deg, last, (uint32_t)off, seg);
            for (uint32_t j = 0; j < need; ++j) g.t_owner[off + j] = t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ membership plan

// Per touched source (after the placement: its batch list is arena[gcur - m,
// gcur)): the thread-per-source tier for tiny adjacencies, else work items of
// IB blocks; sources with more than LIST_MAX batch entries go to the
// block-wide tier (CT_GI items per CTA group) instead of the warp tier.
template <int MODE>
__global__ void __launch_bounds__(256) k_gp_plan_member(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t IB = g.IB;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    __shared__ uint32_t s_ai, s_am, s_at, s_ath, s_ag;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t m = 0, aoff = 0, ni = 0, tiny = 0, ng = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            m = g.vcnt[u];
            aoff = g.gcur[u] - m;
            s = g.sent[u];
            if (s.y > 0) {
                const bool small = MODE == MODE_QUERY
                    ? (s.x <= min(TINY_DEG_Q, TINY_NB_Q * g.C) && s.y <= TINY_NB_Q && m <= TINY_M)
                    : (s.x <= tiny_deg && s.y <= TINY_NB && m <= TINY_M);
                if (small) {
                    tiny = 1;
                } else {
                    ni = (s.y + IB - 1) / IB;
                    if (m > LIST_MAX) ng = (ni + CT_GI - 1) / CT_GI;
                }
            }
        }
        const uint32_t tlo = tiny && s.x <= TINY_SPLIT, thi = tiny && s.x > TINY_SPLIT;
        uint32_t ttot, tthi, gtot;
        const uint32_t tex = block_excl_scan(tlo, &ttot);
        const uint32_t thx = block_excl_scan(thi, &tthi);
        const uint32_t gex = block_excl_scan(ng, &gtot);
        if (threadIdx.x == 0) {
            s_at = ttot ? atomicAdd(&g.dev->n_tiny, ttot) : 0u;
            s_ath = tthi ? atomicAdd(&g.dev->n_tiny_hi, tthi) : 0u;
            s_ag = gtot ? atomicAdd(&g.dev->n_groups, gtot) : 0u;
        }
        const uint32_t item0 = alloc_items(g, ni, &s_ai, &s_am);
        if (t < nt) {
            g.t_a[t] = make_uint4(m, aoff, ng ? CT_FLAG : 0u, item0);
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            if (tlo) g.t_tiny[s_at + tex] = t;
            if (thi) g.t_tiny[g.tiny_cap - 1 - (s_ath + thx)] = t;
            emit_items(g, t, item0, ni);
            for (uint32_t k = 0; k < ng; ++k) g.grp_items[s_ag + gex + k] = make_uint2(t, k * CT_GI);
        }
        __syncthreads();
    }
}

// ------------------------------------------------ block-wide membership tier

// Slot of key v in the shared table of hs slots (buckets of 4; occupied
// slots are a prefix of each bucket), or NIL.
__device__ __forceinline__ uint32_t ct_find(const uint32_t *hk, uint32_t nbk, uint32_t v) {
    uint32_t b = hidx(v, nbk);
    for (uint32_t step = 0; step < nbk; ++step) {
        const uint4 w = *reinterpret_cast<const uint4 *>(hk + 4 * b);
        if (w.x == v) return 4 * b;
        if (w.y == v) return 4 * b + 1;
        if (w.z == v) return 4 * b + 2;
        if (w.w == v) return 4 * b + 3;
        if (w.w == EMPTY_KEY) return NIL;  // the bucket's prefix ended
        b = (b + 1) & (nbk - 1);
    }
    return NIL;
}

// Delete / query for the sources with more than LIST_MAX batch entries:
// one CTA per group of CT_GI work items of one source, one warp per item.
// The source's batch list (contiguous after the placement) is loaded into a
// shared hash set CT_KEYS keys at a time; per slice each warp streams its
// item's entries (16-byte loads) and ORs the hits into a shared bit mask.
// Queries also flag the hit keys and set the list entries' found words.
// Then, as in the warp tier: single-item sources are compacted in place
// (stable) and their emptied blocks returned; items of multi-item sources
// record survivor masks, counts and block ids for the hole filling.
template <int MODE, bool WEIGHTED>
__global__ void __launch_bounds__(256) k_mark_cta(GraphView g) {
    pdl_wait();
    __shared__ __align__(16) uint32_t hk[CT_SLOTS];
    __shared__ uint8_t hf[MODE == MODE_QUERY ? CT_SLOTS : 4];
    __shared__ uint32_t s_bid[CT_GI][32];
    __shared__ uint32_t s_hit[CT_GI][MASK_WORDS];
    __shared__ uint32_t s_free[8][64];
    Dev *dev = g.dev;
    const uint32_t ngroups = dev->n_groups;
    const uint32_t lane = lane_id(), wp = threadIdx.x >> 5;
    const uint32_t C = g.C, IB = g.IB;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    FreeStage fs{s_free[wp], 0u};
    unsigned long long removed = 0;
    for (uint32_t gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        const uint2 grp = g.grp_items[gi];
        const uint32_t t = grp.x;
        const uint4 a = g.t_a[t];
        const uint4 b = g.t_b[t];
        const uint32_t m = a.x, aoff = a.y, item0 = a.w;
        const uint32_t deg = b.x, nb = b.y, root = b.z, ni = b.w;
        const uint32_t c = grp.y + wp;  // this warp's item of the source
        const bool have = wp < CT_GI && c < ni;
        const uint32_t kb = c * IB;
        const uint32_t nblk = have ? min(IB, nb - kb) : 0u;
        uint32_t bid = NIL;
        if (lane < nblk) bid = cbt_walk(g.links, P, root, kb + 1 + lane);
        const bool bad = __any_sync(FULL, lane < nblk && bid == NIL);
        if (bad && lane == 0) latch_status(dev, 5u /* GV_ERR_STATE */);
        const bool work = have && !bad;
        const uint32_t sbase = kb * C;
        const uint32_t nslots = work ? min(nblk * C, deg - sbase) : 0u;
        const uint32_t nquads = (nslots + 3) >> 2;
        if (wp < CT_GI) {
            s_bid[wp][lane] = bid;
            if (lane < MASK_WORDS) s_hit[wp][lane] = 0u;
        }
        for (uint32_t s0 = 0; s0 < m; s0 += CT_KEYS) {
            const uint32_t sm = min(CT_KEYS, m - s0);
            uint32_t hs = 64;
            while (hs < 2 * sm) hs <<= 1;
            const uint32_t nbk = hs / 4;
            __syncthreads();  // the previous slice's readers are done
            for (uint32_t j = threadIdx.x; j < hs; j += blockDim.x) {
                hk[j] = EMPTY_KEY;
                if (MODE == MODE_QUERY) hf[j] = 0;
            }
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < sm; j += blockDim.x) {
                const uint32_t v = g.arena[aoff + s0 + j];
                uint32_t h = 4 * hidx(v, nbk);
                // at most hs / 2 keys: a free or equal slot exists
                for (uint32_t step = 0; step < hs; ++step) {
                    const uint32_t old = atomicCAS(&hk[h], EMPTY_KEY, v);
                    if (old == EMPTY_KEY || old == v) break;
                    h = (h + 1) & (hs - 1);
                }
            }
            __syncthreads();
            for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
                const uint32_t q = q0 + lane;
                const uint32_t x = q << 2;
                uint32_t hit = 0;
                if (q < nquads) {
                    const uint32_t lb = divc(g.cmul, x);
                    const uint4 e4 = ld_stream4(reinterpret_cast<const uint4 *>(
                        g.data + (size_t)s_bid[wp][lb] * C + (x - lb * C)));
                    const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (x + j < nslots) {
                            const uint32_t h = ct_find(hk, nbk, e[j]);
                            if (h != NIL) {
                                hit |= 1u << j;
                                if (MODE == MODE_QUERY) hf[h] = 1;
                            }
                        }
                    }
                }
                uint32_t word = hit << (4u * (lane & 7u));
                word |= __shfl_xor_sync(FULL, word, 1);
                word |= __shfl_xor_sync(FULL, word, 2);
                word |= __shfl_xor_sync(FULL, word, 4);
                if ((lane & 7u) == 0 && word) s_hit[wp][(q0 >> 3) + (lane >> 3)] |= word;
            }
            if (MODE == MODE_QUERY) {
                __syncthreads();
                // every list entry of the slice (repeats included) reads its key's flag
                for (uint32_t j = threadIdx.x; j < sm; j += blockDim.x) {
                    const uint32_t h = ct_find(hk, nbk, g.arena[aoff + s0 + j]);
                    if (h != NIL && hf[h]) g.found[aoff + s0 + j] = 1u;
                }
            }
        }
        __syncwarp();
        if (MODE != MODE_QUERY && work) {
            if (ni == 1) {
                // stable in-place compaction of the single item: each round
                // reads its quads before any lane writes, and targets never
                // pass the slot being read
                uint32_t running = 0;
                for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
                    const uint32_t q = q0 + lane;
                    const uint32_t x = q << 2;
                    uint4 e4 = make_uint4(EMPTY_KEY, EMPTY_KEY, EMPTY_KEY, EMPTY_KEY);
                    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
                    size_t qoff = 0;
                    if (q < nquads) {
                        const uint32_t lb = divc(g.cmul, x);
                        qoff = (size_t)s_bid[wp][lb] * C + (x - lb * C);
                        e4 = ld_stream4(reinterpret_cast<const uint4 *>(g.data + qoff));
                        if (WEIGHTED) w4 = ld_stream4(reinterpret_cast<const uint4 *>(g.wdata + qoff));
                    }
                    const uint32_t hw = (s_hit[wp][(q0 >> 3) + (lane >> 3)] >> (4u * (lane & 7u))) & 0xFu;
                    uint32_t vmask = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (q < nquads && x + j < nslots) vmask |= 1u << j;
                    const uint32_t surv = vmask & ~hw;
                    uint32_t tot;
                    const uint32_t ex = warp_excl_scan(__popc(surv), &tot);
                    uint32_t wpos = running + ex;
                    const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
                    const uint32_t ew[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((surv >> j) & 1u) {
                            if (wpos != x + j) {
                                const uint32_t tq = divc(g.cmul, wpos);
                                const size_t to = (size_t)s_bid[wp][tq] * C + (wpos - tq * C);
                                g.data[to] = e[j];
                                if (WEIGHTED) g.wdata[to] = ew[j];
                            }
                            ++wpos;
                        }
                    }
                    running += tot;
                }
                const uint32_t degn = running;
                if (degn != deg) {
                    const uint32_t nbn = divc(g.cmul, degn + C - 1);
                    const uint32_t k = lane + 1;
                    const bool fr = lane < nblk && k > nbn;
                    fs.push(fr, bid, dev, g.queue, qbb, P);
                    const uint32_t p = k >> 1;
                    const uint32_t pb = __shfl_sync(FULL, bid, (p - 1) & 31u);
                    const uint32_t lastb = __shfl_sync(FULL, bid, (nbn - 1) & 31u);
                    if (fr && p >= 1 && p <= nbn) g.links[2ull * pb + (k & 1u)] = NIL;
                    if (lane == 0) {
                        g.sent[g.t_vid[t]] = make_uint4(degn, nbn, nbn ? root : NIL, nbn ? lastb : NIL);
                        removed += deg - degn;
                    }
                }
            } else {
                const uint32_t it = item0 + c;
                uint32_t cnt = 0;
                if (lane < MASK_WORDS) {
                    const uint32_t lo = lane * 32;
                    uint32_t valid = 0;
                    if (lo < nslots) valid = (nslots - lo >= 32) ? FULL : ((1u << (nslots - lo)) - 1u);
                    const uint32_t sv = valid & ~s_hit[wp][lane];
                    g.it_mask[(size_t)it * MASK_WORDS + lane] = sv;
                    cnt = __popc(sv);
                }
                cnt = warp_sum(cnt);
                if (lane < nblk) g.it_bid[(size_t)it * IB + lane] = bid;
                if (lane == 0) g.it_cnt[it] = cnt;
            }
        }
    }
    if (MODE != MODE_QUERY) {
        fs.flush(fs.n, dev, g.queue, qbb, P);
        if (lane == 0 && removed) atomicAdd(&dev->call_a, removed);
    }
}

// ---------------------------------------------------------------- launch

// Partition CTAs and their range for a batch of n pairs.
void group_shape(unsigned long long n, int num_sms, uint32_t *ctas, unsigned long long *len) {
    unsigned long long c = (n + 32767) / 32768;
    const unsigned long long cap = 2ull * (unsigned long long)num_sms;
    if (c < 1) c = 1;
    if (c > cap) c = cap;
    unsigned long long L = (n + c - 1) / c;
    L = (L + 1023) / 1024 * 1024;
    if (L == 0) L = 1024;
    *ctas = (uint32_t)((n + L - 1) / L);
    if (*ctas == 0) *ctas = 1;
    *len = L;
}

cudaError_t launch_group_hist(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                              unsigned long long n, unsigned long long lo, unsigned long long hi,
                              const LaunchCfg &lc) {
    if (hi <= lo) return cudaSuccess;
    const int ph = mode == MODE_INSERT ? PH_INS_PART : mode == MODE_DELETE ? PH_DEL_PART : PH_QRY_PART;
    PhaseScope ps(lc, ph);
    const uint32_t c0 = (uint32_t)(lo / g.gp_len);
    const uint32_t c1 = (uint32_t)((hi + g.gp_len - 1) / g.gp_len);
    if (mode == MODE_INSERT) launch_pdl(k_gp_hist<MODE_INSERT>, c1 - c0, GP_THREADS, 0, lc.stream, g, src, dst, n, c0);
    else if (mode == MODE_DELETE) launch_pdl(k_gp_hist<MODE_DELETE>, c1 - c0, GP_THREADS, 0, lc.stream, g, src, dst, n, c0);
    else launch_pdl(k_gp_hist<MODE_QUERY>, c1 - c0, GP_THREADS, 0, lc.stream, g, src, dst, n, c0);
    return cudaGetLastError();
}

static cudaError_t place_attr(void (*k)(GraphView), size_t smem) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_group_finish(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                const uint32_t *wts, unsigned long long n, const LaunchCfg &lc) {
    const bool ins = mode == MODE_INSERT, del = mode == MODE_DELETE;
    const int cap = lc.num_sms * GRID_MULT;
    {
        PhaseScope ps(lc, ins ? PH_INS_PART : del ? PH_DEL_PART : PH_QRY_PART);
        launch_pdl(k_gp_colscan, (g.gb_n + 31) / 32, 256, 0, lc.stream, g);
        launch_pdl(k_gp_bktscan, 1, 1024, 0, lc.stream, g);
        if (ins) {
            if (g.wdata) launch_pdl(k_gp_scatter<MODE_INSERT, true>, g.gp_ctas, GP_THREADS, 0, lc.stream, g, src, dst, wts, n);
            else launch_pdl(k_gp_scatter<MODE_INSERT, false>, g.gp_ctas, GP_THREADS, 0, lc.stream, g, src, dst, wts, n);
        } else if (del) {
            launch_pdl(k_gp_scatter<MODE_DELETE, false>, g.gp_ctas, GP_THREADS, 0, lc.stream, g, src, dst, wts, n);
        } else {
            launch_pdl(k_gp_scatter<MODE_QUERY, true>, g.gp_ctas, GP_THREADS, 0, lc.stream, g, src, dst, wts, n);
        }
    }
    {
        PhaseScope ps(lc, ins ? PH_INS_VCOUNT : del ? PH_DEL_VCOUNT : PH_QRY_VCOUNT);
        // chunks: at most n / GP_CHUNK full ones plus one partial per bucket
        const unsigned long long nch = n / GP_CHUNK + g.gb_n;
        launch_pdl(k_gp_count, grid_for(nch, 1, lc.num_sms * 4), GP_THREADS, 0, lc.stream, g);
        launch_pdl(k_gp_vscan, grid_for(g.vmask + 1ull, GP_VPC, cap), 1024, 0, lc.stream, g);
    }
    if (!ins) {
        // deletes and queries: the batch lists now; inserts place after the plan
        cudaError_t e = launch_group_place(mode, g, n, lc);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_group_place(int mode, const GraphView &g, unsigned long long n, const LaunchCfg &lc) {
    static bool attr_done[64] = {};
    int devc = 0;
    if (cudaGetDevice(&devc) != cudaSuccess || devc < 0 || devc >= 64) return cudaErrorInvalidDevice;
    const size_t maxsm = gp_place_smem(GP_WMAX);
    if (!attr_done[devc]) {
        cudaError_t e;
        if ((e = place_attr(k_gp_place<MODE_INSERT, false>, maxsm)) != cudaSuccess) return e;
        if ((e = place_attr(k_gp_place<MODE_INSERT, true>, maxsm)) != cudaSuccess) return e;
        if ((e = place_attr(k_gp_place<MODE_DELETE, false>, maxsm)) != cudaSuccess) return e;
        if ((e = place_attr(k_gp_place<MODE_QUERY, false>, maxsm)) != cudaSuccess) return e;
        attr_done[devc] = true;
    }
    const size_t smem = gp_place_smem(1u << g.gb_shift);
    const unsigned long long nch = n / GP_CHUNK + g.gb_n;
    const int grid = grid_for(nch, 1, lc.num_sms * 4);
    const int ph = mode == MODE_INSERT ? PH_INS_PLACE : mode == MODE_DELETE ? PH_DEL_PLACE : PH_QRY_PLACE;
    PhaseScope ps(lc, ph);
    if (mode == MODE_INSERT) {
        if (g.wdata) launch_pdl(k_gp_place<MODE_INSERT, true>, grid, GP_THREADS, smem, lc.stream, g);
        else launch_pdl(k_gp_place<MODE_INSERT, false>, grid, GP_THREADS, smem, lc.stream, g);
    } else if (mode == MODE_DELETE) {
        launch_pdl(k_gp_place<MODE_DELETE, false>, grid, GP_THREADS, smem, lc.stream, g);
    } else {
        launch_pdl(k_gp_place<MODE_QUERY, false>, grid, GP_THREADS, smem, lc.stream, g);
    }
    return cudaGetLastError();
}

cudaError_t launch_gp_plan_insert(const GraphView &g, int grid, const LaunchCfg &lc) {
    launch_pdl(k_gp_plan_insert, grid, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_gp_plan_member(int mode, const GraphView &g, int grid, const LaunchCfg &lc) {
    if (mode == MODE_DELETE) launch_pdl(k_gp_plan_member<MODE_DELETE>, grid, 256, 0, lc.stream, g);
    else launch_pdl(k_gp_plan_member<MODE_QUERY>, grid, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_mark_cta(int mode, const GraphView &g, unsigned long long nt, const LaunchCfg &lc) {
    // groups: at most the touched sources' items / CT_GI + one per source
    const int grid = grid_for(nt, 1, lc.num_sms * 4);
    const int ph = mode == MODE_DELETE ? PH_DEL_MARK_CTA : PH_QRY_MARK_CTA;
    PhaseScope ps(lc, ph);
    if (mode == MODE_DELETE) {
        if (g.wdata) launch_pdl(k_mark_cta<MODE_DELETE, true>, grid, 256, 0, lc.stream, g);
        else launch_pdl(k_mark_cta<MODE_DELETE, false>, grid, 256, 0, lc.stream, g);
    } else {
        launch_pdl(k_mark_cta<MODE_QUERY, false>, grid, 256, 0, lc.stream, g);
    }
    return cudaGetLastError();
}

}  // namespace gv

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
//   bktscan  one CTA: bucket bases, and the chunk list (every bucket cut into
//            chunks of at most GP_CHUNK pairs; buckets of several chunks get
//            a row of offsets per chunk).
//   scatter  each partition CTA sorts every tile of its range by bucket in
//            shared memory and writes it out bucket run by bucket run, from
//            cursors started at its prefixes: buckets become contiguous.
//   group    per chunk: a counting sort by vertex in shared memory.  A bucket
//            of one chunk is finished here: its vertices' counts, segment
//            starts (bucket base + prefix) and the touched list, and the
//            grouped pairs written out in one contiguous run.  A chunk of a
//            larger bucket adds its per-vertex counts to the vertices' totals
//            with one atomic per (chunk, vertex), whose return value is the
//            chunk's offset inside each vertex's segment (its row).
//   mscan    per bucket of several chunks: segment starts and touched list.
//   mplace   per chunk of such a bucket: the counting sort again, each run
//            written at its vertex's segment start plus the chunk's offset.
// Deletes and queries write the grouped destinations straight into the
// membership arena (the per-source batch lists; queries also record where
// each of their pairs landed); inserts write grouped pairs that the slot
// pass then stores at slot deg + rank of each source (Algorithm 1) after the
// plan and the links, runs of one source landing in consecutive slots.
#include "gv_launch.h"

namespace gv {

__device__ __forceinline__ bool gp_valid(const GraphView &g, uint32_t u, uint32_t v) {
    return u < g.nv && v < g.nv && (g.all_alive || (g.alive[u] && g.alive[v]));
}

// Exclusive scan of cnt[0, n) into out[] by the whole CTA (GP_THREADS
// threads, n a power of two <= 4 * GP_WMAX); all threads call, and every
// entry of out[] is visible to every thread on return.  Returns the total
// to every thread.
__device__ __forceinline__ uint32_t gp_scan_counts(const uint32_t *cnt, uint32_t *out, uint32_t n) {
    const uint32_t per = n > GP_THREADS ? n / GP_THREADS : 1u;
    const uint32_t first = threadIdx.x * per;
    uint32_t s = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (first + k < n) s += cnt[first + k];
    uint32_t tot;
    uint32_t e = block_excl_scan(s, &tot);
    for (uint32_t k = 0; k < per; ++k) {
        if (first + k < n) {
            out[first + k] = e;
            e += cnt[first + k];
        }
    }
    __syncthreads();
    return tot;
}

// ------------------------------------------------------------- partition

constexpr int GP_PER = GP_TILE / GP_THREADS;  // pairs per thread per tile
// Resident CTAs per SM the chunk kernels are compiled for (their occupancy
// is set by registers; overridable for tuning builds).
#ifndef GV_GP_MINB
#define GV_GP_MINB 4
#endif
constexpr int GP_MINB = GV_GP_MINB;

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
    for (unsigned long long i0 = beg + threadIdx.x; i0 < end; i0 += GP_TILE) {
        uint32_t u[GP_PER], v[GP_PER];
#pragma unroll
        for (int j = 0; j < GP_PER; ++j) {
            const unsigned long long i = i0 + (unsigned long long)j * GP_THREADS;
            u[j] = i < end ? ld_stream(src + i) : NIL;
            v[j] = i < end ? ld_stream(dst + i) : NIL;
        }
#pragma unroll
        for (int j = 0; j < GP_PER; ++j) {
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
// All G rows of the CTA's 32 buckets are loaded into shared memory at once
// (dynamic, G * 32 words); warp w then sums rows [w * G / 8, (w + 1) * G / 8).
__global__ void __launch_bounds__(256) k_gp_colscan(GraphView g) {
    pdl_wait();
    extern __shared__ uint32_t s_v[];  // [G][32]
    __shared__ uint32_t s_sum[8][32];
    const uint32_t nb = g.gb_n, G = g.gp_ctas;
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * 32 + lane;
    const bool ok = b < nb;
#pragma unroll 8
    for (uint32_t r = w; r < G; r += 8) s_v[r * 32 + lane] = ok ? g.gp_hist[(size_t)r * nb + b] : 0u;
    __syncthreads();
    const uint32_t r0 = G * w / 8, r1 = G * (w + 1) / 8;
    uint32_t sum = 0;
    for (uint32_t r = r0; r < r1; ++r) sum += s_v[r * 32 + lane];
    s_sum[w][lane] = sum;
    __syncthreads();
    uint32_t run = 0, total = 0;
    for (uint32_t k = 0; k < 8; ++k) {
        if (k < w) run += s_sum[k][lane];
        total += s_sum[k][lane];
    }
    for (uint32_t r = r0; r < r1; ++r) {
        const uint32_t x = s_v[r * 32 + lane];
        if (ok) g.gp_hist[(size_t)r * nb + b] = run;
        run += x;
    }
    if (w == 0 && ok) g.gp_btot[b] = total;
}

// One CTA of 1024 threads, four buckets each: bucket bases, the chunk list
// (chunks of a bucket of several chunks get consecutive rows), the list of
// such buckets, and the number of valid pairs.
__global__ void __launch_bounds__(1024) k_gp_bktscan(GraphView g) {
    pdl_wait();
    const uint32_t nb = g.gb_n;
    uint32_t tot[4], nch[4], st = 0, sc = 0, sr = 0, sm = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t b = threadIdx.x * 4 + j;
        tot[j] = b < nb ? g.gp_btot[b] : 0u;
        nch[j] = (tot[j] + GP_CHUNK - 1) / GP_CHUNK;
        st += tot[j];
        sc += nch[j];
        sr += nch[j] > 1 ? nch[j] : 0u;
        sm += nch[j] > 1 ? 1u : 0u;
    }
    uint32_t all_t, all_c, all_r, all_m;
    uint32_t et = block_excl_scan(st, &all_t);
    uint32_t ec = block_excl_scan(sc, &all_c);
    uint32_t er = block_excl_scan(sr, &all_r);
    uint32_t em = block_excl_scan(sm, &all_m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t b = threadIdx.x * 4 + j;
        if (b < nb) {
            const bool multi = nch[j] > 1;
            g.gp_bbase[b] = et;
            for (uint32_t k = 0; k < nch[j]; ++k)
                g.gp_chunks[ec + k] = make_uint4(et + k * GP_CHUNK, min(GP_CHUNK, tot[j] - k * GP_CHUNK), b,
                                                 multi ? er + k : NIL);
            if (multi) {
                g.gp_mbkt[em] = b;
                er += nch[j];
                ++em;
            }
        }
        et += tot[j];
        ec += nch[j];
    }
    if (threadIdx.x == 0) {
        g.dev->n_chunks = all_c;
        g.dev->n_mbuckets = all_m;
        g.dev->n_grouped = all_t;
    }
}

// Shared memory of k_gp_scatter for nb buckets: cursors, tile counts and
// tile offsets per bucket, and one tile of staged pairs (three words each).
__host__ __device__ constexpr size_t gp_scatter_smem(uint32_t nb) { return (size_t)(3 * nb + 3 * GP_TILE) * 4; }

// Valid pairs of each partition CTA to their buckets, one tile at a time:
// the tile is sorted by bucket in shared memory, then consecutive threads
// write consecutive positions of each bucket's run.  A query's original
// index (or an insert's payload) travels with its pair; an invalid query is
// answered 0 (no arena position).
template <int MODE, bool AUX>
__global__ void __launch_bounds__(GP_THREADS) k_gp_scatter(GraphView g, const uint32_t *__restrict__ src,
                                                           const uint32_t *__restrict__ dst,
                                                           const uint32_t *__restrict__ wts, unsigned long long n) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t psm[];
    const uint32_t nb = g.gb_n, sh = g.gb_shift;
    uint32_t *cur = psm;             // [nb] next position of each bucket for this CTA
    uint32_t *th = cur + nb;         // [nb] pairs of the tile per bucket
    uint32_t *to = th + nb;          // [nb] first staged position of each bucket
    uint32_t *ss = to + nb;          // [GP_TILE] staged sources
    uint32_t *sd = ss + GP_TILE;     // [GP_TILE] staged destinations
    uint32_t *sx = sd + GP_TILE;     // [GP_TILE] staged index / payload
    const uint32_t c = blockIdx.x;
    const uint32_t *row = g.gp_hist + (size_t)c * nb;
    for (uint32_t b = threadIdx.x; b < nb; b += GP_THREADS) {
        cur[b] = g.gp_bbase[b] + row[b];
        th[b] = 0;
    }
    __syncthreads();
    const unsigned long long beg = (unsigned long long)c * g.gp_len;
    const unsigned long long end = min(n, beg + g.gp_len);
    const uint32_t total = g.dev->n_grouped;  // every position written stays below it
    for (unsigned long long t0 = beg; t0 < end; t0 += GP_TILE) {
        uint32_t u[GP_PER], v[GP_PER], x[GP_PER], lr[GP_PER];
#pragma unroll
        for (int j = 0; j < GP_PER; ++j) {
            const unsigned long long i = t0 + threadIdx.x + (unsigned long long)j * GP_THREADS;
            u[j] = i < end ? ld_stream(src + i) : NIL;
            v[j] = i < end ? ld_stream(dst + i) : NIL;
            x[j] = 0u;
            if (AUX && i < end) x[j] = MODE == MODE_QUERY ? (uint32_t)i : (wts ? ld_stream(wts + i) : 0u);
        }
#pragma unroll
        for (int j = 0; j < GP_PER; ++j) {
            const unsigned long long i = t0 + threadIdx.x + (unsigned long long)j * GP_THREADS;
            lr[j] = NIL;
            if (i < end) {
                if (gp_valid(g, u[j], v[j])) lr[j] = atomicAdd(&th[u[j] >> sh], 1u);
                else if (MODE == MODE_QUERY) g.qpos[i] = NIL;
            }
        }
        __syncthreads();
        const uint32_t tv = gp_scan_counts(th, to, nb);
#pragma unroll
        for (int j = 0; j < GP_PER; ++j) {
            if (lr[j] != NIL) {
                const uint32_t p = to[u[j] >> sh] + lr[j];
                if (p < GP_TILE) {
                    ss[p] = u[j];
                    sd[p] = v[j];
                    if (AUX) sx[p] = x[j];
                }
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < tv && j < GP_TILE; j += GP_THREADS) {
            const uint32_t uu = ss[j], b = uu >> sh;
            const uint32_t pos = b < nb ? cur[b] + (j - to[b]) : NIL;
            if (pos < total) {
                g.gp_src[pos] = uu;
                g.gp_dst[pos] = sd[j];
                if (AUX) g.gp_aux[pos] = sx[j];
            } else {
                latch_status(g.dev, 5u /* GV_ERR_STATE */);
            }
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nb; b += GP_THREADS) {
            cur[b] += th[b];
            th[b] = 0;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ grouping by vertex

// Shared memory of the chunk kernels for W vertices per bucket: three words
// per vertex (count, run start, segment offset) and one chunk of staged
// pairs (three words each).
__host__ __device__ constexpr size_t gp_chunk_smem(uint32_t W) { return (size_t)(3 * W + 3 * GP_CHUNK) * 4; }

// One grouped pair out: inserts keep (source, destination, payload) for the
// slot pass; deletes and queries write the destination into the arena (the
// source's batch list), queries also the arena position of their pair.
template <int MODE, bool AUX>
__device__ __forceinline__ void gp_emit(const GraphView &g, uint32_t pos, uint32_t u, uint32_t v, uint32_t x) {
    if (MODE == MODE_INSERT) {
        g.go_src[pos] = u;
        g.go_dst[pos] = v;
        if (AUX) g.go_aux[pos] = x;
    } else {
        g.arena[pos] = v;
        if (MODE == MODE_QUERY) {
            g.found[pos] = 0u;
            g.qpos[x] = pos;
        }
    }
}

// Touched vertices of one bucket (hist[w] > 0 for w < W): each gets its count
// and segment start (base + off[w]), and joins the touched list.  All threads
// call.
__device__ __forceinline__ void gp_list_touched(const GraphView &g, const uint32_t *hist, const uint32_t *off,
                                                uint32_t W, uint32_t vb, uint32_t base, uint32_t *s_t) {
    const uint32_t per = W > GP_THREADS ? W / GP_THREADS : 1u;
    const uint32_t first = threadIdx.x * per;
    uint32_t f = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (first + k < W && hist[first + k]) ++f;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(f, &tot);
    if (threadIdx.x == 0) *s_t = tot ? atomicAdd(&g.dev->n_touched, tot) : 0u;
    __syncthreads();
    uint32_t t = *s_t + ex;
    for (uint32_t k = 0; k < per; ++k) {
        const uint32_t w = first + k;
        if (w < W && hist[w]) {
            const uint32_t u = vb + w;
            g.vcnt[u] = hist[w];
            g.gcur[u] = base + off[w];
            g.t_vid[t++] = u;
        }
    }
}

// Per chunk: a counting sort by vertex in shared memory.  The chunk of a
// bucket that has only this chunk is grouped here (in order of vertices:
// its run of the partitioned order becomes the bucket's grouped run); a
// chunk of a larger bucket adds its counts to the vertices' totals, one
// atomic per (chunk, vertex), and keeps the returned offsets in its row.
template <int MODE, bool AUX>
__global__ void __launch_bounds__(GP_THREADS, GP_MINB) k_gp_group(GraphView g) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t csm[];
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    uint32_t *hist = csm;            // [W]
    uint32_t *loff = hist + W;       // [W] run start inside the chunk
    uint32_t *sv = loff + 2 * W;     // [GP_CHUNK] destinations in run order
    uint32_t *sw = sv + GP_CHUNK;    // [GP_CHUNK] vertex within the bucket
    uint32_t *sx = sw + GP_CHUNK;    // [GP_CHUNK] index / payload
    __shared__ uint32_t s_t;
    constexpr int PER = GP_CHUNK / GP_THREADS;
    const uint32_t nch = g.dev->n_chunks;
    const uint32_t total = g.dev->n_grouped;
    for (uint32_t k = blockIdx.x; k < nch; k += gridDim.x) {
        const uint4 ck = g.gp_chunks[k];  // {start, length, bucket, row or NIL}
        const bool single = ck.w == NIL;
        const uint32_t vb = ck.z << sh;
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS) hist[w] = 0;
        __syncthreads();
        uint32_t wv[PER], vv[PER], xv[PER], lr[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t j = threadIdx.x + e * GP_THREADS;
            if (j < ck.y) {
                wv[e] = ld_stream(g.gp_src + ck.x + j) & (W - 1);
                if (single) {
                    vv[e] = ld_stream(g.gp_dst + ck.x + j);
                    xv[e] = AUX ? ld_stream(g.gp_aux + ck.x + j) : 0u;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < PER; ++e)
            if (threadIdx.x + e * GP_THREADS < ck.y) lr[e] = atomicAdd(&hist[wv[e]], 1u);
        __syncthreads();
        if (single) {
            gp_scan_counts(hist, loff, W);
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                if (threadIdx.x + e * GP_THREADS < ck.y) {
                    const uint32_t p = loff[wv[e]] + lr[e];
                    if (p < GP_CHUNK) {
                        sv[p] = vv[e];
                        sw[p] = wv[e];
                        if (AUX) sx[p] = xv[e];
                    }
                }
            }
            gp_list_touched(g, hist, loff, W, vb, ck.x, &s_t);  // its barriers publish the staging
            for (uint32_t j = threadIdx.x; j < ck.y; j += GP_THREADS) {
                if (ck.x + j < total && sw[j] < W) gp_emit<MODE, AUX>(g, ck.x + j, vb + sw[j], sv[j], AUX ? sx[j] : 0u);
                else latch_status(g.dev, 5u /* GV_ERR_STATE */);
            }
        } else {
            uint32_t *row = g.gp_rows + (size_t)ck.w * W;
            for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS)
                if (hist[w]) row[w] = atomicAdd(&g.vcnt[vb + w], hist[w]);
        }
        __syncthreads();
    }
}

// Per bucket of several chunks (after all its chunks are counted): segment
// starts = bucket base + exclusive prefix of the vertices' totals, and the
// touched list.
// Deletes and queries (HASH): a vertex past CT_KEYS batch entries (only a
// bucket of several chunks holds one) also gets a bucketed hash set of
// member_words(count) words in the arena's hash region, whose offset goes to
// vinfo[u].x; the placement fills it.
template <bool HASH>
__global__ void __launch_bounds__(GP_THREADS) k_gp_mscan(GraphView g) {
    pdl_wait();
    __shared__ uint32_t s_cnt[GP_WMAX];
    __shared__ uint32_t s_off[GP_WMAX];
    __shared__ uint32_t s_t;
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    const uint32_t nm = g.dev->n_mbuckets;
    for (uint32_t i = blockIdx.x; i < nm; i += gridDim.x) {
        const uint32_t b = g.gp_mbkt[i];
        const uint32_t vb = b << sh;
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS) {
            const uint32_t c = g.vcnt[vb + w];
            s_cnt[w] = c;
            if (HASH && c > CT_KEYS) {
                const uint32_t hw = member_words(c);
                const unsigned long long off = atomicAdd(&g.dev->harena_used, (unsigned long long)hw);
                g.vinfo[vb + w].x = (uint32_t)(g.hbase + off);
            }
        }
        __syncthreads();
        gp_scan_counts(s_cnt, s_off, W);
        gp_list_touched(g, s_cnt, s_off, W, vb, g.gp_bbase[b], &s_t);
        __syncthreads();
    }
}

// The arena's hash region (as allocated by k_gp_mscan) to EMPTY; queries
// also clear its hit flags.
template <int MODE>
__global__ void __launch_bounds__(256) k_gp_hash_init(GraphView g) {
    pdl_wait();
    const unsigned long long hused = g.dev->harena_used;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < hused;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        g.arena[g.hbase + k] = EMPTY_KEY;
        if (MODE == MODE_QUERY) g.found[g.hbase + k] = 0u;
    }
}

// Per chunk of a bucket of several chunks: the counting sort again, and each
// vertex's run written at its segment start plus the chunk's offset.
template <int MODE, bool AUX>
__global__ void __launch_bounds__(GP_THREADS, GP_MINB) k_gp_mplace(GraphView g) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t csm[];
    const uint32_t sh = g.gb_shift, W = 1u << sh;
    uint32_t *hist = csm;            // [W]
    uint32_t *loff = hist + W;       // [W] run start inside the chunk
    uint32_t *rbase = loff + W;      // [W] run start in the grouped order
    uint32_t *sv = rbase + W;        // [GP_CHUNK]
    uint32_t *sw = sv + GP_CHUNK;    // [GP_CHUNK]
    uint32_t *sx = sw + GP_CHUNK;    // [GP_CHUNK]
    constexpr int PER = GP_CHUNK / GP_THREADS;
    const uint32_t nch = g.dev->n_chunks;
    const uint32_t total = g.dev->n_grouped;
    for (uint32_t k = blockIdx.x; k < nch; k += gridDim.x) {
        const uint4 ck = g.gp_chunks[k];
        if (ck.w == NIL) continue;  // grouped by k_gp_group (block-uniform)
        const uint32_t vb = ck.z << sh;
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
        const uint32_t *row = g.gp_rows + (size_t)ck.w * W;
        for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS)
            if (hist[w]) rbase[w] = g.gcur[vb + w] + row[w];
        __syncthreads();
        // deletes and queries: hist[w] becomes the vertex's hash-set offset
        // (NIL when its batch keys stay a plain list)
        if (MODE != MODE_INSERT)
            for (uint32_t w = threadIdx.x; w < W; w += GP_THREADS)
                hist[w] = (hist[w] && g.vcnt[vb + w] > CT_KEYS) ? g.vinfo[vb + w].x : NIL;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            if (threadIdx.x + e * GP_THREADS < ck.y) {
                const uint32_t p = loff[wv[e]] + lr[e];
                if (p < GP_CHUNK) {
                    sv[p] = vv[e];
                    sw[p] = wv[e];
                    if (AUX) sx[p] = xv[e];
                }
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < ck.y; j += GP_THREADS) {
            const uint32_t w = sw[j];
            const uint32_t pos = w < W ? rbase[w] + (j - loff[w]) : NIL;
            if (pos < total) gp_emit<MODE, AUX>(g, pos, vb + w, sv[j], AUX ? sx[j] : 0u);
            else latch_status(g.dev, 5u /* GV_ERR_STATE */);
            if (MODE != MODE_INSERT && w < W && hist[w] != NIL) {
                const uint32_t nbk = member_words(g.vcnt[vb + w]) / HB;
                if (bucket_insert(g.arena + hist[w], nbk, sv[j]) == NIL) latch_status(g.dev, 5u /* GV_ERR_STATE */);
            }
        }
        __syncthreads();
    }
}

// Insert slot pass over the grouped pairs: pair i of source u has rank
// i - (segment start of u) and goes to slot deg(u) + rank (Algorithm 1): the
// free slots of the last block first, then the blocks popped for u.
template <bool WEIGHTED>
__global__ void __launch_bounds__(256) k_gp_slots(GraphView g) {
    pdl_wait();
    if (g.dev->abort) return;
    const uint32_t total = g.dev->n_grouped;
    const uint32_t C = g.C;
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(g.dev->q_front, P);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t u = ld_stream(g.go_src + i);
        const uint32_t v = ld_stream(g.go_dst + i);
        if (u > g.vmask) {
            latch_status(g.dev, 5u /* GV_ERR_STATE */);
            continue;
        }
        const uint4 vi = g.vinfo[u];  // {deg, last block, queue offset, segment start}
        const uint32_t r = i - vi.w;
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
            const unsigned long long qo = (unsigned long long)vi.z + jb;
            blk = qo < P ? g.queue[ring(qbase, qo, P)] : NIL;
        }
        if (blk < P && ln < C) {
            const size_t slot = (size_t)blk * C + ln;
            g.data[slot] = v;
            if (WEIGHTED) g.wdata[slot] = ld_stream(g.go_aux + i);
        } else {
            latch_status(g.dev, 5u /* GV_ERR_STATE */);
        }
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

// Per touched source (after the grouping: its batch list is arena[gcur,
// gcur + m)): the thread-per-source tier for tiny adjacencies, else work
// items of IB blocks for the warp tier (up to LIST_MAX batch entries, kept
// as the list), the block-wide tier (up to CT_KEYS batch entries: one shared
// hash set per group of CT_GI items) or, past CT_KEYS, the warp tier over the
// bucketed hash set in the arena's hash region that the grouping filled
// (such sources are also listed from the top of grp_items).
template <int MODE>
__global__ void __launch_bounds__(256) k_gp_plan_member(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t IB = g.IB;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    __shared__ uint32_t s_ai, s_am, s_at, s_ath, s_ag, s_ah;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t m = 0, aoff = 0, ni = 0, tiny = 0, ng = 0, hw = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            m = g.vcnt[u];
            aoff = g.gcur[u];
            s = g.sent[u];
            if (s.y > 0) {
                const bool small = MODE == MODE_QUERY
                    ? (s.x <= min(TINY_DEG_Q, TINY_NB_Q * g.C) && s.y <= TINY_NB_Q && m <= TINY_M)
                    : (s.x <= tiny_deg && s.y <= TINY_NB && m <= TINY_M);
                if (small) {
                    tiny = 1;
                } else {
                    ni = (s.y + IB - 1) / IB;
                    if (m > CT_KEYS) hw = member_words(m);
                    else if (m > LIST_MAX) ng = (ni + CT_GI - 1) / CT_GI;
                }
            }
        }
        const uint32_t tlo = tiny && s.x <= TINY_SPLIT, thi = tiny && s.x > TINY_SPLIT;
        uint32_t ttot, tthi, gtot, htot;
        const uint32_t tex = block_excl_scan(tlo, &ttot);
        const uint32_t thx = block_excl_scan(thi, &tthi);
        const uint32_t gex = block_excl_scan(ng, &gtot);
        const uint32_t hex = block_excl_scan(hw ? 1u : 0u, &htot);
        if (threadIdx.x == 0) {
            s_at = ttot ? atomicAdd(&g.dev->n_tiny, ttot) : 0u;
            s_ath = tthi ? atomicAdd(&g.dev->n_tiny_hi, tthi) : 0u;
            s_ag = gtot ? atomicAdd(&g.dev->n_groups, gtot) : 0u;
            s_ah = htot ? atomicAdd(&g.dev->n_hash, htot) : 0u;
        }
        const uint32_t item0 = alloc_items(g, ni, &s_ai, &s_am);
        if (t < nt) {
            // a hash set (placed by the grouping, vinfo[u].x) or the list
            const uint32_t at = hw ? g.vinfo[g.t_vid[t]].x : aoff;
            g.t_a[t] = make_uint4(m, at, hw ? hw : (ng ? CT_FLAG : 0u), item0);
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            if (tlo) g.t_tiny[s_at + tex] = t;
            if (thi) g.t_tiny[g.tiny_cap - 1 - (s_ath + thx)] = t;
            emit_items(g, t, item0, ni);
            for (uint32_t k = 0; k < ng; ++k) g.grp_items[s_ag + gex + k] = make_uint2(t, k * CT_GI);
            if (hw) g.grp_items[g.grp_cap - 1 - (s_ah + hex)] = make_uint2(t, 0u);
        }
        __syncthreads();
    }
}

// Queries, after the marks: every list entry of a hash-set source takes the
// hit flag of its key's slot.
__global__ void __launch_bounds__(256) k_gp_hash_found(GraphView g) {
    pdl_wait();
    const uint32_t nh = g.dev->n_hash;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = warp; k < nh; k += nwarps) {
        const uint32_t t = g.grp_items[g.grp_cap - 1 - k].x;
        const uint4 a = g.t_a[t];
        const uint32_t seg = g.gcur[g.t_vid[t]];
        const uint32_t *tab = g.arena + a.y;
        const uint32_t nbk = a.z / HB;
        for (uint32_t j = lane; j < a.x; j += 32) {
            const uint32_t h = bucket_find(tab, nbk, g.arena[seg + j]);
            if (h != NIL && g.found[a.y + h]) g.found[seg + j] = 1u;
        }
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
__global__ void __launch_bounds__(32 * CT_GI, 4) k_mark_cta(GraphView g) {
    pdl_wait();
    __shared__ __align__(16) uint32_t hk[CT_SLOTS];
    __shared__ uint8_t hf[MODE == MODE_QUERY ? CT_SLOTS : 4];
    __shared__ uint32_t s_bid[CT_GI][32];
    __shared__ uint32_t s_hit[CT_GI][MASK_WORDS];
    __shared__ uint32_t s_free[CT_GI][64];
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
        __syncwarp();
        // every entry of the item (at most 4 quads per lane) and, for a
        // single-item delete on a weighted graph, every payload: loaded now,
        // in flight while the batch set is built, and all read before any
        // compaction write
        uint4 E[4], Wq[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t q = r * 32 + lane;
            E[r] = make_uint4(EMPTY_KEY, EMPTY_KEY, EMPTY_KEY, EMPTY_KEY);
            Wq[r] = make_uint4(0u, 0u, 0u, 0u);
            if (q < nquads) {
                const uint32_t x = q << 2;
                const uint32_t lb = divc(g.cmul, x);
                const size_t qoff = (size_t)s_bid[wp][lb] * C + (x - lb * C);
                E[r] = ld_stream4(reinterpret_cast<const uint4 *>(g.data + qoff));
                if (WEIGHTED && MODE != MODE_QUERY && ni == 1)
                    Wq[r] = ld_stream4(reinterpret_cast<const uint4 *>(g.wdata + qoff));
            }
        }
        // the source's batch list (planned at most CT_KEYS keys) into the
        // shared hash set
        if (m > CT_KEYS && threadIdx.x == 0) latch_status(dev, 5u /* GV_ERR_STATE */);
        const uint32_t sm = min(CT_KEYS, m);
        uint32_t hs = 64;
        while (hs < 2 * sm) hs <<= 1;
        const uint32_t nbk = hs / 4;
        __syncthreads();  // the previous group's readers are done
        for (uint32_t j = threadIdx.x; j < hs; j += blockDim.x) {
            hk[j] = EMPTY_KEY;
            if (MODE == MODE_QUERY) hf[j] = 0;
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < sm; j += blockDim.x) {
            const uint32_t v = g.arena[aoff + j];
            uint32_t h = 4 * hidx(v, nbk);
            // at most hs / 2 keys: a free or equal slot exists
            for (uint32_t step = 0; step < hs; ++step) {
                const uint32_t old = atomicCAS(&hk[h], EMPTY_KEY, v);
                if (old == EMPTY_KEY || old == v) break;
                h = (h + 1) & (hs - 1);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t q0 = (uint32_t)r * 32;
            if (q0 >= nquads) break;
            const uint32_t q = q0 + lane;
            const uint32_t x = q << 2;
            uint32_t hit = 0;
            if (q < nquads) {
                const uint32_t e[4] = {E[r].x, E[r].y, E[r].z, E[r].w};
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
            // every list entry (repeats included) reads its key's flag
            for (uint32_t j = threadIdx.x; j < sm; j += blockDim.x) {
                const uint32_t h = ct_find(hk, nbk, g.arena[aoff + j]);
                if (h != NIL && hf[h]) g.found[aoff + j] = 1u;
            }
        }
        __syncwarp();
        if (MODE != MODE_QUERY && work) {
            if (ni == 1) {
                // stable in-place compaction of the single item (all of its
                // entries were read above)
                uint32_t running = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t q0 = (uint32_t)r * 32;
                    if (q0 >= nquads) break;
                    const uint32_t q = q0 + lane;
                    const uint32_t x = q << 2;
                    const uint32_t hw = (s_hit[wp][(q0 >> 3) + (lane >> 3)] >> (4u * (lane & 7u))) & 0xFu;
                    uint32_t vmask = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (q < nquads && x + j < nslots) vmask |= 1u << j;
                    const uint32_t surv = vmask & ~hw;
                    uint32_t tot;
                    const uint32_t ex = warp_excl_scan(__popc(surv), &tot);
                    uint32_t wpos = running + ex;
                    const uint32_t e[4] = {E[r].x, E[r].y, E[r].z, E[r].w};
                    const uint32_t ew[4] = {Wq[r].x, Wq[r].y, Wq[r].z, Wq[r].w};
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

// Partition CTAs and their range (a multiple of the tile) for n pairs.
void group_shape(unsigned long long n, int num_sms, uint32_t *ctas, unsigned long long *len) {
    unsigned long long c = (n + 16383) / 16384;
    unsigned long long cap = 3ull * (unsigned long long)num_sms;  // resident partition CTAs per SM
    if (cap > GP_MAXCTAS) cap = GP_MAXCTAS;
    if (c < 1) c = 1;
    if (c > cap) c = cap;
    unsigned long long L = (n + c - 1) / c;
    L = (L + GP_TILE - 1) / GP_TILE * GP_TILE;
    if (L == 0) L = GP_TILE;
    *ctas = (uint32_t)((n + L - 1) / L);
    if (*ctas == 0) *ctas = 1;
    *len = L;
}

// log2 of the vertices per bucket for n pairs over a dictionary of vcap
// vertices (a power of two): about GP_CHUNK pairs per bucket, at most
// GP_BMAX buckets and GP_WMAX vertices per bucket.
uint32_t group_bucket_shift(unsigned long long n, uint32_t vcap) {
    unsigned long long nb = 1;
    while (nb * 2 <= n / GP_CHUNK && nb * 2 <= GP_BMAX) nb *= 2;
    while (nb < GP_BMAX && (unsigned long long)vcap / nb > GP_WMAX) nb *= 2;
    if (nb > vcap) nb = vcap ? vcap : 1;
    uint32_t sh = 0;
    while (((unsigned long long)vcap >> sh) > nb) ++sh;
    return sh;
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

// Dynamic shared-memory opt-in, and the largest shared-memory carveout (the
// kernels' occupancy is set by their shared memory).
template <typename K>
static cudaError_t smem_attr(K k, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// Dynamic shared-memory opt-in of the grouping kernels (once per device).
static cudaError_t group_attrs() {
    static bool done[64] = {};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return cudaErrorInvalidDevice;
    if (done[d]) return cudaSuccess;
    const size_t ps = gp_scatter_smem(GP_BMAX), cs = gp_chunk_smem(GP_WMAX);
    cudaError_t e;
    if ((e = smem_attr(k_gp_colscan, (size_t)GP_MAXCTAS * 32 * 4)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_scatter<MODE_INSERT, false>, ps)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_scatter<MODE_INSERT, true>, ps)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_scatter<MODE_DELETE, false>, ps)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_scatter<MODE_QUERY, true>, ps)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_group<MODE_INSERT, false>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_group<MODE_INSERT, true>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_group<MODE_DELETE, false>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_group<MODE_QUERY, true>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_mplace<MODE_INSERT, false>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_mplace<MODE_INSERT, true>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_mplace<MODE_DELETE, false>, cs)) != cudaSuccess) return e;
    if ((e = smem_attr(k_gp_mplace<MODE_QUERY, true>, cs)) != cudaSuccess) return e;
    done[d] = true;
    return cudaSuccess;
}

template <int MODE, bool AUX>
static void group_rest(const GraphView &g, const uint32_t *src, const uint32_t *dst, const uint32_t *wts,
                       unsigned long long n, const LaunchCfg &lc, int ph_part, int ph_vc) {
    const size_t ps = gp_scatter_smem(g.gb_n), cs = gp_chunk_smem(1u << g.gb_shift);
    // chunks: at most n / GP_CHUNK full ones plus one partial per bucket
    const int gc = grid_for(n / GP_CHUNK + g.gb_n, 1, lc.num_sms * 4);
    {
        PhaseScope p(lc, ph_part);
        launch_pdl(k_gp_colscan, (g.gb_n + 31) / 32, 256, (size_t)g.gp_ctas * 32 * 4, lc.stream, g);
        launch_pdl(k_gp_bktscan, 1, 1024, 0, lc.stream, g);
        launch_pdl(k_gp_scatter<MODE, AUX>, g.gp_ctas, GP_THREADS, ps, lc.stream, g, src, dst, wts, n);
    }
    PhaseScope p(lc, ph_vc);
    constexpr bool HASH = MODE != MODE_INSERT;
    launch_pdl(k_gp_group<MODE, AUX>, gc, GP_THREADS, cs, lc.stream, g);
    launch_pdl(k_gp_mscan<HASH>, grid_for(g.gb_n, 1, lc.num_sms * 4), GP_THREADS, 0, lc.stream, g);
    if (HASH) launch_pdl(k_gp_hash_init<MODE>, grid_for(4 * n + 64, 256, lc.num_sms * GRID_MULT), 256, 0, lc.stream, g);
    launch_pdl(k_gp_mplace<MODE, AUX>, gc, GP_THREADS, cs, lc.stream, g);
}

cudaError_t launch_group_finish(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                const uint32_t *wts, unsigned long long n, const LaunchCfg &lc) {
    cudaError_t e = group_attrs();
    if (e != cudaSuccess) return e;
    if (mode == MODE_INSERT) {
        if (g.wdata) group_rest<MODE_INSERT, true>(g, src, dst, wts, n, lc, PH_INS_PART, PH_INS_GROUP);
        else group_rest<MODE_INSERT, false>(g, src, dst, wts, n, lc, PH_INS_PART, PH_INS_GROUP);
    } else if (mode == MODE_DELETE) {
        group_rest<MODE_DELETE, false>(g, src, dst, wts, n, lc, PH_DEL_PART, PH_DEL_GROUP);
    } else {
        group_rest<MODE_QUERY, true>(g, src, dst, wts, n, lc, PH_QRY_PART, PH_QRY_GROUP);
    }
    return cudaGetLastError();
}

cudaError_t launch_group_place(int mode, const GraphView &g, unsigned long long n, const LaunchCfg &lc) {
    if (mode != MODE_INSERT) return cudaErrorInvalidValue;
    PhaseScope ps(lc, PH_INS_SLOTS);
    const int grid = grid_for(n, 256 * 4, lc.num_sms * GRID_MULT);
    if (g.wdata) launch_pdl(k_gp_slots<true>, grid, 256, 0, lc.stream, g);
    else launch_pdl(k_gp_slots<false>, grid, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_gp_plan_insert(const GraphView &g, int grid, const LaunchCfg &lc) {
    launch_pdl(k_gp_plan_insert, grid, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_gp_hash_found(const GraphView &g, const LaunchCfg &lc) {
    launch_pdl(k_gp_hash_found, lc.num_sms * 4, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_gp_plan_member(int mode, const GraphView &g, int grid, const LaunchCfg &lc) {
    if (mode == MODE_DELETE) launch_pdl(k_gp_plan_member<MODE_DELETE>, grid, 256, 0, lc.stream, g);
    else launch_pdl(k_gp_plan_member<MODE_QUERY>, grid, 256, 0, lc.stream, g);
    return cudaGetLastError();
}

cudaError_t launch_mark_cta(int mode, const GraphView &g, unsigned long long nt, const LaunchCfg &lc) {
    // groups: at most the touched sources' items / CT_GI + one per source
    const int grid = grid_for(nt, 1, lc.num_sms * 6);
    static bool done[64] = {};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return cudaErrorInvalidDevice;
    if (!done[d]) {
        const int co = (int)cudaSharedmemCarveoutMaxShared;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_mark_cta<MODE_DELETE, true>, cudaFuncAttributePreferredSharedMemoryCarveout, co)) !=
            cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_mark_cta<MODE_DELETE, false>, cudaFuncAttributePreferredSharedMemoryCarveout, co)) !=
            cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_mark_cta<MODE_QUERY, false>, cudaFuncAttributePreferredSharedMemoryCarveout, co)) !=
            cudaSuccess) return e;
        done[d] = true;
    }
    const int ph = mode == MODE_DELETE ? PH_DEL_MARK_CTA : PH_QRY_MARK_CTA;
    PhaseScope ps(lc, ph);
    constexpr int T = 32 * CT_GI;
    if (mode == MODE_DELETE) {
        if (g.wdata) launch_pdl(k_mark_cta<MODE_DELETE, true>, grid, T, 0, lc.stream, g);
        else launch_pdl(k_mark_cta<MODE_DELETE, false>, grid, T, 0, lc.stream, g);
    } else {
        launch_pdl(k_mark_cta<MODE_QUERY, false>, grid, T, 0, lc.stream, g);
    }
    return cudaGetLastError();
}

}  // namespace gv

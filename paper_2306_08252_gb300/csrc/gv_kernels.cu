// gv_kernels.cu -- the GraphVine batch kernels for sm_103a.
//
// Every batch operation (insert, delete, query) starts by grouping the batch
// by source vertex on the device.  The paper converts each batch to CSR on
// the host before copying it over ("Initialization and batch updates"); here
// a counting pass gives every valid pair its rank among its source's pairs:
// large batches take one atomic per pair on the source's counter (its return
// value is the rank) and list the touched sources afterwards by a scan of the
// counters; small batches aggregate each tile in a shared-memory table first
// (one atomic per (tile, source)) and list touched sources on the fly.  The
// touched list plays the role of the CSR row list; per-vertex counters are
// indexed through a bijective scramble of the id (see vslot).
//
// Insert (Algorithm 1) then runs per touched source:
//   plan    block demand need(u) = ceil(max(0, cnt - space) / C) with
//           space = nblocks * C - deg (the free slots of the last block), and a
//           block-wide exclusive scan of the demand giving each source its
//           range of edge-queue slots (Figure 3: ranges from a prefix sum,
//           not per-block atomics); one atomicAdd per CTA places the CTA's
//           range.
//   link    one thread per popped block: the block's heap index
//           k = nblocks + 1 + j hangs under heap index k/2 on side k&1 (the
//           bit-string rule, Figure 4); an old parent is found by walking the
//           tree from the root along the bits of k/2.
//   scatter pair of rank r: r < space goes to the last block at slot
//           deg mod C + r, the rest to new block (r - space) / C, slot
//           (r - space) mod C; no atomics.
//   final   sentinels updated; the queue front advances by the blocks popped.
//
// Delete (Algorithm 2) and query (Algorithm 3) share one membership pipeline:
//   plan    per touched source: its batch destinations go to a list (<= 256
//           entries) or a bucketed hash set in an arena; small adjacencies
//           (a few blocks, <= 16 batch entries) go to the thread-per-source
//           tier, the others are cut into work items of IB blocks
//           (IB * C <= 512 slots).
//   scatter batch destinations into the lists (plain store at the rank) or
//           the hash sets (CAS into the first empty slot of the home bucket).
//   mark    one warp per item: resolve the item's block ids by walking the
//           CBT, stream the entries with 16-byte loads (the next round's in
//           flight while a round is tested), test membership (a
//           per-warp shared hash set built from the list, or the arena hash
//           set).  Query sets hit flags.  Delete compacts single-item
//           adjacencies in place (stable) and frees their emptied tail blocks;
//           multi-item adjacencies record a survivor bitmask per item.  The
//           thread-per-source tier does the same for small adjacencies, with
//           the batch entries in registers, on a second stream.
//   vscan   per multi-item source: new degree = survivors; per item the
//           number of holes below the new degree and of survivors at or above
//           it, prefix-summed over the source's items.
//   move    per multi-item item: the g-th hole below the new degree takes the
//           g-th survivor at or above it (sources and targets never overlap,
//           so items run independently); blocks past ceil(deg'/C) return to
//           the queue and their parents' links are cleared.
//   final   counters, queue back pointer, scratch reset.
// Compaction keeps every adjacency's blocks but the last full, so
// nblocks = ceil(deg / C) always holds and the next insert starts at slot deg.
#include "gv_launch.h"

namespace gv {

__device__ __forceinline__ bool valid_pair(const GraphView &g, uint32_t u, uint32_t v) {
    return u < g.nv && v < g.nv && g.alive[u] && g.alive[v];
}

// Insert source u into the tile's shared hash table; returns the slot and the
// pair's rank among this tile's pairs of u.
__device__ __forceinline__ uint32_t agg_insert(uint32_t *keys, uint32_t *cnt, uint32_t u,
                                               uint32_t &rank) {
    uint32_t h = mix32(u) & (AGG_H - 1);
    for (;;) {
        uint32_t k = keys[h];
        if (k == u) break;
        if (k == EMPTY_KEY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY_KEY, u);
            if (old == EMPTY_KEY || old == u) break;
        }
        h = (h + 1) & (AGG_H - 1);
    }
    rank = atomicAdd(&cnt[h], 1u);
    return h;
}

// ---------------------------------------------------------------- grouping

// Loads one tile's pairs and their validity with every global load issued
// before any of them is consumed (memory-level parallelism).  Pair e of this
// thread is pair base + e * AGG_THREADS + threadIdx.x.
__device__ __forceinline__ void load_tile(const GraphView &g, const uint32_t *__restrict__ src,
                                          const uint32_t *__restrict__ dst, unsigned long long n,
                                          unsigned long long base, uint32_t (&us)[AGG_EPT],
                                          uint32_t (&vs)[AGG_EPT], uint32_t &okmask, uint32_t &inmask) {
    okmask = 0;
    inmask = 0;
#pragma unroll
    for (int e = 0; e < AGG_EPT; ++e) {
        const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
        const bool in = i < n;
        us[e] = in ? __ldg(src + i) : NIL;
        vs[e] = in ? __ldg(dst + i) : NIL;
        if (in) inmask |= 1u << e;
    }
#pragma unroll
    for (int e = 0; e < AGG_EPT; ++e)
        if (us[e] < g.nv && vs[e] < g.nv) okmask |= 1u << e;
    if (!g.all_alive) {
        uint8_t au[AGG_EPT], av[AGG_EPT];
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const bool ok = (okmask >> e) & 1u;
            au[e] = ok ? g.alive[us[e]] : 0;
            av[e] = ok ? g.alive[vs[e]] : 0;
        }
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e)
            if (!(au[e] && av[e])) okmask &= ~(1u << e);
    }
    okmask &= inmask;
}

// Counting pass.  Each (tile, source) adds its count with one atomic whose
// return value is the tile's base rank for that source; every valid pair
// records base + its rank inside the tile (prank, NIL for a rejected pair),
// so the later passes need neither aggregation nor atomics to place it.
// The tile that finds a source's count at zero lists the source as touched.
template <int MODE>
__global__ void __launch_bounds__(AGG_THREADS) k_count(GraphView g, const uint32_t *__restrict__ src,
                                                       const uint32_t *__restrict__ dst,
                                                       unsigned long long n) {
    pdl_wait();
    __shared__ uint32_t keys[AGG_H];
    __shared__ uint32_t cnt[AGG_H];
    __shared__ uint32_t s_tbase;
    unsigned long long rej = 0;
    const unsigned long long ntiles = (n + AGG_TILE - 1) / AGG_TILE;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < AGG_H; i += AGG_THREADS) {
            keys[i] = EMPTY_KEY;
            cnt[i] = 0;
        }
        const unsigned long long base = tile * AGG_TILE;
        uint32_t us[AGG_EPT], vs[AGG_EPT], okmask, inmask;
        load_tile(g, src, dst, n, base, us, vs, okmask, inmask);
        rej += __popc(inmask & ~okmask);
        __syncthreads();
        uint32_t sr[AGG_EPT];  // slot | rank in tile << AGG_HBITS
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            sr[e] = NIL;
            if ((okmask >> e) & 1u) {
                uint32_t r;
                const uint32_t sl = agg_insert(keys, cnt, us[e], r);
                sr[e] = sl | (r << AGG_HBITS);
            }
        }
        __syncthreads();
        // one atomic per (tile, source), 8 in flight per thread; the old
        // count becomes the tile's base rank
        uint32_t fresh = 0;
#pragma unroll
        for (int h0 = 0; h0 < AGG_SPT; h0 += AGG_SPT / 2) {
            uint32_t old[AGG_SPT / 2];
#pragma unroll
            for (int i = 0; i < AGG_SPT / 2; ++i) {
                const int s = threadIdx.x + (h0 + i) * AGG_THREADS;
                const uint32_t u = keys[s];
                old[i] = u != EMPTY_KEY ? atomicAdd(&g.vcnt[vslot(g.vmask, u)], cnt[s]) : 1u;
            }
#pragma unroll
            for (int i = 0; i < AGG_SPT / 2; ++i) {
                const int s = threadIdx.x + (h0 + i) * AGG_THREADS;
                if (keys[s] != EMPTY_KEY) cnt[s] = old[i];
                if (old[i] == 0u) fresh |= 1u << (h0 + i);
            }
        }
        uint32_t ntot;
        const uint32_t ex = block_excl_scan(__popc(fresh), &ntot);
        if (threadIdx.x == 0) s_tbase = ntot ? atomicAdd(&g.dev->n_touched, ntot) : 0u;
        __syncthreads();
        uint32_t t = s_tbase + ex;
        while (fresh) {
            const int i = __ffs(fresh) - 1;
            fresh &= fresh - 1u;
            const uint32_t u = keys[threadIdx.x + i * AGG_THREADS];
            g.t_vid[t] = u;
            g.vtid[vslot(g.vmask, u)] = t;
            ++t;
        }
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            if (i < n) g.prank[i] = sr[e] == NIL ? NIL : cnt[sr[e] & (AGG_H - 1)] + (sr[e] >> AGG_HBITS);
        }
        __syncthreads();
    }
    if (MODE != MODE_QUERY) {
        const unsigned long long r = warp_sum_u64(rej);
        if (lane_id() == 0 && r) atomicAdd(&g.dev->call_b, r);
    }
}

// Counting pass for large batches: one atomic per pair, whose return value
// is the pair's rank among its source's pairs; no aggregation, no barriers.
// The touched list is built afterwards by k_touched_scan.
template <int MODE>
__global__ void __launch_bounds__(256) k_count_direct(GraphView g, const uint32_t *__restrict__ src,
                                                      const uint32_t *__restrict__ dst,
                                                      unsigned long long n) {
    pdl_wait();
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long rej = 0;
    for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i0 < n;
         i0 += stride * CD_PER) {
        uint32_t u[CD_PER], v[CD_PER];
        uint32_t ok = 0;
#pragma unroll
        for (int j = 0; j < CD_PER; ++j) {
            const unsigned long long i = i0 + j * stride;
            u[j] = i < n ? ld_stream(src + i) : NIL;
            v[j] = i < n ? ld_stream(dst + i) : NIL;
            if (u[j] < g.nv && v[j] < g.nv) ok |= 1u << j;
        }
        if (!g.all_alive) {
            uint8_t au[CD_PER], av[CD_PER];
#pragma unroll
            for (int j = 0; j < CD_PER; ++j) {
                au[j] = ((ok >> j) & 1u) ? g.alive[u[j]] : 0;
                av[j] = ((ok >> j) & 1u) ? g.alive[v[j]] : 0;
            }
#pragma unroll
            for (int j = 0; j < CD_PER; ++j)
                if (!(au[j] && av[j])) ok &= ~(1u << j);
        }
        uint32_t r[CD_PER];
#pragma unroll
        for (int j = 0; j < CD_PER; ++j) r[j] = ((ok >> j) & 1u) ? atomicAdd(&g.vcnt[vslot(g.vmask, u[j])], 1u) : NIL;
#pragma unroll
        for (int j = 0; j < CD_PER; ++j) {
            const unsigned long long i = i0 + j * stride;
            if (i < n) {
                g.prank[i] = r[j];
                if (r[j] == NIL) ++rej;
            }
        }
    }
    if (MODE != MODE_QUERY) {
        rej = warp_sum_u64(rej);
        if (lane_id() == 0 && rej) atomicAdd(&g.dev->call_b, rej);
    }
}

// Touched list after a direct count: every vertex with a non-zero count
// (vertex order within each chunk; one atomic per CTA chunk).
__global__ void __launch_bounds__(256) k_touched_scan(GraphView g) {
    pdl_wait();
    const uint32_t ncap = g.vmask + 1;
    __shared__ uint32_t s_base;
    for (uint32_t base = blockIdx.x * blockDim.x * 4; base < ncap; base += gridDim.x * blockDim.x * 4) {
        uint32_t flags = 0;
        const uint32_t u0 = base + threadIdx.x * 4;
        if (u0 + 3 < ncap) {
            const uint4 c = *reinterpret_cast<const uint4 *>(g.vcnt + u0);
            flags = (c.x ? 1u : 0u) | (c.y ? 2u : 0u) | (c.z ? 4u : 0u) | (c.w ? 8u : 0u);
        } else {
            for (int j = 0; j < 4; ++j)
                if (u0 + j < ncap && g.vcnt[u0 + j]) flags |= 1u << j;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(__popc(flags), &tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(&g.dev->n_touched, tot) : 0u;
        __syncthreads();
        uint32_t t = s_base + ex;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((flags >> j) & 1u) {
                g.t_vid[t] = vslot_inv(g.vmask, u0 + j);
                g.vtid[u0 + j] = t;
                ++t;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_count_rejects(GraphView g, const uint32_t *__restrict__ src,
                                                       const uint32_t *__restrict__ dst,
                                                       unsigned long long n, unsigned long long *rejected) {
    pdl_wait();
    unsigned long long rej = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        if (!valid_pair(g, src[i], dst[i])) ++rej;
    rej = warp_sum_u64(rej);
    if (lane_id() == 0 && rej) atomicAdd(rejected, rej);
}

// ------------------------------------------------------------------ insert

__global__ void __launch_bounds__(256) k_plan_insert(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t C = g.C;
    __shared__ unsigned long long s_base, s_rbase;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t need = 0, rneed = 0, deg = 0, last = NIL;
        bool run = false;
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            const uint32_t cnt = g.vcnt[vslot(g.vmask, u)];
            const uint4 s = g.sent[u];
            deg = s.x;
            last = s.w;
            // a hub: already in runs, or an empty source whose first
            // allocation takes at least hub_deg entries
            run = g.rs && (is_run(s.z) || (s.y == 0 && cnt >= g.hub_deg));
            if (!run) {
                const uint32_t space = s.y * C - deg;
                need = cnt > space ? divc(g.cmul, cnt - space + C - 1) : 0u;
            } else {
                const uint32_t R = 1u << g.rs;
                const uint32_t nbn = divc(g.cmul, deg + cnt + C - 1);
                rneed = ((nbn + R - 1u) >> g.rs) - ((s.y + R - 1u) >> g.rs);
            }
        }
        uint32_t tot, rtot = 0, rex = 0;
        const uint32_t ex = block_excl_scan(need, &tot);
        if (g.rs) rex = block_excl_scan(rneed, &rtot);
        if (threadIdx.x == 0) {
            s_base = tot ? atomicAdd(&g.dev->alloc_total, (unsigned long long)tot) : 0ull;
            s_rbase = rtot ? atomicAdd(&g.dev->ralloc_total, (unsigned long long)rtot) : 0ull;
        }
        __syncthreads();
        if (t < nt && !run) {
            const unsigned long long off = s_base + ex;
            g.t_a[t] = make_uint4(deg, last, (uint32_t)off, need);
            g.vinfo[vslot(g.vmask, g.t_vid[t])] = make_uint4(deg, last, (uint32_t)off, 0u);
            for (uint32_t j = 0; j < need; ++j) g.t_owner[off + j] = t;
        } else if (t < nt) {
            // run pops: offset into the run queue, count flagged by RUN_BIT
            const unsigned long long roff = s_rbase + rex;
            g.t_a[t] = make_uint4(deg, last, (uint32_t)roff, rneed | RUN_BIT);
            g.vinfo[vslot(g.vmask, g.t_vid[t])] = make_uint4(deg, last, (uint32_t)roff, 1u);
            for (uint32_t j = 0; j < rneed; ++j) g.t_rowner[roff + j] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_link_insert(GraphView g) {
    pdl_wait();
    Dev *dev = g.dev;
    const unsigned long long total = dev->alloc_total;
    const unsigned long long rtotal = g.rs ? dev->ralloc_total : 0ull;
    const unsigned long long qf = dev->q_front, qb = dev->q_back;
    if (total > qb - qf || (rtotal && rtotal > dev->rq_back - dev->rq_front)) {
        // Edge queue exhausted: the whole call becomes a no-op.
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            dev->abort = 1u;
            latch_status(dev, 2u /* GV_ERR_OUT_OF_MEMORY */);
        }
        return;
    }
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(qf, P);
    const uint32_t C = g.C;
    const unsigned long long rqbase = rtotal ? qmod(dev->rq_front, g.RP) : 0ull;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < total + rtotal;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        if (j >= total) {
            // a popped run: its head takes run heap index nr + 1 + (its pop
            // offset) in the tree of run heads, by the same rule as a block
            const unsigned long long jr = j - total;
            const uint32_t t = g.t_rowner[jr];
            const uint4 a = g.t_a[t];
            const uint32_t deg = a.x, roff = a.z, rneed = a.w & ~RUN_BIT;
            const uint32_t R = 1u << g.rs;
            const uint32_t nr = (divc(g.cmul, deg + C - 1) + R - 1u) >> g.rs;
            const uint32_t k = nr + 1 + (uint32_t)(jr - roff);
            const uint32_t nrn = nr + rneed;
            const uint32_t id = g.rqueue[ring(rqbase, jr, g.RP)];
            if (id >= P) {
                latch_status(dev, 5u /* GV_ERR_STATE */);
                continue;
            }
            if (2ull * k > nrn) g.links[2ull * id] = NIL;
            if (2ull * k + 1 > nrn) g.links[2ull * id + 1] = NIL;
            if (k > 1) {
                const uint32_t p = k >> 1;
                const uint32_t pid = p > nr ? g.rqueue[ring(rqbase, roff + (p - nr - 1), g.RP)]
                                            : cbt_walk(g.links, P, g.sent[g.t_vid[t]].z & ~RUN_BIT, p);
                if (pid >= P) {
                    latch_status(dev, 5u /* GV_ERR_STATE */);
                    continue;
                }
                g.links[2ull * pid + (k & 1u)] = id;
            }
            continue;
        }
        const uint32_t t = g.t_owner[j];
        const uint4 a = g.t_a[t];
        const uint32_t deg = a.x, off = a.z, need = a.w;
        const uint32_t nb = divc(g.cmul, deg + C - 1);
        const uint32_t k = nb + 1 + (uint32_t)(j - off);  // heap index of this block
        const uint32_t nbn = nb + need;
        const uint32_t id = g.queue[ring(qbase, j, P)];
        if (id >= P) {
            latch_status(dev, 5u /* GV_ERR_STATE */);
            continue;
        }
        // Child slots that no new block will fill are cleared here; the
        // others are written by the child itself.
        if (2ull * k > nbn) g.links[2ull * id] = NIL;
        if (2ull * k + 1 > nbn) g.links[2ull * id + 1] = NIL;
        if (k > 1) {
            const uint32_t p = k >> 1;
            uint32_t pid;
            if (p > nb) pid = g.queue[ring(qbase, off + (p - nb - 1), P)];
            else pid = cbt_walk(g.links, P, g.sent[g.t_vid[t]].z, p);
            if (pid == NIL || id >= P) {
                latch_status(dev, 5u /* GV_ERR_STATE */);
                continue;
            }
            g.links[2ull * pid + (k & 1u)] = id;
        }
    }
}

// Insert scatter: one pass over the pairs, no aggregation and no atomics.
// Pair i of source u with rank r goes to slot deg(u) + r: the free slots of
// the last block first, then the new blocks popped for u at queue offset
// recorded by the plan in the source's vinfo record.
template <bool WEIGHTED>
__global__ void __launch_bounds__(256) k_scatter_insert(GraphView g, const uint32_t *__restrict__ src,
                                                        const uint32_t *__restrict__ dst,
                                                        const uint32_t *__restrict__ wts,
                                                        unsigned long long n) {
    pdl_wait();
    if (g.dev->abort) return;
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(g.dev->q_front, P);
    const unsigned long long rqbase = g.rs ? qmod(g.dev->rq_front, g.RP) : 0ull;
    const uint32_t C = g.C;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i0 < n;
         i0 += stride * PP) {
        uint32_t r[PP], u[PP], v[PP];
#pragma unroll
        for (int j = 0; j < PP; ++j) {
            const unsigned long long i = i0 + j * stride;
            r[j] = i < n ? ld_stream(g.prank + i) : NIL;
            u[j] = i < n ? ld_stream(src + i) : 0u;
            v[j] = i < n ? ld_stream(dst + i) : 0u;
        }
        uint4 vi[PP];  // {deg, last block, queue offset of the new blocks (or runs), 1 for a run source}
#pragma unroll
        for (int j = 0; j < PP; ++j)
            if (r[j] != NIL) vi[j] = g.vinfo[vslot(g.vmask, u[j])];
        uint32_t blk[PP], ln[PP];
#pragma unroll
        for (int j = 0; j < PP; ++j) {
            blk[j] = NIL;
            ln[j] = 0;
            if (r[j] != NIL) {
                const uint32_t deg = vi[j].x;
                const uint32_t nb = divc(g.cmul, deg + C - 1);
                const uint32_t space = nb * C - deg;
                if (r[j] < space) {
                    blk[j] = vi[j].y;
                    ln[j] = deg - (nb - 1) * C + r[j];
                } else {
                    const uint32_t q = r[j] - space;
                    const uint32_t jb = divc(g.cmul, q);
                    ln[j] = q - jb * C;
                    if (vi[j].w == 0u) {
                        blk[j] = g.queue[ring(qbase, vi[j].z + jb, P)];
                    } else {
                        // block nb + jb of a run source: still inside its last
                        // run (contiguous after the last block), or in run
                        // (nb + jb) >> rs, popped at run offset z + that - nr
                        const uint32_t J = nb + jb, nr = (nb + (1u << g.rs) - 1u) >> g.rs;
                        blk[j] = J < (nr << g.rs) ? vi[j].y + 1u + jb
                                                  : g.rqueue[ring(rqbase, vi[j].z + (J >> g.rs) - nr, g.RP)] +
                                                        (J & ((1u << g.rs) - 1u));
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PP; ++j) {
            if (r[j] != NIL) {
                if (blk[j] < P) {
                    const size_t slot = (size_t)blk[j] * C + ln[j];
                    g.data[slot] = v[j];
                    if (WEIGHTED) g.wdata[slot] = wts ? ld_stream(wts + i0 + j * stride) : 0u;
                } else {
                    latch_status(g.dev, 5u /* GV_ERR_STATE */);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_finalize_insert(GraphView g, unsigned long long n,
                                                         unsigned long long *counts) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t nt = dev->n_touched;
    const bool abort = dev->abort != 0;
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(dev->q_front, P);
    const unsigned long long rqbase = g.rs ? qmod(dev->rq_front, g.RP) : 0ull;
    const uint32_t C = g.C;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint32_t u = g.t_vid[t];
        const uint32_t cnt = g.vcnt[vidx(g, u)];
        if (!abort) {
            const uint4 a = g.t_a[t];
            const uint32_t deg = a.x, off = a.z;
            const uint32_t nb = divc(g.cmul, deg + C - 1);
            uint4 s = g.sent[u];
            s.x = deg + cnt;
            if (!(a.w & RUN_BIT)) {
                const uint32_t need = a.w;
                s.y = nb + need;
                if (need) {
                    if (nb == 0) s.z = g.queue[ring(qbase, off, P)];
                    s.w = g.queue[ring(qbase, off + need - 1, P)];
                }
            } else {
                // run source: the root word is the first run's head with
                // RUN_BIT; the last block is block nbn - 1, found as in the
                // scatter
                const uint32_t R = 1u << g.rs;
                const uint32_t nbn = divc(g.cmul, deg + cnt + C - 1);
                const uint32_t nr = (nb + R - 1u) >> g.rs;
                if (nb == 0) s.z = g.rqueue[ring(rqbase, off, g.RP)] | RUN_BIT;
                if (nbn > nb) {
                    const uint32_t J = nbn - 1u;
                    s.w = J < (nr << g.rs) ? a.y + (J - (nb - 1u))
                                           : g.rqueue[ring(rqbase, off + (J >> g.rs) - nr, g.RP)] + (J & (R - 1u));
                }
                s.y = nbn;
            }
            g.sent[u] = s;
        }
        g.vcnt[vidx(g, u)] = 0;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        unsigned long long rej = dev->call_b;
        unsigned long long ins = n - rej;
        if (abort) {
            ins = 0;
            rej = 0;
        } else {
            dev->q_front += dev->alloc_total;
            dev->rq_front += dev->ralloc_total;
            dev->num_edges += ins;
            dev->tot_ins += ins;
            dev->tot_rej += rej;
        }
        if (counts) {
            counts[0] = ins;
            counts[1] = rej;
        }
        dev->alloc_total = 0;
        dev->call_a = dev->call_b = dev->call_c = 0;
        dev->n_touched = 0;
        dev->n_items = 0;
        dev->n_mitems = 0;
        dev->n_tiny = 0;
        dev->n_tiny_hi = 0;
        dev->arena_used = 0;
        dev->harena_used = 0;
        dev->n_chunks = 0;
        dev->n_groups = 0;
        dev->n_hash = 0;
        dev->free_total = 0;
        dev->ralloc_total = 0;
        dev->rfree_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ------------------------------------------- small insert batches, one CTA

// An insert of at most SMALL_INS pairs in one kernel of one CTA: the chain
// of five dependent kernels of the general path (count, plan, link,
// scatter, finalize) is what a small batch waits for, not its work.  The
// same steps, separated by barriers instead of launches: pairs grouped by
// source in a shared hash table (a returning shared atomic gives each pair
// its rank), block demand per source and one block scan for the queue
// offsets (Figure 3), the pool check before any write (an exhausted queue
// makes the call a no-op), then the new blocks linked at heap indices
// nblocks + 1 .. (Figure 4's bit-string rule) and the pairs written at slot
// deg + rank, and last the sentinels and the call's counters.
constexpr uint32_t SMALL_INS = 2048;
constexpr uint32_t SMALL_HS = 2 * SMALL_INS;  // hash slots (a power of two)
constexpr uint32_t SMALL_THREADS = 1024;
constexpr size_t SMALL_SMEM = SMALL_HS * 3 * 4 + SMALL_INS * (4 + 16 + 4 + 4 + 4 + 4 + 4);

template <bool WEIGHTED>
__global__ void __launch_bounds__(SMALL_THREADS, 1) k_insert_small(GraphView g, const uint32_t *__restrict__ src,
                                                                  const uint32_t *__restrict__ dst,
                                                                  const uint32_t *__restrict__ wts,
                                                                  uint32_t n, unsigned long long *counts) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *hk = sm;                                    // [SMALL_HS] source id per slot
    uint32_t *hc = hk + SMALL_HS;                         // [SMALL_HS] pairs per slot
    uint32_t *ht = hc + SMALL_HS;                         // [SMALL_HS] touched index per slot
    uint4 *ta = reinterpret_cast<uint4 *>(ht + SMALL_HS); // [SMALL_INS] sentinel before the call
    uint32_t *tu = reinterpret_cast<uint32_t *>(ta + SMALL_INS);  // [SMALL_INS] source id
    uint32_t *tslot = tu + SMALL_INS;                     // [SMALL_INS] hash slot
    uint32_t *tneed = tslot + SMALL_INS;                  // [SMALL_INS] new blocks
    uint32_t *toff = tneed + SMALL_INS;                   // [SMALL_INS] queue offset of the new blocks
    uint32_t *pslot = toff + SMALL_INS;                   // [SMALL_INS] hash slot per pair (NIL: rejected)
    uint32_t *prank = pslot + SMALL_INS;                  // [SMALL_INS] rank per pair
    __shared__ uint32_t s_nt, s_rej, s_abort;
    __shared__ unsigned long long s_qbase;
    Dev *dev = g.dev;
    const uint32_t tid = threadIdx.x, C = g.C;
    const unsigned long long P = g.P;
    for (uint32_t h = tid; h < SMALL_HS; h += SMALL_THREADS) {
        hk[h] = EMPTY_KEY;
        hc[h] = 0;
    }
    if (tid == 0) {
        s_nt = 0;
        s_rej = 0;
    }
    __syncthreads();
    // 1. group by source
    uint32_t rej = 0;
    for (uint32_t i = tid; i < n; i += SMALL_THREADS) {
        const uint32_t u = src[i], v = dst[i];
        const bool ok = u < g.nv && v < g.nv && (g.all_alive || (g.alive[u] && g.alive[v]));
        if (!ok) {
            ++rej;
            pslot[i] = NIL;
            continue;
        }
        uint32_t h = hidx(u, SMALL_HS);
        // at most n <= SMALL_HS / 2 keys: a free or equal slot exists
        for (uint32_t step = 0; step < SMALL_HS; ++step) {
            const uint32_t old = atomicCAS(&hk[h], EMPTY_KEY, u);
            if (old == EMPTY_KEY) {
                const uint32_t t = atomicAdd(&s_nt, 1u);
                ht[h] = t;
                tu[t] = u;
                tslot[t] = h;
                break;
            }
            if (old == u) break;
            h = (h + 1) & (SMALL_HS - 1);
        }
        pslot[i] = h;
        prank[i] = atomicAdd(&hc[h], 1u);
    }
    if (rej) atomicAdd(&s_rej, rej);
    __syncthreads();
    const uint32_t nt = s_nt;
    // 2. block demand and queue offsets (two touched sources per thread)
    uint32_t need2[2] = {0, 0};
    for (uint32_t k = 0; k < 2; ++k) {
        const uint32_t t = 2 * tid + k;
        if (t < nt) {
            const uint4 st = g.sent[tu[t]];
            ta[t] = st;
            const uint32_t cnt = hc[tslot[t]];
            const uint32_t space = st.y * C - st.x;
            need2[k] = cnt > space ? divc(g.cmul, cnt - space + C - 1) : 0u;
            tneed[t] = need2[k];
        }
    }
    uint32_t total;
    const uint32_t base = block_excl_scan(need2[0] + need2[1], &total);
    if (2 * tid < nt) toff[2 * tid] = base;
    if (2 * tid + 1 < nt) toff[2 * tid + 1] = base + need2[0];
    // 3. pool check before any write
    if (tid == 0) {
        const unsigned long long qf = dev->q_front, qb = dev->q_back;
        s_abort = total > qb - qf ? 1u : 0u;
        s_qbase = qmod(qf, P);
        if (s_abort) {
            latch_status(dev, 2u /* GV_ERR_OUT_OF_MEMORY */);
            if (counts) {
                counts[0] = 0;
                counts[1] = 0;
            }
        }
    }
    __syncthreads();
    if (s_abort) return;
    const unsigned long long qbase = s_qbase;
    // 4. links of the new blocks, and the pairs' slots
    for (uint32_t j = tid; j < total; j += SMALL_THREADS) {
        // owner: the last touched source whose offset is <= j
        uint32_t lo = 0, hi = nt;  // toff[lo] <= j < toff[hi] (toff[nt] = total)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (toff[mid] <= j) lo = mid;
            else hi = mid;
        }
        const uint32_t t = lo;
        const uint4 st = ta[t];
        const uint32_t nb = st.y, need = tneed[t], off = toff[t];
        const uint32_t k = nb + 1 + (j - off);  // heap index of this block
        const uint32_t nbn = nb + need;
        const uint32_t id = g.queue[ring(qbase, j, P)];
        if (id >= P) {
            latch_status(dev, 5u /* GV_ERR_STATE */);
            continue;
        }
        if (2ull * k > nbn) g.links[2ull * id] = NIL;
        if (2ull * k + 1 > nbn) g.links[2ull * id + 1] = NIL;
        if (k > 1) {
            const uint32_t p = k >> 1;
            const uint32_t pid =
                p > nb ? g.queue[ring(qbase, off + (p - nb - 1), P)] : cbt_walk(g.links, P, st.z, p);
            if (pid >= P) {
                latch_status(dev, 5u /* GV_ERR_STATE */);
                continue;
            }
            g.links[2ull * pid + (k & 1u)] = id;
        }
    }
    for (uint32_t i = tid; i < n; i += SMALL_THREADS) {
        const uint32_t h = pslot[i];
        if (h == NIL) continue;
        const uint32_t t = ht[h], r = prank[i];
        const uint4 st = ta[t];
        const uint32_t deg = st.x, nb = st.y;
        const uint32_t space = nb * C - deg;
        uint32_t blk, ln;
        if (r < space) {
            blk = st.w;
            ln = deg - (nb - 1) * C + r;
        } else {
            const uint32_t q = r - space;
            const uint32_t jb = divc(g.cmul, q);
            ln = q - jb * C;
            blk = g.queue[ring(qbase, toff[t] + jb, P)];
        }
        if (blk < P) {
            const size_t slot = (size_t)blk * C + ln;
            g.data[slot] = dst[i];
            if (WEIGHTED) g.wdata[slot] = wts ? wts[i] : 0u;
        } else {
            latch_status(dev, 5u /* GV_ERR_STATE */);
        }
    }
    // 5. sentinels and counters
    for (uint32_t t = tid; t < nt; t += SMALL_THREADS) {
        uint4 st = ta[t];
        const uint32_t need = tneed[t], off = toff[t], nb = st.y;
        st.x += hc[tslot[t]];
        st.y = nb + need;
        if (need) {
            if (nb == 0) st.z = g.queue[ring(qbase, off, P)];
            st.w = g.queue[ring(qbase, off + need - 1, P)];
        }
        g.sent[tu[t]] = st;
    }
    if (tid == 0) {
        const unsigned long long r2 = s_rej, ins = n - r2;
        dev->q_front += total;
        dev->num_edges += ins;
        dev->tot_ins += ins;
        dev->tot_rej += r2;
        if (counts) {
            counts[0] = ins;
            counts[1] = r2;
        }
    }
}

// ------------------------------------------------------ membership pipeline

// Per touched source: arena words for its batch destinations (a list up to
// LIST_MAX entries, else a hash set), and either the tiny tier (one thread,
// tiny adjacency and few batch entries) or work items of IB blocks.
template <int MODE>
__global__ void __launch_bounds__(256) k_plan_member(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t IB = g.IB;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    __shared__ unsigned long long s_aw, s_hw;
    __shared__ uint32_t s_ai, s_am, s_at, s_ath;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t m = 0, lw = 0, hw = 0, ni = 0, tiny = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            m = g.vcnt[vslot(g.vmask, u)];
            s = g.sent[u];
            if (MODE == MODE_DEDUP) hw = dedup_words(m);
            else if (m <= LIST_MAX) lw = m;
            else hw = member_words(m);
            if (s.y > 0) {
                const bool small = MODE == MODE_QUERY
                    ? (s.x <= min(TINY_DEG_Q, TINY_NB_Q * g.C) && s.y <= TINY_NB_Q && m <= TINY_M)
                    : (MODE != MODE_DEDUP && s.x <= tiny_deg && s.y <= TINY_NB && m <= TINY_M);
                if (small) tiny = 1;
                else ni = (s.y + IB - 1) / IB;
            }
        }
        const uint32_t tlo = tiny && s.x <= TINY_SPLIT, thi = tiny && s.x > TINY_SPLIT;
        uint32_t lt, ht, ttot, tthi;
        const uint32_t lex = block_excl_scan(lw, &lt);
        const uint32_t hex = block_excl_scan(hw, &ht);
        const uint32_t tex = block_excl_scan(tlo, &ttot);
        const uint32_t thx = block_excl_scan(thi, &tthi);
        if (threadIdx.x == 0) {
            s_aw = lt ? atomicAdd(&g.dev->arena_used, (unsigned long long)lt) : 0ull;
            s_hw = ht ? atomicAdd(&g.dev->harena_used, (unsigned long long)ht) : 0ull;
            s_at = ttot ? atomicAdd(&g.dev->n_tiny, ttot) : 0u;
            s_ath = tthi ? atomicAdd(&g.dev->n_tiny_hi, tthi) : 0u;
        }
        const uint32_t item0 = alloc_items(g, ni, &s_ai, &s_am);
        if (t < nt) {
            // hash sets are powers of two >= HB words, so their offsets stay
            // multiples of HB words: every bucket is sector-aligned
            const uint32_t aoff = hw ? (uint32_t)(g.hbase + s_hw + hex) : (uint32_t)(s_aw + lex);
            g.t_a[t] = make_uint4(m, aoff, hw, item0);
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            g.vinfo[vslot(g.vmask, g.t_vid[t])] = make_uint4(m, aoff, hw, 0u);
            if (tlo) g.t_tiny[s_at + tex] = t;
            if (thi) g.t_tiny[g.tiny_cap - 1 - (s_ath + thx)] = t;
            emit_items(g, t, item0, ni);
        }
        __syncthreads();
    }
}

// Segmented deletes: one removed entry for the segment that owns its key
// (shared histogram, flushed to the per-segment counts by the kernel).
__device__ __forceinline__ void seg_count(uint32_t *hist, uint32_t own, uint32_t G, Dev *dev) {
    if (own < G) atomicAdd(&hist[own], 1u);
    else latch_status(dev, 5u /* GV_ERR_STATE */);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_arena_init(GraphView g) {
    pdl_wait();
    // hash region -> EMPTY; query hit flags of both regions -> 0 (list
    // entries are all overwritten by the scatter)
    const unsigned long long lused = g.dev->arena_used, hused = g.dev->harena_used;
    constexpr bool Q = (MODE == MODE_QUERY || MODE == MODE_DEDUP);
    const unsigned long long tot = (Q ? lused : 0ull) + hused;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < tot;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        if (Q && k < lused) {
            g.found[k] = 0u;
        } else {
            const unsigned long long i = g.hbase + (k - (Q ? lused : 0ull));
            g.arena[i] = EMPTY_KEY;
            if (Q) g.found[i] = 0u;
            if (MODE == MODE_DELETE && g.seg_own) g.seg_own[i] = NIL;
        }
    }
}

// Batch destinations into their source's list (plain store at the pair's
// rank) or hash set (a CAS at the home slot, probing on collision); queries
// record where their pair landed.  One pass over the pairs, no aggregation.
template <int MODE>
__global__ void __launch_bounds__(256) k_scatter_member(GraphView g, const uint32_t *__restrict__ src,
                                                        const uint32_t *__restrict__ dst,
                                                        unsigned long long n) {
    constexpr int PPM = PP_MEMBER;
    pdl_wait();
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i0 < n;
         i0 += stride * PPM) {
        uint32_t r[PPM], u[PPM], v[PPM];
#pragma unroll
        for (int j = 0; j < PPM; ++j) {
            const unsigned long long i = i0 + j * stride;
            r[j] = i < n ? ld_stream(g.prank + i) : NIL;
            u[j] = i < n ? ld_stream(src + i) : 0u;
            v[j] = i < n ? ld_stream(dst + i) : 0u;
        }
        uint32_t aoff[PPM], hs[PPM];
#pragma unroll
        for (int j = 0; j < PPM; ++j) {
            if (r[j] != NIL) {
                const uint4 vi = g.vinfo[vslot(g.vmask, u[j])];
                aoff[j] = vi.y;
                hs[j] = vi.z;  // 0: list
            }
        }
        uint32_t pos[PPM];
#pragma unroll
        for (int j = 0; j < PPM; ++j) {
            pos[j] = NIL;
            if (r[j] != NIL && hs[j] == 0) {
                pos[j] = aoff[j] + r[j];
                g.arena[pos[j]] = v[j];
            }
        }
        // bucketed hash sets: read the home bucket of every pair (both
        // halves in flight together; L2, not a possibly stale L1 line), then
        // claim its first empty slot by CAS; occupied slots stay a prefix of
        // each bucket
        uint4 b0[PPM], b1[PPM];
        uint32_t bk[PPM];
        uint32_t rep = 0;  // set-semantics inserts: bit j = pair j claimed its slot
#pragma unroll
        for (int j = 0; j < PPM; ++j) {
            if (r[j] != NIL && hs[j] != 0) {
                bk[j] = hidx(v[j], hs[j] / HB);
                const uint4 *bp = reinterpret_cast<const uint4 *>(g.arena + aoff[j] + bk[j] * HB);
                b0[j] = __ldcg(bp);
                b1[j] = __ldcg(bp + 1);
            }
        }
#pragma unroll
        for (int j = 0; j < PPM; ++j) {
            if (r[j] != NIL && hs[j] != 0) {
                const uint32_t nbk = hs[j] / HB;
                uint32_t *tab = g.arena + aoff[j];
                uint32_t b = bk[j];
                uint32_t w[HB] = {b0[j].x, b0[j].y, b0[j].z, b0[j].w, b1[j].x, b1[j].y, b1[j].z, b1[j].w};
                // each pass ends, moves to the next bucket, or rereads after
                // losing a slot to another insert (which filled that slot):
                // (HB + 1) * nbk passes bound the loop
                for (uint32_t probe = 0; probe < (HB + 1) * nbk; ++probe) {
                    uint32_t hit = NIL, empty = NIL;
#pragma unroll
                    for (uint32_t k = 0; k < HB; ++k) {
                        if (hit == NIL && w[k] == v[j]) hit = k;
                        if (empty == NIL && w[k] == EMPTY_KEY) empty = k;
                    }
                    if (hit != NIL) {
                        pos[j] = aoff[j] + b * HB + hit;
                        break;
                    }
                    if (empty != NIL) {
                        const uint32_t old = atomicCAS(&tab[b * HB + empty], EMPTY_KEY, v[j]);
                        if (old == EMPTY_KEY || old == v[j]) {
                            pos[j] = aoff[j] + b * HB + empty;
                            if (MODE == MODE_DEDUP && old == EMPTY_KEY) rep |= 1u << j;
                            break;
                        }
                        // lost the slot: reread this bucket
                    } else {
                        b = (b + 1) & (nbk - 1);
                    }
                    const uint4 *bp = reinterpret_cast<const uint4 *>(tab + b * HB);
                    const uint4 x0 = __ldcg(bp), x1 = __ldcg(bp + 1);
                    w[0] = x0.x; w[1] = x0.y; w[2] = x0.z; w[3] = x0.w;
                    w[4] = x1.x; w[5] = x1.y; w[6] = x1.z; w[7] = x1.w;
                }
                if (pos[j] == NIL) latch_status(g.dev, 5u /* GV_ERR_STATE */);
            }
        }
        if (MODE == MODE_DELETE && g.seg_own) {
            // segmented delete: each key's owner is the first segment naming it
#pragma unroll
            for (int j = 0; j < PPM; ++j) {
                if (pos[j] != NIL) {
                    const uint32_t sg = segment_of(g.set_off, g.set_G, i0 + j * stride);
                    if (hs[j] == 0) g.seg_own[pos[j]] = sg;
                    else atomicMin(g.seg_own + pos[j], sg);
                }
            }
        }
        if (MODE == MODE_QUERY || MODE == MODE_DEDUP) {
#pragma unroll
            for (int j = 0; j < PPM; ++j) {
                const unsigned long long i = i0 + j * stride;
                if (i < n) {
                    g.qpos[i] = pos[j];
                    if (MODE == MODE_DEDUP) g.pflag[i] = (uint8_t)((rep >> j) & 1u);
                }
            }
        }
    }
}

// ------------------------------------ small delete / query batches, one CTA

// The front of a plain delete or query of at most SMALL_MEM pairs in one
// kernel of one CTA, in place of the counting pass, the plan, the arena
// initialisation and the scatter (four dependent launches that a small batch
// waits for more than it works in): the batch grouped by source in a shared
// hash table (a returning shared atomic gives each pair its rank among its
// source's pairs), then per touched source the plan of the general path
// (batch list or hash set in the arena, thread-per-source tier or work items,
// the same thresholds and the same records), the hash sets cleared, and the
// pairs placed in their lists or sets.  The mark, compaction and finalize
// kernels of the general path follow unchanged.
constexpr uint32_t SMALL_MEM = 2048;
constexpr uint32_t SMALL_MEM_HS = 2 * SMALL_MEM;  // source hash slots (a power of two)
constexpr uint32_t SMALL_MEM_THREADS = 1024;
constexpr size_t SMALL_MEM_SMEM = SMALL_MEM_HS * 3 * 4 + SMALL_MEM * 4 * 4 + SMALL_MEM * 2 * 4;

template <int MODE>
__global__ void __launch_bounds__(SMALL_MEM_THREADS, 1) k_member_small(GraphView g, const uint32_t *__restrict__ src,
                                                                      const uint32_t *__restrict__ dst, uint32_t n) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *hk = sm;                      // [SMALL_MEM_HS] source id per slot
    uint32_t *hc = hk + SMALL_MEM_HS;       // [SMALL_MEM_HS] pairs per slot
    uint32_t *ht = hc + SMALL_MEM_HS;       // [SMALL_MEM_HS] touched index per slot
    uint32_t *tu = ht + SMALL_MEM_HS;       // [SMALL_MEM] source id per touched index
    uint32_t *tslot = tu + SMALL_MEM;       // [SMALL_MEM] hash slot per touched index
    uint32_t *taoff = tslot + SMALL_MEM;    // [SMALL_MEM] arena offset of the source's list or set
    uint32_t *thw = taoff + SMALL_MEM;      // [SMALL_MEM] hash-set words (0: a list)
    uint32_t *pslot = thw + SMALL_MEM;      // [SMALL_MEM] hash slot per pair (NIL: rejected)
    uint32_t *prk = pslot + SMALL_MEM;      // [SMALL_MEM] rank per pair
    __shared__ uint32_t s_nt, s_rej;
    __shared__ unsigned long long s_aw, s_hw;
    __shared__ uint32_t s_ai, s_am, s_at, s_ath;
    __shared__ uint32_t s_lused, s_hused;
    Dev *dev = g.dev;
    const uint32_t tid = threadIdx.x;
    for (uint32_t h = tid; h < SMALL_MEM_HS; h += SMALL_MEM_THREADS) {
        hk[h] = EMPTY_KEY;
        hc[h] = 0;
    }
    if (tid == 0) {
        s_nt = 0;
        s_rej = 0;
        s_lused = 0;
        s_hused = 0;
    }
    __syncthreads();
    // 1. group by source
    uint32_t rej = 0;
    for (uint32_t i = tid; i < n; i += SMALL_MEM_THREADS) {
        const uint32_t u = src[i], v = dst[i];
        if (!valid_pair(g, u, v)) {
            ++rej;
            pslot[i] = NIL;
            if (MODE == MODE_QUERY) g.qpos[i] = NIL;
            continue;
        }
        uint32_t h = hidx(u, SMALL_MEM_HS);
        // at most n <= SMALL_MEM_HS / 2 keys: a free or equal slot exists
        for (uint32_t step = 0; step < SMALL_MEM_HS; ++step) {
            const uint32_t old = atomicCAS(&hk[h], EMPTY_KEY, u);
            if (old == EMPTY_KEY) {
                const uint32_t t = atomicAdd(&s_nt, 1u);
                ht[h] = t;
                tu[t] = u;
                tslot[t] = h;
                break;
            }
            if (old == u) break;
            h = (h + 1) & (SMALL_MEM_HS - 1);
        }
        pslot[i] = h;
        prk[i] = atomicAdd(&hc[h], 1u);
    }
    if (rej) atomicAdd(&s_rej, rej);
    __syncthreads();
    const uint32_t nt = s_nt;
    // 2. plan per touched source (the general path's k_plan_member)
    const uint32_t IB = g.IB;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    for (uint32_t base = 0; base < nt; base += SMALL_MEM_THREADS) {
        const uint32_t t = base + tid;
        uint32_t m = 0, lw = 0, hw = 0, ni = 0, tiny = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            const uint32_t u = tu[t];
            m = hc[tslot[t]];
            s = g.sent[u];
            if (m <= LIST_MAX) lw = m;
            else hw = member_words(m);
            if (s.y > 0) {
                const bool small = MODE == MODE_QUERY
                    ? (s.x <= min(TINY_DEG_Q, TINY_NB_Q * g.C) && s.y <= TINY_NB_Q && m <= TINY_M)
                    : (s.x <= tiny_deg && s.y <= TINY_NB && m <= TINY_M);
                if (small) tiny = 1;
                else ni = (s.y + IB - 1) / IB;
            }
        }
        const uint32_t tlo = tiny && s.x <= TINY_SPLIT, thi = tiny && s.x > TINY_SPLIT;
        uint32_t lt, hts, ttot, tthi;
        const uint32_t lex = block_excl_scan(lw, &lt);
        const uint32_t hex = block_excl_scan(hw, &hts);
        const uint32_t tex = block_excl_scan(tlo, &ttot);
        const uint32_t thx = block_excl_scan(thi, &tthi);
        if (tid == 0) {
            s_aw = lt ? atomicAdd(&dev->arena_used, (unsigned long long)lt) : 0ull;
            s_hw = hts ? atomicAdd(&dev->harena_used, (unsigned long long)hts) : 0ull;
            s_at = ttot ? atomicAdd(&dev->n_tiny, ttot) : 0u;
            s_ath = tthi ? atomicAdd(&dev->n_tiny_hi, tthi) : 0u;
            s_lused += lt;
            s_hused += hts;
        }
        const uint32_t item0 = alloc_items(g, ni, &s_ai, &s_am);
        if (t < nt) {
            const uint32_t aoff = hw ? (uint32_t)(g.hbase + s_hw + hex) : (uint32_t)(s_aw + lex);
            g.t_vid[t] = tu[t];
            g.t_a[t] = make_uint4(m, aoff, hw, item0);
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            taoff[t] = aoff;
            thw[t] = hw;
            if (tlo) g.t_tiny[s_at + tex] = t;
            if (thi) g.t_tiny[g.tiny_cap - 1 - (s_ath + thx)] = t;
            emit_items(g, t, item0, ni);
        }
        __syncthreads();
    }
    // 3. hash sets empty; query hit flags cleared over both regions
    const uint32_t lused = s_lused, hused = s_hused;
    for (uint32_t k = tid; k < hused; k += SMALL_MEM_THREADS) {
        g.arena[g.hbase + k] = EMPTY_KEY;
        if (MODE == MODE_QUERY) g.found[g.hbase + k] = 0u;
    }
    if (MODE == MODE_QUERY)
        for (uint32_t k = tid; k < lused; k += SMALL_MEM_THREADS) g.found[k] = 0u;
    __syncthreads();
    // 4. batch destinations into the lists (at the pair's rank) or the sets
    for (uint32_t i = tid; i < n; i += SMALL_MEM_THREADS) {
        const uint32_t h = pslot[i];
        if (h == NIL) continue;
        const uint32_t t = ht[h];
        const uint32_t v = dst[i];
        uint32_t pos;
        if (thw[t] == 0) {
            pos = taoff[t] + prk[i];
            g.arena[pos] = v;
        } else {
            const uint32_t w = bucket_insert(g.arena + taoff[t], thw[t] / HB, v);
            pos = w == NIL ? NIL : taoff[t] + w;
            if (w == NIL) latch_status(dev, 5u /* GV_ERR_STATE */);
        }
        if (MODE == MODE_QUERY) g.qpos[i] = pos;
    }
    if (tid == 0) {
        dev->n_touched = nt;
        if (MODE != MODE_QUERY && s_rej) dev->call_b += s_rej;
    }
}

// One warp per work item (see the file comment).
// Per multi-item source (one warp, all lanes call): the new degree is the
// sum of the items' survivors; per item, the holes below the new degree and
// the survivors at or above it, prefix-summed over the source's items
// (it_H, it_S); the sentinel gets the new degree and block count.
__device__ __forceinline__ void vscan_source(const GraphView &g, uint32_t t, uint32_t *s_mhist,
                                             unsigned long long &removed) {
    const uint32_t lane = lane_id();
    const uint32_t C = g.C, IB = g.IB, SPI = IB * C;
    const uint4 b = g.t_b[t];
    const uint32_t ni = b.w;
    const uint32_t item0 = g.t_a[t].w;
    const uint32_t deg = b.x, root = b.z;
    uint32_t tot = 0;
    for (uint32_t c = lane; c < ni; c += 32) tot += __ldcg(g.it_cnt + item0 + c);
    const uint32_t degn = warp_sum(tot);
    // The one item that holds position degn (if it starts below it) has
    // survivors on both sides: those below degn, counted from its survivor
    // mask by the whole warp at once (lane w reads word w).
    const uint32_t cs = degn / SPI;
    uint32_t below_cs = 0;
    if (cs < ni) {
        const uint32_t split = degn - cs * SPI;
        uint32_t word = 0;
        if (lane < MASK_WORDS && lane * 32 < split) {
            word = __ldcg(g.it_mask + (size_t)(item0 + cs) * MASK_WORDS + lane);
            const uint32_t nbits = split - lane * 32;
            if (nbits < 32) word &= (1u << nbits) - 1u;
        }
        below_cs = warp_sum(__popc(word));
    }
    uint32_t carryH = 0, carryS = 0;
    for (uint32_t c0 = 0; c0 < ni; c0 += 32) {
        const uint32_t c = c0 + lane;
        uint32_t h = 0, s = 0;
        if (c < ni) {
            const uint32_t sb = c * SPI;
            const uint32_t len = min(SPI, deg - sb);
            const uint32_t cnt = __ldcg(g.it_cnt + item0 + c);
            if (sb + len <= degn) {
                h = len - cnt;
            } else if (sb >= degn) {
                s = cnt;
            } else {
                // c == cs: the item straddling degn
                const uint32_t split = degn - sb;
                h = split - below_cs;
                s = cnt - below_cs;
            }
        }
        uint32_t th, ts;
        const uint32_t eh = warp_excl_scan(h, &th);
        const uint32_t es = warp_excl_scan(s, &ts);
        if (c < ni) {
            g.it_H[item0 + c] = carryH + eh;
            g.it_S[item0 + c] = carryS + es;
        }
        carryH += th;
        carryS += ts;
    }
    if (lane == 0) {
        g.t_a[t].x = degn;
        const uint32_t nbn = divc(g.cmul, degn + C - 1);
        uint32_t lastb = NIL;
        if (nbn) {
            const uint32_t k = nbn - 1;
            lastb = __ldcg(g.it_bid + (size_t)(item0 + k / IB) * IB + (k % IB));
        }
        const uint32_t u = g.t_vid[t];
        g.sent[u] = make_uint4(degn, nbn, nbn ? root : NIL, lastb);
        removed += deg - degn;
        if (g.set_G && !g.seg_own) atomicAdd(&s_mhist[member_of(g.set_vbase, g.set_G, u)], deg - degn);
    }
}

template <int MODE, bool WEIGHTED = false>
__global__ void __launch_bounds__(256, 4) k_mark(GraphView g) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t nlo = dev->n_items, nhi = dev->n_mitems;
    const uint32_t nitems = nlo + nhi;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    const unsigned long long rqbb = g.rs ? qmod(dev->rq_back, g.RP) : 0ull;
    __shared__ uint32_t s_free[8][64];
    __shared__ uint32_t s_bid[8][32];
    __shared__ __align__(16) uint32_t s_hkey[8][2 * LIST_MAX];
    // queries: hit flag per list key; segmented deletes: owner segment per key
    __shared__ uint32_t s_hfound[8][(MODE == MODE_QUERY || MODE == MODE_DELETE) ? 2 * LIST_MAX : 1];
    const bool segd = MODE == MODE_DELETE && g.seg_own != nullptr;
    __shared__ uint32_t s_mhist[(MODE == MODE_QUERY) ? 1 : SET_MAX_G];
    if (MODE != MODE_QUERY && g.set_G) {
        for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x) s_mhist[i] = 0;
        __syncthreads();
    }
    FreeStage fs{s_free[threadIdx.x >> 5], 0u};
    unsigned long long removed = 0;  // entries deleted by this warp (lane 0)
    for (uint32_t vi = warp; vi < nitems; vi += nwarps) {
        const uint32_t it = item_at(g, vi, nlo, nhi);
        const uint2 itm = g.items[it];
        const uint32_t t = itm.x, c = itm.y;
        const uint4 a = g.t_a[t];
        if (a.z == CT_FLAG) continue;  // a source of the block-wide tier (k_mark_cta)
        const uint4 b = g.t_b[t];
        const uint32_t deg = b.x, nb = b.y, root = b.z, ni = b.w;
        const uint32_t kb = c * IB;
        const uint32_t nblk = min(IB, nb - kb);
        uint32_t bid = NIL;
        if (lane < nblk) bid = blk_at(g, root, kb + 1 + lane);
        if (__any_sync(FULL, lane < nblk && bid == NIL)) {
            if (lane == 0) latch_status(dev, 5u /* GV_ERR_STATE */);
            continue;
        }

        // Block ids of the item, one per lane, mirrored in shared memory so
        // that lanes can look up any block without a shuffle.
        uint32_t *sb_ids = s_bid[threadIdx.x >> 5];
        sb_ids[lane] = bid;
        __syncwarp();
        const uint32_t sbase = kb * C;
        const uint32_t nslots = min(nblk * C, deg - sbase);
        const uint32_t nquads = (nslots + 3) >> 2;
        // Each round streams 32 quads of the item's entries; the next
        // round's quad is loaded while this one is tested (software
        // pipelining: one load latency exposed per item instead of per
        // round), and the first round's is in flight while the batch list
        // below is built.  Prefetching is safe under compaction: a round's
        // writes go to slots at or below the slot it reads, never to the
        // next round's.
        uint4 e4n = make_uint4(EMPTY_KEY, EMPTY_KEY, EMPTY_KEY, EMPTY_KEY);
        if (lane < nquads) {
            const uint32_t xn = lane << 2, lbn = divc(g.cmul, xn);
            e4n = ld_stream4(reinterpret_cast<const uint4 *>(g.data + (size_t)sb_ids[lbn] * C + (xn - lbn * C)));
        }
        // Batch list of this source (<= LIST_MAX entries): a shared hash set
        // per warp of nsb buckets of 4 slots (nsb * 4 a power of two >= 2m,
        // at least 64 slots).  A key takes the first empty slot of its home
        // bucket (then of the next ones), so occupied slots are a prefix of
        // each bucket and a lookup is one 16-byte shared load.
        bool listmode = false;
        uint32_t nsb = 16;
        uint32_t *hk = s_hkey[threadIdx.x >> 5];
        uint32_t *hf = s_hfound[threadIdx.x >> 5];
        if (MODE == MODE_DELETE || MODE == MODE_QUERY) {
            listmode = (a.z == 0);
            if (listmode) {
                while (4 * nsb < 2 * a.x) nsb *= 2;
                for (uint32_t j = lane; j < 4 * nsb; j += 32) {
                    hk[j] = EMPTY_KEY;
                    if (MODE == MODE_QUERY) hf[j] = 0u;
                    if (segd) hf[j] = NIL;
                }
                __syncwarp();
                for (uint32_t j = lane; j < a.x; j += 32) {
                    const uint32_t v = g.arena[a.y + j];
                    uint32_t h = 4 * hidx(v, nsb);
                    // at most 2m keys in 4 * nsb >= 2m slots: a free or equal
                    // slot exists, so the walk ends within 4 * nsb steps
                    for (uint32_t step = 0; step < 4 * nsb; ++step) {
                        const uint32_t old = atomicCAS(&hk[h], EMPTY_KEY, v);
                        if (old == EMPTY_KEY || old == v) break;
                        h = (h + 1) & (4 * nsb - 1);
                    }
                    if (segd) atomicMin(&hf[h], g.seg_own[a.y + j]);
                }
            }
        }
        __syncwarp();
        const bool single = (ni == 1);
        uint32_t running = 0;
        for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
            const uint32_t q = q0 + lane;
            const bool qv = q < nquads;
            const uint32_t x = q << 2;
            const uint32_t lb = divc(g.cmul, x);
            const size_t qoff = qv ? (size_t)sb_ids[lb] * C + (x - lb * C) : 0;
            const uint4 e4 = e4n;
            e4n = make_uint4(EMPTY_KEY, EMPTY_KEY, EMPTY_KEY, EMPTY_KEY);
            if (q + 32 < nquads) {
                const uint32_t xn = (q + 32) << 2, lbn = divc(g.cmul, xn);
                e4n = ld_stream4(reinterpret_cast<const uint4 *>(g.data + (size_t)sb_ids[lbn] * C + (xn - lbn * C)));
            }
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
            // payloads of a weighted graph move with their entries: read in
            // the same round as the entries, before any compaction write
            uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
            if (WEIGHTED && MODE != MODE_QUERY && single && qv)
                w4 = ld_stream4(reinterpret_cast<const uint4 *>(g.wdata + qoff));
            uint32_t vmask = 0;  // bit j: entry j is a stored entry of this item
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (qv && (x + j < nslots)) vmask |= 1u << j;
            uint32_t hitm = 0;   // bit j: entry j is in the batch set
            if (MODE == MODE_VDEL) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (((vmask >> j) & 1u) && ((g.dead[e[j] >> 5] >> (e[j] & 31u)) & 1u)) hitm |= 1u << j;
            } else if (listmode) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((vmask >> j) & 1u) {
                        uint32_t b = hidx(e[j], nsb);
                        for (uint32_t step = 0; step < nsb; ++step) {
                            const uint4 w = *reinterpret_cast<const uint4 *>(hk + 4 * b);
                            const uint32_t k = w.x == e[j] ? 0u : w.y == e[j] ? 1u : w.z == e[j] ? 2u
                                             : w.w == e[j] ? 3u : NIL;
                            if (k != NIL) {
                                hitm |= 1u << j;
                                if (MODE == MODE_QUERY) hf[4 * b + k] = 1u;
                                if (segd) seg_count(s_mhist, hf[4 * b + k], g.set_G, dev);
                                break;
                            }
                            if (w.w == EMPTY_KEY) break;  // the bucket's prefix ended
                            b = (b + 1) & (nsb - 1);
                        }
                    }
                }
            } else {
                // global bucketed hash set.  Occupied slots of a bucket are a
                // prefix (inserts claim the first empty slot), so a lookup
                // reads the first half-bucket of the home buckets of all four
                // entries together and goes on to the second half, or the
                // next bucket, only past four occupied slots without the key
                const uint32_t *tab = g.arena + a.y;
                const uint32_t nbk = a.z / HB;
                const uint32_t need = vmask;
                uint4 x0[4];
                uint32_t bk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    bk[j] = hidx(e[j], nbk);
                    if ((need >> j) & 1u) x0[j] = *reinterpret_cast<const uint4 *>(tab + bk[j] * HB);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((need >> j) & 1u) {
                        uint4 w = x0[j];
                        uint32_t half = 0;  // 0: slots 0-3 of bucket bk[j]; 1: slots 4-7
                        for (uint32_t probe = 0; probe < 2 * nbk; ++probe) {
                            const uint32_t k = w.x == e[j] ? 0u : w.y == e[j] ? 1u : w.z == e[j] ? 2u
                                             : w.w == e[j] ? 3u : NIL;
                            if (k != NIL) {
                                hitm |= 1u << j;
                                if (MODE == MODE_QUERY) g.found[a.y + bk[j] * HB + half * 4 + k] = 1u;
                                if (segd) seg_count(s_mhist, g.seg_own[a.y + bk[j] * HB + half * 4 + k], g.set_G, dev);
                                break;
                            }
                            if (w.w == EMPTY_KEY) break;  // the prefix ended in this half
                            if (half == 0) {
                                half = 1;
                            } else {
                                half = 0;
                                bk[j] = (bk[j] + 1) & (nbk - 1);
                            }
                            w = *reinterpret_cast<const uint4 *>(tab + bk[j] * HB + half * 4);
                        }
                    }
                }
            }
            const uint32_t surv = vmask & ~hitm;
            if (MODE == MODE_QUERY) continue;
            uint32_t tot;
            const uint32_t ex = warp_excl_scan(__popc(surv), &tot);
            if (single) {
                // Stable in-place compaction: targets never pass the slot
                // being read, and each round reads before it writes.
                uint32_t w = running + ex;
                const uint32_t ew[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((surv >> j) & 1u) {
                        if (w != x + j) {
                            const uint32_t tq = divc(g.cmul, w);
                            const size_t to = (size_t)sb_ids[tq] * C + (w - tq * C);
                            g.data[to] = e[j];
                            if (WEIGHTED) g.wdata[to] = ew[j];
                        }
                        ++w;
                    }
                }
            } else {
                uint32_t word = surv << (4u * (lane & 7u));
                word |= __shfl_xor_sync(FULL, word, 1);
                word |= __shfl_xor_sync(FULL, word, 2);
                word |= __shfl_xor_sync(FULL, word, 4);
                if ((lane & 7u) == 0) g.it_mask[(size_t)it * MASK_WORDS + (q0 >> 3) + (lane >> 3)] = word;
            }
            running += tot;
        }
        if (MODE == MODE_QUERY) {
            __syncwarp();
            // every list entry (repeated queries included) reads its key's flag
            if (listmode) {
                for (uint32_t j = lane; j < a.x; j += 32) {
                    const uint32_t v = g.arena[a.y + j];
                    uint32_t h = 4 * hidx(v, nsb);
                    for (uint32_t step = 0; step < 4 * nsb && hk[h] != v; ++step) h = (h + 1) & (4 * nsb - 1);
                    if (hk[h] == v && hf[h]) g.found[a.y + j] = 1u;
                }
            }
            __syncwarp();
            continue;
        }
        if (single) {
            const uint32_t degn = running;
            if (degn != deg) {
                const uint32_t nbn = divc(g.cmul, degn + C - 1);
                const uint32_t k = lane + 1;
                const bool fr = lane < nblk && k > nbn;
                const bool run = is_run(root);  // a run source returns whole runs
                fs.push(fr && !run, bid, dev, g.queue, qbb, P);
                const uint32_t p = k >> 1;
                const uint32_t pb = __shfl_sync(FULL, bid, (p - 1) & 31u);
                const uint32_t lastb = __shfl_sync(FULL, bid, (nbn - 1) & 31u);
                if (fr && !run && p >= 1 && p <= nbn) g.links[2ull * pb + (k & 1u)] = NIL;
                if (fr && run) release_run(g, root, k, bid, nbn, rqbb);
                if (lane == 0) {
                    const uint32_t u = g.t_vid[t];
                    g.sent[u] = make_uint4(degn, nbn, nbn ? root : NIL, nbn ? lastb : NIL);
                    removed += deg - degn;
                    if (g.set_G && !g.seg_own) atomicAdd(&s_mhist[member_of(g.set_vbase, g.set_G, u)], deg - degn);
                }
            }
        } else {
            if (lane < nblk) g.it_bid[(size_t)it * IB + lane] = bid;
            if (lane == 0) g.it_cnt[it] = running;
        }
    }
    if (MODE != MODE_QUERY) {
        fs.flush(fs.n, dev, g.queue, qbb, P);
        if (lane == 0 && removed) atomicAdd(&dev->call_a, removed);
        if (g.set_G) {
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x)
                if (s_mhist[i]) atomicAdd(&g.set_counts[2 * i], (unsigned long long)s_mhist[i]);
        }
    }
}

// Tiny adjacencies, one thread per source: at most TINY_NB (8) blocks and
// min(TINY_DEG, TINY_NB * C) entries, at most TINY_M batch entries (held in
// registers).  Delete / vertex delete compact in place (stable) and return
// emptied blocks; query sets the hit flag of every matching batch entry.
struct Blocks8 {
    uint32_t b[TINY_NB];
    __device__ __forceinline__ uint32_t get(uint32_t i) const {
        uint32_t r = b[0];
#pragma unroll
        for (uint32_t k = 1; k < TINY_NB; ++k)
            if (i == k) r = b[k];
        return r;
    }
};

template <int MODE>
__global__ void __launch_bounds__(256) k_mark_tiny(GraphView g) {
    pdl_wait();
    // Vertex deletes visit every vertex id directly (no touched list: the
    // incoming-edge pass covers all live vertices); other modes visit the
    // planned tiny sources.
    constexpr bool DIRECT = MODE == MODE_VDEL;
    Dev *dev = g.dev;
    const uint32_t nlo = DIRECT ? g.nv : dev->n_tiny, nhi = DIRECT ? 0u : dev->n_tiny_hi;
    const uint32_t ntiny = nlo + nhi;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    const uint32_t C = g.C;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    const unsigned long long rqbb = g.rs ? qmod(dev->rq_back, g.RP) : 0ull;
    __shared__ uint32_t s_free[8][64];
    __shared__ uint32_t s_mhist[(MODE == MODE_QUERY) ? 1 : SET_MAX_G];
    if (MODE != MODE_QUERY && g.set_G) {
        for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x) s_mhist[i] = 0;
        __syncthreads();
    }
    FreeStage fs{s_free[threadIdx.x >> 5], 0u};
    unsigned long long removed = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // the loop bound is uniform per warp: the queue staging needs all lanes
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < ntiny; base += stride) {
        const uint32_t k = base + lane_id();
        bool act = k < ntiny;
        uint32_t t = 0, deg = 0, nb = 0, root = NIL, m = 0, aoff = 0;
        if (DIRECT) {
            if (act) act = g.alive[k] != 0;
            if (act) {
                const uint4 sv = g.sent[k];
                deg = sv.x;
                nb = sv.y;
                root = sv.z;
                act = deg > 0 && deg <= tiny_deg && nb <= TINY_NB;
            }
        } else if (act) {
            t = g.t_tiny[k < nlo ? k : (uint32_t)(g.tiny_cap - nhi + (k - nlo))];
            const uint4 a = g.t_a[t];
            const uint4 b = g.t_b[t];
            deg = b.x;
            nb = b.y;
            root = b.z;
            m = a.x;
            aoff = a.y;
        }
        // heap index h (1-based) lives in bl.b[h-1]; children of h are 2h, 2h+1
        // (a run source's first TINY_NB blocks all lie in its first run,
        // R >= TINY_NB: consecutive ids from the head)
        const bool run = is_run(root);
        Blocks8 bl;
#pragma unroll
        for (uint32_t h = 0; h < TINY_NB; ++h) bl.b[h] = NIL;
        bl.b[0] = run ? root & ~RUN_BIT : root;
        bool bad = act && bl.b[0] >= P;
#pragma unroll
        for (uint32_t h = 2; h <= TINY_NB; ++h) {
            if (act && !bad && h <= nb) {
                const uint32_t parent = bl.b[h / 2 - 1];
                const uint32_t c = run ? bl.b[0] + (h - 1) : g.links[2ull * parent + (h & 1u)];
                bl.b[h - 1] = c;
                if (c >= P) bad = true;
            }
        }
        if (bad) {
            latch_status(dev, 5u /* GV_ERR_STATE */);
            act = false;
        }
        uint32_t d[TINY_M];
        // 64-bit signature of the batch entries (bit hidx(v, 64) per entry):
        // a stored entry whose bit is clear is in no batch entry, which
        // spares the 16 comparisons for most entries
        unsigned long long sig = 0;
#pragma unroll
        for (int j = 0; j < (int)TINY_M; ++j) {
            d[j] = (MODE != MODE_VDEL && act && (uint32_t)j < m) ? g.arena[aoff + j] : EMPTY_KEY;
            if (d[j] != EMPTY_KEY) sig |= 1ull << hidx(d[j], 64);
        }
        uint32_t qhit = 0;
        uint32_t w = 0;
        // Two quads of stored entries in flight per step: both are read
        // before either is processed, which is safe because the stable
        // in-place compaction writes only to slots w <= the slot being read.
        for (uint32_t x0 = 0; act && x0 < deg; x0 += 8) {
            uint4 eq[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t x = x0 + 4 * h;
                eq[h] = make_uint4(NIL, NIL, NIL, NIL);
                if (x < deg) {
                    const uint32_t bi = divc(g.cmul, x);
                    eq[h] = ld_stream4(reinterpret_cast<const uint4 *>(g.data + (size_t)bl.get(bi) * C + (x - bi * C)));
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t x = x0 + 4 * h;
                const uint32_t e[4] = {eq[h].x, eq[h].y, eq[h].z, eq[h].w};
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (x + jj < deg) {
                        bool hit;
                        if (MODE == MODE_VDEL) {
                            hit = (g.dead[e[jj] >> 5] >> (e[jj] & 31u)) & 1u;
                        } else {
                            uint32_t hm = 0;
                            if ((sig >> hidx(e[jj], 64)) & 1ull) {
#pragma unroll
                                for (int j = 0; j < (int)TINY_M; ++j) hm |= (uint32_t)(d[j] == e[jj]) << j;
                            }
                            hit = hm != 0;
                            if (MODE == MODE_QUERY) qhit |= hm;
                            if (MODE == MODE_DELETE && hit && g.seg_own) {
                                uint32_t own = NIL;
                                for (uint32_t r = hm; r; r &= r - 1) own = min(own, g.seg_own[aoff + __ffs(r) - 1]);
                                seg_count(s_mhist, own, g.set_G, dev);
                            }
                        }
                        if (MODE != MODE_QUERY && !hit) {
                            if (w != x + jj) {
                                const uint32_t wi = divc(g.cmul, w);
                                const size_t to = (size_t)bl.get(wi) * C + (w - wi * C);
                                g.data[to] = e[jj];
                                if (g.wdata) {
                                    // one thread owns the adjacency and no write has reached
                                    // slot x + jj yet: its payload is still in place
                                    const uint32_t bi = divc(g.cmul, x);
                                    g.wdata[to] = g.wdata[(size_t)bl.get(bi) * C + (x - bi * C) + jj];
                                }
                            }
                            ++w;
                        }
                    }
                }
            }
        }
        if (MODE == MODE_QUERY) {
            if (act)
                for (uint32_t j = 0; j < m; ++j)
                    if ((qhit >> j) & 1u) g.found[aoff + j] = 1u;
            continue;
        }
        const bool changed = act && w != deg;
        const uint32_t nbn = divc(g.cmul, w + C - 1);
        // blocks past the new count return to the queue; a freed block's
        // parent, if still owned, forgets it
#pragma unroll
        for (uint32_t h = TINY_NB; h >= 1; --h) {
            const bool fr = changed && h <= nb && h > nbn;
            fs.push(fr && !run, bl.b[h - 1], dev, g.queue, qbb, P);
            if (fr && !run && h >= 2 && h / 2 <= nbn) g.links[2ull * bl.b[h / 2 - 1] + (h & 1u)] = NIL;
        }
        if (changed && run && nbn == 0) push_run(g, bl.b[0], rqbb);  // emptied: its only run returns
        if (changed) {
            const uint32_t u = DIRECT ? k : g.t_vid[t];
            g.sent[u] = make_uint4(w, nbn, nbn ? root : NIL, nbn ? bl.get(nbn - 1) : NIL);
            removed += deg - w;
            if (g.set_G && !g.seg_own) atomicAdd(&s_mhist[member_of(g.set_vbase, g.set_G, u)], deg - w);
        }
    }
    if (MODE != MODE_QUERY) {
        fs.flush(fs.n, dev, g.queue, qbb, P);
        removed = warp_sum_u64(removed);
        if (lane_id() == 0 && removed) atomicAdd(&dev->call_a, removed);
        if (g.set_G) {
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x)
                if (s_mhist[i]) atomicAdd(&g.set_counts[2 * i], (unsigned long long)s_mhist[i]);
        }
    }
}

// One warp per multi-item source.
// One warp per multi-item source.
template <int MODE>
__global__ void __launch_bounds__(256) k_vscan(GraphView g) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    __shared__ uint32_t s_mhist[SET_MAX_G];
    if (g.set_G) {
        for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x) s_mhist[i] = 0;
        __syncthreads();
    }
    unsigned long long removed = 0;
    // multi-item sources own the top nhi items; visit each source once, at
    // its first item
    const uint32_t nhi = dev->n_mitems;
    for (uint32_t vi = warp; vi < nhi; vi += nwarps) {
        const uint2 first = g.items[g.max_items - nhi + vi];
        if (first.y != 0) continue;
        const uint32_t t = first.x;
        if (g.t_b[t].w <= 1) continue;
        vscan_source(g, t, s_mhist, removed);
    }
    if (lane == 0 && removed) atomicAdd(&dev->call_a, removed);
    if (g.set_G) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < g.set_G; i += blockDim.x)
            if (s_mhist[i]) atomicAdd(&g.set_counts[2 * i], (unsigned long long)s_mhist[i]);
    }
}

// One warp per item of a multi-item source.
template <int MODE>
__global__ void __launch_bounds__(256) k_move(GraphView g) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t nhi = dev->n_mitems;  // items of multi-item sources (top region)
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB, SPI = IB * C;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    const unsigned long long rqbb = g.rs ? qmod(dev->rq_back, g.RP) : 0ull;
    __shared__ uint32_t s_free[8][64];
    FreeStage fs{s_free[threadIdx.x >> 5], 0u};
    for (uint32_t vi = warp; vi < nhi; vi += nwarps) {
        const uint32_t it = (uint32_t)(g.max_items - nhi + vi);
        const uint2 itm = g.items[it];
        const uint32_t t = itm.x, c = itm.y;
        const uint4 b = g.t_b[t];
        const uint32_t ni = b.w;
        if (ni <= 1) continue;
        const uint4 a = g.t_a[t];
        const uint32_t degn = a.x, item0 = a.w, deg = b.x, nb = b.y;
        const uint32_t nbn = divc(g.cmul, degn + C - 1);
        const uint32_t sb = c * SPI;
        const uint32_t len = min(SPI, deg - sb);
        const uint32_t *mk = g.it_mask + (size_t)it * MASK_WORDS;
        const uint32_t *bids = g.it_bid + (size_t)it * IB;
        if (sb < degn) {
            const uint32_t lim = min(len, degn - sb);
            uint32_t hrank = g.it_H[it];
            for (uint32_t w0 = 0; w0 < lim; w0 += 32) {
                const uint32_t x = w0 + lane;
                const uint32_t word = mk[w0 >> 5];
                const bool hole = x < lim && !((word >> lane) & 1u);
                const unsigned bal = __ballot_sync(FULL, hole);
                if (hole) {
                    const uint32_t gr = hrank + __popc(bal & ((1u << lane) - 1u));
                    uint32_t lo = 0, hi = ni;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (g.it_S[item0 + mid] <= gr) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo == 0) {
                        latch_status(dev, 5u /* GV_ERR_STATE */);
                        continue;
                    }
                    const uint32_t cs = lo - 1;
                    uint32_t r = gr - g.it_S[item0 + cs];
                    const uint32_t sbs = cs * SPI;
                    const uint32_t split = degn > sbs ? degn - sbs : 0u;
                    const uint32_t lens = min(SPI, deg - sbs);
                    const uint32_t *mks = g.it_mask + (size_t)(item0 + cs) * MASK_WORDS;
                    uint32_t pos = NIL;
                    for (uint32_t w = split >> 5; w * 32 < lens; ++w) {
                        uint32_t word2 = mks[w];
                        if (w == (split >> 5)) word2 &= ~((1u << (split & 31u)) - 1u);
                        const uint32_t remain = lens - w * 32;
                        if (remain < 32) word2 &= (1u << remain) - 1u;
                        const uint32_t pc = __popc(word2);
                        if (r < pc) {
                            for (uint32_t z = 0; z < r; ++z) word2 &= word2 - 1u;
                            pos = w * 32 + (uint32_t)(__ffs(word2) - 1);
                            break;
                        }
                        r -= pc;
                    }
                    const uint32_t pq = pos != NIL ? divc(g.cmul, pos) : 0u, xq = divc(g.cmul, x);
                    const uint32_t srcb = pos != NIL ? g.it_bid[(size_t)(item0 + cs) * IB + pq] : NIL;
                    const uint32_t dstb = bids[xq];
                    if (pos != NIL && srcb < P && dstb < P) {
                        const size_t from = (size_t)srcb * C + (pos - pq * C);
                        const size_t to = (size_t)dstb * C + (x - xq * C);
                        g.data[to] = g.data[from];
                        if (g.wdata) g.wdata[to] = g.wdata[from];
                    } else {
                        latch_status(dev, 5u /* GV_ERR_STATE */);
                    }
                }
                hrank += __popc(bal);
            }
        }
        const uint32_t kb = c * IB;
        const uint32_t nblk = min(IB, nb - kb);
        const uint32_t k = kb + 1 + lane;
        const bool fr = lane < nblk && k > nbn;
        const bool run = is_run(b.z);  // a run source returns whole runs
        fs.push(fr && !run, fr ? bids[lane] : NIL, dev, g.queue, qbb, P);
        if (fr && run) release_run(g, b.z, k, bids[lane], nbn, rqbb);
        if (fr && !run) {
            const uint32_t p = k >> 1;
            if (p >= 1 && p <= nbn) {
                const uint32_t pb = g.it_bid[(size_t)(item0 + (p - 1) / IB) * IB + (p - 1) % IB];
                g.links[2ull * pb + (k & 1u)] = NIL;
            }
        }
    }
    fs.flush(fs.n, dev, g.queue, qbb, P);
}

__global__ void __launch_bounds__(256) k_query_out(GraphView g, unsigned long long n, uint8_t *out) {
    pdl_wait();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = g.qpos[i];
        out[i] = (p != NIL && g.found[p]) ? 1 : 0;
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_finalize_member(GraphView g, unsigned long long *counts) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t nt = dev->n_touched;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint32_t u = g.t_vid[t];
        g.vcnt[vidx(g, u)] = 0;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        if (MODE == MODE_DELETE) {
            const unsigned long long del = dev->call_a, rej = dev->call_b;
            dev->q_back += dev->free_total;
            dev->rq_back += dev->rfree_total;
            dev->num_edges -= del;
            dev->tot_del += del;
            dev->tot_rej += rej;
            if (counts) {
                counts[0] = del;
                counts[1] = rej;
            }
        }
        dev->alloc_total = 0;
        dev->call_a = dev->call_b = dev->call_c = 0;
        dev->n_touched = 0;
        dev->n_items = 0;
        dev->n_mitems = 0;
        dev->n_tiny = 0;
        dev->n_tiny_hi = 0;
        dev->arena_used = 0;
        dev->harena_used = 0;
        dev->n_chunks = 0;
        dev->n_groups = 0;
        dev->n_hash = 0;
        dev->free_total = 0;
        dev->ralloc_total = 0;
        dev->rfree_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ----------------------------------------------------------- vertex delete

__global__ void __launch_bounds__(256) k_vdel_mark(GraphView g, const uint32_t *__restrict__ ids,
                                                   uint32_t k) {
    pdl_wait();
    for (uint32_t base = blockIdx.x * blockDim.x; base < k; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool own = false;
        uint32_t id = NIL;
        if (i < k) {
            id = ids[i];
            if (id < g.nv) {
                const uint32_t bit = 1u << (id & 31u);
                const uint32_t old = atomicOr(&g.dead[id >> 5], bit);
                own = !(old & bit) && g.alive[id];
            }
        }
        const uint32_t t = warp_atomic_add<unsigned int>(&g.dev->n_touched, 1u, own);
        if (own) {
            g.alive[id] = 0;
            g.t_vid[t] = id;
        }
    }
}

// Deleted vertices: their blocks become items to free; sentinels cleared.
__global__ void __launch_bounds__(256) k_plan_vfree(GraphView g) {
    pdl_wait();
    const uint32_t nt = g.dev->n_touched;
    const uint32_t IB = g.IB;
    __shared__ uint32_t s_ai;
    unsigned long long removed = 0;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t ni = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            s = g.sent[g.t_vid[t]];
            ni = (s.y + IB - 1) / IB;
            removed += s.x;
        }
        uint32_t itot;
        const uint32_t iex = block_excl_scan(ni, &itot);
        if (threadIdx.x == 0) s_ai = itot ? atomicAdd(&g.dev->n_items, itot) : 0u;
        __syncthreads();
        if (t < nt) {
            const uint32_t item0 = s_ai + iex;
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            g.t_a[t] = make_uint4(0, 0, 0, item0);
            emit_items(g, t, item0, ni);
            g.sent[g.t_vid[t]] = make_uint4(0, 0, NIL, NIL);
        }
        __syncthreads();
    }
    const unsigned long long r = warp_sum_u64(removed);
    if (lane_id() == 0 && r) atomicAdd(&g.dev->call_a, r);
}

__global__ void __launch_bounds__(256) k_free_items(GraphView g) {
    pdl_wait();
    Dev *dev = g.dev;
    const uint32_t nitems = dev->n_items;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t IB = g.IB;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    const unsigned long long rqbb = g.rs ? qmod(dev->rq_back, g.RP) : 0ull;
    __shared__ uint32_t s_free[8][64];
    FreeStage fs{s_free[threadIdx.x >> 5], 0u};
    for (uint32_t it = warp; it < nitems; it += nwarps) {
        const uint2 itm = g.items[it];
        const uint4 b = g.t_b[itm.x];
        const uint32_t kb = itm.y * IB;
        const uint32_t nblk = min(IB, b.y - kb);
        const bool fr = lane < nblk;
        const bool run = is_run(b.z);
        uint32_t bid = NIL;
        if (fr) bid = blk_at(g, b.z, kb + 1 + lane);
        if (fr && bid == NIL) latch_status(dev, 5u /* GV_ERR_STATE */);
        fs.push(fr && bid != NIL && !run, bid, dev, g.queue, qbb, P);
        // a run source: each run's head block returns the run
        if (fr && bid != NIL && run && ((kb + lane) & ((1u << g.rs) - 1u)) == 0u) push_run(g, bid, rqbb);
    }
    fs.flush(fs.n, dev, g.queue, qbb, P);
}

// Between the two phases of a vertex delete: the touched list and the item
// list are rebuilt for the incoming-edge pass.
__global__ void k_reset_lists(GraphView g) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        g.dev->n_touched = 0;
        g.dev->n_items = 0;
        g.dev->n_mitems = 0;
        g.dev->n_tiny = 0;
        g.dev->n_tiny_hi = 0;
    }
}

// Every live vertex with edges becomes a touched source of the incoming-edge
// pass (its entries are tested against the deleted-id bitmap).
__global__ void __launch_bounds__(256) k_plan_vdel_in(GraphView g) {
    pdl_wait();
    const uint32_t nv = g.nv;
    const uint32_t IB = g.IB;
    const uint32_t tiny_deg = min(TINY_DEG, TINY_NB * g.C);
    __shared__ uint32_t s_at, s_ai, s_am;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nv; base += gridDim.x * blockDim.x) {
        const uint32_t u = base + threadIdx.x;
        uint32_t take = 0, ni = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (u < nv && g.alive[u]) {
            s = g.sent[u];
            // tiny adjacencies are handled by k_mark_tiny straight from the
            // dictionary; only the others become touched sources with items
            if (s.x && !(s.x <= tiny_deg && s.y <= TINY_NB)) {
                take = 1;
                ni = (s.y + IB - 1) / IB;
            }
        }
        uint32_t ttot;
        const uint32_t tex = block_excl_scan(take, &ttot);
        if (threadIdx.x == 0) s_at = ttot ? atomicAdd(&g.dev->n_touched, ttot) : 0u;
        const uint32_t item0 = alloc_items(g, ni, &s_ai, &s_am);
        if (take) {
            const uint32_t t = s_at + tex;
            g.t_vid[t] = u;
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            g.t_a[t] = make_uint4(0, 0, 0, item0);
            emit_items(g, t, item0, ni);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_finalize_vdel(GraphView g, const uint32_t *__restrict__ ids,
                                                       uint32_t k) {
    pdl_wait();
    Dev *dev = g.dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t id = ids[i];
        if (id < g.nv) g.dead[id >> 5] = 0u;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        const unsigned long long del = dev->call_a;
        dev->q_back += dev->free_total;
        dev->rq_back += dev->rfree_total;
        dev->num_edges -= del;
        dev->tot_del += del;
        dev->alloc_total = 0;
        dev->call_a = dev->call_b = dev->call_c = 0;
        dev->n_touched = 0;
        dev->n_items = 0;
        dev->n_mitems = 0;
        dev->n_tiny = 0;
        dev->n_tiny_hi = 0;
        dev->arena_used = 0;
        dev->harena_used = 0;
        dev->n_chunks = 0;
        dev->n_groups = 0;
        dev->n_hash = 0;
        dev->free_total = 0;
        dev->ralloc_total = 0;
        dev->rfree_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ------------------------------------------------------ set-semantics insert

// After the membership pass over the batch (hit flags = value already
// stored): pair i is inserted iff it claimed its value's slot (first of its
// repeats in the batch) and the value is not stored yet; every other pair
// gets source NIL so that the insert that follows skips it.
__global__ void __launch_bounds__(256) k_dedup_select(GraphView g, const uint32_t *__restrict__ src,
                                                      unsigned long long n, uint32_t *src2,
                                                      unsigned long long *cnt) {
    pdl_wait();
    unsigned long long k = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = g.qpos[i];
        const bool take = p != NIL && g.pflag[i] && !g.found[p];
        src2[i] = take ? src[i] : NIL;
        k += take;
    }
    k = warp_sum_u64(k);
    if (lane_id() == 0 && k) atomicAdd(cnt, k);
}

__global__ void k_copy_rejects(Dev *dev, unsigned long long *tmp) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) tmp[0] = dev->call_b;
}

// Final counts of a set-semantics insert: {inserted, rejected pairs of the
// caller's batch}; the insert's own reject count (which includes the skipped
// repeats) is taken back out of the running total.
__global__ void k_dedup_counts(Dev *dev, const unsigned long long *tmp, unsigned long long n,
                               unsigned long long *counts) {
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        // tmp[0] = rejected by the grouping pass, tmp[2..3] = {inserted, rejected} of the insert
        const unsigned long long ins = tmp[2], rej2 = tmp[3], rej = tmp[0];
        if (rej2 >= rej) dev->tot_rej -= rej2 - rej;
        if (counts) {
            counts[0] = ins;
            counts[1] = (ins == 0 && rej2 == 0 && n != 0) ? 0ull : rej;  // {0, 0} when the insert aborted
        }
    }
}

// ---------------------------------------------------------------- graph sets

// Concatenated member batches -> one batch over the set's shared dictionary:
// the source becomes base(member) + u, the destination stays member-local
// (stored entries of a member are its own ids).  A pair with an endpoint
// outside its member's range is rejected here (source NIL) and counted for
// its member.
__global__ void __launch_bounds__(256) k_set_remap(GraphView g, const uint32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ dst, unsigned long long n,
                                                   uint32_t *gsrc, uint32_t *gdst) {
    pdl_wait();
    __shared__ unsigned long long s_off[SET_MAX_G + 1];
    __shared__ uint32_t s_base[SET_MAX_G + 1];
    __shared__ uint32_t s_rej[SET_MAX_G];
    const uint32_t G = g.set_G;
    for (uint32_t i = threadIdx.x; i <= G; i += blockDim.x) {
        s_off[i] = g.set_off[i];
        s_base[i] = g.set_vbase[i];
        if (i < G) s_rej[i] = 0;
    }
    __syncthreads();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = G;  // s_off[lo] <= i < s_off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_off[mid] <= i) lo = mid;
            else hi = mid;
        }
        const uint32_t u = ld_stream(src + i), v = ld_stream(dst + i);
        const uint32_t nvm = s_base[lo + 1] - s_base[lo];
        const bool ok = u < nvm && v < nvm;
        gsrc[i] = ok ? s_base[lo] + u : NIL;
        gdst[i] = v;
        if (!ok) atomicAdd(&s_rej[lo], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x)
        if (s_rej[i]) atomicAdd(&g.set_counts[2 * i + 1], (unsigned long long)s_rej[i]);
}

// Per-segment counts of a batch made of several requests on one graph:
// {valid pairs, rejected pairs} per segment (segments = consecutive pair
// ranges, offsets in set_off; multiset inserts insert every valid pair).
__global__ void __launch_bounds__(256) k_segment_counts(GraphView g, const uint32_t *__restrict__ src,
                                                        const uint32_t *__restrict__ dst, unsigned long long n) {
    pdl_wait();
    __shared__ unsigned long long s_off[SET_MAX_G + 1];
    __shared__ uint32_t s_rej[SET_MAX_G];
    const uint32_t G = g.set_G;
    for (uint32_t i = threadIdx.x; i <= G; i += blockDim.x) {
        s_off[i] = g.set_off[i];
        if (i < G) s_rej[i] = 0;
    }
    __syncthreads();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t u = src[i], v = dst[i];
        const bool ok = u < g.nv && v < g.nv && (g.all_alive || (g.alive[u] && g.alive[v]));
        if (!ok) {
            uint32_t lo = 0, hi = G;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_off[mid] <= i) lo = mid;
                else hi = mid;
            }
            atomicAdd(&s_rej[lo], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x)
        if (s_rej[i]) atomicAdd(&g.set_counts[2 * i + 1], (unsigned long long)s_rej[i]);
}

// Inserted pairs per member (multiset): its batch size minus its rejects.
__global__ void k_set_insert_counts(GraphView g) {
    pdl_wait();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.set_G; i += gridDim.x * blockDim.x)
        g.set_counts[2 * i] = (g.set_off[i + 1] - g.set_off[i]) - g.set_counts[2 * i + 1];
}

cudaError_t launch_set_remap(const GraphView &g, const uint32_t *src, const uint32_t *dst, unsigned long long n,
                             uint32_t *gsrc, uint32_t *gdst, const LaunchCfg &lc);
cudaError_t launch_set_insert_counts(const GraphView &g, const LaunchCfg &lc);

// ------------------------------------------------------------------ launch


// Counting pass over pairs [lo, hi) of a batch of n_total pairs (the path --
// per-pair atomics or per-tile aggregation -- follows n_total, so the
// pieces of one batch all take the same one).
cudaError_t launch_count_range(int mode, const GraphView &g0, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n_total, unsigned long long lo, unsigned long long hi,
                               const LaunchCfg &lc) {
    const int ph = mode == MODE_INSERT ? PH_INS_COUNT : mode == MODE_DELETE ? PH_DEL_COUNT : PH_QRY_COUNT;
    if (hi <= lo) return cudaSuccess;
    GraphView g = g0;
    g.prank = g0.prank + lo;  // ranks are written at the pair's index
    src += lo;
    dst += lo;
    const unsigned long long n = hi - lo;
    PhaseScope ps(lc, ph);
    if (n_total >= ((unsigned long long)g.nv >> g.dense_shift)) {
        // large batch: per-pair atomics (the touched list follows the pass)
        const int grid = grid_for(n, 256 * CD_PER, lc.num_sms * GRID_MULT);
        switch (mode) {
        case MODE_INSERT: launch_pdl(k_count_direct<MODE_INSERT>, grid, 256, 0, lc.stream, g, src, dst, n); break;
        case MODE_DELETE: launch_pdl(k_count_direct<MODE_DELETE>, grid, 256, 0, lc.stream, g, src, dst, n); break;
        default: launch_pdl(k_count_direct<MODE_QUERY>, grid, 256, 0, lc.stream, g, src, dst, n); break;
        }
    } else {
        // small batch: per-tile aggregation, touched list appended on the fly
        const int grid = grid_for(n, AGG_TILE, lc.num_sms * GRID_MULT);
        switch (mode) {
        case MODE_INSERT: launch_pdl(k_count<MODE_INSERT>, grid, AGG_THREADS, 0, lc.stream, g, src, dst, n); break;
        case MODE_DELETE: launch_pdl(k_count<MODE_DELETE>, grid, AGG_THREADS, 0, lc.stream, g, src, dst, n); break;
        default: launch_pdl(k_count<MODE_QUERY>, grid, AGG_THREADS, 0, lc.stream, g, src, dst, n); break;
        }
    }
    return cudaGetLastError();
}

// After every piece of a batch is counted: the touched list of a large
// batch (a pass over the vertex counters).
cudaError_t launch_count_finish(int mode, const GraphView &g, unsigned long long n_total, const LaunchCfg &lc) {
    const int ph = mode == MODE_INSERT ? PH_INS_COUNT : mode == MODE_DELETE ? PH_DEL_COUNT : PH_QRY_COUNT;
    if (n_total >= ((unsigned long long)g.nv >> g.dense_shift)) {
        PhaseScope ps(lc, ph + 1);  // the touched-list phase follows each count phase
        launch_pdl(k_touched_scan, grid_for(g.vmask + 1ull, 1024, lc.num_sms * GRID_MULT), 256, 0, lc.stream, g);
    }
    return cudaGetLastError();
}

cudaError_t launch_count(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                         unsigned long long n, const LaunchCfg &lc) {
    cudaError_t e = launch_count_range(mode, g, src, dst, n, 0, n, lc);
    if (e != cudaSuccess) return e;
    return launch_count_finish(mode, g, n, lc);
}

cudaError_t launch_count_rejects(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                 unsigned long long n, unsigned long long *rejected,
                                 const LaunchCfg &lc) {
    launch_pdl(k_count_rejects, grid_for(n, 256, lc.num_sms * GRID_MULT), 256, 0, lc.stream, g, src, dst, n, rejected);
    return cudaGetLastError();
}

cudaError_t launch_insert_small(const GraphView &g, const uint32_t *src, const uint32_t *dst, const uint32_t *wts,
                                unsigned long long n, unsigned long long *counts, const LaunchCfg &lc) {
    if (n == 0 || n > SMALL_INS) return cudaErrorInvalidValue;
    // the shared-memory opt-in is per function and device
    static bool attr_set[64][2] = {};
    int devc = 0;
    if (cudaGetDevice(&devc) != cudaSuccess || devc < 0 || devc >= 64) return cudaErrorInvalidDevice;
    const int w = g.wdata ? 1 : 0;
    if (!attr_set[devc][w]) {
        const cudaError_t e = w ? cudaFuncSetAttribute(k_insert_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)SMALL_SMEM)
                                : cudaFuncSetAttribute(k_insert_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)SMALL_SMEM);
        if (e != cudaSuccess) return e;
        attr_set[devc][w] = true;
    }
    PhaseScope ps(lc, PH_INS_SMALL);
    if (w) launch_pdl(k_insert_small<true>, 1, SMALL_THREADS, SMALL_SMEM, lc.stream, g, src, dst, wts, (uint32_t)n, counts);
    else launch_pdl(k_insert_small<false>, 1, SMALL_THREADS, SMALL_SMEM, lc.stream, g, src, dst, wts, (uint32_t)n, counts);
    return cudaGetLastError();
}

uint32_t small_insert_max() { return SMALL_INS; }

cudaError_t launch_insert_tail(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, const LaunchCfg &lc, const uint32_t *wts) {
    const int cap = lc.num_sms * GRID_MULT;
    // a batch of n pairs touches at most n sources: small batches launch
    // small grids (grid-stride loops cover any count)
    const int gt = grid_for(tcap < n ? tcap : n, 256, cap);
    {
        PhaseScope ps(lc, PH_INS_PLAN);
        if (g.grouped) launch_gp_plan_insert(g, gt, lc);
        else launch_pdl(k_plan_insert, gt, 256, 0, lc.stream, g);
    }
    const unsigned long long max_pops = n / g.C + (tcap < n ? tcap : n) + 1;  // new blocks: <= n/C + sources
    {
        PhaseScope ps(lc, PH_INS_LINK);
        launch_pdl(k_link_insert, grid_for(max_pops, 256, cap), 256, 0, lc.stream, g);
    }
    if (g.grouped) {
        // the grouped batch goes straight from its chunks into the slots
        const cudaError_t e = launch_group_place(MODE_INSERT, g, n, lc);
        if (e != cudaSuccess) return e;
    } else {
        PhaseScope ps(lc, PH_INS_SCATTER);
        if (g.wdata) launch_pdl(k_scatter_insert<true>, grid_for(n, 256 * PP, cap), 256, 0, lc.stream, g, src, dst, wts, n);
        else launch_pdl(k_scatter_insert<false>, grid_for(n, 256 * PP, cap), 256, 0, lc.stream, g, src, dst, wts, n);
    }
    {
        PhaseScope ps(lc, PH_INS_FINALIZE);
        launch_pdl(k_finalize_insert, gt, 256, 0, lc.stream, g, n, counts);
    }
    return cudaGetLastError();
}

template <int MODE>
static void member_tail(const GraphView &g0, const uint32_t *src, const uint32_t *dst,
                        unsigned long long n, unsigned long long tcap, unsigned long long *counts,
                        uint8_t *qout, const LaunchCfg &lc, bool small) {
    GraphView g = g0;
    g.hbase = (uint32_t)((n + 63) / 64 * 64);  // lists below (at most n words), hash sets above

    const int cap = lc.num_sms * GRID_MULT;
    // grids follow the batch: at most n touched sources; work items start at
    // one per source (grid-stride loops cover sources with many items)
    const unsigned long long nt = tcap < n ? tcap : n;
    const int gt = grid_for(nt, 256, cap);
    const int gi = grid_for(4 * nt + 256, 8, lc.num_sms * GRID_MULT);  // warp-per-item kernels: 8 warps per CTA
    const bool del = MODE == MODE_DELETE;
    if (g.grouped) {
        // the grouping already placed every source's batch list in the arena
        // (and filled the hash sets of sources past CT_KEYS batch entries)
        PhaseScope ps(lc, del ? PH_DEL_PLAN : PH_QRY_PLAN);
        launch_gp_plan_member(MODE, g, gt, lc);
    } else if (small) {
        // one CTA groups, plans and places the batch (k_member_small)
        PhaseScope ps(lc, del ? PH_DEL_PLAN : PH_QRY_PLAN);
        launch_pdl(k_member_small<MODE>, 1, SMALL_MEM_THREADS, SMALL_MEM_SMEM, lc.stream, g, src, dst, (uint32_t)n);
    } else {
        {
            PhaseScope ps(lc, del ? PH_DEL_PLAN : PH_QRY_PLAN);
            launch_pdl(k_plan_member<MODE>, gt, 256, 0, lc.stream, g);
        }
        {
            PhaseScope ps(lc, del ? PH_DEL_ARENA : PH_QRY_ARENA);
            launch_pdl(k_arena_init<MODE>, grid_for(5 * n + 64, 256, cap), 256, 0, lc.stream, g);
        }
        PhaseScope ps(lc, del ? PH_DEL_SCATTER : PH_QRY_SCATTER);
        launch_pdl(k_scatter_member<MODE>, grid_for(n, 256 * PP_MEMBER, cap), 256, 0, lc.stream, g, src, dst, n);
    }
    // The two tiers touch disjoint sources (their blocks, sentinels and list
    // ranges) and share only atomically updated counters, so the thread-per-
    // source tier runs on the graph's second stream beside the warp tier
    // (measured faster at every batch size from 1K pairs up, L2 cold).
    const bool fork = lc.side && lc.fork && lc.join;
    if (fork) {
        cudaEventRecord(lc.fork, lc.stream);
        cudaStreamWaitEvent(lc.side, lc.fork, 0);
        LaunchCfg ls = lc;
        ls.stream = lc.side;
        PhaseScope ps(ls, del ? PH_DEL_MARK_TINY : PH_QRY_MARK_TINY);
        k_mark_tiny<MODE><<<gt, 256, 0, lc.side>>>(g);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_MARK : PH_QRY_MARK);
        if (MODE != MODE_QUERY && g.wdata) launch_pdl(k_mark<MODE, true>, gi, 256, 0, lc.stream, g);
        else launch_pdl(k_mark<MODE>, gi, 256, 0, lc.stream, g);
    }
    // sources with more than LIST_MAX batch entries (grouped path only):
    // disjoint from the warp tier's sources
    if (g.grouped) {
        launch_mark_cta(MODE, g, nt, lc);
        if (!del) launch_gp_hash_found(g, lc);
    }
    if (!fork) {
        PhaseScope ps(lc, del ? PH_DEL_MARK_TINY : PH_QRY_MARK_TINY);
        launch_pdl(k_mark_tiny<MODE>, gt, 256, 0, lc.stream, g);
    }
    if (del) {
        // the hole filling of multi-item sources does not touch tiny sources
        // either: the side stream joins only before the finalize
        {
            PhaseScope ps(lc, PH_DEL_VSCAN);
            launch_pdl(k_vscan<MODE>, grid_for(nt, 8, cap), 256, 0, lc.stream, g);
        }
        PhaseScope ps(lc, PH_DEL_MOVE);
        launch_pdl(k_move<MODE>, gi, 256, 0, lc.stream, g);
    }
    if (fork) {
        cudaEventRecord(lc.join, lc.side);
        cudaStreamWaitEvent(lc.stream, lc.join, 0);
    }
    // the first kernel after the join is an ordinary launch: it waits for
    // the side stream's work through the event, not for one predecessor grid
    if (!del) {
        PhaseScope ps(lc, PH_QRY_OUT);
        if (fork) k_query_out<<<grid_for(n, 256, cap), 256, 0, lc.stream>>>(g, n, qout);
        else launch_pdl(k_query_out, grid_for(n, 256, cap), 256, 0, lc.stream, g, n, qout);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_FINALIZE : PH_QRY_FINALIZE);
        if (fork && del) k_finalize_member<MODE><<<gt, 256, 0, lc.stream>>>(g, counts);
        else launch_pdl(k_finalize_member<MODE>, gt, 256, 0, lc.stream, g, counts);
    }
}

cudaError_t launch_member_tail(int mode, const GraphView &g, const uint32_t *src,
                               const uint32_t *dst, unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, uint8_t *qout, const LaunchCfg &lc) {
    if (mode == MODE_DELETE) member_tail<MODE_DELETE>(g, src, dst, n, tcap, counts, qout, lc, false);
    else member_tail<MODE_QUERY>(g, src, dst, n, tcap, counts, qout, lc, false);
    return cudaGetLastError();
}

uint64_t small_member_max() { return SMALL_MEM; }

cudaError_t launch_member_small(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                unsigned long long n, unsigned long long tcap, unsigned long long *counts,
                                uint8_t *qout, const LaunchCfg &lc) {
    if (n == 0 || n > SMALL_MEM || g.grouped || g.set_G || g.seg_own) return cudaErrorInvalidValue;
    // the shared-memory opt-in is per function and device
    static bool attr_set[64][2] = {};
    int devc = 0;
    if (cudaGetDevice(&devc) != cudaSuccess || devc < 0 || devc >= 64) return cudaErrorInvalidDevice;
    const int q = mode == MODE_QUERY ? 1 : 0;
    if (!attr_set[devc][q]) {
        const cudaError_t e = q ? cudaFuncSetAttribute(k_member_small<MODE_QUERY>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_MEM_SMEM)
                                : cudaFuncSetAttribute(k_member_small<MODE_DELETE>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_MEM_SMEM);
        if (e != cudaSuccess) return e;
        attr_set[devc][q] = true;
    }
    if (mode == MODE_DELETE) member_tail<MODE_DELETE>(g, src, dst, n, tcap, counts, qout, lc, true);
    else member_tail<MODE_QUERY>(g, src, dst, n, tcap, counts, qout, lc, true);
    return cudaGetLastError();
}

cudaError_t launch_vertex_delete(const GraphView &g, const uint32_t *ids, uint32_t k,
                                 const LaunchCfg &lc) {
    const int cap = lc.num_sms * GRID_MULT;
    const int gi = lc.num_sms * GRID_MULT;
    PhaseScope ps(lc, PH_VDEL);
    k_vdel_mark<<<grid_for(k, 256, cap), 256, 0, lc.stream>>>(g, ids, k);
    launch_pdl(k_plan_vfree, grid_for(k, 256, cap), 256, 0, lc.stream, g);
    launch_pdl(k_free_items, gi, 256, 0, lc.stream, g);
    launch_pdl(k_reset_lists, 1, 32, 0, lc.stream, g);
    launch_pdl(k_plan_vdel_in, grid_for(g.nv, 256, cap), 256, 0, lc.stream, g);
    // disjoint tiers, as in deletes: the thread-per-source one on the side stream
    const bool fork = lc.side && lc.fork && lc.join;
    if (fork) {
        cudaEventRecord(lc.fork, lc.stream);
        cudaStreamWaitEvent(lc.side, lc.fork, 0);
        k_mark_tiny<MODE_VDEL><<<grid_for(g.nv, 256, cap), 256, 0, lc.side>>>(g);
        cudaEventRecord(lc.join, lc.side);
    }
    if (g.wdata) launch_pdl(k_mark<MODE_VDEL, true>, gi, 256, 0, lc.stream, g);
    else launch_pdl(k_mark<MODE_VDEL>, gi, 256, 0, lc.stream, g);
    if (!fork) launch_pdl(k_mark_tiny<MODE_VDEL>, grid_for(g.nv, 256, cap), 256, 0, lc.stream, g);
    launch_pdl(k_vscan<MODE_VDEL>, grid_for(g.nv, 8, cap), 256, 0, lc.stream, g);
    launch_pdl(k_move<MODE_VDEL>, gi, 256, 0, lc.stream, g);
    if (fork) cudaStreamWaitEvent(lc.stream, lc.join, 0);
    k_finalize_vdel<<<grid_for(k, 256, cap), 256, 0, lc.stream>>>(g, ids, k);
    return cudaGetLastError();
}

}  // namespace gv

namespace gv {
cudaError_t launch_set_remap(const GraphView &g, const uint32_t *src, const uint32_t *dst, unsigned long long n,
                             uint32_t *gsrc, uint32_t *gdst, const LaunchCfg &lc) {
    if (n == 0) return cudaSuccess;
    PhaseScope ps(lc, PH_OTHER);
    unsigned long long blocks = (n + 2047) / 2048;
    const unsigned long long cap = (unsigned long long)lc.num_sms * GRID_MULT;
    if (blocks > cap) blocks = cap;
    k_set_remap<<<(int)blocks, 256, 0, lc.stream>>>(g, src, dst, n, gsrc, gdst);
    return cudaGetLastError();
}
cudaError_t launch_segment_counts(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                  unsigned long long n, const LaunchCfg &lc) {
    if (n == 0) return cudaSuccess;
    unsigned long long blocks = (n + 2047) / 2048;
    const unsigned long long cap = (unsigned long long)lc.num_sms * GRID_MULT;
    if (blocks > cap) blocks = cap;
    k_segment_counts<<<(int)blocks, 256, 0, lc.stream>>>(g, src, dst, n);
    return cudaGetLastError();
}
// After a segmented insert: its totals {inserted, rejected} are {0, 0} only
// when the call was a no-op (pool exhausted); then every segment gets {0, 0}.
__global__ void k_segment_noop_check(GraphView g, const unsigned long long *tot, unsigned long long n) {
    pdl_wait();
    if (tot[0] != 0 || tot[1] != 0 || n == 0) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * g.set_G; i += gridDim.x * blockDim.x)
        g.set_counts[i] = 0;
}

cudaError_t launch_segment_noop_check(const GraphView &g, const unsigned long long *tot, unsigned long long n,
                                      const LaunchCfg &lc) {
    launch_pdl(k_segment_noop_check, (2 * g.set_G + 255) / 256, 256, 0, lc.stream, g, tot, n);
    return cudaGetLastError();
}

cudaError_t launch_set_insert_counts(const GraphView &g, const LaunchCfg &lc) {
    launch_pdl(k_set_insert_counts, (g.set_G + 255) / 256, 256, 0, lc.stream, g);
    return cudaGetLastError();
}
}  // namespace gv

namespace gv {
cudaError_t launch_dedup_insert_prepare(const GraphView &g0, const uint32_t *src, const uint32_t *dst,
                                        unsigned long long n, unsigned long long tcap, uint32_t *src2,
                                        unsigned long long *tmp, const LaunchCfg &lc) {
    // tmp[0]: pairs rejected by the grouping pass; tmp[1]: pairs selected
    // Every source gets a hash set (no list region): dedup_words(m) <= 8m
    // words, so the arena needs at most 8n words from hbase = 0.
    GraphView g = g0;
    g.hbase = 0;
    const int cap = lc.num_sms * GRID_MULT;
    const unsigned long long nt = tcap < n ? tcap : n;
    const int gt = grid_for(nt, 256, cap);
    const int gi = grid_for(4 * nt + 256, 8, cap);
    launch_pdl(k_plan_member<MODE_DEDUP>, gt, 256, 0, lc.stream, g);
    launch_pdl(k_arena_init<MODE_DEDUP>, grid_for(8 * n + 64, 256, cap), 256, 0, lc.stream, g);
    launch_pdl(k_scatter_member<MODE_DEDUP>, grid_for(n, 256 * PP_MEMBER, cap), 256, 0, lc.stream, g, src, dst, n);
    launch_pdl(k_mark<MODE_QUERY>, gi, 256, 0, lc.stream, g);
    launch_pdl(k_dedup_select, grid_for(n, 256, cap), 256, 0, lc.stream, g, src, n, src2, tmp + 1);
    launch_pdl(k_copy_rejects, 1, 32, 0, lc.stream, g.dev, tmp);
    launch_pdl(k_finalize_member<MODE_QUERY>, gt, 256, 0, lc.stream, g, nullptr);
    return cudaGetLastError();
}
cudaError_t launch_dedup_counts(Dev *dev, const unsigned long long *tmp, unsigned long long n,
                                unsigned long long *counts, const LaunchCfg &lc) {
    launch_pdl(k_dedup_counts, 1, 32, 0, lc.stream, dev, tmp, n, counts);
    return cudaGetLastError();
}
}  // namespace gv

namespace gv {
// Clears the per-call state of a counting pass whose batch is not applied
// (the first batch of a set-semantics graph, counted only to fix C).
cudaError_t launch_finalize_count_only(const GraphView &g, const LaunchCfg &lc) {
    launch_pdl(k_finalize_member<MODE_QUERY>, grid_for(g.nv, 256, lc.num_sms * GRID_MULT), 256, 0, lc.stream, g, nullptr);
    return cudaGetLastError();
}
}  // namespace gv

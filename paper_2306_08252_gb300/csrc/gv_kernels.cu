// gv_kernels.cu -- the GraphVine batch kernels for sm_103a.
//
// Every batch operation (insert, delete, query) starts by grouping the batch
// by source vertex on the device.  The paper converts each batch to CSR on
// the host before copying it over ("Initialization and batch updates"); here
// a counting pass aggregates each tile of pairs in a shared-memory hash table
// and adds one count per (tile, source) into a per-vertex counter, so hub
// vertices do not serialise on one global atomic per edge.  The first source
// to see a zero count appends itself to the call's touched list, which plays
// the role of the CSR row list.
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
//   scatter each pair gets rank r among its source's batch pairs (per-tile
//           rank + one atomic cursor per (tile, source)); r < space goes to
//           the last block at slot deg mod C + r, the rest to new block
//           (r - space) / C, slot (r - space) mod C.
//   final   sentinels updated; the queue front advances by the blocks popped.
//
// Delete (Algorithm 2) and query (Algorithm 3) share one membership pipeline:
//   plan    per touched source: its batch destinations go to a list (<= 32
//           entries) or an open-addressing hash set (> 32) in an arena; its
//           blocks are cut into work items of IB blocks (IB * C <= 512 slots).
//   scatter batch destinations into the lists / hash sets.
//   mark    one warp per item: resolve the item's block ids by walking the
//           CBT, stream the entries with 16-byte loads, test membership
//           (binary search over a warp-sorted list, or a hash probe).  Query
//           sets hit flags.  Delete compacts single-item adjacencies in place
//           (stable) and frees their emptied tail blocks; multi-item
//           adjacencies record a survivor bitmask per item.
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

__device__ __forceinline__ unsigned long long ring(unsigned long long base, unsigned long long off,
                                                   unsigned long long P) {
    unsigned long long q = base + off;
    return q >= P ? q - P : q;
}

// ---------------------------------------------------------------- grouping

template <int MODE>
__global__ void __launch_bounds__(AGG_THREADS) k_count(GraphView g, const uint32_t *__restrict__ src,
                                                       const uint32_t *__restrict__ dst,
                                                       unsigned long long n) {
    __shared__ uint32_t keys[AGG_H];
    __shared__ uint32_t cnt[AGG_H];
    unsigned long long rej = 0;
    const unsigned long long ntiles = (n + AGG_TILE - 1) / AGG_TILE;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < AGG_H; i += AGG_THREADS) {
            keys[i] = EMPTY_KEY;
            cnt[i] = 0;
        }
        __syncthreads();
        const unsigned long long base = tile * AGG_TILE;
        uint32_t us[AGG_EPT], vs[AGG_EPT];
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            us[e] = i < n ? __ldg(src + i) : NIL;
            vs[e] = i < n ? __ldg(dst + i) : NIL;
        }
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            if (i < n) {
                if (valid_pair(g, us[e], vs[e])) {
                    uint32_t r;
                    agg_insert(keys, cnt, us[e], r);
                } else {
                    ++rej;
                }
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < AGG_H; s += AGG_THREADS) {
            const uint32_t u = keys[s];
            bool isnew = false;
            if (u != EMPTY_KEY) isnew = atomicAdd(&g.vcnt[u], cnt[s]) == 0u;
            const uint32_t t = warp_atomic_add<unsigned int>(&g.dev->n_touched, 1u, isnew);
            if (isnew) {
                g.t_vid[t] = u;
                g.vtid[u] = t;
            }
        }
        __syncthreads();
    }
    if (MODE != MODE_QUERY) {
        const unsigned long long r = warp_sum_u64(rej);
        if (lane_id() == 0 && r) atomicAdd(&g.dev->call_b, r);
    }
}

__global__ void __launch_bounds__(256) k_count_rejects(GraphView g, const uint32_t *__restrict__ src,
                                                       const uint32_t *__restrict__ dst,
                                                       unsigned long long n, unsigned long long *rejected) {
    unsigned long long rej = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        if (!valid_pair(g, src[i], dst[i])) ++rej;
    rej = warp_sum_u64(rej);
    if (lane_id() == 0 && rej) atomicAdd(rejected, rej);
}

// ------------------------------------------------------------------ insert

__global__ void __launch_bounds__(256) k_plan_insert(GraphView g) {
    const uint32_t nt = g.dev->n_touched;
    const uint32_t C = g.C;
    __shared__ unsigned long long s_base;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t need = 0, deg = 0, last = NIL;
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            const uint32_t cnt = g.vcnt[u];
            const uint4 s = g.sent[u];
            deg = s.x;
            last = s.w;
            const uint32_t space = s.y * C - deg;
            need = cnt > space ? (cnt - space + C - 1) / C : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(need, &tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(&g.dev->alloc_total, (unsigned long long)tot) : 0ull;
        __syncthreads();
        const unsigned long long off = s_base + ex;
        if (t < nt) {
            g.t_a[t] = make_uint4(deg, last, (uint32_t)off, need);
            for (uint32_t j = 0; j < need; ++j) g.t_owner[off + j] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_link_insert(GraphView g) {
    Dev *dev = g.dev;
    const unsigned long long total = dev->alloc_total;
    const unsigned long long qf = dev->q_front, qb = dev->q_back;
    if (total > qb - qf) {
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
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < total;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t t = g.t_owner[j];
        const uint4 a = g.t_a[t];
        const uint32_t deg = a.x, off = a.z, need = a.w;
        const uint32_t nb = (deg + C - 1) / C;
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

__global__ void __launch_bounds__(AGG_THREADS) k_scatter_insert(GraphView g,
                                                                const uint32_t *__restrict__ src,
                                                                const uint32_t *__restrict__ dst,
                                                                unsigned long long n) {
    if (g.dev->abort) return;
    __shared__ uint32_t keys[AGG_H];
    __shared__ uint32_t cnt[AGG_H];
    __shared__ uint32_t tid[AGG_H];
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(g.dev->q_front, P);
    const uint32_t C = g.C;
    const unsigned long long ntiles = (n + AGG_TILE - 1) / AGG_TILE;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < AGG_H; i += AGG_THREADS) {
            keys[i] = EMPTY_KEY;
            cnt[i] = 0;
        }
        __syncthreads();
        const unsigned long long base = tile * AGG_TILE;
        uint32_t vs[AGG_EPT], slot[AGG_EPT], rank[AGG_EPT];
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            const uint32_t u = i < n ? __ldg(src + i) : NIL;
            vs[e] = i < n ? __ldg(dst + i) : NIL;
            slot[e] = NIL;
            if (i < n && valid_pair(g, u, vs[e])) slot[e] = agg_insert(keys, cnt, u, rank[e]);
        }
        __syncthreads();
        for (int s = threadIdx.x; s < AGG_H; s += AGG_THREADS) {
            const uint32_t u = keys[s];
            if (u != EMPTY_KEY) {
                cnt[s] = atomicAdd(&g.vcur[u], cnt[s]);
                tid[s] = g.vtid[u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            if (slot[e] != NIL) {
                const uint32_t r = cnt[slot[e]] + rank[e];
                const uint4 a = g.t_a[tid[slot[e]]];
                const uint32_t deg = a.x, last = a.y, off = a.z;
                const uint32_t nb = (deg + C - 1) / C;
                const uint32_t space = nb * C - deg;
                uint32_t b, lane;
                if (r < space) {
                    b = last;
                    lane = deg - (nb - 1) * C + r;
                } else {
                    const uint32_t q = r - space;
                    const uint32_t jb = q / C;
                    lane = q - jb * C;
                    b = g.queue[ring(qbase, off + jb, P)];
                }
                if (b < P) g.data[(size_t)b * C + lane] = vs[e];
                else latch_status(g.dev, 5u /* GV_ERR_STATE */);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_finalize_insert(GraphView g, unsigned long long n,
                                                         unsigned long long *counts) {
    Dev *dev = g.dev;
    const uint32_t nt = dev->n_touched;
    const bool abort = dev->abort != 0;
    const unsigned long long P = g.P;
    const unsigned long long qbase = qmod(dev->q_front, P);
    const uint32_t C = g.C;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint32_t u = g.t_vid[t];
        const uint32_t cnt = g.vcnt[u];
        if (!abort) {
            const uint4 a = g.t_a[t];
            const uint32_t deg = a.x, off = a.z, need = a.w;
            const uint32_t nb = (deg + C - 1) / C;
            uint4 s = g.sent[u];
            s.x = deg + cnt;
            s.y = nb + need;
            if (need) {
                if (nb == 0) s.z = g.queue[ring(qbase, off, P)];
                s.w = g.queue[ring(qbase, off + need - 1, P)];
            }
            g.sent[u] = s;
        }
        g.vcnt[u] = 0;
        g.vcur[u] = 0;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        unsigned long long rej = dev->call_b;
        unsigned long long ins = n - rej;
        if (abort) {
            ins = 0;
            rej = 0;
        } else {
            dev->q_front += dev->alloc_total;
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
        dev->arena_used = 0;
        dev->free_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ------------------------------------------------------ membership pipeline

// Items over the blocks of one touched source: t_b[t] = {deg, nblocks, root,
// items}; t_a[t].w = first item.  Returns nothing; writes the item list.
__device__ __forceinline__ void emit_items(const GraphView &g, uint32_t t, uint32_t item0,
                                           uint32_t ni) {
    for (uint32_t c = 0; c < ni; ++c) g.items[item0 + c] = make_uint2(t, c);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_plan_member(GraphView g) {
    const uint32_t nt = g.dev->n_touched;
    const uint32_t IB = g.IB;
    __shared__ unsigned long long s_aw;
    __shared__ uint32_t s_ai;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nt; base += gridDim.x * blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t m = 0, words = 0, hs = 0, ni = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (t < nt) {
            const uint32_t u = g.t_vid[t];
            m = g.vcnt[u];
            s = g.sent[u];
            if (m <= 32) {
                words = m;
            } else {
                hs = 64;
                while (hs < 2 * m) hs <<= 1;
                words = hs;
            }
            ni = (s.y + IB - 1) / IB;
        }
        uint32_t wt, itot;
        const uint32_t wex = block_excl_scan(words, &wt);
        const uint32_t iex = block_excl_scan(ni, &itot);
        if (threadIdx.x == 0) {
            s_aw = wt ? atomicAdd(&g.dev->arena_used, (unsigned long long)wt) : 0ull;
            s_ai = itot ? atomicAdd(&g.dev->n_items, itot) : 0u;
        }
        __syncthreads();
        if (t < nt) {
            const uint32_t item0 = s_ai + iex;
            g.t_a[t] = make_uint4(m, (uint32_t)(s_aw + wex), hs, item0);
            g.t_b[t] = make_uint4(s.x, s.y, s.z, ni);
            emit_items(g, t, item0, ni);
        }
        __syncthreads();
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_arena_init(GraphView g) {
    const unsigned long long used = g.dev->arena_used;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < used;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        g.arena[i] = EMPTY_KEY;
        if (MODE == MODE_QUERY) g.found[i] = 0u;
    }
}

template <int MODE>
__global__ void __launch_bounds__(AGG_THREADS) k_scatter_member(GraphView g,
                                                                const uint32_t *__restrict__ src,
                                                                const uint32_t *__restrict__ dst,
                                                                unsigned long long n) {
    __shared__ uint32_t keys[AGG_H];
    __shared__ uint32_t cnt[AGG_H];
    __shared__ uint32_t tid[AGG_H];
    const unsigned long long ntiles = (n + AGG_TILE - 1) / AGG_TILE;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < AGG_H; i += AGG_THREADS) {
            keys[i] = EMPTY_KEY;
            cnt[i] = 0;
        }
        __syncthreads();
        const unsigned long long base = tile * AGG_TILE;
        uint32_t vs[AGG_EPT], slot[AGG_EPT], rank[AGG_EPT];
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            const uint32_t u = i < n ? __ldg(src + i) : NIL;
            vs[e] = i < n ? __ldg(dst + i) : NIL;
            slot[e] = NIL;
            if (i < n && valid_pair(g, u, vs[e])) slot[e] = agg_insert(keys, cnt, u, rank[e]);
        }
        __syncthreads();
        for (int s = threadIdx.x; s < AGG_H; s += AGG_THREADS) {
            const uint32_t u = keys[s];
            if (u != EMPTY_KEY) {
                cnt[s] = atomicAdd(&g.vcur[u], cnt[s]);
                tid[s] = g.vtid[u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < AGG_EPT; ++e) {
            const unsigned long long i = base + (unsigned long long)e * AGG_THREADS + threadIdx.x;
            if (slot[e] != NIL) {
                const uint32_t r = cnt[slot[e]] + rank[e];
                const uint4 a = g.t_a[tid[slot[e]]];
                uint32_t pos;
                if (a.z == 0) {
                    pos = a.y + r;
                    g.arena[pos] = vs[e];
                } else {
                    pos = a.y + hash_insert(g.arena + a.y, a.z, vs[e]);
                }
                if (MODE == MODE_QUERY) g.qpos[i] = pos;
            } else if (MODE == MODE_QUERY && i < n) {
                g.qpos[i] = NIL;
            }
        }
        __syncthreads();
    }
}

// One warp per work item (see the file comment).
template <int MODE>
__global__ void __launch_bounds__(256) k_mark(GraphView g) {
    Dev *dev = g.dev;
    const uint32_t nitems = dev->n_items;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    for (uint32_t it = warp; it < nitems; it += nwarps) {
        const uint2 itm = g.items[it];
        const uint32_t t = itm.x, c = itm.y;
        const uint4 a = g.t_a[t];
        const uint4 b = g.t_b[t];
        const uint32_t deg = b.x, nb = b.y, root = b.z, ni = b.w;
        const uint32_t kb = c * IB;
        const uint32_t nblk = min(IB, nb - kb);
        uint32_t bid = NIL;
        if (lane < nblk) bid = cbt_walk(g.links, P, root, kb + 1 + lane);
        if (__any_sync(FULL, lane < nblk && bid == NIL)) {
            if (lane == 0) latch_status(dev, 5u /* GV_ERR_STATE */);
            continue;
        }

        bool listmode = false;
        uint32_t skey = EMPTY_KEY, spay = lane;
        if (MODE == MODE_DELETE || MODE == MODE_QUERY) {
            listmode = (a.z == 0);
            if (listmode) {
                if (lane < a.x) skey = g.arena[a.y + lane];
                warp_sort_pairs(skey, spay);
            }
        }
        const uint32_t sbase = kb * C;
        const uint32_t nslots = min(nblk * C, deg - sbase);
        const uint32_t nquads = (nslots + 3) >> 2;
        const bool single = (ni == 1);
        uint32_t running = 0;
        uint32_t qfound = 0;
        for (uint32_t q0 = 0; q0 < nquads; q0 += 32) {
            const uint32_t q = q0 + lane;
            const bool qv = q < nquads;
            const uint32_t x = q << 2;
            const uint32_t lb = x / C;
            const uint32_t myb = __shfl_sync(FULL, bid, lb & 31u);
            uint4 e4 = make_uint4(EMPTY_KEY, EMPTY_KEY, EMPTY_KEY, EMPTY_KEY);
            if (qv) e4 = *reinterpret_cast<const uint4 *>(g.data + (size_t)myb * C + (x - lb * C));
            const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
            uint32_t surv = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool valid = qv && (x + j < nslots);
                bool hit = false;
                if (MODE == MODE_VDEL) {
                    if (valid) hit = (g.dead[e[j] >> 5] >> (e[j] & 31u)) & 1u;
                } else if (listmode) {
                    const uint32_t pos = warp_lower_bound(skey, e[j]);
                    const uint32_t kk = __shfl_sync(FULL, skey, pos);
                    hit = valid && kk == e[j];
                    if (MODE == MODE_QUERY) qfound |= __reduce_or_sync(FULL, hit ? (1u << pos) : 0u);
                } else if (valid) {
                    const uint32_t h = hash_find(g.arena + a.y, a.z, e[j]);
                    hit = h != NIL;
                    if (MODE == MODE_QUERY && hit) g.found[a.y + h] = 1u;
                }
                if (valid && !hit) surv |= 1u << j;
            }
            if (MODE == MODE_QUERY) continue;
            uint32_t tot;
            const uint32_t ex = warp_excl_scan(__popc(surv), &tot);
            if (single) {
                // Stable in-place compaction: targets never pass the slot
                // being read, and each round reads before it writes.
                uint32_t w = running + ex;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool sj = (surv >> j) & 1u;
                    const uint32_t tq = w / C;
                    const uint32_t tb = __shfl_sync(FULL, bid, tq & 31u);
                    if (sj && w != x + j) g.data[(size_t)tb * C + (w - tq * C)] = e[j];
                    if (sj) ++w;
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
            if (listmode) {
                // Hits were recorded at the first sorted position of each key;
                // equal keys (repeated queries) share that position's bit.
                const uint32_t first = warp_lower_bound(skey, skey);
                if (lane < a.x && ((qfound >> first) & 1u)) g.found[a.y + spay] = 1u;
            }
            continue;
        }
        if (single) {
            const uint32_t degn = running;
            if (degn != deg) {
                const uint32_t nbn = (degn + C - 1) / C;
                const uint32_t k = lane + 1;
                const bool fr = lane < nblk && k > nbn;
                const unsigned long long fpos = warp_atomic_add<unsigned long long>(&dev->free_total, 1u, fr);
                const uint32_t p = k >> 1;
                const uint32_t pb = __shfl_sync(FULL, bid, (p - 1) & 31u);
                const uint32_t lastb = __shfl_sync(FULL, bid, (nbn - 1) & 31u);
                if (fr) {
                    g.queue[ring(qbb, fpos, P)] = bid;
                    if (p >= 1 && p <= nbn) g.links[2ull * pb + (k & 1u)] = NIL;
                }
                if (lane == 0) {
                    g.sent[g.t_vid[t]] = make_uint4(degn, nbn, nbn ? root : NIL, nbn ? lastb : NIL);
                    atomicAdd(&dev->call_a, (unsigned long long)(deg - degn));
                }
            }
        } else {
            if (lane < nblk) g.it_bid[(size_t)it * IB + lane] = bid;
            if (lane == 0) g.it_cnt[it] = running;
        }
    }
}

// One warp per multi-item source.
template <int MODE>
__global__ void __launch_bounds__(256) k_vscan(GraphView g) {
    Dev *dev = g.dev;
    const uint32_t nt = dev->n_touched;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB, SPI = IB * C;
    for (uint32_t t = warp; t < nt; t += nwarps) {
        const uint4 b = g.t_b[t];
        const uint32_t ni = b.w;
        if (ni <= 1) continue;
        const uint32_t item0 = g.t_a[t].w;
        const uint32_t deg = b.x, root = b.z;
        uint32_t tot = 0;
        for (uint32_t c = lane; c < ni; c += 32) tot += g.it_cnt[item0 + c];
        const uint32_t degn = warp_sum(tot);
        uint32_t carryH = 0, carryS = 0;
        for (uint32_t c0 = 0; c0 < ni; c0 += 32) {
            const uint32_t c = c0 + lane;
            uint32_t h = 0, s = 0;
            if (c < ni) {
                const uint32_t sb = c * SPI;
                const uint32_t len = min(SPI, deg - sb);
                const uint32_t cnt = g.it_cnt[item0 + c];
                if (sb + len <= degn) {
                    h = len - cnt;
                } else if (sb >= degn) {
                    s = cnt;
                } else {
                    const uint32_t split = degn - sb;
                    const uint32_t *mk = g.it_mask + (size_t)(item0 + c) * MASK_WORDS;
                    uint32_t below = 0;
                    for (uint32_t w = 0; w * 32 < split; ++w) {
                        uint32_t word = mk[w];
                        const uint32_t nbits = split - w * 32;
                        if (nbits < 32) word &= (1u << nbits) - 1u;
                        below += __popc(word);
                    }
                    h = split - below;
                    s = cnt - below;
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
            const uint32_t nbn = (degn + C - 1) / C;
            uint32_t lastb = NIL;
            if (nbn) {
                const uint32_t k = nbn - 1;
                lastb = g.it_bid[(size_t)(item0 + k / IB) * IB + (k % IB)];
            }
            g.sent[g.t_vid[t]] = make_uint4(degn, nbn, nbn ? root : NIL, lastb);
            if (deg != degn) atomicAdd(&dev->call_a, (unsigned long long)(deg - degn));
        }
    }
}

// One warp per item of a multi-item source.
template <int MODE>
__global__ void __launch_bounds__(256) k_move(GraphView g) {
    Dev *dev = g.dev;
    const uint32_t nitems = dev->n_items;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t C = g.C, IB = g.IB, SPI = IB * C;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    for (uint32_t it = warp; it < nitems; it += nwarps) {
        const uint2 itm = g.items[it];
        const uint32_t t = itm.x, c = itm.y;
        const uint4 b = g.t_b[t];
        const uint32_t ni = b.w;
        if (ni <= 1) continue;
        const uint4 a = g.t_a[t];
        const uint32_t degn = a.x, item0 = a.w, deg = b.x, nb = b.y;
        const uint32_t nbn = (degn + C - 1) / C;
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
                    if (pos != NIL) {
                        const uint32_t srcb = g.it_bid[(size_t)(item0 + cs) * IB + pos / C];
                        const uint32_t val = g.data[(size_t)srcb * C + pos % C];
                        const uint32_t dstb = bids[x / C];
                        g.data[(size_t)dstb * C + x % C] = val;
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
        const unsigned long long fpos = warp_atomic_add<unsigned long long>(&dev->free_total, 1u, fr);
        if (fr) {
            g.queue[ring(qbb, fpos, P)] = bids[lane];
            const uint32_t p = k >> 1;
            if (p >= 1 && p <= nbn) {
                const uint32_t pb = g.it_bid[(size_t)(item0 + (p - 1) / IB) * IB + (p - 1) % IB];
                g.links[2ull * pb + (k & 1u)] = NIL;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_query_out(GraphView g, unsigned long long n, uint8_t *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = g.qpos[i];
        out[i] = (p != NIL && g.found[p]) ? 1 : 0;
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_finalize_member(GraphView g, unsigned long long *counts) {
    Dev *dev = g.dev;
    const uint32_t nt = dev->n_touched;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint32_t u = g.t_vid[t];
        g.vcnt[u] = 0;
        g.vcur[u] = 0;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        if (MODE == MODE_DELETE) {
            const unsigned long long del = dev->call_a, rej = dev->call_b;
            dev->q_back += dev->free_total;
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
        dev->arena_used = 0;
        dev->free_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ----------------------------------------------------------- vertex delete

__global__ void __launch_bounds__(256) k_vdel_mark(GraphView g, const uint32_t *__restrict__ ids,
                                                   uint32_t k) {
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
    Dev *dev = g.dev;
    const uint32_t nitems = dev->n_items;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t IB = g.IB;
    const unsigned long long P = g.P;
    const unsigned long long qbb = qmod(dev->q_back, P);
    for (uint32_t it = warp; it < nitems; it += nwarps) {
        const uint2 itm = g.items[it];
        const uint4 b = g.t_b[itm.x];
        const uint32_t kb = itm.y * IB;
        const uint32_t nblk = min(IB, b.y - kb);
        const bool fr = lane < nblk;
        uint32_t bid = NIL;
        if (fr) bid = cbt_walk(g.links, P, b.z, kb + 1 + lane);
        if (fr && bid == NIL) latch_status(dev, 5u /* GV_ERR_STATE */);
        const unsigned long long fpos = warp_atomic_add<unsigned long long>(&dev->free_total, 1u, fr);
        if (fr && bid != NIL) g.queue[ring(qbb, fpos, P)] = bid;
    }
}

// Between the two phases of a vertex delete: the touched list and the item
// list are rebuilt for the incoming-edge pass.
__global__ void k_reset_lists(GraphView g) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        g.dev->n_touched = 0;
        g.dev->n_items = 0;
    }
}

// Every live vertex with edges becomes a touched source of the incoming-edge
// pass (its entries are tested against the deleted-id bitmap).
__global__ void __launch_bounds__(256) k_plan_vdel_in(GraphView g) {
    const uint32_t nv = g.nv;
    const uint32_t IB = g.IB;
    __shared__ uint32_t s_at, s_ai;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nv; base += gridDim.x * blockDim.x) {
        const uint32_t u = base + threadIdx.x;
        uint32_t take = 0, ni = 0;
        uint4 s = make_uint4(0, 0, NIL, NIL);
        if (u < nv && g.alive[u]) {
            s = g.sent[u];
            if (s.x) {
                take = 1;
                ni = (s.y + IB - 1) / IB;
            }
        }
        uint32_t ttot, itot;
        const uint32_t tex = block_excl_scan(take, &ttot);
        const uint32_t iex = block_excl_scan(ni, &itot);
        if (threadIdx.x == 0) {
            s_at = ttot ? atomicAdd(&g.dev->n_touched, ttot) : 0u;
            s_ai = itot ? atomicAdd(&g.dev->n_items, itot) : 0u;
        }
        __syncthreads();
        if (take) {
            const uint32_t t = s_at + tex;
            const uint32_t item0 = s_ai + iex;
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
    Dev *dev = g.dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t id = ids[i];
        if (id < g.nv) g.dead[id >> 5] = 0u;
    }
    if (last_cta(dev) && threadIdx.x == 0) {
        const unsigned long long del = dev->call_a;
        dev->q_back += dev->free_total;
        dev->num_edges -= del;
        dev->tot_del += del;
        dev->alloc_total = 0;
        dev->call_a = dev->call_b = dev->call_c = 0;
        dev->n_touched = 0;
        dev->n_items = 0;
        dev->arena_used = 0;
        dev->free_total = 0;
        dev->abort = 0;
        dev->done_ctas = 0;
    }
}

// ------------------------------------------------------------------ launch

namespace {
inline int grid_for(unsigned long long work, int per_block, int cap) {
    unsigned long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (unsigned long long)cap) g = cap;
    return (int)g;
}
}  // namespace

cudaError_t launch_count(int mode, const GraphView &g, const uint32_t *src, const uint32_t *dst,
                         unsigned long long n, const LaunchCfg &lc) {
    const int grid = grid_for(n, AGG_TILE, lc.num_sms * 8);
    const int ph = mode == MODE_INSERT ? PH_INS_COUNT : mode == MODE_DELETE ? PH_DEL_COUNT : PH_QRY_COUNT;
    PhaseScope ps(lc, ph);
    switch (mode) {
    case MODE_INSERT: k_count<MODE_INSERT><<<grid, AGG_THREADS, 0, lc.stream>>>(g, src, dst, n); break;
    case MODE_DELETE: k_count<MODE_DELETE><<<grid, AGG_THREADS, 0, lc.stream>>>(g, src, dst, n); break;
    default: k_count<MODE_QUERY><<<grid, AGG_THREADS, 0, lc.stream>>>(g, src, dst, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_count_rejects(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                                 unsigned long long n, unsigned long long *rejected,
                                 const LaunchCfg &lc) {
    k_count_rejects<<<grid_for(n, 256, lc.num_sms * 8), 256, 0, lc.stream>>>(g, src, dst, n, rejected);
    return cudaGetLastError();
}

cudaError_t launch_insert_tail(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                               unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, const LaunchCfg &lc) {
    const int cap = lc.num_sms * 8;
    const int gt = grid_for(tcap, 256, cap);
    {
        PhaseScope ps(lc, PH_INS_PLAN);
        k_plan_insert<<<gt, 256, 0, lc.stream>>>(g);
    }
    const unsigned long long max_pops = n / g.C + tcap + 1;
    {
        PhaseScope ps(lc, PH_INS_LINK);
        k_link_insert<<<grid_for(max_pops, 256, cap), 256, 0, lc.stream>>>(g);
    }
    {
        PhaseScope ps(lc, PH_INS_SCATTER);
        k_scatter_insert<<<grid_for(n, AGG_TILE, cap), AGG_THREADS, 0, lc.stream>>>(g, src, dst, n);
    }
    {
        PhaseScope ps(lc, PH_INS_FINALIZE);
        k_finalize_insert<<<gt, 256, 0, lc.stream>>>(g, n, counts);
    }
    return cudaGetLastError();
}

template <int MODE>
static void member_tail(const GraphView &g, const uint32_t *src, const uint32_t *dst,
                        unsigned long long n, unsigned long long tcap, unsigned long long *counts,
                        uint8_t *qout, const LaunchCfg &lc) {
    const int cap = lc.num_sms * 8;
    const int gt = grid_for(tcap, 256, cap);
    const int gi = lc.num_sms * 8;  // warp-per-item kernels: 8 warps per CTA
    const bool del = MODE == MODE_DELETE;
    {
        PhaseScope ps(lc, del ? PH_DEL_PLAN : PH_QRY_PLAN);
        k_plan_member<MODE><<<gt, 256, 0, lc.stream>>>(g);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_ARENA : PH_QRY_ARENA);
        k_arena_init<MODE><<<grid_for(4 * n + 64, 256, cap), 256, 0, lc.stream>>>(g);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_SCATTER : PH_QRY_SCATTER);
        k_scatter_member<MODE><<<grid_for(n, AGG_TILE, cap), AGG_THREADS, 0, lc.stream>>>(g, src, dst, n);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_MARK : PH_QRY_MARK);
        k_mark<MODE><<<gi, 256, 0, lc.stream>>>(g);
    }
    if (del) {
        {
            PhaseScope ps(lc, PH_DEL_VSCAN);
            k_vscan<MODE><<<grid_for(tcap, 8, cap), 256, 0, lc.stream>>>(g);
        }
        PhaseScope ps(lc, PH_DEL_MOVE);
        k_move<MODE><<<gi, 256, 0, lc.stream>>>(g);
    } else {
        PhaseScope ps(lc, PH_QRY_OUT);
        k_query_out<<<grid_for(n, 256, cap), 256, 0, lc.stream>>>(g, n, qout);
    }
    {
        PhaseScope ps(lc, del ? PH_DEL_FINALIZE : PH_QRY_FINALIZE);
        k_finalize_member<MODE><<<gt, 256, 0, lc.stream>>>(g, counts);
    }
}

cudaError_t launch_member_tail(int mode, const GraphView &g, const uint32_t *src,
                               const uint32_t *dst, unsigned long long n, unsigned long long tcap,
                               unsigned long long *counts, uint8_t *qout, const LaunchCfg &lc) {
    if (mode == MODE_DELETE) member_tail<MODE_DELETE>(g, src, dst, n, tcap, counts, qout, lc);
    else member_tail<MODE_QUERY>(g, src, dst, n, tcap, counts, qout, lc);
    return cudaGetLastError();
}

cudaError_t launch_vertex_delete(const GraphView &g, const uint32_t *ids, uint32_t k,
                                 const LaunchCfg &lc) {
    const int cap = lc.num_sms * 8;
    const int gi = lc.num_sms * 8;
    PhaseScope ps(lc, PH_VDEL);
    k_vdel_mark<<<grid_for(k, 256, cap), 256, 0, lc.stream>>>(g, ids, k);
    k_plan_vfree<<<grid_for(k, 256, cap), 256, 0, lc.stream>>>(g);
    k_free_items<<<gi, 256, 0, lc.stream>>>(g);
    k_reset_lists<<<1, 32, 0, lc.stream>>>(g);
    k_plan_vdel_in<<<grid_for(g.nv, 256, cap), 256, 0, lc.stream>>>(g);
    k_mark<MODE_VDEL><<<gi, 256, 0, lc.stream>>>(g);
    k_vscan<MODE_VDEL><<<grid_for(g.nv, 8, cap), 256, 0, lc.stream>>>(g);
    k_move<MODE_VDEL><<<gi, 256, 0, lc.stream>>>(g);
    k_finalize_vdel<<<grid_for(k, 256, cap), 256, 0, lc.stream>>>(g, ids, k);
    return cudaGetLastError();
}

}  // namespace gv

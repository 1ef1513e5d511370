// gv_internal.cuh -- device-side layout and helpers of the GraphVine GB300 library.
//
// Layout in HBM (one graph):
//   sent[vcap]      uint4 per vertex, the edge sentinel: {deg, nblocks, root, last}.
//                   deg = stored entries, nblocks = ceil(deg / C) (adjacencies are
//                   kept compacted), root = block id of heap index 1 of the CBT,
//                   last = block id of heap index nblocks (where the next insert
//                   starts, "last insert edge block" of the paper).  NIL when empty.
//   alive[vcap]     uint8 per vertex.
//   data[P * C]     uint32 destination ids; block b holds slots data[b*C .. b*C+C).
//   links[2 * P]    uint32 child block ids of block b: links[2b] left, links[2b+1]
//                   right; heap index k has children 2k and 2k+1 (Figure 2).
//   queue[P]        uint32 ring of free block ids (the paper's edge queue); the
//                   free ids sit at positions [q_front, q_back) modulo P.
//   gv_dev          control block: queue positions, counters, status word.
// Block ids are uint32 indices into data/links, so the pool may hold up to
// 2^32 - 1 blocks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gv {

constexpr uint32_t NIL = 0xFFFFFFFFu;
constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;
constexpr uint32_t FULL = 0xFFFFFFFFu;

// Device control block (one per graph, device memory).
struct Dev {
    unsigned long long q_front;     // edge queue: next pop position
    unsigned long long q_back;      // edge queue: next push position
    unsigned long long num_edges;   // stored entries
    unsigned long long tot_ins, tot_del, tot_rej;
    // per-call scratch counters (reset by the finalize kernels)
    unsigned long long alloc_total; // blocks popped by this call
    unsigned long long free_total;  // blocks pushed by this call
    unsigned long long arena_used;  // words of the membership arena used
    unsigned long long call_a;      // inserted / deleted entries of this call
    unsigned long long call_b;      // rejected pairs of this call
    unsigned long long call_c;      // extra per-call counter (sums)
    unsigned int n_touched;         // touched sources of this call
    unsigned int n_items;           // work items of this call
    unsigned int done_ctas;         // last-CTA ticket of the finalize kernels
    unsigned int status;            // latched device status (gv_status), sticky
    unsigned int abort;             // set when this call must not mutate the graph
    unsigned int n_tiny;            // touched sources handled one per thread
    unsigned int n_mitems;          // work items of multi-item sources (top of the item array)
    unsigned int n_tiny_hi;         // tiny sources with more than TINY_SPLIT entries (top of t_tiny)
    unsigned long long harena_used; // words of the arena's hash region used
    // grouped path (large batches): chunks of the partitioned batch, and
    // work groups of the block-wide membership tier
    unsigned int n_chunks;
    unsigned int n_groups;
    unsigned int n_mbuckets;        // buckets of more than one chunk
    unsigned int n_grouped;         // valid pairs of the grouped batch
    unsigned int n_hash;            // grouped path: sources whose batch keys go to an arena hash set
    // hub runs (see GraphView::rs): ring of free run heads, and the runs
    // popped / pushed by the current call
    unsigned long long rq_front, rq_back;
    unsigned long long ralloc_total, rfree_total;
};

// Everything a kernel needs to know about one graph (passed by value).
struct GraphView {
    uint4 *sent;
    uint8_t *alive;
    uint32_t *data;
    uint32_t *wdata;  // per-slot 32-bit payload (weights), parallel to data; NULL when unweighted
    uint32_t *links;
    uint32_t *queue;
    Dev *dev;
    unsigned long long P;   // pool blocks
    uint32_t C;             // entries per block
    uint32_t IB;            // blocks per work item (IB * C <= 512)
    uint32_t nv;            // vertex count
    uint32_t all_alive;     // 1 while no vertex has ever been deleted (alive[] need not be read)
    uint32_t vmask;         // dictionary capacity - 1 (capacity is a power of two)
    unsigned long long cmul;  // ceil(2^40 / C): x / C == (x * cmul) >> 40 for x < 2^31
    uint32_t dense_shift;   // batches with n >= nv >> dense_shift use per-pair counting
    // vertex-indexed scratch (zero between calls), indexed by vslot(u)
    uint32_t *vcnt;         // batch entries per source
    uint4 *vinfo;           // per-source plan record read by the scatters (one 16-byte load per pair)
    uint32_t *vtid;         // touched index of a source (valid while vcnt > 0)
    // touched-indexed scratch
    uint32_t *t_vid;        // touched source ids
    uint4 *t_a;             // per-touched info A (op specific)
    uint4 *t_b;             // per-touched info B (op specific)
    uint32_t *t_owner;      // insert: pop index -> touched index
    uint32_t *t_tiny;       // touched indices of tiny adjacencies (one thread each)
    uint32_t *prank;        // per pair: rank among its source's batch pairs (NIL = rejected)
    // work items (membership ops)
    uint2 *items;           // {touched index, chunk}
    uint32_t *it_mask;      // 16 words per item: survivor bits by slot
    uint32_t *it_cnt;       // survivors per item
    uint32_t *it_H;         // exclusive prefix of holes below the new degree
    uint32_t *it_S;         // exclusive prefix of survivors at/above the new degree
    uint32_t *it_bid;       // IB block ids per item
    // membership arena
    uint32_t *arena;        // list entries, then (from hbase) bucketed hash sets
    uint32_t hbase;         // first word of the hash region (a multiple of 64)
    uint32_t *found;        // query: hit flags, parallel to arena
    uint32_t *qpos;         // query: arena position of each query (NIL if invalid)
    uint8_t *pflag;         // set-semantics insert: 1 if the pair claimed its value's slot
    uint32_t *dead;         // vertex delete: bitmap of deleted ids
    unsigned long long max_items;
    unsigned long long tiny_cap;       // entries of t_tiny (touched capacity)
    unsigned long long arena_cap;
    // graph sets (many member graphs in one structure); set_G == 0 otherwise
    uint32_t set_G;                    // members
    const uint32_t *set_vbase;         // G+1 first vertex of each member (device)
    const unsigned long long *set_off; // G+1 first pair of each member's batch (device)
    unsigned long long *set_counts;    // 2G per-member counts of this call (device)
    // segmented deletes (set_G segments of one batch, set_vbase unused): the
    // segment that first names each batch key, one word per arena word;
    // NULL otherwise
    uint32_t *seg_own;
    // Grouped path (large plain batches): the batch is grouped by source on
    // the device by a radix partition (bucket = u >> gb_shift) and a
    // counting sort per chunk of a bucket; per-vertex scratch is then indexed
    // by the vertex id itself (no scramble: no per-pair atomics remain).
    uint32_t grouped;           // 1 during a grouped call
    uint32_t gb_shift;          // log2(vertices per bucket)
    uint32_t gb_n;              // buckets (vcap >> gb_shift)
    uint32_t gp_ctas;           // CTAs of the partition passes
    unsigned long long gp_len;  // pairs per partition CTA (a multiple of GP_TILE)
    uint32_t *gp_src;           // partitioned pairs, bucket by bucket
    uint32_t *gp_dst;
    uint32_t *gp_aux;           // query: original index; weighted insert: payload
    uint32_t *gp_hist;          // [gp_ctas][gb_n]: counts, then prefixes over the CTAs
    uint32_t *gp_btot;          // [gb_n] valid pairs per bucket
    uint32_t *gp_bbase;         // [gb_n] first partitioned position of each bucket
    uint4 *gp_chunks;           // {start, length, bucket, row of a multi-chunk bucket's chunk or NIL}
    uint32_t *gp_mbkt;          // buckets of more than one chunk
    uint32_t *gp_rows;          // [row][vertex of the bucket]: a chunk's offset in each vertex's segment
    uint32_t *go_src;           // insert: the grouped pairs (source order)
    uint32_t *go_dst;
    uint32_t *go_aux;
    uint32_t *gcur;             // per vertex: start of its segment in the grouped order
    uint2 *grp_items;           // block-wide membership tier: {touched index, first item} from
                                // the bottom; hash-set sources {touched index, -} from the top
    unsigned long long grp_cap; // entries of grp_items
    // Hub runs (a per-vertex block size): a source whose first allocation
    // takes at least hub_deg entries gets its blocks in runs of R = 2^rs
    // contiguous, R-aligned blocks of the run region [0, RP * R) instead of
    // one at a time, so its blocks are C * R slots long for the tree: the
    // tree links run heads only (heap index of a run), its height drops by
    // rs, and every slot computation (degree, slot index, block index in
    // units of C) stays as for the other sources.  Marked by RUN_BIT in the
    // sentinel's root word; kept until the source is emptied.  rs == 0: no
    // runs (the bit is never set).
    uint32_t rs;
    uint32_t hub_deg;
    unsigned long long RP;      // runs in the run region
    uint32_t *rqueue;           // ring of RP free run heads (block ids, multiples of R)
    uint32_t *t_rowner;         // insert: run pop index -> touched index
};

// Grouped path limits and sizes.
constexpr uint32_t GP_BMAX = 4096;     // buckets at most
constexpr uint32_t GP_WMAX = 4096;     // vertices per bucket at most
constexpr uint32_t GP_TILE = 4096;     // pairs per tile of a partition CTA
constexpr uint32_t GP_CHUNK = 4096;    // pairs per chunk of a bucket
constexpr uint32_t GP_THREADS = 512;   // threads of the partition and chunk CTAs
constexpr uint32_t GP_MAXCTAS = 1024;  // partition CTAs at most (rows of the column scan)
// Sources with more batch entries than LIST_MAX go to the block-wide
// membership tier: CT_GI work items per CTA share one shared-memory hash set
// of the source's batch entries, built CT_KEYS keys at a time.
constexpr uint32_t CT_GI = 8;          // items per group = warps per CTA
constexpr uint32_t CT_SLOTS = 8192;
constexpr uint32_t CT_KEYS = CT_SLOTS / 2;
constexpr uint32_t CT_FLAG = 0xFFFFFFFFu;  // t_a[t].z of a block-wide-tier source

// Index of vertex u in the per-call vertex scratch (vcnt, vinfo).
__device__ __forceinline__ uint32_t vidx(const GraphView &g, uint32_t u);

// Segment of pair i: the last s with off[s] <= i (off has G+1 entries).
__device__ __forceinline__ uint32_t segment_of(const unsigned long long *off, uint32_t G, unsigned long long i) {
    uint32_t lo = 0, hi = G;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Largest number of members of a graph set (per-CTA shared histograms).
constexpr uint32_t SET_MAX_G = 1024;

// Member owning global vertex u: the last i with vbase[i] <= u.
__device__ __forceinline__ uint32_t member_of(const uint32_t *vbase, uint32_t G, uint32_t u) {
    uint32_t lo = 0, hi = G;  // vbase[lo] <= u < vbase[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (vbase[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

enum Mode : int { MODE_INSERT = 0, MODE_DELETE = 1, MODE_QUERY = 2, MODE_VDEL = 3, MODE_DEDUP = 4 };

// A source's batch destinations are kept as a plain list up to LIST_MAX
// entries (tested through a shared-memory hash set built per work item) and
// as a bucketed hash set in the arena above it: buckets of HB = 8 words (one
// 32-byte sector) whose occupied slots are always a prefix.  An insert reads
// its whole home bucket in one round trip (two 16-byte loads in flight); a
// lookup reads the first half and goes on only past four occupied slots; only
// a full bucket sends either to the next one.
constexpr uint32_t LIST_MAX = 256;
constexpr uint32_t HB = 8;

// Arena words of a source under set-semantics inserts: every source gets a
// bucketed hash set (which also merges repeated pairs of the batch), the
// power of two at or above 2m, at least one bucket.
__host__ __device__ __forceinline__ uint32_t dedup_words(uint32_t m) {
    uint32_t h = HB;
    while (h < 2 * m) h <<= 1;
    return h;
}

// Tiny adjacencies (one thread per source): at most TINY_DEG entries in at
// most TINY_NB blocks, at most TINY_M batch entries.
constexpr uint32_t TINY_DEG = 128;
constexpr uint32_t TINY_NB = 8;
constexpr uint32_t TINY_M = 16;
// Tiny sources of up to TINY_SPLIT entries are listed from the bottom of
// t_tiny, larger ones from the top, so that a warp's 32 threads walk
// adjacencies of similar length (loop trip counts diverge less).
constexpr uint32_t TINY_SPLIT = 32;
// Queries only read: their thread-per-source tier stops at four blocks (a
// longer serial walk costs more than a warp item saves).
constexpr uint32_t TINY_DEG_Q = 64;
constexpr uint32_t TINY_NB_Q = 4;

// Arena words of a source with m batch entries: m (list) or the hash set
// size, the power of two at or above 2m.
__host__ __device__ __forceinline__ uint32_t member_words(uint32_t m) {
    if (m <= LIST_MAX) return m;
    uint32_t h = 2 * LIST_MAX;
    while (h < 2 * m) h <<= 1;
    return h;
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // "lowbias32" integer hash (C. Wellons, 2018).
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Home slot of key v in a table of `size` slots or buckets (a power of two):
// the top bits of v times an odd constant (multiplicative hashing, Knuth,
// TAOCP vol. 3, 6.4), two instructions where a full mixer takes seven; the
// membership tables it indexes are probed once per stored entry.
__device__ __forceinline__ uint32_t hidx(uint32_t v, uint32_t size) {
    return __umulhi(v * 0x9E3779B1u, size);
}

// Slot of vertex u in the per-call vertex scratch arrays: a bijection of
// [0, capacity) (multiplication by an odd constant modulo the power-of-two
// capacity).  Power-law graphs put most updates on a few low ids; without
// the scramble their counters share a handful of L2 slices, whose atomic
// units (about 1.5 G operations/s each) then serialise the whole batch.
constexpr uint32_t VSCRAMBLE = 0x9E3779B1u;
constexpr uint32_t inverse_odd(uint32_t a) {
    uint32_t x = a;  // Newton iteration for the inverse modulo 2^32
    for (int i = 0; i < 5; ++i) x *= 2u - a * x;
    return x;
}
constexpr uint32_t VSCRAMBLE_INV = inverse_odd(VSCRAMBLE);
static_assert(VSCRAMBLE * VSCRAMBLE_INV == 1u, "scramble inverse");

__device__ __forceinline__ uint32_t vslot(uint32_t vmask, uint32_t u) { return (u * VSCRAMBLE) & vmask; }
__device__ __forceinline__ uint32_t vidx(const GraphView &g, uint32_t u) { return g.grouped ? u : vslot(g.vmask, u); }
__device__ __forceinline__ uint32_t vslot_inv(uint32_t vmask, uint32_t i) { return (i * VSCRAMBLE_INV) & vmask; }

// Programmatic dependent launch: a kernel launched with the attribute may be
// scheduled while its predecessor on the stream drains; it waits here,
// before touching anything the predecessor wrote, until that grid has
// completed and its memory is visible.  A no-op for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void latch_status(Dev *dev, unsigned int code) {
    atomicCAS(&dev->status, 0u, code);
}

// Block id at heap index k (k >= 1) of the CBT rooted at `root`: follow the
// bits of k below its leading 1, most significant first, 0 = left, 1 = right
// (the bit-string rule of "Dynamic edge inserts").  Every id on the path is
// checked against the pool size; an id outside the pool (a corrupted tree)
// yields NIL, which callers treat as an error instead of dereferencing it.
__device__ __forceinline__ uint32_t cbt_walk(const uint32_t *__restrict__ links,
                                             unsigned long long P, uint32_t root, uint32_t k) {
    uint32_t b = root;
    if (b >= P) return NIL;
    int top = 31 - __clz(k);
    for (int i = top - 1; i >= 0; --i) {
        b = links[2ull * b + ((k >> i) & 1u)];
        if (b >= P) return NIL;
    }
    return b;
}

// Hub runs: the sentinel's root word is the id of the root block, or of the
// head of the first run with RUN_BIT set (block ids then stay below 2^31 - 1,
// so that no root word of a run equals NIL).
constexpr uint32_t RUN_BIT = 0x80000000u;

__device__ __forceinline__ bool is_run(uint32_t rw) { return rw != NIL && (rw & RUN_BIT); }

// Block id of the block at heap index k (k >= 1, in blocks of C slots) of
// the adjacency whose sentinel root word is rw: a tree walk for a plain
// adjacency; for a run adjacency a walk to the run holding block k - 1
// (run heap index ((k - 1) >> rs) + 1), then the offset inside the run.
__device__ __forceinline__ uint32_t blk_at(const GraphView &g, uint32_t rw, uint32_t k) {
    if (!is_run(rw)) return cbt_walk(g.links, g.P, rw, k);
    const uint32_t j = k - 1;
    const uint32_t h = cbt_walk(g.links, g.P, rw & ~RUN_BIT, (j >> g.rs) + 1);
    return h == NIL ? NIL : h + (j & ((1u << g.rs) - 1u));
}

// x mod P for a pool of P blocks (0 for an empty pool).
__device__ __forceinline__ unsigned long long qmod(unsigned long long x, unsigned long long P) {
    return P ? x % P : 0ull;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// x / C by multiply and shift.  With M = ceil(2^40 / C) and e = M*C - 2^40
// < C <= 512, floor(x*M / 2^40) = floor(x / C) whenever x*e < 2^40, i.e. for
// every x < 2^31 (degrees and slot indices stay below that).
__device__ __forceinline__ uint32_t divc(unsigned long long cmul, uint32_t x) {
    return (uint32_t)(((unsigned long long)x * cmul) >> 40);
}

// Loads of data read exactly once (batch pairs, ranks, adjacency entries
// streamed by a scan): evict-first, so that they do not push the per-vertex
// records and hash sets that many pairs share out of L2.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream4(const uint4 *p) { return __ldcs(p); }

// Full-warp exclusive scan of a uint32 (all 32 lanes must call).
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t *total) {
    uint32_t lane = lane_id();
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    *total = __shfl_sync(FULL, incl, 31);
    return incl - v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

// Warp-aggregated atomicAdd (all 32 lanes must call): every lane with `want`
// adds `v`; each gets the counter value before its own share.
template <typename T>
__device__ __forceinline__ T warp_atomic_add(T *ctr, uint32_t v, bool want) {
    uint32_t val = want ? v : 0u;
    uint32_t total;
    uint32_t excl = warp_excl_scan(val, &total);
    T base = 0;
    if (lane_id() == 0 && total) base = atomicAdd(ctr, (T)total);
    base = __shfl_sync(FULL, base, 0);
    return base + (T)excl;
}

// Block-wide exclusive scan (blockDim.x a multiple of 32, <= 1024; all
// threads must call).  Returns the exclusive prefix and the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t s_w[33];
    uint32_t wt;
    uint32_t ex = warp_excl_scan(v, &wt);
    uint32_t w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0) s_w[w] = wt;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane_id() < nw ? s_w[lane_id()] : 0u;
        uint32_t t2;
        uint32_t e2 = warp_excl_scan(x, &t2);
        if (lane_id() < nw) s_w[lane_id()] = e2;
        if (lane_id() == 0) s_w[32] = t2;
    }
    __syncthreads();
    uint32_t r = ex + s_w[w];
    *total = s_w[32];
    __syncthreads();
    return r;
}

// Block-wide sum of a 64-bit value (all threads must call).
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v) {
    __shared__ unsigned long long s_p[32];
    v = warp_sum_u64(v);
    uint32_t w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0) s_p[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (threadIdx.x == 0)
        for (uint32_t i = 0; i < nw; ++i) r += s_p[i];
    __syncthreads();
    return r;  // valid in thread 0
}


// Open-addressing hash set in a global arena region of `hsize` (power of two)
// words: insert, returning the slot of `v`.
__device__ __forceinline__ uint32_t hash_insert(uint32_t *tab, uint32_t hsize, uint32_t v) {
    uint32_t h = mix32(v) & (hsize - 1);
    for (uint32_t probe = 0; probe < hsize; ++probe) {
        uint32_t cur = tab[h];
        if (cur == v) return h;
        if (cur == EMPTY_KEY) {
            uint32_t old = atomicCAS(&tab[h], EMPTY_KEY, v);
            if (old == EMPTY_KEY || old == v) return h;
        }
        h = (h + 1) & (hsize - 1);
    }
    return NIL;  // unreachable: tables are sized at twice the entries
}

__device__ __forceinline__ uint32_t hash_find(const uint32_t *tab, uint32_t hsize, uint32_t v) {
    uint32_t h = mix32(v) & (hsize - 1);
    for (uint32_t probe = 0; probe < hsize; ++probe) {
        uint32_t cur = tab[h];
        if (cur == v) return h;
        if (cur == EMPTY_KEY) return NIL;
        h = (h + 1) & (hsize - 1);
    }
    return NIL;
}

// Bucketed hash set of nbk buckets of HB words at tab (occupied slots are a
// prefix of each bucket): insert v, returning its word index in tab (NIL if
// the table is full, which sizing at twice the keys rules out).  Each pass
// ends, moves to the next bucket, or rereads after losing a slot to another
// insert (which filled that slot): (HB + 1) * nbk passes bound the loop.
__device__ __forceinline__ uint32_t bucket_insert(uint32_t *tab, uint32_t nbk, uint32_t v) {
    uint32_t b = hidx(v, nbk);
    for (uint32_t probe = 0; probe < (HB + 1) * nbk; ++probe) {
        const uint4 *bp = reinterpret_cast<const uint4 *>(tab + b * HB);
        const uint4 x0 = __ldcg(bp), x1 = __ldcg(bp + 1);
        const uint32_t w[HB] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        uint32_t hit = NIL, empty = NIL;
#pragma unroll
        for (uint32_t k = 0; k < HB; ++k) {
            if (hit == NIL && w[k] == v) hit = k;
            if (empty == NIL && w[k] == EMPTY_KEY) empty = k;
        }
        if (hit != NIL) return b * HB + hit;
        if (empty != NIL) {
            const uint32_t old = atomicCAS(&tab[b * HB + empty], EMPTY_KEY, v);
            if (old == EMPTY_KEY || old == v) return b * HB + empty;
        } else {
            b = (b + 1) & (nbk - 1);
        }
    }
    return NIL;
}

// Word index of v in the bucketed hash set (NIL if absent).
__device__ __forceinline__ uint32_t bucket_find(const uint32_t *tab, uint32_t nbk, uint32_t v) {
    uint32_t b = hidx(v, nbk);
    for (uint32_t step = 0; step < nbk; ++step) {
        const uint4 *bp = reinterpret_cast<const uint4 *>(tab + b * HB);
        const uint4 x0 = __ldcg(bp), x1 = __ldcg(bp + 1);
        const uint32_t w[HB] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (uint32_t k = 0; k < HB; ++k)
            if (w[k] == v) return b * HB + k;
        if (w[HB - 1] != EMPTY_KEY) {
            b = (b + 1) & (nbk - 1);
            continue;
        }
        return NIL;  // the bucket's prefix ended without v
    }
    return NIL;
}

// Last-CTA detection for a finalize kernel: returns true in exactly one CTA,
// after every CTA has passed this point.  Uses dev->done_ctas, which the last
// CTA resets.
__device__ __forceinline__ bool last_cta(Dev *dev) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(&dev->done_ctas, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Position off past base in a ring of P slots (base < P, off <= P).
__device__ __forceinline__ unsigned long long ring(unsigned long long base, unsigned long long off,
                                                   unsigned long long P) {
    unsigned long long q = base + off;
    return q >= P ? q - P : q;
}

// A run freed by a delete goes back onto the run queue at rq_back + the
// call's run counter (published by the finalize kernel).  Runs return
// rarely (a hub shrinking by whole runs), so no staging.
__device__ __forceinline__ void push_run(const GraphView &g, uint32_t head, unsigned long long rqbb) {
    const unsigned long long pos = atomicAdd(&g.dev->rfree_total, 1ull);
    g.rqueue[ring(rqbb, pos, g.RP)] = head;
}

// Delete-side release for a run adjacency (root word rw) shrinking to nbn
// blocks: the block at heap index k with id bid gives its whole run back
// when it is the run's head and the run lies past the runs still needed;
// a kept parent run forgets it.  The walk to the parent passes only kept
// runs, whose links to kept children no thread clears.
__device__ __forceinline__ void release_run(const GraphView &g, uint32_t rw, uint32_t k, uint32_t bid,
                                            uint32_t nbn, unsigned long long rqbb) {
    const uint32_t j = k - 1, R = 1u << g.rs;
    if (j & (R - 1u)) return;
    const uint32_t kr = (j >> g.rs) + 1u;         // heap index of the run
    const uint32_t nrn = (nbn + R - 1u) >> g.rs;  // runs kept
    if (kr <= nrn) return;
    push_run(g, bid, rqbb);
    const uint32_t pr = kr >> 1;
    if (kr >= 2u && pr <= nrn) {
        const uint32_t ph = cbt_walk(g.links, g.P, rw & ~RUN_BIT, pr);
        if (ph != NIL) g.links[2ull * ph + (kr & 1u)] = NIL;
        else latch_status(g.dev, 5u /* GV_ERR_STATE */);
    }
}

// Freed block ids of one warp, staged in shared memory and pushed onto the
// edge queue 32 at a time with one atomic on the call's free counter (the
// queue positions are q_back + counter, published by the finalize kernel).
struct FreeStage {
    uint32_t *buf;  // 64 ids: this warp's slice of shared memory
    uint32_t n;     // ids held (warp-uniform)

    __device__ __forceinline__ void flush(uint32_t cnt, Dev *dev, uint32_t *queue, unsigned long long qbb,
                                          unsigned long long P) {
        unsigned long long base = 0;
        if (lane_id() == 0 && cnt) base = atomicAdd(&dev->free_total, (unsigned long long)cnt);
        base = __shfl_sync(FULL, base, 0);
        if (lane_id() < cnt) queue[ring(qbb, base + lane_id(), P)] = buf[lane_id()];
        __syncwarp();
    }

    // All 32 lanes call; lanes with `want` add `id`.
    __device__ __forceinline__ void push(bool want, uint32_t id, Dev *dev, uint32_t *queue, unsigned long long qbb,
                                         unsigned long long P) {
        const uint32_t lane = lane_id();
        const unsigned bal = __ballot_sync(FULL, want);
        if (want) buf[n + __popc(bal & ((1u << lane) - 1u))] = id;
        n += __popc(bal);
        __syncwarp();
        if (n >= 32) {
            flush(32, dev, queue, qbb, P);
            const uint32_t rem = n - 32;
            const uint32_t x = lane < rem ? buf[32 + lane] : 0u;
            __syncwarp();
            if (lane < rem) buf[lane] = x;
            __syncwarp();
            n = rem;
        }
    }
};

// ------------------------------------------------------------ work items

// Items over the blocks of one touched source: t_b[t] = {deg, nblocks, root,
// items}; t_a[t].w = first item.  Returns nothing; writes the item list.
__device__ __forceinline__ void emit_items(const GraphView &g, uint32_t t, uint32_t item0,
                                           uint32_t ni) {
    for (uint32_t c = 0; c < ni; ++c) g.items[item0 + c] = make_uint2(t, c);
}

// First work item of a source with ni items, for every thread of the block
// (all threads call): single-item sources count up from the bottom of the
// item array, multi-item sources down from the top (so the kernels that
// handle only multi-item sources visit only their items).
__device__ __forceinline__ uint32_t alloc_items(const GraphView &g, uint32_t ni, uint32_t *s_lo, uint32_t *s_hi) {
    uint32_t ltot, htot;
    const uint32_t lex = block_excl_scan(ni == 1 ? 1u : 0u, &ltot);
    const uint32_t hex = block_excl_scan(ni > 1 ? ni : 0u, &htot);
    if (threadIdx.x == 0) {
        *s_lo = ltot ? atomicAdd(&g.dev->n_items, ltot) : 0u;
        *s_hi = htot ? atomicAdd(&g.dev->n_mitems, htot) : 0u;
    }
    __syncthreads();
    if (ni == 1) return *s_lo + lex;
    if (ni > 1) return (uint32_t)(g.max_items - (*s_hi + hex + ni));
    return 0u;
}

// Work item of virtual index vi over both regions ([0, nlo) bottom, then the
// nhi top items).
__device__ __forceinline__ uint32_t item_at(const GraphView &g, uint32_t vi, uint32_t nlo, uint32_t nhi) {
    return vi < nlo ? vi : (uint32_t)(g.max_items - nhi + (vi - nlo));
}

}  // namespace gv

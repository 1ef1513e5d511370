/*
 * graphvine.h -- C ABI of the GB300 (sm_103a) GraphVine dynamic-graph library.
 *
 * GraphVine ("A Data Structure to Optimize Dynamic Graph Processing on GPUs",
 * Krishnan S, Tavva, Nasre) stores a directed graph as a vertex dictionary
 * whose entries point at per-vertex sentinels; each sentinel roots a complete
 * binary tree (CBT) of fixed-capacity edge blocks taken from a pre-allocated
 * pool, the "edge queue".  Edge updates arrive in batches.  This library keeps
 * that structure resident in device memory and runs every step of the batch
 * operations in its own CUDA kernels.
 *
 * Conventions (all entry points):
 *   - Array arguments are plain pointers.  Unless an entry point says
 *     otherwise, an array may live in device memory (cudaMalloc, a torch CUDA
 *     tensor) or in host memory (pinned or pageable).  Host arrays are copied
 *     to and from library-owned device staging buffers.  The edge batches of
 *     gv_bulk_build, gv_insert_edges, gv_insert_edges_weighted,
 *     gv_delete_edges and gv_query_edges are copied on a copy stream the
 *     library owns, into one of three rotating staging sets, so that a
 *     call's copies overlap the kernels of the calls before it; `stream`
 *     waits for them.  Their host
 *     OUTPUT arrays (counts, query results) are written in stream order: a
 *     page-locked output holds its values once `stream` has reached the
 *     end of the call (synchronise `stream`, or gv_sync, before reading it);
 *     a pageable output is complete when the call returns.  Other calls with
 *     a host output array synchronise `stream` before they return.
 *   - The caller owns every array it passes; it must stay valid, and a host
 *     input unchanged, until the call's work on `stream` has completed (a
 *     pageable host input may be reused once the call returns).  The
 *     library owns the graph state, the block pool (unless
 *     gv_config.pool_mem is given) and its scratch memory.
 *   - Calls are asynchronous and ordered on `stream` (a cudaStream_t, passed
 *     as void*; NULL = the legacy default stream).  Calls on one graph must
 *     be ordered by the caller (one stream, or explicit dependencies): the
 *     graph's scratch memory is shared by its calls.  Different graphs are
 *     independent and may be used from different threads.  Inside a call the
 *     library may fork part of the work onto a second stream it owns; that
 *     work joins back onto `stream` before the call's last kernel, so the
 *     ordering on `stream` (and stream capture into a CUDA graph) holds.
 *     Consecutive kernels of a call are launched with programmatic stream
 *     serialization: each may be scheduled while its predecessor drains and
 *     waits, at its first instruction, for the predecessor's results.
 *   - The return value reports host-detectable errors at once (NULL graph,
 *     NULL array with n > 0, n too large, CUDA launch or allocation failure).
 *     Errors found on the device (edge pool exhausted, structure
 *     inconsistency) turn the operation into a no-op -- the graph is left
 *     exactly as it was -- and are latched in a device status word that the
 *     next gv_sync() or gv_stats() returns and clears.
 *   - Vertex ids and edge endpoints are uint32_t; valid ids are < the vertex
 *     count.  An edge whose endpoint is out of range or not alive is rejected
 *     and counted; the rest of its batch proceeds.
 *   - Multiset semantics by default: inserting a pair that is already stored
 *     adds another copy (Algorithm 1 appends without a duplicate check); a
 *     delete removes every stored copy of each (u, v) it names (Algorithm 2
 *     marks every matching entry).  With GV_DEDUP an insert adds a pair only
 *     if it is not stored yet and not already added by the same batch.
 *   - With GV_WEIGHTED every entry carries a 32-bit payload that stays with
 *     it; deletes match (u, v) whatever the payload.
 */
#ifndef GRAPHVINE_H
#define GRAPHVINE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gv_graph gv_graph; /* opaque, owned by the library */

typedef enum gv_status {
    GV_OK = 0,
    GV_ERR_INVALID_ARG = 1,   /* bad argument, detected on the host */
    GV_ERR_OUT_OF_MEMORY = 2, /* device allocation failed, or edge pool exhausted (op is a no-op) */
    GV_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    GV_ERR_TIMEOUT = 4,       /* a bounded device wait gave up (op is a no-op) */
    GV_ERR_STATE = 5          /* inconsistent structure detected on the device, or call out of order */
} gv_status;

/* gv_config.flags */
#define GV_DEDUP 1u /* set semantics for inserts (cuSTINGER/Hornet-style duplicate check) */
/* Pool growth ("Edge Queue": when 80% of the pool is used it grows by 25%).
 * Checked on the host before each insert against an upper bound of the
 * blocks in use plus the insert's worst-case demand ceil(n/C) + min(n, |V|);
 * when the bound passes 80% the call synchronises its stream once, reads the
 * exact count and, if needed, moves the pool into an allocation 25% larger
 * (repeatedly, until the exact count plus the demand is under 80%).  Block
 * ids are kept.  Library-owned pools only (pool_mem must be NULL); a failed
 * allocation keeps the old pool. */
#define GV_GROW 2u
/* Weighted entries: every stored entry carries a 32-bit payload (a weight,
 * or any 32-bit value) that moves with it through deletes and compaction.
 * The pool then holds 8*C + 12 bytes per block.  Excludes GV_DEDUP (which of
 * several repeated pairs a set-semantics batch keeps is not defined). */
#define GV_WEIGHTED 4u
/* Large batches (see dense_shift below) of plain inserts, deletes and
 * queries are grouped by source with one atomic per pair on the source's
 * counter.  With this flag they are grouped instead by a radix partition of
 * the source ids (no per-pair global atomic; dictionaries of at most 2^24
 * vertices): the batch becomes contiguous per-source runs, inserts write
 * each source's new entries as consecutive slots and deletes and queries
 * test stored entries against the runs (sources of more than 256 and at
 * most 4096 batch entries through a shared-memory hash set per CTA).  Same
 * results; measured slower on the 10M-edge RMAT step (1.32 against 1.14
 * ms), so not the default. */
#define GV_RADIX_GROUPING 8u

typedef struct gv_config {
    /* C, the number of edge entries per edge block (multiple of 4, 4..512).
     * 0 = the paper's rule ("Initialization"): the average degree of the
     * vertices with non-zero degree in the first edge batch, rounded up to a
     * multiple of 4; fixed from then on. */
    uint32_t block_capacity;
    uint32_t flags;          /* GV_DEDUP | GV_GROW | GV_WEIGHTED | GV_RADIX_GROUPING, or 0 */
    /* Bytes reserved for the edge-block pool: block storage (4*C bytes per
     * block), tree links (8 bytes per block) and the edge queue (4 bytes per
     * block).  0 = half of the free device memory ("Edge Queue": at least
     * half of GPU memory is reserved with one allocation). */
    uint64_t pool_bytes;
    /* Optional caller-owned device buffer of pool_bytes bytes (16-byte
     * aligned) to hold the pool instead of a library allocation.  It must
     * outlive the graph. */
    void *pool_mem;
    /* Hint for the dictionary capacity; rounded up to a power of two
     * ("Vertex dictionary": 453 vertices -> 512). */
    uint32_t vertex_capacity;
    /* Tuning (0 = default).  item_blocks: blocks of one adjacency that one
     * warp handles per work item in deletes and queries (1 .. min(32, 512/C);
     * default the maximum) -- fewer blocks put more warps on a long
     * adjacency.  dense_shift: batches of n pairs with n >= vertices >> s
     * (dictionary capacity) are grouped with one atomic per pair plus a pass
     * over all vertices (or, with GV_RADIX_GROUPING, by a radix partition of
     * the source ids: buckets by the high bits, then a counting sort of each
     * chunk of a bucket by the low bits), smaller ones with per-tile
     * aggregation (default s = 3). */
    uint32_t item_blocks;
    uint32_t dense_shift;
    /* Hub runs: a per-vertex edge-block size ("Conclusion and future work":
     * changing the block size; "Performance Evaluation": deletes on graphs
     * with a large maximum degree pay for the height of the hubs' trees).
     * hub_shift s in 3..8 (0 = off): a vertex whose first allocation (the
     * first insert, or bulk build, that gives it entries) takes at least
     * hub_degree entries (0 = C * 2^s) receives its edge blocks in runs of
     * R = 2^s contiguous blocks, so that for its tree a block holds C * R
     * entries: the tree links run heads only and is s levels shallower.  The
     * vertex keeps runs until it is emptied.  hub_percent (1..90, 0 = 50)
     * of the pool's blocks, rounded down to whole runs, form the run region,
     * with its own queue of free runs; an insert that needs more runs than
     * are free fails like an exhausted pool (GV_ERR_OUT_OF_MEMORY, nothing
     * changes).  gv_reblock re-decides every vertex: after it, exactly the
     * vertices of degree >= the threshold (at the new C) are hubs, so it also
     * serves to promote vertices that grew past the threshold after their
     * first allocation.  With GV_GROW the pool grows by single blocks only
     * (the growth rule applies to the blocks outside the run region, whose
     * size stays as created).  Results never depend on the setting.
     * Excludes GV_RADIX_GROUPING and graph sets; block ids stay below
     * 2^31 - 1 (the pool is capped there). */
    uint32_t hub_shift;
    uint32_t hub_degree;
    uint32_t hub_percent;
    uint32_t reserved;
} gv_config;

typedef struct gv_stats_t {
    uint32_t num_vertices;     /* ids 0 .. num_vertices-1 exist (alive or deleted) */
    uint32_t vertex_capacity;  /* dictionary capacity, a power of two */
    uint32_t block_capacity;   /* C (0 until fixed by the first edge batch) */
    uint32_t flags;
    uint64_t num_edges;        /* stored edge entries (a multigraph counts copies) */
    uint64_t pool_blocks;      /* blocks in the pool */
    uint64_t pool_blocks_used; /* blocks owned by adjacencies */
    uint64_t pool_blocks_free; /* blocks in the edge queue */
    uint64_t pool_bytes;       /* device bytes of the pool (blocks, links, queue) */
    uint64_t device_bytes;     /* all device bytes held by the graph, scratch included */
    uint64_t total_inserted;   /* since creation */
    uint64_t total_deleted;
    uint64_t total_rejected;
    uint32_t device_status;    /* latched device status (gv_status), cleared by the read */
    uint32_t hub_shift;        /* log2 of the blocks per run (0: no hub runs) */
    uint64_t pool_runs;        /* runs of the run region (its blocks count in pool_blocks) */
    uint64_t pool_runs_free;   /* runs in the run queue (their blocks count in pool_blocks_free) */
} gv_stats_t;

/*
 * gv_create -- vertex dictionary, sentinels and block pool ("Dynamic vertex
 * updates": dictionary, sentinels and one kernel attaching a sentinel to each
 * vertex; "Edge Queue": the pool is reserved once and every block id pushed
 * onto the queue).
 *   cfg           configuration (NULL = all defaults).
 *   num_vertices  initial vertex count; ids 0 .. num_vertices-1, all alive.
 *   stream        stream for the initialisation kernels.
 *   out           receives the graph handle.
 * When C is given the pool is allocated here; with C = 0 it is allocated by
 * the first edge batch, once C is known.  Errors: GV_ERR_INVALID_ARG (bad C,
 * NULL out, misaligned pool_mem, pool too small for one block),
 * GV_ERR_OUT_OF_MEMORY, GV_ERR_CUDA.
 */
gv_status gv_create(const gv_config *cfg, uint32_t num_vertices, void *stream, gv_graph **out);

/* gv_destroy -- synchronises the graph's last stream and frees everything the
 * library allocated.  NULL is a no-op. */
gv_status gv_destroy(gv_graph *g);

/*
 * gv_bulk_build -- the first edge batch ("Initialization and batch updates";
 * Table 3 "Bulk" rows): fixes C by the paper's rule if the configuration left
 * it 0 (this reads two counters back, so the call synchronises `stream`
 * once), allocates the pool if needed, then inserts the n pairs exactly as
 * gv_insert_edges does.  On a graph that already holds edges it is a plain
 * insert.
 *   src, dst  n uint32 endpoints each (device or host).
 *   d_counts  optional, 2 uint64 written on the device: {inserted, rejected}.
 */
gv_status gv_bulk_build(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                        uint64_t *d_counts, void *stream);

/*
 * gv_insert_edges -- batched edge insert (Algorithm 1, "Dynamic edge
 * inserts").  The batch is grouped by source on the device; each source's
 * new edges fill the free slots of its last block, then blocks popped from
 * the edge queue at offsets given by a prefix sum of per-source block demand
 * (Figure 3); each new block hangs in the source's CBT at the place the bit
 * string of its 1-based index names (Figure 4).  A batch of at most 2,048
 * pairs (without GV_DEDUP) runs all of it in one kernel of one thread block
 * (grouping in shared memory); larger ones in a chain of grid-wide kernels.
 *   src, dst  n uint32 endpoints each (device or host), any order, any
 *             duplicates.
 *   d_counts  optional, 2 uint64 (device or host): {inserted, rejected}.
 * If the batch needs more blocks than the queue holds, nothing is inserted,
 * d_counts gets {0, 0} and the device status latches GV_ERR_OUT_OF_MEMORY.
 * With GV_DEDUP a membership pass runs first (the batch's destinations per
 * source in a hash set, every stored block of each touched source scanned as
 * in gv_query_edges) and only pairs that are neither stored nor repeated
 * within the batch are inserted; repeats count as neither inserted nor
 * rejected.  Such a batch holds at most 2^28 pairs (GV_ERR_INVALID_ARG).
 */
gv_status gv_insert_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                          uint64_t *d_counts, void *stream);

/*
 * gv_delete_edges -- batched edge delete (Algorithm 2, "Dynamic edge
 * deletes").  Every stored entry (u, v) with (u, v) in the batch is removed,
 * all copies of it; pairs that are not stored are ignored.  Each touched
 * adjacency is compacted so that all its blocks but the last are full, and
 * the emptied blocks are pushed back onto the edge queue ("Edge Queue":
 * emptied blocks return to the queue for reuse).
 *   src, dst  n uint32 endpoints each (device or host).
 *   d_counts  optional, 2 uint64: {deleted entries, rejected pairs}.
 */
gv_status gv_delete_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                          uint64_t *d_counts, void *stream);

/*
 * gv_query_edges -- batched edge-existence query (Algorithm 3, "Querying
 * operations"): out[i] = 1 if src[i] and dst[i] are valid, alive ids and
 * (src[i], dst[i]) is stored, else 0.
 *   src, dst  n uint32 each (device or host).
 *   out       n uint8 results (device or host).
 */
gv_status gv_query_edges(gv_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                         uint8_t *out, void *stream);

/*
 * gv_neighbors -- the current out-neighbours of n vertices, as CSR in each
 * adjacency's storage order (the in-order walk of the block tree that
 * Algorithms 2 and 3 perform).  Invalid or deleted ids give empty lists.
 *   vids          n uint32 vertex ids (device or host).
 *   offsets       n+1 uint64 (device or host): offsets[i] .. offsets[i+1]
 *                 index vids[i]'s neighbours in nbrs.
 *   nbrs          nbr_capacity uint32 (device or host).
 *   total         host pointer, receives the number of neighbours; required.
 * Synchronises `stream` (the total is read back).  If the total exceeds
 * nbr_capacity, offsets are written, nbrs is not, and GV_ERR_INVALID_ARG is
 * returned with *total set.
 */
gv_status gv_neighbors(gv_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets,
                       uint32_t *nbrs, uint64_t nbr_capacity, uint64_t *total, void *stream);

/*
 * gv_insert_vertices -- append k vertices with ids num_vertices ..
 * num_vertices+k-1, alive and without edges ("Dynamic vertex updates": when
 * the dictionary is full it is reallocated at twice the size and copied by
 * one kernel; new vertices get sentinels by the initialisation kernel).
 *   new_ids  optional, k uint32 (device or host) receiving the new ids.
 */
gv_status gv_insert_vertices(gv_graph *g, uint32_t k, uint32_t *new_ids, void *stream);

/*
 * gv_delete_vertices -- delete k vertices: each valid, alive id in ids is
 * marked dead, its blocks return to the edge queue, and every edge pointing
 * at it is removed from every other adjacency (incoming and outgoing edges,
 * as the paper describes for faimGraph in "Prior Work"; GraphVine itself
 * keeps the dictionary slot, "Dynamic vertex updates").  Ids are not reused.
 * Invalid, dead or repeated ids are ignored.
 *   ids  k uint32 (device or host).
 * Cost: one pass over every live adjacency.
 */
gv_status gv_delete_vertices(gv_graph *g, const uint32_t *ids, uint32_t k, void *stream);

/*
 * gv_export_csr -- the whole graph as CSR in storage order: offsets has
 * num_vertices+1 uint64 entries, nbrs nbr_capacity uint32 entries (device or
 * host), total (host) receives the edge count.  Same contract as
 * gv_neighbors over ids 0 .. num_vertices-1.
 */
gv_status gv_export_csr(gv_graph *g, uint64_t *offsets, uint32_t *nbrs, uint64_t nbr_capacity,
                        uint64_t *total, void *stream);

/* gv_degrees -- num_vertices uint32 out-degrees and, if alive is not NULL,
 * num_vertices uint8 alive flags (device or host; host outputs synchronise). */
gv_status gv_degrees(gv_graph *g, uint32_t *deg, uint8_t *alive, void *stream);

/* gv_reserve -- grow the graph's scratch memory for batches of up to
 * max_batch pairs now, so that later calls with at most that many pairs
 * allocate nothing (a prerequisite for capturing them in a CUDA graph). */
gv_status gv_reserve(gv_graph *g, uint64_t max_batch);

/* gv_sync -- wait for the graph's last stream; return and clear the latched
 * device status. */
gv_status gv_sync(gv_graph *g);

/* gv_stats -- synchronise, then fill *out (host pointer).  Returns and
 * clears the latched device status like gv_sync. */
gv_status gv_stats(gv_graph *g, gv_stats_t *out);

/*
 * gv_validate -- structural self-check on the device, for tests: every
 * adjacency holds ceil(deg/C) blocks, every tree walk stays inside the pool,
 * no block is owned twice or both owned and queued, and owned + queued =
 * pool.  Writes the number of violations to *violations (host) and
 * synchronises.
 */
gv_status gv_validate(gv_graph *g, uint64_t *violations, void *stream);

/*
 * Per-phase device timing (tracing).  While enabled, the library records a
 * CUDA event pair on the call's stream around every kernel it launches for
 * this graph; each pair is attributed to a named phase (e.g.
 * "insert.scatter", "delete.mark").  Off by default; costs one event record
 * per launch when on.
 *   gv_profile            enable (1) or disable (0).
 *   gv_profile_read       synchronises the recorded events, writes for phases
 *                         0 .. n-1 the summed device milliseconds (ms, may be
 *                         NULL) and launch counts (launches, may be NULL)
 *                         since the previous read, then resets them.
 *   gv_profile_num_phases number of phases.
 *   gv_profile_phase_name static name of a phase, NULL if out of range.
 */
gv_status gv_profile(gv_graph *g, int enable);
gv_status gv_profile_read(gv_graph *g, double *ms, uint64_t *launches, uint32_t n);
uint32_t gv_profile_num_phases(void);
const char *gv_profile_phase_name(uint32_t phase);

/*
 * gv_insert_edges_segmented -- gv_insert_edges on a batch made of nseg
 * requests (pairs d_offsets[i] .. d_offsets[i+1]-1 belong to request i), with
 * per-request counts: d_counts[2i] = inserted, d_counts[2i+1] = rejected.
 * The result equals inserting the requests one after another (multiset
 * inserts commute), which lets a server merge queued insert requests into
 * one launch sequence.  nseg in 1 .. 1024; all arrays device memory; the
 * graph's C must already be fixed (after gv_bulk_build or with a configured
 * C).  If the merged batch does not fit the pool, nothing is inserted and
 * every request gets {0, 0}.
 */
gv_status gv_insert_edges_segmented(gv_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    const uint64_t *d_offsets, uint32_t nseg, uint64_t *d_counts, void *stream);

/*
 * gv_insert_edges_weighted -- gv_insert_edges on a graph created with
 * GV_WEIGHTED, each pair with its 32-bit payload w[i] (device or host, n
 * entries).  Plain gv_insert_edges (and gv_bulk_build) on such a graph store
 * payload 0.  Deletes remove entries by (u, v) whatever their payload.  The
 * paper's entries are plain destination ids; weighted entries are its
 * "future work" extension (weighted edge entries).
 * Errors: GV_ERR_INVALID_ARG on an unweighted graph or a graph set.
 */
gv_status gv_insert_edges_weighted(gv_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                                   uint64_t n, uint64_t *d_counts, void *stream);

/*
 * gv_neighbors_weighted -- gv_neighbors with the payloads: weights[k] belongs
 * to nbrs[k] (same layout and capacity rules).  Weighted graphs only.
 */
gv_status gv_neighbors_weighted(gv_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets, uint32_t *nbrs,
                                uint32_t *weights, uint64_t nbr_capacity, uint64_t *total, void *stream);

/*
 * gv_delete_edges_segmented -- one delete call for nseg consecutive batches
 * (segments) of the same graph, with the result of applying them one call
 * each, in segment order: segment s holds pairs d_offsets[s] ..
 * d_offsets[s+1]-1.  The graph ends as after the nseg deletes (Algorithm 2
 * removes every stored copy of each named pair, so a pair named again by a
 * later segment finds nothing left); d_counts[2s] = stored entries removed
 * for pairs whose key segment s is the first to name, d_counts[2s+1] = pairs
 * of segment s rejected (endpoint out of range or dead).  A serving loop uses
 * it to run queued delete requests as one batch.
 *   d_offsets  nseg+1 uint64 (device), ascending, d_offsets[0] = 0,
 *              d_offsets[nseg] = n.
 *   nseg       1 .. 1024.
 *   d_counts   2*nseg uint64 (device), written.
 * Device arrays only; not on graph sets.  The paper has no segmented call
 * (its batches are one call each).
 */
gv_status gv_delete_edges_segmented(gv_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    const uint64_t *d_offsets, uint32_t nseg, uint64_t *d_counts, void *stream);

/*
 * Graph sets: many independent graphs ("members") in one device structure
 * that shares one dictionary (members own consecutive vertex ranges), one
 * block pool and one scratch area, so that an update touching every member
 * runs as one launch sequence whatever the number of members (and can be
 * captured in a CUDA graph once gv_reserve has sized the scratch).  Member
 * batches use member-local vertex ids.  Vertex insert/delete is not
 * available on a set; gv_stats, gv_validate, gv_sync, gv_reserve,
 * gv_profile and gv_destroy work on it as on a graph.
 *
 * gv_set_create -- cfg must give C (block_capacity != 0) and no GV_DEDUP;
 *   num_vertices is a host array of num_graphs (1 .. 1024) vertex counts.
 * gv_set_insert_edges / gv_set_delete_edges / gv_set_query_edges -- the
 *   members' batches concatenated: pairs d_offsets[i] .. d_offsets[i+1]-1 of
 *   d_src/d_dst belong to member i (d_offsets: num_graphs+1 uint64, device;
 *   n = d_offsets[num_graphs], given by the caller).  d_counts (device,
 *   2*num_graphs uint64) receives per member {inserted, rejected} /
 *   {deleted, rejected} / {0, rejected}; d_out (query, device, n uint8) the
 *   answers.  All arrays must be device memory (GV_ERR_INVALID_ARG
 *   otherwise): the calls allocate nothing once scratch is reserved and
 *   never synchronise.  Semantics per member are those of the single-graph
 *   calls (Algorithms 1-3).
 * gv_set_member_neighbors -- member `member`'s CSR (member-local ids),
 *   contract of gv_neighbors over all of its vertices.
 */
gv_status gv_set_create(const gv_config *cfg, uint32_t num_graphs, const uint32_t *num_vertices, void *stream,
                        gv_graph **out);
gv_status gv_set_insert_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              const uint64_t *d_offsets, uint64_t *d_counts, void *stream);
gv_status gv_set_delete_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              const uint64_t *d_offsets, uint64_t *d_counts, void *stream);
gv_status gv_set_query_edges(gv_graph *set, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                             const uint64_t *d_offsets, uint64_t *d_counts, uint8_t *d_out, void *stream);
gv_status gv_set_member_neighbors(gv_graph *set, uint32_t member, uint64_t *offsets, uint32_t *nbrs,
                                  uint64_t nbr_capacity, uint64_t *total, void *stream);

/*
 * gv_degree_offsets_noalloc -- CSR offsets of the listed vertices' current
 * out-degrees, computed without allocating any memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory at the point of the call: serving loops that must not stall
 * on an allocation (cudaFree synchronises the whole device), processes whose
 * device memory is all held by another allocator (a framework's caching
 * allocator), and code that runs under a fixed device-memory budget.
 *   d_vids     n uint32 vertex ids, DEVICE memory only.
 *   n          at most 67,108,864 (2^26); larger n returns GV_ERR_INVALID_ARG
 *              and does nothing.
 *   d_offsets  n+1 uint64, DEVICE memory only: offsets[i] = sum of the degrees
 *              of vids[0 .. i-1], offsets[n] = the total.  Invalid or deleted
 *              ids count 0.  The same offsets gv_neighbors returns.
 * Host arrays are rejected with GV_ERR_INVALID_ARG (staging them would
 * allocate).  Asynchronous on `stream`; nothing is read back.
 * Scratch: the scan's chunk sums live in one fixed 512 KiB device array that
 * every GPU loading this library holds until the process exits.  All calls
 * on a device share it and it keeps the last call's contents (every call
 * overwrites the part it uses, so nothing needs clearing); calls whose work
 * overlaps on the GPU -- on different streams without ordering, from any
 * graph -- race on it and must be serialised by the caller.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress),
 * and so does the first call after the device's context was replaced (for
 * example by cudaDeviceReset); make that first call before any stream
 * capture begins.  An error already pending in the CUDA runtime when the
 * call starts (from the caller's own launches) is returned as GV_ERR_CUDA
 * and left pending, not cleared.
 */
gv_status gv_degree_offsets_noalloc(gv_graph *g, const uint32_t *d_vids, uint32_t n, uint64_t *d_offsets,
                                    void *stream);

/*
 * gv_reblock -- change the edge-block size C of a built graph ("dynamically
 * changing the edge block size", the paper's future work: the average
 * degree, and with it the best C, drifts over many batch updates).  Every
 * stored entry (with its payload) stays; only the blocking changes: each
 * vertex gets ceil(deg / C) blocks of the new size, taken as one contiguous
 * run of the pool, and the pool memory (the same bytes: library-owned,
 * grown, or the caller's pool_mem) is laid out again for the new C.
 *   block_capacity  the new C: a multiple of 4 in [4, 512]; 0 for the
 *                   paper's rule over the current degrees ("Initialization":
 *                   the average degree of the vertices with at least one
 *                   entry, rounded up to a multiple of 4, at least 4); or
 *                   GV_REBLOCK_MIN_FOOTPRINT for the C of least pool
 *                   footprint over the current degrees: a block costs 4C
 *                   bytes of slots (8C on a weighted graph) plus 12 bytes of
 *                   links and queue entry, a vertex of degree d holds
 *                   ceil(d / C) blocks, and the C in {4, 8, ..., 512} of
 *                   least total wins (the smallest on ties).
 *   h_block_capacity optional host uint32: the C now in use.
 * Returns GV_ERR_STATE if no edge batch has fixed C yet, a latched device
 * error if one is pending, GV_ERR_OUT_OF_MEMORY if the entries do not fit
 * the pool at the new size or the scratch cannot be allocated -- all three
 * before anything changes -- and GV_ERR_CUDA if a copy fails after the
 * layout was switched (the graph is then undefined).
 * Scratch: 4 bytes per slot of the new layout (8 on a weighted graph) in
 * the graph's delete/query scratch, plus 12 bytes per vertex in its staging
 * buffers; like all of the graph's scratch it grows when needed and is kept
 * until gv_destroy.
 * With hub runs (gv_config.hub_shift), the run region is laid out again
 * for the new C with the same share of the pool; every vertex whose degree
 * reaches the hub threshold at the new C (hub_degree, or C * 2^s) gets its
 * blocks as whole runs there, every other vertex as plain blocks outside
 * it; GV_ERR_OUT_OF_MEMORY (nothing changed) if either part does not fit.
 * Synchronises `stream` (it reads the degree totals).
 */
#define GV_REBLOCK_MIN_FOOTPRINT 1u
gv_status gv_reblock(gv_graph *g, uint32_t block_capacity, uint32_t *h_block_capacity, void *stream);

/*
 * gv_serve -- continuous batching of a stream of requests on one graph (the
 * serving form of the batched update path: requests arriving while earlier
 * work runs are merged into runs whose device work overlaps).  Each request
 * is an insert, delete or query batch of n (src, dst) pairs with an arrival
 * time; once arrived, consecutive requests of one kind (at most max_reqs
 * requests and merge_pairs pairs) form one run: one segmented insert
 * (gv_insert_edges_segmented), one segmented delete
 * (gv_delete_edges_segmented) or one query batch, so every request gets the
 * result it would get alone, applied in arrival order.  Up to `slots` runs
 * are in flight: the upload of a run's pairs, its call and the download of
 * its results run on three streams of the loop's own, ordered by events, so
 * that one run's copies overlap another's kernels.  Calls stay in arrival
 * order.  An insert run is admitted while its worst-case block demand
 * (ceil(n / C) blocks plus one per touched source, a whole run per source
 * with hub runs) fits the free blocks last read; else the loop waits for the
 * runs in flight and reads the pool again; a run that still does not fit
 * fails (status GV_ERR_OUT_OF_MEMORY, counts {0, 0}) unless the graph has
 * GV_GROW.
 *   reqs     n_reqs requests (host memory, caller-owned): the kind, n, src,
 *            dst, answers and arrival fields are inputs; status, done and
 *            counts are outputs.  src and dst in pinned host memory are
 *            uploaded as they are; other host memory is copied into the
 *            loop's pinned staging first.  Query answers (1 = stored) go to
 *            `answers` (n bytes of host memory).
 *   cfg      NULL for the defaults: slots 4 (1..64), max_reqs 1024
 *            (1..1024), merge_pairs 2,000,000 (every request must hold at
 *            most this many pairs); realtime 1 honours the arrival times
 *            (seconds after the call starts, non-decreasing), 0 treats
 *            every request as arrived at the start.
 *   h_stats  optional host uint64[2]: runs launched, requests merged.
 *   stream   the stream of the library calls (as for every other entry
 *            point; it stays the graph's stream after the loop).  Uploads
 *            and downloads run on two streams the loop creates and
 *            destroys.
 * Allocates the loop's device and pinned buffers (slots of merge_pairs
 * pairs) and reserves the graph's scratch for merge_pairs pairs at the
 * start; frees the loop's buffers before returning.  Returns when every
 * request has completed (or failed); GV_ERR_INVALID_ARG for a malformed
 * request or configuration, before anything runs.
 */
#define GV_SERVE_INSERT 0u
#define GV_SERVE_DELETE 1u
#define GV_SERVE_QUERY 2u
typedef struct gv_serve_request {
    uint32_t kind;          /* GV_SERVE_INSERT, GV_SERVE_DELETE or GV_SERVE_QUERY */
    int32_t status;         /* out: GV_OK, or GV_ERR_OUT_OF_MEMORY for an insert that did not fit */
    uint64_t n;             /* pairs */
    const uint32_t *src;    /* n source ids (host) */
    const uint32_t *dst;    /* n destination ids (host) */
    uint8_t *answers;       /* queries: n answers (host); unused otherwise */
    double arrival;         /* seconds after the start of the call */
    double done;            /* out: when the loop saw the request's run complete (same clock) */
    uint64_t counts[2];     /* out: inserts and deletes, {done, rejected} */
} gv_serve_request;
typedef struct gv_serve_config {
    uint32_t slots;
    uint32_t max_reqs;
    uint64_t merge_pairs;
    uint32_t realtime;
    uint32_t reserved;
} gv_serve_config;
gv_status gv_serve(gv_graph *g, gv_serve_request *reqs, uint64_t n_reqs, const gv_serve_config *cfg,
                   uint64_t *h_stats, void *stream);

/* gv_status_string -- a static, human-readable name for a status code. */
const char *gv_status_string(gv_status s);

/*
 * Graph analytics over the stored structure.  The paper lists analytics on
 * the dynamic structure as future work ("Conclusion and future work") and
 * defines none; these calls compute the textbook quantities, reading each
 * adjacency through its tree of edge blocks as the delete and query paths do.
 *
 * gv_bfs -- unweighted single-source distances (level-synchronous
 * breadth-first search over stored entries).
 *   source    a vertex id < the vertex count (else GV_ERR_INVALID_ARG); a
 *             deleted source reaches nothing.
 *   dist      n uint32 (device or host), n = vertex count: dist[source] = 0,
 *             dist[v] = length of a shortest path of stored edges, and
 *             0xFFFFFFFF for unreached vertices.
 *   h_levels  optional host uint32: number of distinct finite distances.
 * Synchronises `stream` once per four levels (it reads the frontier size).
 */
gv_status gv_bfs(gv_graph *g, uint32_t source, uint32_t *dist, uint32_t *h_levels, void *stream);

/*
 * gv_sssp -- single-source shortest path lengths (the paper's future work
 * names shortest paths beside BFS).  The length of a stored entry is its
 * 32-bit payload on a graph created with GV_WEIGHTED (0 for entries inserted
 * without one) and 1 otherwise, so on an unweighted graph the result equals
 * gv_bfs's distances.  Computed by Bellman-Ford rounds over a frontier of
 * vertices whose distance fell; the distances are unique, the number of
 * rounds depends on the order of the atomic minima.
 *   source    a vertex id < the vertex count (else GV_ERR_INVALID_ARG); a
 *             deleted source reaches nothing.
 *   dist      n uint64 (device or host), n = vertex count: dist[source] = 0,
 *             dist[v] = minimum over paths of stored entries of the summed
 *             lengths, and 0xFFFFFFFFFFFFFFFF for unreached vertices.
 *   h_rounds  optional host uint32: relaxation rounds that had a non-empty
 *             frontier.
 * Synchronises `stream` once per four rounds (it reads the frontier size).
 */
gv_status gv_sssp(gv_graph *g, uint32_t source, uint64_t *dist, uint32_t *h_rounds, void *stream);

/*
 * gv_pagerank -- `iterations` steps of PageRank power iteration in fp64 over
 * the N live vertices: r_0 = 1/N; r'(v) = (1 - d)/N + d * (sum over stored
 * entries (u, v) of r(u)/deg(u) + (sum of r(u) over live u with deg(u) = 0)/N),
 * where every stored copy of a pair counts.  Deleted vertices get 0.
 *   damping   d in [0, 1] (else GV_ERR_INVALID_ARG).
 *   rank      n doubles (device or host), n = vertex count.
 * The per-entry sums are fp64 atomic additions, so the summation order (and
 * the last bits) can differ from run to run.
 */
gv_status gv_pagerank(gv_graph *g, uint32_t iterations, double damping, double *rank, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHVINE_H */

/*
 * GraphVine CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU model of what the dynamic-graph hot
 * path computes (GraphVine, "A Data Structure to Optimize Dynamic Graph
 * Processing on GPUs", sections "Dynamic vertex updates", "Dynamic edge
 * updates" and "Querying operations"; Algorithms 1, 2 and 3).  It keeps one
 * sorted array of destination ids per source vertex plus an alive flag per
 * vertex and applies one operation at a time, in call order.  An entry may
 * carry a 32-bit payload (a weight; 0 for unweighted inserts) that stays
 * with it through deletes and compaction.  There is no
 * blocking, no block pool, no tree: only the result the paper's structure
 * must reproduce.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The GPU library shares no code with it.
 *
 * Readings of the paper fixed here (the paper is silent or ambiguous):
 *   - inserts are multiset appends (Algorithm 1 appends without a duplicate
 *     check); with ORC_DEDUP a pair is added only if absent from the
 *     adjacency and not already added by the same batch;
 *   - a delete removes every stored copy of each (u, v) in the batch
 *     (Algorithm 2 marks every stored entry equal to a batch entry); repeated
 *     batch entries are idempotent; deleting an absent pair is a no-op;
 *   - a pair with an endpoint out of range or not alive is rejected and
 *     counted, for inserts and deletes alike;
 *   - a vertex delete clears the vertex's adjacency and removes every edge
 *     pointing at it; ids are never reused (the dictionary keeps its slot,
 *     section "Dynamic vertex updates").
 *
 * Pure C99; builds with gcc on x86-64 and AArch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gv_oracle_internal.h"

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

void adj_reserve(orc_adj *a, uint64_t need) {
    if (need <= a->cap) return;
    uint64_t c = a->cap ? a->cap : 4;
    while (c < need) c *= 2;
    a->v = (uint32_t *)realloc(a->v, c * sizeof(uint32_t));
    a->w = (uint32_t *)realloc(a->w, c * sizeof(uint32_t));
    a->cap = c;
}

/* Sorts an adjacency by (v, w): the canonical order of its entries. */
void adj_sort(orc_adj *a) {
    uint64_t *k = (uint64_t *)malloc((a->n ? a->n : 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < a->n; ++i) k[i] = ((uint64_t)a->v[i] << 32) | a->w[i];
    qsort(k, a->n, sizeof(uint64_t), cmp_u64);
    for (uint64_t i = 0; i < a->n; ++i) {
        a->v[i] = (uint32_t)(k[i] >> 32);
        a->w[i] = (uint32_t)(k[i] & 0xFFFFFFFFu);
    }
    free(k);
}

/* 1 if x occurs in the sorted array a[0..n). */
int sorted_contains(const uint32_t *a, uint64_t n, uint32_t x) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == x;
}

static void ensure_cap(orc_graph *g, uint32_t need) {
    if (need <= g->cap) return;
    uint32_t c = g->cap ? g->cap : 1;
    while (c < need) c *= 2;
    g->alive = (uint8_t *)realloc(g->alive, c);
    g->adj = (orc_adj *)realloc(g->adj, (size_t)c * sizeof(orc_adj));
    memset(g->alive + g->cap, 0, c - g->cap);
    memset(g->adj + g->cap, 0, (size_t)(c - g->cap) * sizeof(orc_adj));
    g->cap = c;
}

/* create(nv): nv live vertices, no edges. */
orc_graph *orc_create(uint32_t nv, uint32_t flags) {
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    g->flags = flags;
    ensure_cap(g, nv ? nv : 1);
    g->nv = nv;
    for (uint32_t i = 0; i < nv; ++i) g->alive[i] = 1;
    return g;
}

void orc_destroy(orc_graph *g) {
    if (!g) return;
    for (uint32_t i = 0; i < g->cap; ++i) {
        free(g->adj[i].v);
        free(g->adj[i].w);
    }
    free(g->adj);
    free(g->alive);
    free(g);
}

int valid_pair(const orc_graph *g, uint32_t u, uint32_t v) {
    return u < g->nv && v < g->nv && g->alive[u] && g->alive[v];
}

/*
 * Sort the batch's valid pairs by (u, v) so that each source's batch entries
 * form one run.  This is plain preparation of the input, the CSR form that
 * the paper assumes for every batch (section "Initialization and batch
 * updates"); rejected pairs are counted here.
 */
static uint64_t *sorted_valid_keys(const orc_graph *g, const uint32_t *src, const uint32_t *dst,
                                   uint64_t n, uint64_t *n_valid, uint64_t *rejected) {
    uint64_t *k = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t m = 0, rej = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (valid_pair(g, src[i], dst[i])) k[m++] = ((uint64_t)src[i] << 32) | dst[i];
        else ++rej;
    }
    qsort(k, m, sizeof(uint64_t), cmp_u64);
    *n_valid = m;
    *rejected = rej;
    return k;
}

int cmp_triple(const void *a, const void *b) {
    const orc_triple *x = (const orc_triple *)a, *y = (const orc_triple *)b;
    if (x->u != y->u) return (x->u > y->u) - (x->u < y->u);
    if (x->v != y->v) return (x->v > y->v) - (x->v < y->v);
    return (x->w > y->w) - (x->w < y->w);
}

/*
 * insert_edges (Algorithm 1): every valid (u, v) is appended to u's
 * adjacency, with its payload w (0 when w is NULL).  Under ORC_DEDUP the
 * pair is added only when v is not yet in adj[u] and was not already added
 * by this batch.  The batch's valid pairs are sorted by (u, v, w) first (the
 * CSR form the paper assumes for a batch, "Initialization and batch
 * updates").
 */
void orc_insert_edges_weighted(orc_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                               uint64_t n, uint64_t *inserted, uint64_t *rejected) {
    orc_triple *k = (orc_triple *)malloc((n ? n : 1) * sizeof(orc_triple));
    uint64_t m = 0, rej = 0, ins = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (valid_pair(g, src[i], dst[i])) {
            k[m].u = src[i];
            k[m].v = dst[i];
            k[m].w = w ? w[i] : 0u;
            ++m;
        } else {
            ++rej;
        }
    }
    qsort(k, m, sizeof(orc_triple), cmp_triple);
    uint64_t i = 0;
    while (i < m) {
        uint32_t u = k[i].u;
        uint64_t j = i;
        while (j < m && k[j].u == u) ++j;
        orc_adj *a = &g->adj[u];
        uint64_t old_n = a->n;
        adj_reserve(a, a->n + (j - i));
        for (uint64_t t = i; t < j; ++t) {
            uint32_t v = k[t].v;
            if (g->flags & ORC_DEDUP) {
                if (sorted_contains(a->v, old_n, v)) continue;          /* already in the graph */
                if (a->n > old_n && a->v[a->n - 1] == v) continue;     /* already added (batch sorted) */
            }
            a->v[a->n] = v;
            a->w[a->n] = k[t].w;
            ++a->n;
            ++ins;
        }
        adj_sort(a);
        i = j;
    }
    free(k);
    g->num_edges += ins;
    if (inserted) *inserted = ins;
    if (rejected) *rejected = rej;
}

void orc_insert_edges(orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                      uint64_t *inserted, uint64_t *rejected) {
    orc_insert_edges_weighted(g, src, dst, NULL, n, inserted, rejected);
}

/*
 * delete_edges (Algorithm 2): for each source u, D(u) is the set of batch
 * destinations; every stored entry of adj[u] equal to a member of D(u) is
 * removed.  deleted counts removed entries.
 */
void orc_delete_edges(orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                      uint64_t *deleted, uint64_t *rejected) {
    uint64_t m, rej, del = 0;
    uint64_t *k = sorted_valid_keys(g, src, dst, n, &m, &rej);
    uint32_t *dset = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t i = 0;
    while (i < m) {
        uint32_t u = (uint32_t)(k[i] >> 32);
        uint64_t j = i;
        while (j < m && (uint32_t)(k[j] >> 32) == u) ++j;
        uint64_t nd = 0;
        for (uint64_t t = i; t < j; ++t) dset[nd++] = (uint32_t)(k[t] & 0xFFFFFFFFu); /* sorted */
        orc_adj *a = &g->adj[u];
        uint64_t w = 0;
        for (uint64_t r = 0; r < a->n; ++r) {
            if (sorted_contains(dset, nd, a->v[r])) {
                ++del;
            } else {
                a->w[w] = a->w[r];
                a->v[w++] = a->v[r];
            }
        }
        a->n = w;
        i = j;
    }
    free(dset);
    free(k);
    g->num_edges -= del;
    if (deleted) *deleted = del;
    if (rejected) *rejected = rej;
}

/* query (Algorithm 3): out[i] = 1 iff the pair is valid and dst is in adj[src]. */
void orc_query_edges(const orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n,
                     uint8_t *out) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t u = src[i], v = dst[i];
        out[i] = (uint8_t)(valid_pair(g, u, v) && sorted_contains(g->adj[u].v, g->adj[u].n, v));
    }
}

/* insert_vertices (section "Dynamic vertex updates"): ids nv .. nv+k-1, alive. */
uint32_t orc_insert_vertices(orc_graph *g, uint32_t k, uint32_t *new_ids) {
    uint32_t first = g->nv;
    ensure_cap(g, g->nv + k);
    for (uint32_t i = 0; i < k; ++i) {
        g->alive[first + i] = 1;
        if (new_ids) new_ids[i] = first + i;
    }
    g->nv += k;
    return first;
}

/*
 * delete_vertices: every valid, alive id in ids is marked dead, its adjacency
 * is cleared, and every entry pointing at it is removed from all adjacencies.
 * Returns the number of vertices that were deleted (invalid or already-dead
 * ids are ignored).
 */
uint32_t orc_delete_vertices(orc_graph *g, const uint32_t *ids, uint32_t k) {
    uint8_t *gone = (uint8_t *)calloc(g->nv ? g->nv : 1, 1);
    uint32_t cnt = 0;
    for (uint32_t i = 0; i < k; ++i) {
        uint32_t s = ids[i];
        if (s < g->nv && g->alive[s] && !gone[s]) { gone[s] = 1; ++cnt; }
    }
    for (uint32_t s = 0; s < g->nv; ++s) {
        if (!gone[s]) continue;
        g->alive[s] = 0;
        g->num_edges -= g->adj[s].n;
        g->adj[s].n = 0;
    }
    for (uint32_t u = 0; u < g->nv; ++u) {
        orc_adj *a = &g->adj[u];
        uint64_t w = 0;
        for (uint64_t r = 0; r < a->n; ++r) {
            if (gone[a->v[r]]) {
                g->num_edges -= 1;
            } else {
                a->w[w] = a->w[r];
                a->v[w++] = a->v[r];
            }
        }
        a->n = w;
    }
    free(gone);
    return cnt;
}

uint32_t orc_num_vertices(const orc_graph *g) { return g->nv; }
uint64_t orc_num_edges(const orc_graph *g) { return g->num_edges; }

void orc_degrees(const orc_graph *g, uint32_t *deg) {
    for (uint32_t u = 0; u < g->nv; ++u) deg[u] = (uint32_t)g->adj[u].n;
}

void orc_alive(const orc_graph *g, uint8_t *out) { memcpy(out, g->alive, g->nv); }

/*
 * neighbors: CSR of the listed vertices' adjacencies in canonical (sorted)
 * order.  offsets has n+1 entries.  Returns the total; writes nbrs only when
 * the total fits in cap.  Invalid or dead ids get an empty list.
 */
uint64_t orc_neighbors(const orc_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets,
                       uint32_t *nbrs, uint64_t cap) {
    uint64_t tot = 0;
    for (uint32_t i = 0; i < n; ++i) {
        offsets[i] = tot;
        uint32_t u = vids[i];
        if (u < g->nv && g->alive[u]) tot += g->adj[u].n;
    }
    offsets[n] = tot;
    if (tot > cap || !nbrs) return tot;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u = vids[i];
        if (u < g->nv && g->alive[u] && g->adj[u].n)
            memcpy(nbrs + offsets[i], g->adj[u].v, g->adj[u].n * sizeof(uint32_t));
    }
    return tot;
}

/* neighbors with payloads: as orc_neighbors, plus wts[] aligned with nbrs
 * (entries in (v, w) order). */
uint64_t orc_neighbors_weighted(const orc_graph *g, const uint32_t *vids, uint32_t n, uint64_t *offsets,
                                uint32_t *nbrs, uint32_t *wts, uint64_t cap) {
    uint64_t tot = orc_neighbors(g, vids, n, offsets, nbrs, cap);
    if (tot > cap || !nbrs || !wts) return tot;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u = vids[i];
        if (u < g->nv && g->alive[u] && g->adj[u].n)
            memcpy(wts + offsets[i], g->adj[u].w, g->adj[u].n * sizeof(uint32_t));
    }
    return tot;
}

/* Full canonical CSR: offsets[nv+1], nbrs[num_edges]. */
void orc_export_csr(const orc_graph *g, uint64_t *offsets, uint32_t *nbrs) {
    uint64_t tot = 0;
    for (uint32_t u = 0; u < g->nv; ++u) {
        offsets[u] = tot;
        if (g->adj[u].n) memcpy(nbrs + tot, g->adj[u].v, g->adj[u].n * sizeof(uint32_t));
        tot += g->adj[u].n;
    }
    offsets[g->nv] = tot;
}

/* ------------------------------------------------------------------------
 * Structural sizing rules of the paper.  They fix the shape of the GPU
 * structure (how many blocks, where each block hangs in the tree), not the
 * graph it stores, and are pinned against the paper's worked examples.
 * ------------------------------------------------------------------------ */

/* Vertex dictionary capacity: the power of two at or above n (section
 * "Vertex dictionary and adjacency list structure": 453 vertices -> 512). */
uint64_t orc_dictionary_capacity(uint64_t n) {
    uint64_t c = 1;
    while (c < n) c <<= 1;
    return c;
}

/* Edge blocks an adjacency of degree deg occupies when every block but the
 * last is full: ceil(deg / C). */
uint64_t orc_blocks_for_degree(uint64_t deg, uint32_t C) { return (deg + C - 1) / C; }

/*
 * Edge-block size rule (section "Initialization"): the average degree of the
 * vertices with non-zero degree in the first batch.  Rounding is not stated;
 * the reading taken: ceil of the average, rounded up to a multiple of 4, at
 * least 4 (so that blocks hold whole 16-byte vectors) and at most 512 (the
 * paper bounds neither end; 512 slots is the largest block the structure
 * takes, so a mean degree above 512 gives C = 512).
 */
uint32_t orc_block_capacity_rule(const uint32_t *deg, uint32_t nv) {
    uint64_t sum = 0, nz = 0;
    for (uint32_t u = 0; u < nv; ++u) if (deg[u]) { sum += deg[u]; ++nz; }
    if (nz == 0) return 4;
    uint64_t avg = (sum + nz - 1) / nz;
    uint64_t c = (avg + 3) / 4 * 4;
    if (c < 4) c = 4;
    if (c > 512) c = 512;
    return (uint32_t)c;
}

/*
 * Block size of least pool footprint (the paper's future work: changing the
 * edge-block size to cut the internal fragmentation of the blocks).  A block
 * of C slots costs 4C bytes of slots (8C with a 32-bit payload per slot)
 * plus 12 bytes of tree links and queue entry; a vertex of degree d holds
 * ceil(d / C) blocks.  Returns the C in {4, 8, ..., 512} of least total
 * bytes over the given degrees, the smallest such C on ties.
 */
uint32_t orc_min_footprint_capacity(const uint32_t *deg, uint32_t nv, int weighted) {
    uint32_t best_c = 4;
    uint64_t best = UINT64_MAX;
    for (uint32_t c = 4; c <= 512; c += 4) {
        uint64_t blocks = 0;
        for (uint32_t u = 0; u < nv; ++u) blocks += ((uint64_t)deg[u] + c - 1) / c;
        const uint64_t bytes = blocks * (4ull * c * (weighted ? 2u : 1u) + 12u);
        if (bytes < best) {
            best = bytes;
            best_c = c;
        }
    }
    return best_c;
}

/*
 * Bit string placing the k-th block (1-based) of a complete binary tree
 * (section "Dynamic edge inserts"): the binary form of k without its leading
 * 1; '0' = go left, '1' = go right, the last step names the side on which
 * the block hangs (the ninth block gets "001").  Writes a NUL-terminated
 * string and returns its length.
 */
uint32_t orc_cbt_path(uint64_t k, char *out) {
    int top = 63;
    while (top > 0 && !((k >> top) & 1u)) --top;
    uint32_t len = 0;
    for (int b = top - 1; b >= 0; --b) out[len++] = ((k >> b) & 1u) ? '1' : '0';
    out[len] = '\0';
    return len;
}

/*
 * Parallel pop ranges (section "Dynamic edge inserts", Figure 3): with
 * incl[] the inclusive prefix sum of per-vertex block demand, thread i pops
 * queue slots [incl[i-1], incl[i]) (thread 0: [0, incl[0])).
 */
void orc_pop_ranges(const uint32_t *need, uint32_t n, uint64_t *begin, uint64_t *end) {
    uint64_t run = 0;
    for (uint32_t i = 0; i < n; ++i) {
        begin[i] = run;
        run += need[i];
        end[i] = run;
    }
}

/*
 * Blocks a source needs for an insert of cnt edges when its adjacency has
 * degree deg and every block but the last is full (Algorithm 1: the free
 * slots of the last block are used first): ceil(max(0, cnt - space) / C)
 * with space = (C - deg mod C) mod C.
 */
uint64_t orc_insert_block_demand(uint64_t deg, uint64_t cnt, uint32_t C) {
    uint64_t space = (C - deg % C) % C;
    if (cnt <= space) return 0;
    return (cnt - space + C - 1) / C;
}

/*
 * Graph analytics over the stored structure.  The paper names analytics on
 * the dynamic structure as future work ("Conclusion and future work") and
 * defines none; these are the textbook definitions.
 *
 * orc_bfs: unweighted single-source distances (breadth-first search, level
 * by level): dist[source] = 0 if the source is alive, dist[v] = 1 + min over
 * stored entries (u, v) with u at distance dist[u]; unreached (and every
 * vertex when the source is dead) = 0xFFFFFFFF.  Returns the number of
 * levels (largest finite distance + 1; 0 when nothing is reached).
 */
uint32_t orc_bfs(const orc_graph *g, uint32_t source, uint32_t *dist) {
    for (uint32_t v = 0; v < g->nv; ++v) dist[v] = 0xFFFFFFFFu;
    if (source >= g->nv || !g->alive[source]) return 0;
    uint32_t *cur = (uint32_t *)malloc(sizeof(uint32_t) * (g->nv + 1));
    uint32_t *nxt = (uint32_t *)malloc(sizeof(uint32_t) * (g->nv + 1));
    uint32_t ncur = 1, level = 0;
    cur[0] = source;
    dist[source] = 0;
    while (ncur > 0) {
        uint32_t nnxt = 0;
        for (uint32_t i = 0; i < ncur; ++i) {
            const orc_adj *a = &g->adj[cur[i]];
            for (uint64_t j = 0; j < a->n; ++j) {
                const uint32_t v = a->v[j];
                if (dist[v] == 0xFFFFFFFFu) {
                    dist[v] = level + 1;
                    nxt[nnxt++] = v;
                }
            }
        }
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
        ncur = nnxt;
        ++level;
    }
    free(cur);
    free(nxt);
    return level;
}

/*
 * orc_pagerank: power iteration of PageRank with damping d over the alive
 * vertices (N of them), in fp64.  r_0 = 1/N; each iteration
 *   r'(v) = (1 - d)/N + d * ( sum over stored entries (u, v) of r(u)/deg(u)
 *                             + (sum of r(u) over alive u with deg(u) = 0)/N )
 * (a stored entry counts once per copy, so a multigraph weights parallel
 * edges by their multiplicity).  Dead vertices get 0.  N = 0: all 0.
 */
void orc_pagerank(const orc_graph *g, uint32_t iterations, double damping, double *rank) {
    uint64_t N = 0;
    for (uint32_t v = 0; v < g->nv; ++v) N += g->alive[v] ? 1u : 0u;
    for (uint32_t v = 0; v < g->nv; ++v) rank[v] = (N && g->alive[v]) ? 1.0 / (double)N : 0.0;
    if (N == 0) return;
    double *acc = (double *)malloc(sizeof(double) * (g->nv + 1));
    for (uint32_t it = 0; it < iterations; ++it) {
        double dangling = 0.0;
        for (uint32_t v = 0; v < g->nv; ++v) acc[v] = 0.0;
        for (uint32_t u = 0; u < g->nv; ++u) {
            if (!g->alive[u]) continue;
            const orc_adj *a = &g->adj[u];
            if (a->n == 0) {
                dangling += rank[u];
                continue;
            }
            for (uint64_t j = 0; j < a->n; ++j) acc[a->v[j]] += rank[u] / (double)a->n;
        }
        for (uint32_t v = 0; v < g->nv; ++v)
            rank[v] = g->alive[v] ? (1.0 - damping) / (double)N + damping * (acc[v] + dangling / (double)N) : 0.0;
    }
    free(acc);
}

/*
 * orc_sssp: single-source shortest path lengths (Dijkstra's algorithm with a
 * binary heap and lazy deletion), the third analytic the paper's future work
 * names beside BFS.  The length of a stored entry (u, v) is its payload when
 * `weighted` is non-zero, else 1 (so the result equals orc_bfs's distances).
 * dist[source] = 0 if the source is alive; dist[v] = min over stored entries
 * (u, v) of dist[u] + length; unreached (and every vertex when the source is
 * dead) = UINT64_MAX.  Returns the number of reached vertices.
 */
typedef struct {
    uint64_t d;
    uint32_t v;
} orc_heap_item;

static void heap_push(orc_heap_item *h, uint64_t *n, orc_heap_item x) {
    uint64_t i = (*n)++;
    while (i > 0) {
        const uint64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static orc_heap_item heap_pop(orc_heap_item *h, uint64_t *n) {
    const orc_heap_item top = h[0];
    const orc_heap_item last = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && h[c + 1].d < h[c].d) ++c;
        if (last.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    if (*n > 0) h[i] = last;
    return top;
}

uint32_t orc_sssp(const orc_graph *g, uint32_t source, int weighted, uint64_t *dist) {
    for (uint32_t v = 0; v < g->nv; ++v) dist[v] = UINT64_MAX;
    if (source >= g->nv || !g->alive[source]) return 0;
    /* one heap entry per improvement: at most num_edges + 1 */
    orc_heap_item *h = (orc_heap_item *)malloc(sizeof(orc_heap_item) * (g->num_edges + 1));
    uint8_t *done = (uint8_t *)calloc(g->nv, 1);
    uint64_t n = 0;
    uint32_t reached = 0;
    dist[source] = 0;
    heap_push(h, &n, (orc_heap_item){0, source});
    while (n > 0) {
        const orc_heap_item x = heap_pop(h, &n);
        if (done[x.v] || x.d != dist[x.v]) continue;
        done[x.v] = 1;
        ++reached;
        const orc_adj *a = &g->adj[x.v];
        for (uint64_t j = 0; j < a->n; ++j) {
            const uint32_t v = a->v[j];
            const uint64_t nd = x.d + (weighted ? (uint64_t)a->w[j] : 1u);
            if (nd < dist[v]) {
                dist[v] = nd;
                heap_push(h, &n, (orc_heap_item){nd, v});
            }
        }
    }
    free(h);
    free(done);
    return reached;
}

/*
 * Parallel CPU baseline -- MEASUREMENT INFRASTRUCTURE ONLY.
 *
 * The oracle's sorted-vector algorithm (one sorted array per source; a batch
 * is grouped by source, inserts append and re-sort, deletes filter against
 * the sorted batch set, queries binary-search), run with OpenMP over all host
 * cores: the batch's valid pairs are bucketed by source range with a
 * parallel counting sort, and each bucket (a disjoint set of sources) is
 * processed by one thread, so no two threads touch the same adjacency.  It
 * works on the oracle's graph object and gives the oracle's results (the
 * tests check that); it exists to time a multi-core CPU against the GPU path
 * on the same step.  Only the benchmark's CPU-baseline leg and the tests
 * load it.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gv_oracle_internal.h"

/* Sources per bucket: buckets are contiguous id ranges. */
static uint32_t bucket_shift(uint32_t nv, int threads) {
    uint32_t shift = 0;
    const uint64_t want = (uint64_t)threads * 64; /* enough buckets to balance */
    while ((((uint64_t)nv + (1ull << shift) - 1) >> shift) > want && shift < 31) ++shift;
    return shift;
}

/*
 * Valid pairs of the batch as (u, v, w) triples grouped by bucket (stable
 * within a thread's range of the input), with bucket offsets boff[nb + 1].
 * Returns the triples; *rejected = pairs with an invalid or dead endpoint.
 */
static orc_triple *bucket_pairs(const orc_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                                uint64_t n, int threads, uint32_t shift, uint32_t nb, uint64_t **boff_out,
                                uint64_t *rejected) {
    uint64_t *cnt = (uint64_t *)calloc((size_t)threads * nb + 1, sizeof(uint64_t));
    uint64_t rej = 0;
#pragma omp parallel num_threads(threads) reduction(+ : rej)
    {
        const int t = omp_get_thread_num();
        const uint64_t lo = n * t / threads, hi = n * (t + 1) / threads;
        uint64_t *c = cnt + (size_t)t * nb;
        for (uint64_t i = lo; i < hi; ++i) {
            if (valid_pair(g, src[i], dst[i])) ++c[src[i] >> shift];
            else ++rej;
        }
    }
    /* exclusive offsets in (bucket, thread) order */
    uint64_t *boff = (uint64_t *)malloc(((size_t)nb + 1) * sizeof(uint64_t));
    uint64_t run = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        boff[b] = run;
        for (int t = 0; t < threads; ++t) {
            const uint64_t x = cnt[(size_t)t * nb + b];
            cnt[(size_t)t * nb + b] = run;
            run += x;
        }
    }
    boff[nb] = run;
    orc_triple *k = (orc_triple *)malloc((run ? run : 1) * sizeof(orc_triple));
#pragma omp parallel num_threads(threads)
    {
        const int t = omp_get_thread_num();
        const uint64_t lo = n * t / threads, hi = n * (t + 1) / threads;
        uint64_t *c = cnt + (size_t)t * nb;
        for (uint64_t i = lo; i < hi; ++i) {
            if (!valid_pair(g, src[i], dst[i])) continue;
            orc_triple *o = &k[c[src[i] >> shift]++];
            o->u = src[i];
            o->v = dst[i];
            o->w = w ? w[i] : 0u;
        }
    }
    free(cnt);
    *boff_out = boff;
    *rejected = rej;
    return k;
}

/* Batch insert (the oracle's Algorithm 1 reading, multiset or set semantics). */
void orc_par_insert_edges(orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, int threads,
                          uint64_t *inserted, uint64_t *rejected) {
    if (threads < 1) threads = 1;
    const uint32_t shift = bucket_shift(g->nv, threads);
    const uint32_t nb = (uint32_t)(((uint64_t)g->nv + (1ull << shift) - 1) >> shift) + 1;
    uint64_t *boff, rej, ins = 0;
    orc_triple *k = bucket_pairs(g, src, dst, NULL, n, threads, shift, nb, &boff, &rej);
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1) reduction(+ : ins)
    for (uint32_t b = 0; b < nb; ++b) {
        orc_triple *kb = k + boff[b];
        const uint64_t m = boff[b + 1] - boff[b];
        if (m == 0) continue;
        qsort(kb, m, sizeof(orc_triple), cmp_triple);
        uint64_t i = 0;
        while (i < m) {
            const uint32_t u = kb[i].u;
            uint64_t j = i;
            while (j < m && kb[j].u == u) ++j;
            orc_adj *a = &g->adj[u];
            const uint64_t old_n = a->n;
            adj_reserve(a, a->n + (j - i));
            for (uint64_t t = i; t < j; ++t) {
                const uint32_t v = kb[t].v;
                if (g->flags & ORC_DEDUP) {
                    if (sorted_contains(a->v, old_n, v)) continue;
                    if (a->n > old_n && a->v[a->n - 1] == v) continue;
                }
                a->v[a->n] = v;
                a->w[a->n] = kb[t].w;
                ++a->n;
                ++ins;
            }
            adj_sort(a);
            i = j;
        }
    }
    free(k);
    free(boff);
    g->num_edges += ins;
    if (inserted) *inserted = ins;
    if (rejected) *rejected = rej;
}

/* Batch delete (the oracle's Algorithm 2 reading: every stored copy goes). */
void orc_par_delete_edges(orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, int threads,
                          uint64_t *deleted, uint64_t *rejected) {
    if (threads < 1) threads = 1;
    const uint32_t shift = bucket_shift(g->nv, threads);
    const uint32_t nb = (uint32_t)(((uint64_t)g->nv + (1ull << shift) - 1) >> shift) + 1;
    uint64_t *boff, rej, del = 0;
    orc_triple *k = bucket_pairs(g, src, dst, NULL, n, threads, shift, nb, &boff, &rej);
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1) reduction(+ : del)
    for (uint32_t b = 0; b < nb; ++b) {
        orc_triple *kb = k + boff[b];
        const uint64_t m = boff[b + 1] - boff[b];
        if (m == 0) continue;
        qsort(kb, m, sizeof(orc_triple), cmp_triple);
        uint32_t *dset = (uint32_t *)malloc(m * sizeof(uint32_t));
        uint64_t i = 0;
        while (i < m) {
            const uint32_t u = kb[i].u;
            uint64_t j = i, nd = 0;
            while (j < m && kb[j].u == u) ++j;
            for (uint64_t t = i; t < j; ++t) dset[nd++] = kb[t].v; /* sorted */
            orc_adj *a = &g->adj[u];
            uint64_t wpos = 0;
            for (uint64_t r = 0; r < a->n; ++r) {
                if (sorted_contains(dset, nd, a->v[r])) {
                    ++del;
                } else {
                    a->w[wpos] = a->w[r];
                    a->v[wpos++] = a->v[r];
                }
            }
            a->n = wpos;
            i = j;
        }
        free(dset);
    }
    free(k);
    free(boff);
    g->num_edges -= del;
    if (deleted) *deleted = del;
    if (rejected) *rejected = rej;
}

/* Queries (the oracle's Algorithm 3 reading), one binary search each. */
void orc_par_query_edges(const orc_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, int threads,
                         uint8_t *out) {
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t u = src[i], v = dst[i];
        out[i] = (uint8_t)(valid_pair(g, u, v) && sorted_contains(g->adj[u].v, g->adj[u].n, v));
    }
}

/*
 * Shared declarations of the CPU oracle (gv_oracle.c) and the parallel CPU
 * baseline (gv_cpu_parallel.c) -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY.
 * The GPU library shares nothing with either.
 */
#ifndef GV_ORACLE_INTERNAL_H
#define GV_ORACLE_INTERNAL_H

#include <stdint.h>

#define ORC_DEDUP 1u

typedef struct {
    uint32_t *v;     /* destination ids, sorted by (v, w) (multiset) */
    uint32_t *w;     /* 32-bit payload (weight) of each entry; 0 when unweighted */
    uint64_t n;
    uint64_t cap;
} orc_adj;

typedef struct orc_graph {
    uint32_t nv;        /* vertex ids in [0, nv) exist */
    uint32_t cap;       /* allocated vertex slots */
    uint32_t flags;
    uint8_t *alive;
    orc_adj *adj;
    uint64_t num_edges;
} orc_graph;

typedef struct {
    uint32_t u, v, w;
} orc_triple;

/* Room for `need` entries in an adjacency (geometric growth). */
void adj_reserve(orc_adj *a, uint64_t need);
/* Sorts an adjacency by (v, w): the canonical order of its entries. */
void adj_sort(orc_adj *a);
/* 1 if x occurs in the sorted array a[0..n). */
int sorted_contains(const uint32_t *a, uint64_t n, uint32_t x);
/* 1 if both endpoints are in range and alive. */
int valid_pair(const orc_graph *g, uint32_t u, uint32_t v);
/* qsort order of triples by (u, v, w). */
int cmp_triple(const void *a, const void *b);

#endif

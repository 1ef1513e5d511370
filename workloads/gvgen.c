/*
 * Seeded synthetic workload generators for dynamic-graph batches.
 *
 * This file draws random numbers and nothing else: it holds none of the graph
 * data structure's arithmetic (no grouping, no block sizing, no adjacency
 * logic).  Both the CPU oracle side and the GPU side of every test and of the
 * benchmark take their inputs from here, so that both see identical batches.
 *
 * Generators (all public, named algorithms):
 *   - splitmix64 (Steele, Lea, Flood 2014) expands a (seed, stream) pair into
 *     a xoshiro256** state;
 *   - xoshiro256** (Blackman, Vigna 2018) produces the 64-bit stream;
 *   - bounded integers use the high half of a 64x64->128 multiply
 *     (Lemire 2019, without the rejection step: the bias is below 2^-32 for
 *     bounds below 2^32 and is irrelevant for synthetic inputs);
 *   - RMAT (Chakrabarti, Zhan, Faloutsos 2004): per level one 32-bit uniform
 *     picks a quadrant with probabilities (a, b, c, d), most significant bit
 *     first; quadrant a = (0,0), b = (src 0, dst 1), c = (src 1, dst 0),
 *     d = (1,1).  No noise, no vertex permutation.
 *   - Fisher-Yates shuffle for permutations and samples without replacement.
 *
 * Pure C99, no platform intrinsics: identical output on x86-64 and AArch64.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

typedef struct { uint64_t s[4]; } xo_state;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo_state *st) {
    uint64_t *s = st->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void xo_seed(xo_state *st, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull) ^ 0x5851F42D4C957F2Dull;
    for (int i = 0; i < 4; ++i) st->s[i] = splitmix64_next(&x);
}

static inline uint32_t bounded32(xo_state *st, uint32_t bound) {
    return (uint32_t)(((unsigned __int128)xo_next(st) * bound) >> 64);
}

static inline uint64_t bounded64(xo_state *st, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)xo_next(st) * bound) >> 64);
}

/* n raw 64-bit words (for tests of the generator itself). */
void gvgen_raw(uint64_t seed, uint64_t stream, uint64_t n, uint64_t *out) {
    xo_state st; xo_seed(&st, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = xo_next(&st);
}

/* n pairs with src, dst uniform in [lo, lo + nv). */
void gvgen_uniform_pairs(uint64_t seed, uint64_t stream, uint64_t n, uint32_t lo, uint32_t nv,
                         uint32_t *src, uint32_t *dst) {
    xo_state st; xo_seed(&st, seed, stream);
    for (uint64_t i = 0; i < n; ++i) {
        src[i] = lo + bounded32(&st, nv);
        dst[i] = lo + bounded32(&st, nv);
    }
}

/* n values uniform in [lo, lo + range). */
void gvgen_uniform_u32(uint64_t seed, uint64_t stream, uint64_t n, uint32_t lo, uint32_t range,
                       uint32_t *out) {
    xo_state st; xo_seed(&st, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = lo + bounded32(&st, range);
}

/* n values uniform in [0, 1) with 53-bit resolution. */
void gvgen_uniform_f64(uint64_t seed, uint64_t stream, uint64_t n, double *out) {
    xo_state st; xo_seed(&st, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = (double)(xo_next(&st) >> 11) * 0x1.0p-53;
}

/*
 * n RMAT pairs at the given scale (ids in [0, 2^scale)).  Thresholds are the
 * cumulative probabilities a, a+b, a+b+c scaled to 2^32.  If limit < 2^scale,
 * pairs with an endpoint >= limit are redrawn (used for graphs whose vertex
 * count is not a power of two).
 */
void gvgen_rmat_pairs(uint64_t seed, uint64_t stream, uint64_t n, uint32_t scale,
                      double a, double b, double c, uint32_t limit,
                      uint32_t *src, uint32_t *dst) {
    xo_state st; xo_seed(&st, seed, stream);
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)floor(a * two32);
    uint64_t tab = (uint64_t)floor((a + b) * two32);
    uint64_t tabc = (uint64_t)floor((a + b + c) * two32);
    uint64_t full = (scale >= 32) ? 0xFFFFFFFFull + 1 : (1ull << scale);
    uint64_t lim = (limit == 0 || (uint64_t)limit > full) ? full : (uint64_t)limit;
    uint64_t i = 0;
    while (i < n) {
        uint32_t s = 0, d = 0;
        uint64_t word = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            uint64_t r;
            if ((lvl & 1u) == 0) { word = xo_next(&st); r = word & 0xFFFFFFFFull; }
            else { r = word >> 32; }
            uint32_t sb, db;
            if (r < ta) { sb = 0; db = 0; }
            else if (r < tab) { sb = 0; db = 1; }
            else if (r < tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        if ((uint64_t)s < lim && (uint64_t)d < lim) {
            src[i] = s; dst[i] = d; ++i;
        }
    }
}

/* In-place Fisher-Yates shuffle of a uint64 array (used on pair keys). */
void gvgen_shuffle_u64(uint64_t seed, uint64_t stream, uint64_t n, uint64_t *a) {
    xo_state st; xo_seed(&st, seed, stream);
    if (n < 2) return;
    for (uint64_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded64(&st, i + 1);
        uint64_t t = a[i]; a[i] = a[j]; a[j] = t;
    }
}

/* In-place Fisher-Yates shuffle of a uint32 array. */
void gvgen_shuffle_u32(uint64_t seed, uint64_t stream, uint64_t n, uint32_t *a) {
    xo_state st; xo_seed(&st, seed, stream);
    if (n < 2) return;
    for (uint64_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded64(&st, i + 1);
        uint32_t t = a[i]; a[i] = a[j]; a[j] = t;
    }
}

/* k indices drawn uniformly with replacement from [0, n). */
void gvgen_sample_with_replacement(uint64_t seed, uint64_t stream, uint64_t n, uint64_t k,
                                   uint64_t *out) {
    xo_state st; xo_seed(&st, seed, stream);
    for (uint64_t i = 0; i < k; ++i) out[i] = bounded64(&st, n);
}

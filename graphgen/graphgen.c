/*
 * graphgen.c -- seeded synthetic graph generators shared by the tests, the
 * oracle checks and the benchmark.  Holds no arithmetic of the shortest-path
 * method: it only builds directed CSR graphs (row_ptr u64[n+1], col u32[m],
 * w u32[m]) with positive integer weights.
 *
 * Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written here from its
 * published definition; only 64-bit integer arithmetic, so the same seed gives
 * the same graph on every host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t n;
    uint64_t m;
    uint64_t* row_ptr;
    uint32_t* col;
    uint32_t* w;
} gg_graph;

typedef struct { uint64_t state; } rng_t;

static uint64_t rng_next(rng_t* r) {
    uint64_t z = (r->state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* Uniform integer in [lo, hi] (modulo reduction; bias below 2^-40 here). */
static uint64_t rng_range(rng_t* r, uint64_t lo, uint64_t hi) {
    return lo + rng_next(r) % (hi - lo + 1);
}
/* Uniform double in [0, 1) with 53 random bits (exact, host independent). */
static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

static rng_t rng_seed(uint64_t seed, uint64_t stream) {
    rng_t r;
    r.state = seed ^ (stream * 0xD1B54A32D192ED03ull);
    rng_next(&r);
    return r;
}

static gg_graph* gg_alloc(uint32_t n, uint64_t m) {
    gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    g->n = n;
    g->m = m;
    g->row_ptr = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    g->col = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    g->w = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!g->row_ptr || !g->col || !g->w) {
        free(g->row_ptr); free(g->col); free(g->w); free(g);
        return NULL;
    }
    return g;
}

void gg_free(gg_graph* g) {
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->w); free(g);
}
uint32_t gg_n(const gg_graph* g) { return g->n; }
uint64_t gg_m(const gg_graph* g) { return g->m; }
void gg_copy(const gg_graph* g, uint64_t* row_ptr, uint32_t* col, uint32_t* w) {
    memcpy(row_ptr, g->row_ptr, sizeof(uint64_t) * ((size_t)g->n + 1));
    memcpy(col, g->col, sizeof(uint32_t) * g->m);
    memcpy(w, g->w, sizeof(uint32_t) * g->m);
}

/* LSD radix sort of u64 keys, 16-bit digits, passes limited to key_bits. */
static int radix_sort_u64(uint64_t* a, uint64_t cnt, int key_bits) {
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * 65536);
    if (!tmp || !hist) { free(tmp); free(hist); return -1; }
    uint64_t* src = a;
    uint64_t* dst = tmp;
    for (int shift = 0; shift < key_bits; shift += 16) {
        memset(hist, 0, sizeof(uint64_t) * 65536);
        for (uint64_t i = 0; i < cnt; ++i) hist[(src[i] >> shift) & 0xFFFF]++;
        uint64_t run = 0;
        for (int d = 0; d < 65536; ++d) { uint64_t c = hist[d]; hist[d] = run; run += c; }
        for (uint64_t i = 0; i < cnt; ++i) dst[hist[(src[i] >> shift) & 0xFFFF]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * cnt);
    free(tmp);
    free(hist);
    return 0;
}

/* Builds a CSR from sorted unique (u << 32 | v) keys; weights U[wlo, whi]. */
static gg_graph* csr_from_sorted_keys(uint32_t n, const uint64_t* key, uint64_t m,
                                      uint32_t wlo, uint32_t whi, rng_t* r) {
    gg_graph* g = gg_alloc(n, m);
    if (!g) return NULL;
    for (uint64_t i = 0; i < m; ++i) g->row_ptr[(key[i] >> 32) + 1]++;
    for (uint32_t u = 0; u < n; ++u) g->row_ptr[u + 1] += g->row_ptr[u];
    for (uint64_t i = 0; i < m; ++i) {
        g->col[i] = (uint32_t)(key[i] & 0xFFFFFFFFu);
        g->w[i] = (uint32_t)rng_range(r, wlo, whi);
    }
    return g;
}

static int bits_for(uint64_t x) { int b = 0; while (b < 64 && (x >> b)) ++b; return b; }

/* Random directed graph: every vertex gets `deg` distinct uniform targets
 * other than itself; weights U[wlo, whi]. */
gg_graph* gg_random(uint32_t n, uint32_t deg, uint32_t wlo, uint32_t whi, uint64_t seed) {
    if (n < 2 || deg >= n) return NULL;
    rng_t r = rng_seed(seed, 1);
    gg_graph* g = gg_alloc(n, (uint64_t)n * deg);
    if (!g) return NULL;
    uint64_t e = 0;
    for (uint32_t u = 0; u < n; ++u) {
        g->row_ptr[u] = e;
        uint64_t first = e;
        while (e - first < deg) {
            uint32_t v = (uint32_t)rng_range(&r, 0, n - 1);
            if (v == u) continue;
            int dup = 0;
            for (uint64_t k = first; k < e; ++k) if (g->col[k] == v) { dup = 1; break; }
            if (dup) continue;
            g->col[e++] = v;
        }
        /* keep targets sorted within a row */
        for (uint64_t i = first + 1; i < e; ++i) {
            uint32_t t = g->col[i]; uint64_t j = i;
            while (j > first && g->col[j - 1] > t) { g->col[j] = g->col[j - 1]; --j; }
            g->col[j] = t;
        }
    }
    g->row_ptr[n] = e;
    for (uint64_t k = 0; k < e; ++k) g->w[k] = (uint32_t)rng_range(&r, wlo, whi);
    return g;
}

/* Random graph with per-vertex out-degree U[dmin, dmax] (distinct, non-self
 * targets), weights U[wlo, whi]. */
gg_graph* gg_random_var(uint32_t n, uint32_t dmin, uint32_t dmax, uint32_t wlo, uint32_t whi,
                        uint64_t seed) {
    if (n < 2 || dmin > dmax || dmax >= n) return NULL;
    rng_t r = rng_seed(seed, 2);
    uint32_t* degs = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!degs) return NULL;
    uint64_t m = 0;
    for (uint32_t u = 0; u < n; ++u) { degs[u] = (uint32_t)rng_range(&r, dmin, dmax); m += degs[u]; }
    gg_graph* g = gg_alloc(n, m);
    if (!g) { free(degs); return NULL; }
    uint64_t e = 0;
    for (uint32_t u = 0; u < n; ++u) {
        g->row_ptr[u] = e;
        uint64_t first = e;
        while (e - first < degs[u]) {
            uint32_t v = (uint32_t)rng_range(&r, 0, n - 1);
            if (v == u) continue;
            int dup = 0;
            for (uint64_t k = first; k < e; ++k) if (g->col[k] == v) { dup = 1; break; }
            if (dup) continue;
            g->col[e++] = v;
        }
        for (uint64_t i = first + 1; i < e; ++i) {
            uint32_t t = g->col[i]; uint64_t j = i;
            while (j > first && g->col[j - 1] > t) { g->col[j] = g->col[j - 1]; --j; }
            g->col[j] = t;
        }
    }
    g->row_ptr[n] = e;
    for (uint64_t k = 0; k < e; ++k) g->w[k] = (uint32_t)rng_range(&r, wlo, whi);
    free(degs);
    return g;
}

/* R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of
 * edge_factor * 2^scale edges picks one of four quadrants per level with
 * probabilities (a, b, c, 1-a-b-c).  Vertex ids are then relabelled by a
 * seeded random permutation; self-loops and duplicate edges are removed;
 * weights U[wlo, whi] are drawn per remaining edge in (src, dst) order. */
gg_graph* gg_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c,
                  uint32_t wlo, uint32_t whi, uint64_t seed) {
    if (scale < 1 || scale > 30) return NULL;
    uint32_t n = 1u << scale;
    uint64_t cnt = (uint64_t)edge_factor << scale;
    rng_t r = rng_seed(seed, 3);
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    if (!perm || !key) { free(perm); free(key); return NULL; }
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n - 1; i > 0; --i) {          /* Fisher-Yates */
        uint32_t j = (uint32_t)rng_range(&r, 0, i);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    const double ab = a + b, abc = a + b + c;
    uint64_t kept = 0;
    for (uint64_t e = 0; e < cnt; ++e) {
        uint32_t u = 0, v = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            double p = rng_unit(&r);
            uint32_t bu = 0, bv = 0;
            if (p < a) { bu = 0; bv = 0; }
            else if (p < ab) { bu = 0; bv = 1; }
            else if (p < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        u = perm[u];
        v = perm[v];
        if (u == v) continue;
        key[kept++] = ((uint64_t)u << 32) | v;
    }
    if (radix_sort_u64(key, kept, 32 + bits_for(n - 1)) != 0) { free(perm); free(key); return NULL; }
    uint64_t m = 0;
    for (uint64_t i = 0; i < kept; ++i)
        if (m == 0 || key[i] != key[m - 1]) key[m++] = key[i];
    gg_graph* g = csr_from_sorted_keys(n, key, m, wlo, whi, &r);
    free(perm);
    free(key);
    return g;
}

/* 2-D grid rows x cols, 4-neighbour, both directions, each directed edge
 * with its own weight U[wlo, whi].  Vertex (i, j) has id i * cols + j. */
gg_graph* gg_grid(uint32_t rows, uint32_t cols, uint32_t wlo, uint32_t whi, uint64_t seed) {
    uint64_t n64 = (uint64_t)rows * cols;
    if (rows < 1 || cols < 1 || n64 > 0xFFFFFFFEull) return NULL;
    uint32_t n = (uint32_t)n64;
    uint64_t m = 2ull * ((uint64_t)rows * (cols - 1) + (uint64_t)cols * (rows - 1));
    rng_t r = rng_seed(seed, 4);
    gg_graph* g = gg_alloc(n, m);
    if (!g) return NULL;
    uint64_t e = 0;
    for (uint32_t i = 0; i < rows; ++i)
        for (uint32_t j = 0; j < cols; ++j) {
            uint32_t u = i * cols + j;
            g->row_ptr[u] = e;
            /* ascending target order: up, left, right, down */
            if (i > 0) g->col[e++] = u - cols;
            if (j > 0) g->col[e++] = u - 1;
            if (j + 1 < cols) g->col[e++] = u + 1;
            if (i + 1 < rows) g->col[e++] = u + cols;
        }
    g->row_ptr[n] = e;
    for (uint64_t k = 0; k < e; ++k) g->w[k] = (uint32_t)rng_range(&r, wlo, whi);
    return g;
}

/* Layered DAG: `layers` layers of `width` vertices (layer-major ids).  Every
 * vertex draws `deg` edges; each edge goes to layer + U{1..maxskip} and a
 * uniform vertex of that layer; edges past the last layer are dropped;
 * duplicate targets are redrawn.  Weights U[wlo, whi]. */
gg_graph* gg_dag(uint32_t layers, uint32_t width, uint32_t deg, uint32_t maxskip,
                 uint32_t wlo, uint32_t whi, uint64_t seed) {
    uint64_t n64 = (uint64_t)layers * width;
    if (layers < 1 || width < 1 || n64 > 0xFFFFFFFEull || deg > width) return NULL;
    uint32_t n = (uint32_t)n64;
    rng_t r = rng_seed(seed, 5);
    gg_graph* g = gg_alloc(n, (uint64_t)n * deg);
    if (!g) return NULL;
    uint64_t e = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint32_t lay = u / width;
        g->row_ptr[u] = e;
        uint64_t first = e;
        for (uint32_t d = 0; d < deg; ++d) {
            for (;;) {
                uint32_t skip = (uint32_t)rng_range(&r, 1, maxskip);
                uint32_t pos = (uint32_t)rng_range(&r, 0, width - 1);
                if (lay + skip >= layers) break;  /* dropped */
                uint32_t v = (lay + skip) * width + pos;
                int dup = 0;
                for (uint64_t k = first; k < e; ++k) if (g->col[k] == v) { dup = 1; break; }
                if (dup) continue;
                g->col[e++] = v;
                break;
            }
        }
        for (uint64_t i = first + 1; i < e; ++i) {
            uint32_t t = g->col[i]; uint64_t j = i;
            while (j > first && g->col[j - 1] > t) { g->col[j] = g->col[j - 1]; --j; }
            g->col[j] = t;
        }
    }
    g->row_ptr[n] = e;
    g->m = e;
    for (uint64_t k = 0; k < e; ++k) g->w[k] = (uint32_t)rng_range(&r, wlo, whi);
    return g;
}

/* Stream of seeded uniform integers in [lo, hi] (sources, sizes, arrivals). */
void gg_uniform(uint64_t seed, uint64_t stream, uint64_t count, uint64_t lo, uint64_t hi,
                uint64_t* out) {
    rng_t r = rng_seed(seed, 100 + stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = rng_range(&r, lo, hi);
}

/* Stream of seeded uniform doubles in [0, 1). */
void gg_unit(uint64_t seed, uint64_t stream, uint64_t count, double* out) {
    rng_t r = rng_seed(seed, 200 + stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = rng_unit(&r);
}

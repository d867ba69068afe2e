/*
 * graphgen.c -- seeded synthetic graph inputs for SCAN: R-MAT and Chung-Lu
 * edge samplers and a CSR builder (drop self-loops, symmetrise, sort, dedup).
 *
 * This module holds none of the clustering arithmetic. It is shared by the
 * CPU oracle, the tests and the benchmark so that both sides of every parity
 * check see the same graph.
 *
 * Random numbers: every edge i draws from its own xoshiro256** stream whose
 * state is filled by SplitMix64 from (seed, i) (both generators are published
 * by Blackman and Vigna). Sampling is integer-only for R-MAT, so an R-MAT
 * graph is bit-identical on every platform and for any thread count.
 * Chung-Lu weights use libm pow(), so those graphs are reproducible on one
 * platform (glibc) but may differ by a rounding between architectures.
 *
 * Output: offsets int64[n+1], adj int32[nnz], rows sorted ascending, no
 * duplicates, no self-loops, symmetric. Arrays are malloc'd and owned by the
 * returned handle (gg_free).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct gg_graph {
    int64_t n;
    int64_t nnz;
    int64_t *offsets;
    int32_t *adj;
} gg_graph;

/* ---------------------------------------------------------------- RNG */
static inline uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo256 *r) {
    uint64_t *s = r->s;
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

/* Stream `stream` of generator `seed`: SplitMix64 fills the 256-bit state. */
static inline void xo_seed(xo256 *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed;
    (void)splitmix64_next(&x);
    x ^= stream * 0xD1342543DE82EF95ULL;
    for (int k = 0; k < 4; ++k) r->s[k] = splitmix64_next(&x);
}

/* Uniform integer in [0, bound) by Lemire's multiply-shift. */
static inline uint64_t xo_below(xo256 *r, uint64_t bound) {
    unsigned __int128 p = (unsigned __int128)xo_next(r) * bound;
    return (uint64_t)(p >> 64);
}

/* ------------------------------------------------------------ helpers */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t *p, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t v = p[i];
            int64_t j = i - 1;
            while (j >= 0 && p[j] > v) { p[j + 1] = p[j]; --j; }
            p[j + 1] = v;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/* Seeded random permutation of [0, n) (Fisher-Yates). */
static uint32_t *make_perm(int64_t n, uint64_t seed) {
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!perm) return NULL;
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    xo256 r;
    xo_seed(&r, seed, 0xFFFFFFFFFFFFFFFFULL);
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)xo_below(&r, (uint64_t)(i + 1));
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return perm;
}

/*
 * Edge source: fills (src, dst) for edge index i. Both passes of the CSR
 * build regenerate edges from their counters, so no edge list is stored.
 */
typedef void (*edge_fn)(const void *ctx, int64_t i, uint32_t *u, uint32_t *v);

static gg_graph *build_csr(int64_t n, int64_t num_edges, edge_fn fn, const void *ctx) {
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g || !deg) { free(g); free(deg); return NULL; }
    g->n = n;

    /* pass 1: degree of the symmetrised multigraph */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < num_edges; ++i) {
        uint32_t u, v;
        fn(ctx, i, &u, &v);
        if (u == v) continue;
        __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
    }
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!start) { free(deg); free(g); return NULL; }
    start[0] = 0;
    for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + deg[i];
    int64_t total = start[n];
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!tmp) { free(deg); free(start); free(g); return NULL; }
    memcpy(deg, start, sizeof(int64_t) * (size_t)n); /* deg becomes the cursor */

    /* pass 2: scatter both directions (order inside a row is fixed by the sort) */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < num_edges; ++i) {
        uint32_t u, v;
        fn(ctx, i, &u, &v);
        if (u == v) continue;
        int64_t pu = __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        int64_t pv = __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
        tmp[pu] = (int32_t)v;
        tmp[pv] = (int32_t)u;
    }

    /* sort + dedup each row in place; deg[i] := unique count */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *p = tmp + start[i];
        int64_t len = start[i + 1] - start[i];
        sort_row(p, len);
        int64_t w = 0;
        for (int64_t k = 0; k < len; ++k)
            if (w == 0 || p[k] != p[w - 1]) p[w++] = p[k];
        deg[i] = w;
    }
    g->offsets = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g->offsets) { free(deg); free(start); free(tmp); free(g); return NULL; }
    g->offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) g->offsets[i + 1] = g->offsets[i] + deg[i];
    g->nnz = g->offsets[n];
    g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nnz > 0 ? g->nnz : 1));
    if (!g->adj) { free(deg); free(start); free(tmp); free(g->offsets); free(g); return NULL; }
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i)
        memcpy(g->adj + g->offsets[i], tmp + start[i], sizeof(int32_t) * (size_t)deg[i]);
    free(tmp);
    free(start);
    free(deg);
    return g;
}

/* --------------------------------------------------------------- R-MAT */
typedef struct {
    int scale;
    uint64_t seed;
    uint32_t ta, tab, tabc; /* cumulative quadrant thresholds on 32-bit draws */
    const uint32_t *perm;   /* NULL: no relabelling */
} rmat_ctx;

static void rmat_edge(const void *vctx, int64_t i, uint32_t *pu, uint32_t *pv) {
    const rmat_ctx *c = (const rmat_ctx *)vctx;
    xo256 r;
    xo_seed(&r, c->seed, (uint64_t)i);
    uint32_t u = 0, v = 0;
    for (int l = 0; l < c->scale; ++l) {
        uint32_t x = (uint32_t)(xo_next(&r) >> 32);
        uint32_t bu, bv;
        if (x < c->ta) { bu = 0; bv = 0; }
        else if (x < c->tab) { bu = 0; bv = 1; }
        else if (x < c->tabc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
    }
    if (c->perm) { u = c->perm[u]; v = c->perm[v]; }
    *pu = u;
    *pv = v;
}

static uint32_t prob_to_u32(double p) {
    double x = p * 4294967296.0;
    if (x <= 0.0) return 0;
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)x;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): edge_factor * 2^scale edge
 * samples; each descends `scale` levels choosing a quadrant with
 * probabilities (a, b, c, 1-a-b-c). No noise. With relabel != 0 the vertex
 * ids pass through a seeded random permutation (Graph500 style).
 */
gg_graph *gg_rmat(int scale, int64_t edge_factor, double a, double b, double c,
                  uint64_t seed, int relabel) {
    if (scale < 1 || scale > 31 || edge_factor < 0) return NULL;
    int64_t n = (int64_t)1 << scale;
    rmat_ctx ctx;
    ctx.scale = scale;
    ctx.seed = seed;
    ctx.ta = prob_to_u32(a);
    ctx.tab = prob_to_u32(a + b);
    ctx.tabc = prob_to_u32(a + b + c);
    uint32_t *perm = NULL;
    if (relabel) {
        perm = make_perm(n, seed);
        if (!perm) return NULL;
    }
    ctx.perm = perm;
    gg_graph *g = build_csr(n, edge_factor * n, rmat_edge, &ctx);
    free(perm);
    return g;
}

/* ------------------------------------------------------------ Chung-Lu */
typedef struct {
    int64_t n;
    uint64_t seed;
    const double *prob;
    const uint32_t *alias;
    const uint32_t *perm;
} cl_ctx;

static inline uint32_t alias_draw(const cl_ctx *c, xo256 *r) {
    uint64_t col = xo_below(r, (uint64_t)c->n);
    double coin = (double)(xo_next(r) >> 11) * (1.0 / 9007199254740992.0);
    return coin < c->prob[col] ? (uint32_t)col : c->alias[col];
}

static void cl_edge(const void *vctx, int64_t i, uint32_t *pu, uint32_t *pv) {
    const cl_ctx *c = (const cl_ctx *)vctx;
    xo256 r;
    xo_seed(&r, c->seed, (uint64_t)i);
    uint32_t u = alias_draw(c, &r);
    uint32_t v = alias_draw(c, &r);
    if (c->perm) { u = c->perm[u]; v = c->perm[v]; }
    *pu = u;
    *pv = v;
}

/*
 * Chung-Lu (sampling form): weights w_i = (i+1)^(-1/(gamma-1)), scaled to
 * mean avg_deg and capped at sqrt(n * avg_deg); ceil(n*avg_deg/2) endpoint
 * pairs are drawn i.i.d. from a Vose alias table over w; self-loops and
 * duplicates are dropped, so the realised degree is below avg_deg.
 */
gg_graph *gg_chung_lu(int64_t n, double avg_deg, double gamma, uint64_t seed, int relabel) {
    if (n < 1 || n > 2147483647LL || avg_deg < 0.0 || gamma <= 1.0) return NULL;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *prob = (double *)malloc(sizeof(double) * (size_t)n);
    uint32_t *alias = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *large = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!w || !prob || !alias || !small || !large) {
        free(w); free(prob); free(alias); free(small); free(large);
        return NULL;
    }
    double expo = -1.0 / (gamma - 1.0), sum = 0.0;
    for (int64_t i = 0; i < n; ++i) { w[i] = pow((double)(i + 1), expo); sum += w[i]; }
    double scale = avg_deg * (double)n / sum, cap = sqrt((double)n * avg_deg), tot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        w[i] *= scale;
        if (w[i] > cap) w[i] = cap;
        tot += w[i];
    }
    /* Vose's alias method */
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / tot;
        if (prob[i] < 1.0) small[ns++] = (uint32_t)i; else large[nl++] = (uint32_t)i;
    }
    while (ns > 0 && nl > 0) {
        uint32_t s = small[--ns], l = large[--nl];
        alias[s] = l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { uint32_t l = large[--nl]; prob[l] = 1.0; alias[l] = l; }
    while (ns > 0) { uint32_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
    free(w); free(small); free(large);

    uint32_t *perm = NULL;
    if (relabel) {
        perm = make_perm(n, seed);
        if (!perm) { free(prob); free(alias); return NULL; }
    }
    cl_ctx ctx = {n, seed, prob, alias, perm};
    int64_t m = (int64_t)ceil((double)n * avg_deg / 2.0);
    gg_graph *g = build_csr(n, m, cl_edge, &ctx);
    free(prob); free(alias); free(perm);
    return g;
}

/* ------------------------------------------------- explicit edge lists */
typedef struct { const int32_t *src, *dst; } list_ctx;

static void list_edge(const void *vctx, int64_t i, uint32_t *pu, uint32_t *pv) {
    const list_ctx *c = (const list_ctx *)vctx;
    *pu = (uint32_t)c->src[i];
    *pv = (uint32_t)c->dst[i];
}

/* CSR of an explicit undirected edge list (ids in [0, n)); repairs as above. */
gg_graph *gg_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    if (n < 0) return NULL;
    for (int64_t i = 0; i < m; ++i)
        if (src[i] < 0 || dst[i] < 0 || src[i] >= n || dst[i] >= n) return NULL;
    list_ctx ctx = {src, dst};
    return build_csr(n, m, list_edge, &ctx);
}

int64_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_nnz(const gg_graph *g) { return g->nnz; }
int64_t *gg_offsets(gg_graph *g) { return g->offsets; }
int32_t *gg_adj(gg_graph *g) { return g->adj; }

void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->offsets);
    free(g->adj);
    free(g);
}

/* Uniform draws for workload recipes (parameter mixes, arrival times). */
void gg_uniform_u64(uint64_t seed, uint64_t stream, int64_t count, uint64_t *out) {
    xo256 r;
    xo_seed(&r, seed, stream);
    for (int64_t i = 0; i < count; ++i) out[i] = xo_next(&r);
}

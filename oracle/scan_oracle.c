/*
 * scan_oracle.c -- CPU oracle for exact structural graph clustering (SCAN).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this file; the product path
 * never does. It shares no code with the CUDA library.
 *
 * This is the plain definition written out, single pass, slow and obvious.
 * Paper: GPUSCAN++ (Efficient Structural Graph Clustering on GPUs),
 * Section 2.1 (Definitions 2.1-2.3, Core, Structural Reachability,
 * Cluster, Hub and Outlier). Readings taken where the paper is loose:
 *   - sigma >= eps is inclusive and is tested exactly in integers: with
 *     eps = p/q, S(u,v) <=> c^2 q^2 >= p^2 |N[u]| |N[v]| (unsigned 128-bit),
 *     instead of the floating-point test of Algorithm 2 (checkSim).
 *   - neighbourhoods are closed: |N[v]| = deg(v) + 1 and, for adjacent u, v,
 *     |N[u] cap N[v]| = |nbr(u) cap nbr(v)| + 2 (the "+2" of checkSim).
 *   - a core u satisfies |N_eps[u]| >= mu with u itself counted (Definition
 *     Core), not the "mu-1 neighbours" of Example 2.1.
 *   - a cluster contains at least one core; its id is its smallest core id.
 *   - a non-core vertex eps-similar to cores of several clusters belongs to
 *     all of them (Definition Cluster, maximality); all pairs are reported.
 *   - hub: a vertex in no cluster whose neighbours' cluster memberships
 *     (borders included, each with all its clusters) span >= 2 distinct
 *     clusters (Definition Hub and Outlier); otherwise outlier. No degree
 *     guard as in Algorithm 4.
 *   - isolated vertices have |N_eps| = 1 < mu and are outliers.
 *
 * Parity status: pinned (worked values of Example 3.1 and Example 4.2,
 * reconstructed Figure-1 fixture, closed forms, brute force over all graphs
 * with up to 7 vertices and sampled 8-12 vertex graphs). The per-slot
 * counts of oracle_counts_for_slots are pinned to the sparse matrix square
 * (A^2)[u, v] + 2 on every slot of graphs with empty rows and with degree
 * ratios above 32 (its binary-search branch).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

enum { LABEL_CORE = 0, LABEL_BORDER = 1, LABEL_HUB = 2, LABEL_OUTLIER = 3 };

/*
 * Input contract of Section 2.1: a simple undirected graph. Rows must be
 * sorted strictly ascending (so no duplicates), ids in [0, n), no self-loops,
 * and symmetric. Returns ORACLE_OK, or ORACLE_EINVAL with *bad set to the
 * first offending slot (or -1 for a bad offsets array).
 */
int oracle_validate(int64_t n, const int64_t *off, const int32_t *adj, int64_t nnz, int64_t *bad) {
    *bad = -1;
    if (n < 0 || nnz < 0) return ORACLE_EINVAL;
    if (off[0] != 0 || off[n] != nnz) return ORACLE_EINVAL;
    for (int64_t u = 0; u < n; ++u)
        if (off[u + 1] < off[u]) return ORACLE_EINVAL;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = adj[e];
            if (v < 0 || v >= n || v == u) { *bad = e; return ORACLE_EINVAL; }
            if (e > off[u] && adj[e - 1] >= adj[e]) { *bad = e; return ORACLE_EINVAL; }
        }
    }
    /* symmetry: v in nbr(u) => u in nbr(v) (binary search in row v) */
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = adj[e], lo = off[v], hi = off[v + 1];
            int found = 0;
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (adj[mid] < u) lo = mid + 1;
                else if (adj[mid] > u) hi = mid;
                else { found = 1; break; }
            }
            if (!found) { *bad = e; return ORACLE_EINVAL; }
        }
    }
    return ORACLE_OK;
}

/* |A cap B| of two ascending lists by a linear merge. */
static int64_t count_merge(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

static int contains(const int32_t *b, int64_t nb, int32_t x) {
    int64_t lo = 0, hi = nb;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (b[mid] < x) lo = mid + 1;
        else if (b[mid] > x) hi = mid;
        else return 1;
    }
    return 0;
}

/* |A cap B| by looking up each element of the shorter list in the longer. */
static int64_t count_search(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
    if (na > nb) { const int32_t *t = a; a = b; b = t; int64_t k = na; na = nb; nb = k; }
    int64_t c = 0;
    for (int64_t i = 0; i < na; ++i) c += contains(b, nb, a[i]);
    return c;
}

/* Position of x in row v (x must be present). */
static int64_t find_slot(const int64_t *off, const int32_t *adj, int64_t v, int32_t x) {
    int64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (adj[mid] < x) lo = mid + 1;
        else if (adj[mid] > x) hi = mid;
        else return mid;
    }
    return -1;
}

/*
 * Definition 2.2 (Eq. 1) numerator for every adjacent pair: for the slot of
 * (u, v), cn[slot] = |N[u] cap N[v]| = |nbr(u) cap nbr(v)| + 2 (u and v are
 * both in both closed neighbourhoods). Each undirected edge is counted once
 * (u < v) and copied to the slot of (v, u). Threads only split the edge loop.
 */
void oracle_common_counts(int64_t n, const int64_t *off, const int32_t *adj, int32_t *cn, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t u = 0; u < n; ++u) {
        const int32_t *ru = adj + off[u];
        int64_t du = off[u + 1] - off[u];
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = adj[e];
            if (v < u) continue;
            const int32_t *rv = adj + off[v];
            int64_t dv = off[v + 1] - off[v];
            int64_t big = du > dv ? du : dv, small = du > dv ? dv : du;
            int64_t c = (small == 0 || big / (small ? small : 1) <= 32)
                            ? count_merge(ru, du, rv, dv)
                            : count_search(ru, du, rv, dv);
            cn[e] = (int32_t)(c + 2);
            cn[find_slot(off, adj, v, (int32_t)u)] = (int32_t)(c + 2);
        }
    }
}

/*
 * Definition 2.3 with eps = p/q: v in N_eps[u] <=> sigma(u,v) >= p/q
 * <=> c * q >= p * sqrt(|N[u]| |N[v]|) <=> c^2 q^2 >= p^2 |N[u]| |N[v]|
 * (all terms non-negative). Exact in unsigned 128-bit: c < 2^31, q < 2^32,
 * |N| < 2^31 keep both sides below 2^126.
 */
static int eps_similar(int64_t c, int64_t du1, int64_t dv1, uint32_t p, uint32_t q) {
    unsigned __int128 lhs = (unsigned __int128)((uint64_t)c * (uint64_t)c) * ((uint64_t)q * (uint64_t)q);
    unsigned __int128 rhs = (unsigned __int128)((uint64_t)p * (uint64_t)p) * ((uint64_t)du1 * (uint64_t)dv1);
    return lhs >= rhs;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sort + unique in place; returns the new length */
static int64_t sort_unique(int32_t *a, int64_t k) {
    if (k <= 1) return k;
    qsort(a, (size_t)k, sizeof(int32_t), cmp_i32);
    int64_t w = 1;
    for (int64_t i = 1; i < k; ++i)
        if (a[i] != a[w - 1]) a[w++] = a[i];
    return w;
}

/*
 * Full SCAN(eps = p/q, mu) of Section 2.1.
 *   core[n]   : 1 if |N_eps[u]| >= mu (Definition Core).
 *   cid[n]    : smallest core id of the core's cluster; -1 for non-cores.
 *   label[n]  : 0 core, 1 border (non-core in >= 1 cluster), 2 hub, 3 outlier.
 *   pairs     : (v, c) for each non-core v and each cluster c containing it,
 *               ascending by (v, c); capacity 2*nnz int32; *npairs = count.
 *   cn_out    : optional per-slot |N[u] cap N[v]| (NULL to skip).
 * threads only parallelises the common-count loop (deterministic).
 */
int oracle_scan_from_counts(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *cn, uint32_t p,
                            uint32_t q, uint32_t mu, uint8_t *core, int32_t *cid, uint8_t *label, int32_t *pairs,
                            int64_t *npairs);

int oracle_scan(int64_t n, const int64_t *off, const int32_t *adj, uint32_t p, uint32_t q, uint32_t mu,
                int threads, uint8_t *core, int32_t *cid, uint8_t *label, int32_t *pairs, int64_t *npairs,
                int32_t *cn_out) {
    *npairs = 0;
    if (p == 0 || q == 0 || p > q || mu < 2) return ORACLE_EINVAL;
    int64_t nnz = off[n], bad;
    if (oracle_validate(n, off, adj, nnz, &bad) != ORACLE_OK) return ORACLE_EINVAL;
    int32_t *cn = cn_out ? cn_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!cn) return ORACLE_ENOMEM;

    /* Definition 2.2: common closed-neighbour counts per adjacent pair */
    oracle_common_counts(n, off, adj, cn, threads);

    int rc = oracle_scan_from_counts(n, off, adj, cn, p, q, mu, core, cid, label, pairs, npairs);
    if (!cn_out) free(cn);
    return rc;
}

/*
 * The rest of SCAN(eps = p/q, mu) once the per-slot closed common counts
 * cn[nnz] of Definition 2.2 are known (outputs as for oracle_scan).
 */
int oracle_scan_from_counts(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *cn, uint32_t p,
                            uint32_t q, uint32_t mu, uint8_t *core, int32_t *cid, uint8_t *label, int32_t *pairs,
                            int64_t *npairs) {
    *npairs = 0;
    if (p == 0 || q == 0 || p > q || mu < 2) return ORACLE_EINVAL;
    int64_t nnz = off[n];
    uint8_t *sim = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *boff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *scratch = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!sim || !queue || !boff || !scratch) {
        free(sim); free(queue); free(boff); free(scratch);
        return ORACLE_ENOMEM;
    }

    /* Definition 2.3: S(u,v) per slot */
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = adj[e];
            sim[e] = (uint8_t)eps_similar(cn[e], off[u + 1] - off[u] + 1, off[v + 1] - off[v] + 1, p, q);
        }

    /* Definition Core: |N_eps[u]| = 1 (u itself, sigma(u,u) = 1) + #similar neighbours */
    for (int64_t u = 0; u < n; ++u) {
        int64_t e_u = 1;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) e_u += sim[e];
        core[u] = (uint8_t)(e_u >= (int64_t)mu);
    }

    /* Definitions Structural Reachability + Cluster: the cores reachable from
     * a core through eps-similar core-core steps form one cluster. Visit cores
     * in increasing id; each unlabelled one starts a BFS, so its id is the
     * smallest core id of the cluster. */
    for (int64_t u = 0; u < n; ++u) cid[u] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (!core[s] || cid[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        cid[s] = (int32_t)s;
        while (head < tail) {
            int64_t x = queue[head++];
            for (int64_t e = off[x]; e < off[x + 1]; ++e) {
                int64_t y = adj[e];
                if (sim[e] && core[y] && cid[y] < 0) {
                    cid[y] = (int32_t)s;
                    queue[tail++] = (int32_t)y;
                }
            }
        }
    }

    /* Definition Cluster (maximality): a non-core v belongs to the cluster of
     * every core u with v in N_eps[u]. B(v) = sorted unique cluster ids. */
    boff[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t k = 0;
        if (!core[v]) {
            int32_t *b = scratch; /* temporary list */
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                int64_t u = adj[e];
                if (core[u] && sim[e]) b[k++] = cid[u];
            }
            k = sort_unique(b, k);
            for (int64_t i = 0; i < k; ++i) {
                pairs[2 * (boff[v] + i)] = (int32_t)v;
                pairs[2 * (boff[v] + i) + 1] = b[i];
            }
        }
        boff[v + 1] = boff[v] + k;
    }
    *npairs = boff[n];

    /* Definition Hub and Outlier: clusters(w) = {cid(w)} for a core, B(w) for
     * a non-core. A vertex in no cluster is a hub iff the union over its
     * neighbours has >= 2 distinct ids. */
    for (int64_t u = 0; u < n; ++u) {
        if (core[u]) { label[u] = LABEL_CORE; continue; }
        if (boff[u + 1] > boff[u]) { label[u] = LABEL_BORDER; continue; }
        int64_t k = 0;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t w = adj[e];
            if (core[w]) scratch[k++] = cid[w];
            else
                for (int64_t i = boff[w]; i < boff[w + 1]; ++i) scratch[k++] = pairs[2 * i + 1];
        }
        k = sort_unique(scratch, k);
        label[u] = (uint8_t)(k >= 2 ? LABEL_HUB : LABEL_OUTLIER);
    }

    free(sim); free(queue); free(boff); free(scratch);
    return ORACLE_OK;
}

/*
 * Definition 2.2 numerator for selected slots only (sampled full-size
 * checks): out[i] = |N[u] cap N[v]| for the slot slots[i] = (u, v), where u
 * is the row holding the slot. Each count is computed independently.
 */
void oracle_counts_for_slots(int64_t n, const int64_t *off, const int32_t *adj, const int64_t *slots, int64_t k,
                             int32_t *out, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < k; ++i) {
        int64_t s = slots[i], lo = 0, hi = n;
        while (hi - lo > 1) { /* row u with off[u] <= s < off[u+1] */
            int64_t mid = lo + (hi - lo) / 2;
            if (off[mid] <= s) lo = mid; else hi = mid;
        }
        while (lo + 1 <= n && off[lo + 1] <= s) ++lo; /* skip empty rows sharing the offset */
        int64_t u = lo, v = adj[s];
        int64_t du = off[u + 1] - off[u], dv = off[v + 1] - off[v];
        int64_t big = du > dv ? du : dv, small = du > dv ? dv : du;
        int64_t c = (small == 0 || big / small <= 32) ? count_merge(adj + off[u], du, adj + off[v], dv)
                                                       : count_search(adj + off[u], du, adj + off[v], dv);
        out[i] = (int32_t)(c + 2);
    }
}

/*
 * brute.c -- literal set-definition SCAN for tiny graphs (n <= 32), and an
 * exhaustive driver that compares it with the oracle on every graph of a
 * given order.
 *
 * TEST INFRASTRUCTURE ONLY (pins the oracle; never used by the product).
 *
 * Every set is a 32-bit mask. The steps follow Section 2.1 of the paper
 * literally, without the oracle's shortcuts (no BFS, no per-edge loop):
 *   Definition 2.1: N[v] = nbr(v) + {v}.
 *   Definition 2.2/2.3: N_eps[u] = {v in N[u] : sigma(u,v) >= eps}, with
 *     sigma compared exactly as |N[u] & N[v]|^2 q^2 >= p^2 |N[u]| |N[v]|.
 *   Definition Core: |N_eps[u]| >= mu.
 *   Definition Structural Reachability: R(u) for a core u is the closure of
 *     {u} under "add N_eps[x] for every core x already in the set"; a
 *     non-core reaches only itself.
 *   Definition Cluster: the distinct sets R(u) over cores u (a cluster must
 *     hold a core); connectivity and maximality are then checked literally.
 *   Definition Hub and Outlier: a vertex in no cluster is a hub iff at least
 *     two distinct clusters contain one of its neighbours.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_scan(int64_t n, const int64_t *off, const int32_t *adj, uint32_t p, uint32_t q, uint32_t mu,
                int threads, uint8_t *core, int32_t *cid, uint8_t *label, int32_t *pairs, int64_t *npairs,
                int32_t *cn_out);

#define BRUTE_OK 0
#define BRUTE_EINVAL 1
#define BRUTE_EDEF 3 /* a definition check failed: the reading is inconsistent */

static int pop(uint32_t x) { return __builtin_popcount(x); }

static int sim(uint32_t Nu, uint32_t Nv, uint32_t p, uint32_t q) {
    uint64_t c = (uint64_t)pop(Nu & Nv), du = (uint64_t)pop(Nu), dv = (uint64_t)pop(Nv);
    unsigned __int128 lhs = (unsigned __int128)(c * c) * ((uint64_t)q * q);
    unsigned __int128 rhs = (unsigned __int128)((uint64_t)p * p) * (du * dv);
    return lhs >= rhs;
}

/*
 * nbr[v]: neighbour mask of v (symmetric, no self bit). Outputs in the
 * oracle's format: core[n], cid[n] (-1 for non-cores), label[n] (0 core,
 * 1 border, 2 hub, 3 outlier), pairs (v, c) ascending, *npairs.
 */
int brute_scan(int n, const uint32_t *nbr, uint32_t p, uint32_t q, uint32_t mu,
               uint8_t *core, int32_t *cid, uint8_t *label, int32_t *pairs, int64_t *npairs) {
    *npairs = 0;
    if (n < 0 || n > 32 || p == 0 || q == 0 || p > q || mu < 2) return BRUTE_EINVAL;
    uint32_t N[32], Neps[32], R[32], clusters[32];
    uint32_t coremask = 0;
    int nclusters = 0;
    for (int v = 0; v < n; ++v) N[v] = nbr[v] | (1u << v);
    for (int u = 0; u < n; ++u) {
        Neps[u] = 0;
        for (int v = 0; v < n; ++v)
            if (((N[u] >> v) & 1u) && sim(N[u], N[v], p, q)) Neps[u] |= 1u << v;
        if ((uint32_t)pop(Neps[u]) >= mu) coremask |= 1u << u;
    }
    for (int u = 0; u < n; ++u) {
        if (!((coremask >> u) & 1u)) { R[u] = 1u << u; continue; }
        uint32_t set = 1u << u, prev;
        do {
            prev = set;
            for (int x = 0; x < n; ++x)
                if (((set & coremask) >> x) & 1u) set |= Neps[x];
        } while (set != prev);
        R[u] = set;
        int seen = 0;
        for (int k = 0; k < nclusters; ++k) seen |= clusters[k] == set;
        if (!seen) clusters[nclusters++] = set;
    }
    /* literal check of Definition Cluster on every candidate */
    for (int k = 0; k < nclusters; ++k) {
        uint32_t C = clusters[k];
        for (int v1 = 0; v1 < n; ++v1)
            for (int v2 = 0; v2 < n; ++v2) {
                if (!((C >> v1) & 1u) || !((C >> v2) & 1u)) continue;
                int ok = 0;
                for (int x = 0; x < n && !ok; ++x)
                    if (((C >> x) & 1u) && ((R[x] >> v1) & 1u) && ((R[x] >> v2) & 1u)) ok = 1;
                if (!ok) return BRUTE_EDEF;
            }
        for (int u = 0; u < n; ++u)
            if (((C & coremask) >> u) & 1u)
                if ((R[u] & ~C) != 0) return BRUTE_EDEF;
    }
    /* cluster id = smallest core id in the cluster */
    int32_t ccid[32];
    for (int k = 0; k < nclusters; ++k) ccid[k] = __builtin_ctz(clusters[k] & coremask);
    int64_t np = 0;
    for (int v = 0; v < n; ++v) {
        core[v] = (uint8_t)((coremask >> v) & 1u);
        cid[v] = -1;
        int32_t mine[32];
        int nm = 0;
        for (int k = 0; k < nclusters; ++k)
            if ((clusters[k] >> v) & 1u) mine[nm++] = ccid[k];
        for (int i = 1; i < nm; ++i) { /* insertion sort of the member ids */
            int32_t t = mine[i];
            int j = i - 1;
            while (j >= 0 && mine[j] > t) { mine[j + 1] = mine[j]; --j; }
            mine[j + 1] = t;
        }
        if (core[v]) {
            if (nm != 1) return BRUTE_EDEF; /* a core lies in exactly one cluster */
            cid[v] = mine[0];
            label[v] = 0;
        } else if (nm > 0) {
            for (int i = 0; i < nm; ++i) { pairs[2 * np] = v; pairs[2 * np + 1] = mine[i]; ++np; }
            label[v] = 1;
        } else {
            int touched = 0;
            for (int k = 0; k < nclusters; ++k) touched += (clusters[k] & nbr[v]) != 0;
            label[v] = (uint8_t)(touched >= 2 ? 2 : 3);
        }
    }
    *npairs = np;
    return BRUTE_OK;
}

/*
 * Compare oracle_scan with brute_scan on every simple graph with n vertices
 * whose edge mask lies in [mask_lo, mask_hi) (bit k of the mask is the k-th
 * pair (i, j), i < j, in row-major order). Returns the number of graphs that
 * disagree (or that fail a definition check); *first_bad = first such mask.
 */
int64_t brute_exhaustive(int n, uint32_t p, uint32_t q, uint32_t mu, int64_t mask_lo, int64_t mask_hi,
                         int threads, int64_t *first_bad) {
    if (n < 1 || n > 11) return -1;
    int pi[64], pj[64], np = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) { pi[np] = i; pj[np] = j; ++np; }
    int64_t bad = 0, first = -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    #pragma omp parallel for schedule(dynamic, 4096) reduction(+:bad)
    for (int64_t mask = mask_lo; mask < mask_hi; ++mask) {
        uint32_t nbr[32] = {0};
        for (int k = 0; k < np; ++k)
            if ((mask >> k) & 1) { nbr[pi[k]] |= 1u << pj[k]; nbr[pj[k]] |= 1u << pi[k]; }
        int64_t off[33];
        int32_t adj[128];
        off[0] = 0;
        for (int v = 0; v < n; ++v) {
            int64_t e = off[v];
            for (int w = 0; w < n; ++w)
                if ((nbr[v] >> w) & 1u) adj[e++] = w;
            off[v + 1] = e;
        }
        uint8_t c1[32], c2[32], l1[32], l2[32];
        int32_t d1[32], d2[32], p1[256], p2[256];
        int64_t n1 = 0, n2 = 0;
        int r1 = oracle_scan(n, off, adj, p, q, mu, 0, c1, d1, l1, p1, &n1, NULL);
        int r2 = brute_scan(n, nbr, p, q, mu, c2, d2, l2, p2, &n2);
        int diff = r1 != 0 || r2 != 0 || n1 != n2 ||
                   memcmp(c1, c2, (size_t)n) != 0 || memcmp(d1, d2, sizeof(int32_t) * (size_t)n) != 0 ||
                   memcmp(l1, l2, (size_t)n) != 0 ||
                   (n1 == n2 && n1 > 0 && memcmp(p1, p2, sizeof(int32_t) * 2 * (size_t)n1) != 0);
        if (diff) {
            ++bad;
            #pragma omp critical
            { if (first < 0 || mask < first) first = mask; }
        }
    }
    *first_bad = first;
    return bad;
}

// k_query.cu -- one SCAN query on a resident graph.
//
// Steps (GPUSCAN++ Algorithm 1's three phases, restated):
//   similarity  per degree-oriented edge: closed common count, exact eps-test,
//               result mirrored to both slots (Algorithm 2 / checkSim);
//   cores       |N_eps[u]| = 1 + #similar slots of row u, early exit at mu;
//   clusters    lock-free union-find over core-core similar edges, hooking
//               the larger root under the smaller one, so each root is the
//               smallest core id of its cluster (Algorithm 3 replaced);
//   borders     every (non-core v, cluster of an eps-similar core) pair,
//               sorted and unique per vertex;
//   labels      core / border / hub / outlier (Algorithm 4, by definition).
#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr int kBlock = 256;
constexpr int kUfLimit = 1 << 22;

// ------------------------------------------------------------------ similarity
// Binary search of x in the ascending row r[0, len).
__device__ __forceinline__ int contains(const int32_t *__restrict__ r, int32_t len, int32_t x) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t y = __ldg(r + mid);
        if (y < x) lo = mid + 1;
        else if (y > x) hi = mid;
        else return 1;
    }
    return 0;
}

// Warp per degree-oriented edge (u, v), deg(u) <= deg(v): each lane takes
// elements of nbr(u) and binary-searches them in nbr(v) (checkSim of
// Algorithm 2, with the exact test). PRUNE skips edges whose outcome the
// degrees fix; WRITE_SIM / WRITE_CN select the outputs.
template <bool PRUNE, bool WRITE_SIM, bool WRITE_CN>
__global__ void __launch_bounds__(kBlock) k_isect_bsearch(
    const int64_t *__restrict__ off, const int32_t *__restrict__ adj, const int32_t *__restrict__ src,
    const uint32_t *__restrict__ rev, const int32_t *__restrict__ deg, const uint32_t *__restrict__ oe, int64_t m,
    QParams qp, uint8_t *__restrict__ sim, int32_t *__restrict__ cn) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kBlock / kWarp);
    for (int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kWarp; i < m; i += warps) {
        const uint32_t e = oe[i];
        const int32_t u = src[e], v = adj[e];
        const int32_t du = deg[u], dv = deg[v];
        uint64_t pp, qq;
        qp.eps(u, pp, qq);
        if (PRUNE) {
            if (dev::prune_dissimilar((uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) continue;
            if (dev::prune_similar((uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) {
                if (lane == 0) { sim[e] = 1; sim[rev[e]] = 1; }
                continue;
            }
        }
        const int32_t *ru = adj + off[u];
        const int32_t *rv = adj + off[v];
        int c = 0;
        for (int32_t k = lane; k < du; k += kWarp) c += contains(rv, dv, __ldg(ru + k));
        c = __reduce_add_sync(0xffffffffu, c) + 2;
        if (lane == 0) {
            if (WRITE_CN) { cn[e] = c; cn[rev[e]] = c; }
            if (WRITE_SIM && dev::eps_similar((uint64_t)c, (uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) {
                sim[e] = 1;
                sim[rev[e]] = 1;
            }
        }
    }
}

// eps-test from cached closed common counts, one thread per oriented edge
__global__ void __launch_bounds__(kBlock) k_sim_from_counts(
    const int32_t *__restrict__ adj, const int32_t *__restrict__ src, const uint32_t *__restrict__ rev,
    const int32_t *__restrict__ deg, const uint32_t *__restrict__ oe, int64_t m, const int32_t *__restrict__ cn,
    QParams qp, uint8_t *__restrict__ sim) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < m; i += (int64_t)gridDim.x * kBlock) {
        const uint32_t e = oe[i];
        const int32_t u = src[e], v = adj[e];
        uint64_t pp, qq;
        qp.eps(u, pp, qq);
        if (dev::eps_similar((uint64_t)cn[e], (uint64_t)deg[u] + 1, (uint64_t)deg[v] + 1, pp, qq)) {
            sim[e] = 1;
            sim[rev[e]] = 1;
        }
    }
}

// ------------------------------------------------------------------ cores
// Warp per vertex: count similar slots, stop once 1 + count >= mu.
__global__ void __launch_bounds__(kBlock) k_core(const int64_t *__restrict__ off, const uint8_t *__restrict__ sim,
                                                 int32_t n, QParams qp, uint8_t *__restrict__ core) {
    const int64_t u = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const uint32_t mu = qp.mu_of((int32_t)u);
    const int64_t b = off[u], e = off[u + 1];
    uint32_t cnt = 1;  // u itself: sigma(u, u) = 1
    for (int64_t s0 = b; s0 < e && cnt < mu; s0 += kWarp) {
        const int64_t s = s0 + lane;
        const bool hit = s < e && sim[s];
        cnt += __popc(__ballot_sync(0xffffffffu, hit));
    }
    if (lane == 0) core[u] = cnt >= mu ? 1 : 0;
}

// ------------------------------------------------------------------ union-find
__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x, uint32_t *err) {
    for (int it = 0; it < kUfLimit; ++it) {
        int32_t p = ((volatile int32_t *)parent)[x];
        if (p == x) return x;
        int32_t gp = ((volatile int32_t *)parent)[p];
        if (gp != p) ((volatile int32_t *)parent)[x] = gp;  // path halving; gp is an ancestor of x
        x = gp;
    }
    atomicOr(err, ERR_FIND_LIMIT);
    return x;
}

// Hook the larger root under the smaller one (CAS on the root's own entry).
__device__ __forceinline__ void uf_unite(int32_t *parent, int32_t a, int32_t b, uint32_t *err) {
    for (int it = 0; it < kUfLimit; ++it) {
        a = uf_find(parent, a, err);
        b = uf_find(parent, b, err);
        if (a == b) return;
        if (a > b) { int32_t t = a; a = b; b = t; }
        int32_t old = atomicCAS(parent + b, b, a);
        if (old == b) return;
    }
    atomicOr(err, ERR_UF_LIMIT);
}

__global__ void k_uf_init(const uint8_t *__restrict__ core, int32_t n, int32_t *__restrict__ parent) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) parent[u] = core[u] ? (int32_t)u : -1;
}

// one thread per oriented edge: core-core similar edges join clusters
__global__ void __launch_bounds__(kBlock) k_uf_hook(const int32_t *__restrict__ adj, const int32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ oe, int64_t m,
                                                   const uint8_t *__restrict__ sim, const uint8_t *__restrict__ core,
                                                   int32_t *parent, uint32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < m; i += (int64_t)gridDim.x * kBlock) {
        const uint32_t e = oe[i];
        if (!sim[e]) continue;
        const int32_t u = src[e], v = adj[e];
        if (core[u] && core[v]) uf_unite(parent, u, v, err);
    }
}

__global__ void k_uf_final(const uint8_t *__restrict__ core, int32_t n, int32_t *parent, int32_t *__restrict__ cid,
                           uint32_t *err) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    cid[u] = core[u] ? uf_find(parent, (int32_t)u, err) : -1;
}

// ------------------------------------------------------------------ borders
// Warp per non-core vertex: number of eps-similar core neighbours (< mu - 1).
__global__ void __launch_bounds__(kBlock) k_border_count(const int64_t *__restrict__ off,
                                                        const int32_t *__restrict__ adj,
                                                        const uint8_t *__restrict__ sim,
                                                        const uint8_t *__restrict__ core, int32_t n,
                                                        int32_t *__restrict__ cnt) {
    const int64_t v = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    int c = 0;
    if (!core[v]) {
        const int64_t b = off[v], e = off[v + 1];
        for (int64_t s = b + lane; s < e; s += kWarp) c += (sim[s] && core[adj[s]]) ? 1 : 0;
        c = __reduce_add_sync(0xffffffffu, c);
    }
    if (lane == 0) cnt[v] = c;
}

// Warp per non-core vertex: write the candidate cluster ids, then lane 0
// sorts the (short) segment and removes duplicates.
__global__ void __launch_bounds__(kBlock) k_border_fill(const int64_t *__restrict__ off,
                                                       const int32_t *__restrict__ adj,
                                                       const uint8_t *__restrict__ sim,
                                                       const uint8_t *__restrict__ core,
                                                       const int32_t *__restrict__ cid, int32_t n,
                                                       const int64_t *__restrict__ raw_off, int32_t *__restrict__ raw,
                                                       int32_t *__restrict__ ucnt) {
    const int64_t v = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const int64_t base = raw_off[v], k = raw_off[v + 1] - base;
    if (k == 0) {
        if (lane == 0) ucnt[v] = 0;
        return;
    }
    const int64_t b = off[v], e = off[v + 1];
    int64_t w = base;
    for (int64_t s0 = b; s0 < e; s0 += kWarp) {
        const int64_t s = s0 + lane;
        int32_t x = -1;
        bool f = false;
        if (s < e && sim[s]) {
            const int32_t u = adj[s];
            if (core[u]) { f = true; x = cid[u]; }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, f);
        if (f) raw[w + __popc(mask & ((1u << lane) - 1u))] = x;
        w += __popc(mask);
    }
    __syncwarp();
    if (lane == 0) {
        int32_t *a = raw + base;
        for (int64_t i = 1; i < k; ++i) {  // insertion sort: k < mu - 1
            int32_t t = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > t) { a[j + 1] = a[j]; --j; }
            a[j + 1] = t;
        }
        int64_t u = 1;
        for (int64_t i = 1; i < k; ++i)
            if (a[i] != a[u - 1]) a[u++] = a[i];
        ucnt[v] = (int32_t)u;
    }
}

__global__ void k_border_emit(const int64_t *__restrict__ raw_off, const int32_t *__restrict__ raw,
                              const int32_t *__restrict__ ucnt, const int64_t *__restrict__ pair_off, int32_t n,
                              int32_t *__restrict__ pairs, int64_t pairs_cap, int64_t *__restrict__ npairs) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) *npairs = pair_off[n];
    if (v >= n) return;
    const int64_t b = raw_off[v], o = pair_off[v];
    for (int32_t i = 0; i < ucnt[v]; ++i) {
        if (o + i >= pairs_cap) break;
        pairs[2 * (o + i)] = (int32_t)v;
        pairs[2 * (o + i) + 1] = raw[b + i];
    }
}

// ------------------------------------------------------------------ labels
// Warp per vertex. A vertex in no cluster is a hub iff the union of its
// neighbours' memberships holds two distinct ids: some neighbour is itself
// in >= 2 clusters, or two neighbours' single ids differ (min != max).
__global__ void __launch_bounds__(kBlock) k_label(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                 const uint8_t *__restrict__ core, const int32_t *__restrict__ cid,
                                                 const int32_t *__restrict__ ucnt, const int64_t *__restrict__ raw_off,
                                                 const int32_t *__restrict__ raw, int32_t n,
                                                 uint8_t *__restrict__ label) {
    const int64_t u = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    if (core[u]) { if (lane == 0) label[u] = SCAN_CORE; return; }
    if (ucnt[u] > 0) { if (lane == 0) label[u] = SCAN_BORDER; return; }
    const int64_t b = off[u], e = off[u + 1];
    int32_t lo = INT32_MAX, hi = -1;
    bool multi = false;
    for (int64_t s0 = b; s0 < e; s0 += kWarp) {
        const int64_t s = s0 + lane;
        if (s < e) {
            const int32_t w = adj[s];
            int32_t id = -1;
            if (core[w]) id = cid[w];
            else if (ucnt[w] > 0) {
                id = raw[raw_off[w]];
                multi |= ucnt[w] > 1;
            }
            if (id >= 0) { lo = min(lo, id); hi = max(hi, id); }
        }
        const bool any_multi = __any_sync(0xffffffffu, multi);
        const int32_t glo = __reduce_min_sync(0xffffffffu, lo);
        const int32_t ghi = __reduce_max_sync(0xffffffffu, hi);
        if (any_multi || (ghi >= 0 && glo != ghi)) {
            if (lane == 0) label[u] = SCAN_HUB;
            return;
        }
    }
    if (lane == 0) label[u] = SCAN_OUTLIER;
}

}  // namespace

static scan_status launch_isect(Graph *g, bool prune, bool write_sim, bool write_cn, const QParams &qp,
                                int32_t *cn) {
    Ctx *c = g->ctx;
    if (g->m == 0) return SCAN_OK;
    const unsigned grid = grid_for(g->m * kWarp, kBlock, c->num_sms * 64);
    auto *off = (const int64_t *)g->off.ptr;
    auto *adj = (const int32_t *)g->adj.ptr;
    auto *src = (const int32_t *)g->src.ptr;
    auto *rev = (const uint32_t *)g->rev.ptr;
    auto *deg = (const int32_t *)g->deg.ptr;
    auto *oe = (const uint32_t *)g->oe.ptr;
    auto *sim = (uint8_t *)g->sim.ptr;
    if (prune)
        k_isect_bsearch<true, true, false><<<grid, kBlock, 0, c->stream>>>(off, adj, src, rev, deg, oe, g->m, qp, sim, cn);
    else if (write_cn && !write_sim)
        k_isect_bsearch<false, false, true><<<grid, kBlock, 0, c->stream>>>(off, adj, src, rev, deg, oe, g->m, qp, sim, cn);
    else
        k_isect_bsearch<false, true, false><<<grid, kBlock, 0, c->stream>>>(off, adj, src, rev, deg, oe, g->m, qp, sim, cn);
    c->launches++;
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status build_count_cache(Graph *g) {
    Ctx *c = g->ctx;
    if (!g->cn_cache.ptr) SCAN_TRY(dev_alloc(c, g->cn_cache, sizeof(int32_t) * (size_t)(g->nnz > 0 ? g->nnz : 1)));
    int32_t *cn = (int32_t *)g->cn_cache.ptr;
    if (g->strategy == SCAN_STRATEGY_OWNER) SCAN_TRY(launch_owner_isect(g, false, false, true, QParams{}, cn));
    else if (g->strategy == SCAN_STRATEGY_BSEARCH) SCAN_TRY(launch_isect(g, false, false, true, QParams{}, cn));
    else SCAN_TRY(launch_fwd_counts(g, false, true, QParams{}, cn));
    g->cache_valid = true;
    return SCAN_OK;
}

scan_status query_pipeline(Graph *g, const QParams &qp, uint32_t mode, uint8_t *core, int32_t *cid,
                           uint8_t *label, int32_t *pairs, int64_t pairs_cap, int64_t *npairs) {
    Ctx *c = g->ctx;
    cudaStream_t st = c->stream;
    const int32_t n = g->n;
    const int64_t nnz = g->nnz, m = g->m;
    auto *off = (const int64_t *)g->off.ptr;
    auto *adj = (const int32_t *)g->adj.ptr;
    auto *src = (const int32_t *)g->src.ptr;
    auto *rev = (const uint32_t *)g->rev.ptr;
    auto *deg = (const int32_t *)g->deg.ptr;
    auto *oe = (const uint32_t *)g->oe.ptr;
    auto *sim = (uint8_t *)g->sim.ptr;
    auto *err = (uint32_t *)g->err.ptr;

    {
        StageTimer t(c, SCAN_STAGE_SIMILARITY);
        if (nnz > 0) SCAN_CUDA(cudaMemsetAsync(sim, 0, (size_t)nnz, st));
        if (mode & SCAN_Q_BUILD_CACHE) SCAN_TRY(build_count_cache(g));
        const bool use_cache = g->cache_valid && !(mode & (SCAN_Q_RECOMPUTE | SCAN_Q_PLAIN));
        if (use_cache) {
            if (m > 0) {
                k_sim_from_counts<<<grid_for(m, kBlock, c->num_sms * 32), kBlock, 0, st>>>(
                    adj, src, rev, deg, oe, m, (const int32_t *)g->cn_cache.ptr, qp, sim);
                c->launches++;
            }
        } else if (mode & SCAN_Q_PLAIN) {
            SCAN_TRY(launch_isect(g, false, true, false, qp, nullptr));
        } else if (g->strategy == SCAN_STRATEGY_OWNER) {
            SCAN_TRY(launch_owner_isect(g, true, true, false, qp, nullptr));
        } else if (g->strategy == SCAN_STRATEGY_BSEARCH) {
            SCAN_TRY(launch_isect(g, true, true, false, qp, nullptr));
        } else {
            SCAN_TRY(launch_fwd_counts(g, true, false, qp, nullptr));
        }
    }

    if (n == 0) {
        SCAN_CUDA(cudaMemsetAsync(npairs, 0, sizeof(int64_t), st));
        SCAN_CUDA(cudaGetLastError());
        return SCAN_OK;
    }
    const unsigned gw = grid_for((int64_t)n * kWarp, kBlock);
    const unsigned gt = grid_for(n, kBlock);
    {
        StageTimer t(c, SCAN_STAGE_CORE);
        k_core<<<gw, kBlock, 0, st>>>(off, sim, n, qp, core);
        c->launches++;
    }
    {
        StageTimer t(c, SCAN_STAGE_CLUSTER);
        int32_t *parent = (int32_t *)g->parent.ptr;
        k_uf_init<<<gt, kBlock, 0, st>>>(core, n, parent);
        if (m > 0)
            k_uf_hook<<<grid_for(m, kBlock, c->num_sms * 32), kBlock, 0, st>>>(adj, src, oe, m, sim, core, parent,
                                                                                err);
        k_uf_final<<<gt, kBlock, 0, st>>>(core, n, parent, cid, err);
        c->launches += 2 + (m > 0);
    }
    int32_t *cnt = (int32_t *)g->cnt.ptr;
    int64_t *cnt_off = (int64_t *)g->cnt_off.ptr;
    int32_t *ucnt = (int32_t *)g->ucnt.ptr;
    int64_t *pair_off = (int64_t *)g->pair_off.ptr;
    int32_t *raw = (int32_t *)g->raw.ptr;
    {
        StageTimer t(c, SCAN_STAGE_BORDER);
        k_border_count<<<gw, kBlock, 0, st>>>(off, adj, sim, core, n, cnt);
        c->launches++;
        SCAN_TRY(launch_exclusive_scan_i32_to_i64(c, cnt, cnt_off, n, g->scan_tmp));
        k_border_fill<<<gw, kBlock, 0, st>>>(off, adj, sim, core, cid, n, cnt_off, raw, ucnt);
        c->launches++;
        SCAN_TRY(launch_exclusive_scan_i32_to_i64(c, ucnt, pair_off, n, g->scan_tmp));
        k_border_emit<<<gt, kBlock, 0, st>>>(cnt_off, raw, ucnt, pair_off, n, pairs, pairs_cap, npairs);
        c->launches++;
    }
    {
        StageTimer t(c, SCAN_STAGE_LABEL);
        k_label<<<gw, kBlock, 0, st>>>(off, adj, core, cid, ucnt, cnt_off, raw, n, label);
        c->launches++;
    }
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

}  // namespace scan

// scan_internal.cuh -- internal structures and device helpers of libscan.so.
//
// Layout in HBM of a resident graph (n vertices, nnz = 2m directed slots):
//   off   int64[n+1]  CSR offsets (vertex array, Section 4.1)
//   adj   int32[nnz]  neighbour ids, rows ascending (adjacency array)
//   src   int32[nnz]  row of each slot (COO expansion of off)
//   rev   uint32[nnz] slot of (v,u) for the slot of (u,v) (plays the Eid role:
//                     it ties the two directions of one edge together)
//   deg   int32[n]
//   oe    uint32[m]   degree-oriented edges: the slot in the row of the lower
//                     (deg, id) endpoint, i.e. the degree-oriented edge array
//                     of Section 4.1 expressed as slot ids
// Per-query scratch lives on the graph and is reused between queries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "scan.h"

namespace scan {

// device error word bits
enum : uint32_t {
    ERR_UF_LIMIT = 1u,     // union-find retry bound hit
    ERR_FIND_LIMIT = 2u,   // root walk bound hit
    ERR_LOOP_LIMIT = 4u,   // any other bounded device loop
};

constexpr int kWarp = 32;

struct Ctx;
struct Part;  // out-of-core state of a graph kept in host memory (partition.cu)

// Device allocation accounted against the context's budget.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Graph {
    Ctx *ctx = nullptr;
    int32_t n = 0;
    int64_t nnz = 0;
    int64_t m = 0;          // undirected edges = nnz / 2
    DevBuf off, adj, src, rev, deg, oe;
    DevBuf cn_cache;        // int32[m] closed common counts per oriented edge (cached-count serving)
    DevBuf cdd;             // uint64[m] (deg u + 1)(deg v + 1) per oriented edge (same cache)
    bool cache_valid = false;
    // owner schedule of the shared-memory intersection (built on first use)
    bool owner_ready = false;
    DevBuf owners_small;    // int32[n_small] owners with deg <= 128
    DevBuf items[4];        // work items of classes 1..3
    int64_t n_items[4] = {0, 0, 0, 0};
    int32_t n_small = 0;
    DevBuf owners_chunked;  // int32[n_chunked] owners whose row is split in value chunks
    int32_t n_chunked = 0;
    DevBuf acc;             // int32[nnz] partial counts of chunked owners (kept zero between queries)
    // degree-oriented (forward) lists for triangle-based counting
    DevBuf foff;            // int64[n+1] offsets of out(x) in oe / fadj (built at load)
    DevBuf fadj;            // int32[m] out(x) neighbour ids, ascending
    DevBuf fin;             // uint32[nnz] for a slot (b, a) with a below b: index of a->b in fadj
    DevBuf fcnt;            // int32[m] triangle counts per oriented edge
    DevBuf fsrc;            // int32[m] lower endpoint of each oriented edge, in fadj order
    DevBuf fhid;            // int32[m] dense id of each out-list element (degree level first): bitmap tables
    DevBuf fwd_owners;      // warp-level owners
    DevBuf fwd_items[3];    // CTA items, by table class 1..2
    int64_t fwd_items_n[3] = {0, 0, 0};
    int32_t fwd_small = 0;
    bool fwd_ready = false;
    DevBuf fwd_ebase, fwd_elen, fwd_efin;  // precomputed entries of the CTA items (start in fadj, length, (a, b) index)
    bool fwd_entries = false;              // entries built (else the kernel derives them per round)
    bool fwd_entries_tried = false;        // a build was attempted (it is skipped when it does not fit)
    bool fwd_rank_sorted = false;  // out-lists ordered by (deg, id) instead of id
    int32_t fwd_smem_words[3] = {0, 0, 0};  // shared memory the largest table of each item class needs
    bool fwd_queue = false;  // count in one persistent launch over a work queue (else one launch per class)
    DevBuf fwd_qctr;        // its take counters
    // the per-class launches: class 2 and the warp owners run on a side
    // stream beside classes 1 and 0 (forked from and joined to the query's stream)
    cudaStream_t fwd_side = nullptr;
    cudaEvent_t fwd_fork = nullptr, fwd_join = nullptr;
    int64_t fwd_small_work = 1 << 15;  // owners with out-degree <= 64 and at most this many probes: one warp
    int64_t fwd_item_work = 1 << 20;   // target probes per CTA work item
    int strategy = 0;       // similarity kernel family: SCAN_STRATEGY_*
    // one captured query pipeline, replayed as a CUDA graph (query_replay)
    cudaGraphExec_t qexec = nullptr;
    uint64_t qkey = 0;
    uint64_t qlaunches = 0;   // kernels in the captured graph (added to the launch counter per replay)
    bool qgraph_off = false;  // capture failed once: no more attempts
    DevBuf qparams;           // uint64[3] parameters the replayed graph reads
    uint64_t *h_qparams = nullptr;  // pinned staging of the same
    DevBuf heavy;           // int32[n_heavy] vertices whose rows are walked by a whole CTA
    int32_t n_heavy = 0;
    bool heavy_ready = false;
    Part *part = nullptr;   // non-null: the CSR stays in host memory and is streamed in blocks
    // per-query scratch
    DevBuf sim;             // uint8[nnz] 1 = eps-similar (per-slot output of the per-edge families; on first use)
    DevBuf simo;            // uint8[m] 1 = oriented edge oe[i] is eps-similar
    DevBuf nsim;            // int32[n+1] open eps-degree
    DevBuf hst;             // int32[n+1] hub test state of the label stage's push direction
    DevBuf mslots;          // uint64[1] row slots of the vertices in a cluster
    DevBuf core, cid, parent, label;
    DevBuf cnt, cnt_off;    // int32[n+1] counts, int64[n+1] exclusive offsets
    DevBuf ucnt, pair_off;  // unique membership counts / offsets
    DevBuf raw;             // int32[nnz] raw border candidates
    DevBuf pairs;           // int32[2*nnz]
    DevBuf npairs;          // int64[1]
    DevBuf scan_tmp;        // block partials for the prefix scan
    DevBuf err;             // uint32[1]
    // host staging
    int64_t *h_npairs = nullptr; // pinned
    uint32_t *h_err = nullptr;   // pinned
    // the second output set of a parameter sweep (scan_query_sweep), made on
    // first use: one query writes it while the other set is copied to the host
    DevBuf core2, cid2, label2, pairs2, npairs2;
    cudaStream_t sweep_stream = nullptr;    // the copies to the host
    cudaEvent_t sweep_done[2] = {nullptr, nullptr};    // a set's query finished
    cudaEvent_t sweep_copied[2] = {nullptr, nullptr};  // a set's copies finished
    int64_t *h_sweep_np = nullptr;          // pinned int64[2]: pair counts of the two sets

    template <class F>
    void for_each_buf(F f) {
        DevBuf *bufs[] = {&off, &adj, &src, &rev, &deg, &oe, &cn_cache, &cdd, &owners_small, &items[0], &items[1],
                          &items[2], &items[3], &owners_chunked, &acc, &foff, &fadj, &fin, &fcnt, &fsrc, &fhid, &fwd_qctr, &fwd_owners,
                          &fwd_items[0], &fwd_items[1], &fwd_items[2], &fwd_ebase, &fwd_elen, &fwd_efin, &heavy,
                          &qparams, &sim, &simo, &nsim, &hst, &mslots, &core, &cid, &parent, &label,
                          &cnt, &cnt_off, &ucnt, &pair_off, &raw, &pairs, &npairs, &scan_tmp, &err,
                          &core2, &cid2, &label2, &pairs2, &npairs2};
        for (DevBuf *b : bufs) f(*b);
    }
};

// Query parameters seen by the kernels: either one (eps, mu) for the whole
// graph, or -- for a batch of graphs stored as one disjoint union -- a graph
// index per vertex and per-graph parameter arrays in device memory.
struct QParams {
    uint64_t pp = 0, qq = 0;        // eps_num^2, eps_den^2
    uint32_t mu = 0;
    const int32_t *gid = nullptr;   // [n] graph index of every vertex, or null
    const uint64_t *gpp = nullptr;  // [k] per-graph eps_num^2
    const uint64_t *gqq = nullptr;  // [k] per-graph eps_den^2
    const uint32_t *gmu = nullptr;  // [k] per-graph mu
    const uint64_t *dev = nullptr;  // or one (eps_num^2, eps_den^2, mu) in device memory (graph replays)
    __device__ __forceinline__ void eps(int32_t v, uint64_t &p2, uint64_t &q2) const {
        if (gid) {
            const int32_t g = gid[v];
            p2 = gpp[g];
            q2 = gqq[g];
        } else if (dev) {
            p2 = dev[0];
            q2 = dev[1];
        } else {
            p2 = pp;
            q2 = qq;
        }
    }
    __device__ __forceinline__ uint32_t mu_of(int32_t v) const {
        return gid ? gmu[gid[v]] : (dev ? (uint32_t)dev[2] : mu);
    }
};

struct StageMark {
    int stage;
    cudaEvent_t start, stop;
};

struct Ctx {
    int device = 0;
    uint64_t budget = 0;   // 0 = no cap
    uint64_t used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t launches = 0;
    int num_sms = 0;
    int smem_optin = 0;
    uint32_t loop_limit = 0;  // union-find iteration cap of later queries; 0 = the compiled bound
    // per-stage timing
    bool profiling = false;
    std::vector<StageMark> marks;
    double stage_ms[SCAN_STAGE_COUNT] = {0};
    int64_t stage_n[SCAN_STAGE_COUNT] = {0};
};

// Records CUDA events around one stage when the context is profiling.
struct StageTimer {
    Ctx *c;
    StageMark mark{};
    bool on;
    StageTimer(Ctx *ctx, int stage) : c(ctx), on(ctx->profiling) {
        if (!on) return;
        mark.stage = stage;
        cudaEventCreate(&mark.start);
        cudaEventCreate(&mark.stop);
        cudaEventRecord(mark.start, c->stream);
    }
    ~StageTimer() {
        if (!on) return;
        cudaEventRecord(mark.stop, c->stream);
        c->marks.push_back(mark);
    }
};

}  // namespace scan

// The opaque ABI handles are the internal objects.
struct scan_ctx : scan::Ctx {};
struct scan_graph : scan::Graph {};

// Host result of one query (library-owned until scan_result_free).
struct scan_result {
    int32_t n = 0;
    int64_t k = 0;
    uint8_t *core = nullptr;
    int32_t *cid = nullptr;
    uint8_t *label = nullptr;
    int32_t *pairs = nullptr;
    bool pinned = false;  // arrays from the pinned block pool (else malloc)
    size_t cap[4] = {0, 0, 0, 0};  // pinned block sizes of core, cid, label, pairs
};

namespace scan {

// ---- host helpers (abi.cu)
void set_error(const std::string &msg);
scan_status cuda_fail(cudaError_t e, const char *what);
scan_status dev_alloc(Ctx *c, DevBuf &b, size_t bytes);
void dev_free(Ctx *c, DevBuf &b);
scan_status check_params(const scan_params *p);
scan_status take_device_error(Graph *g);
// Allocates and prepares a resident graph. The CSR comes from offsets/adj
// (host, or device with on_dev), or -- when fill is given -- fill writes it
// into g->off and g->adj on the context's stream (offsets/adj unused).
scan_status graph_create(Ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz, bool on_dev,
                         Graph **out, const std::function<scan_status(Graph *)> &fill = nullptr);
void graph_destroy(Graph *g);
// pinned host blocks from a pool: at least `bytes` (block size in *cap), null if out of memory
void *pinned_get(size_t bytes, size_t *cap);
void pinned_put(void *p, size_t cap);  // back to the pool (p may be null)
scan_result *result_new(int32_t n, int64_t k, bool pinned);
bool result_set_pairs(scan_result *r, int64_t k);  // room for k pairs (r->k = k); false if out of memory
// out of core (partition.cu)
scan_status part_create(Ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz, Graph **out,
                        int64_t block_slots_hint);
scan_status part_query(Graph *g, const scan_params &p, scan_result **out);
void sweep_release(Graph *g);  // the sweep's stream, events and pinned counts (sweep.cu)
void fwd_release(Graph *g);    // the counting stage's side stream and events (k_fwd.cu)
void part_release(Graph *g);
int32_t part_block_count(const Graph *g);
uint64_t part_transfer_bytes(const Graph *g);
scan_status part_set_zero_copy(Graph *g, bool on);
scan_status plan_edge_extended(int32_t n, const int64_t *off, const int32_t *adj, int64_t nnz, uint64_t mem,
                               int64_t *subgraphs, uint64_t *bytes);
scan_status plan_triangle_blocks(int32_t n, const int64_t *off, const int32_t *adj, int64_t nnz, uint64_t mem,
                                 int32_t *blocks, int64_t *pairs, uint64_t *bytes);

#define SCAN_CUDA(call)                                              \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::scan::cuda_fail(_e, #call);  \
    } while (0)

#define SCAN_TRY(call)                       \
    do {                                     \
        scan_status _s = (call);             \
        if (_s != SCAN_OK) return _s;        \
    } while (0)

// ---- launchers (k_*.cu); every launcher counts its kernels in ctx->launches
scan_status launch_exclusive_scan_i32_to_i64(Ctx *c, const int32_t *in, int64_t *out, int64_t count,
                                             DevBuf &tmp);
scan_status graph_prepare(Graph *g);                    // deg, src, rev, validation, oe
scan_status query_pipeline(Graph *g, const QParams &qp, uint32_t mode, uint8_t *core, int32_t *cid,
                           uint8_t *label, int32_t *pairs, int64_t pairs_cap, int64_t *npairs);
// The same pipeline for one graph and uniform parameters, replayed as a CUDA
// graph once it has run once with the same mode and output buffers.
scan_status query_replay(Graph *g, const scan_params &p, uint32_t mode, uint8_t *core, int32_t *cid, uint8_t *label,
                         int32_t *pairs, int64_t pairs_cap, int64_t *npairs);
void query_graph_drop(Graph *g);  // forget the captured graph (buffers or kernel choice changed)
uint64_t replay_key(uint32_t mode, const void *a, const void *b, const void *c, const void *d, int64_t cap,
                    const void *e);  // identity of a captured launch sequence
// The count cache: per oriented edge oe[i], its closed common count and the
// product of its endpoints' closed degrees, so that a cached query's eps-test
// reads 12 contiguous bytes per edge and no vertex data.
scan_status cache_reserve(Graph *g);  // allocate both arrays (no-op when present)
void cache_free(Graph *g);            // free them; the cache is no longer valid
scan_status build_count_cache(Graph *g);
scan_status cache_to_slots(Graph *g, int32_t *slot_counts);  // int32[nnz] device, counts per slot
scan_status owner_schedule_build(Graph *g);
scan_status launch_owner_isect(Graph *g, bool prune, bool write_sim, bool write_cn, const QParams &qp, int32_t *cn);
scan_status fwd_prepare(Graph *g);
// write_cn: cn[i] and dd[i] of every oriented edge (the count cache)
scan_status launch_fwd_counts(Graph *g, bool write_sim, bool write_cn, const QParams &qp, int32_t *cn,
                              uint64_t *dd = nullptr);

inline QParams uniform_params(const scan_params &p) {
    QParams q;
    q.pp = (uint64_t)p.eps_num * p.eps_num;
    q.qq = (uint64_t)p.eps_den * p.eps_den;
    q.mu = p.mu;
    return q;
}

inline unsigned grid_for(int64_t items, int per_block, int max_blocks = 1 << 30) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

}  // namespace scan

// ---------------------------------------------------------------- device
namespace scan {
namespace dev {

// Exact eps-test of Definition 2.3 with eps = p/q on closed sizes:
// sigma(u,v) >= p/q  <=>  c^2 q^2 >= p^2 du dv  (c < 2^31, du dv < 2^62).
__device__ __forceinline__ bool eps_similar(uint64_t c, uint64_t du1, uint64_t dv1, uint64_t pp, uint64_t qq) {
    unsigned __int128 lhs = (unsigned __int128)(c * c) * qq;
    unsigned __int128 rhs = (unsigned __int128)pp * (du1 * dv1);
    return lhs >= rhs;
}
// the same test on the product dd = du1 * dv1
__device__ __forceinline__ bool eps_similar_dd(uint64_t c, uint64_t dd, uint64_t pp, uint64_t qq) {
    return (unsigned __int128)(c * c) * qq >= (unsigned __int128)pp * dd;
}

// Degree-only outcomes (|N[u] cap N[v]| lies in [2, min(du, dv)]):
// sigma <= sqrt(dmin/dmax) < eps  <=>  dmin q^2 < p^2 dmax  -> never similar
__device__ __forceinline__ bool prune_dissimilar(uint64_t dmin1, uint64_t dmax1, uint64_t pp, uint64_t qq) {
    return (unsigned __int128)dmin1 * qq < (unsigned __int128)pp * dmax1;
}
// sigma >= 2/sqrt(du dv) >= eps  <=>  4 q^2 >= p^2 du dv  -> always similar
__device__ __forceinline__ bool prune_similar(uint64_t du1, uint64_t dv1, uint64_t pp, uint64_t qq) {
    return (unsigned __int128)4u * qq >= (unsigned __int128)pp * (du1 * dv1);
}

// (deg, id) orientation of Section 4.1: u precedes v.
__device__ __forceinline__ bool rank_less(int32_t du, int32_t u, int32_t dv, int32_t v) {
    return du < dv || (du == dv && u < v);
}

// |a cap b| of two ascending rows of distinct ids, computed by a whole warp
// (every lane gets the count). Rows of similar length are merged 32 ids at a
// time: each step loads a window of each row (coalesced), every id of the
// window with the smaller maximum is looked up in the other window by a
// 5-step search over the lanes' registers, and both windows advance past
// that maximum, so each step settles at least one window. A row more than
// 16 times shorter than the other is probed instead, each lane binary
// searching its ids in the longer row. Bounded by na + nb steps.
__device__ __forceinline__ int32_t warp_common(const int32_t *__restrict__ a, int32_t na,
                                               const int32_t *__restrict__ b, int32_t nb) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (na > nb) {
        const int32_t *t = a;
        a = b;
        b = t;
        const int32_t tn = na;
        na = nb;
        nb = tn;
    }
    int c = 0;
    if ((int64_t)nb > 16 * (int64_t)na) {
        for (int32_t k = lane; k < na; k += 32) {
            const int32_t x = __ldg(a + k);
            int32_t lo = 0, hi = nb;
            for (int it = 0; it < 40 && lo < hi; ++it) {
                const int32_t mid = (lo + hi) >> 1;
                const int32_t y = __ldg(b + mid);
                if (y < x) lo = mid + 1;
                else if (y > x) hi = mid;
                else {
                    ++c;
                    break;
                }
            }
        }
        return __reduce_add_sync(full, c);
    }
    int32_t ia = 0, ib = 0;
    for (int64_t guard = 0; guard <= (int64_t)na + nb && ia < na && ib < nb; ++guard) {
        const int32_t x = ia + lane < na ? __ldg(a + ia + lane) : INT32_MAX;
        const int32_t y = ib + lane < nb ? __ldg(b + ib + lane) : INT32_MAX;
        const int32_t lim = min(__shfl_sync(full, x, 31), __shfl_sync(full, y, 31));
        int pos = 0;  // ids of the y window below x (the window is ascending)
#pragma unroll
        for (int s = 16; s; s >>= 1)
            if (__shfl_sync(full, y, pos + s - 1) < x) pos += s;
        const int32_t yp = __shfl_sync(full, y, pos);
        c += (x <= lim && x != INT32_MAX && yp == x) ? 1 : 0;
        ia += __popc(__ballot_sync(full, x <= lim && ia + lane < na));
        ib += __popc(__ballot_sync(full, y <= lim && ib + lane < nb));
    }
    return __reduce_add_sync(full, c);
}

}  // namespace dev
}  // namespace scan

// abi.cu -- the C ABI of libscan.so (declared in include/scan.h).
//
// Every entry point catches C++ exceptions and CUDA errors and maps them to
// a scan_status; the detail goes to a thread-local message.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "scan_internal.cuh"

namespace scan {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

scan_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    return SCAN_ECUDA;
}

scan_status dev_alloc(Ctx *c, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->budget && c->used + bytes > c->budget) {
        set_error("device budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                  std::to_string(c->used) + " of " + std::to_string(c->budget) + " in use");
        return SCAN_EBUDGET;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        return SCAN_ENOMEM;
    }
    b.ptr = p;
    b.bytes = bytes;
    c->used += bytes;
    return SCAN_OK;
}

void dev_free(Ctx *c, DevBuf &b) {
    if (b.ptr) {
        cudaFree(b.ptr);
        c->used -= b.bytes;
    }
    b.ptr = nullptr;
    b.bytes = 0;
}

static void graph_release(Graph *g) {
    Ctx *c = g->ctx;
    query_graph_drop(g);
    sweep_release(g);
    fwd_release(g);
    g->for_each_buf([c](DevBuf &b) { dev_free(c, b); });
    if (g->h_npairs) cudaFreeHost(g->h_npairs);
    if (g->h_err) cudaFreeHost(g->h_err);
    if (g->h_qparams) cudaFreeHost(g->h_qparams);
    g->h_npairs = nullptr;
    g->h_err = nullptr;
    g->h_qparams = nullptr;
}

scan_status check_params(const scan_params *p) {
    if (!p) { set_error("params is NULL"); return SCAN_EINVAL; }
    if (p->eps_num == 0 || p->eps_den == 0 || p->eps_num > p->eps_den) {
        set_error("eps must satisfy 0 < eps_num <= eps_den (0 < eps <= 1)");
        return SCAN_EINVAL;
    }
    if (p->mu < 2) { set_error("mu must be >= 2"); return SCAN_EINVAL; }
    return SCAN_OK;
}

// Reads and clears the graph's device error word after a synchronisation.
scan_status take_device_error(Graph *g) {
    Ctx *c = g->ctx;
    SCAN_CUDA(cudaMemcpyAsync(g->h_err, g->err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    if (*g->h_err) {
        uint32_t e = *g->h_err;
        SCAN_CUDA(cudaMemsetAsync(g->err.ptr, 0, sizeof(uint32_t), c->stream));
        set_error("a bounded device loop gave up (error bits " + std::to_string(e) + ")");
        return SCAN_ETIMEOUT;
    }
    return SCAN_OK;
}

}  // namespace scan

using namespace scan;


#define ABI_GUARD_BEGIN try {
#define ABI_GUARD_END                                   \
    }                                                   \
    catch (const std::bad_alloc &) {                    \
        set_error("host allocation failed");            \
        return SCAN_ENOMEM;                             \
    }                                                   \
    catch (...) {                                       \
        set_error("internal error");                    \
        return SCAN_EINVAL;                             \
    }

extern "C" {

const char *scan_last_error(void) { return g_last_error.c_str(); }

scan_status scan_ctx_create(const scan_ctx_opts *opts, scan_ctx **out) {
    ABI_GUARD_BEGIN
    if (!out) { set_error("out is NULL"); return SCAN_EINVAL; }
    *out = nullptr;
    int dev = opts ? opts->device : 0;
    int count = 0;
    SCAN_CUDA(cudaGetDeviceCount(&count));
    if (dev < 0 || dev >= count) {
        set_error("device ordinal " + std::to_string(dev) + " out of range (" + std::to_string(count) + " devices)");
        return SCAN_EINVAL;
    }
    SCAN_CUDA(cudaSetDevice(dev));
    scan_ctx *c = new scan_ctx();
    c->device = dev;
    c->budget = opts ? opts->budget_bytes : 0;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) {
        if (opts && opts->stream) {
            c->stream = (cudaStream_t)opts->stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "context setup");
    }
    *out = c;
    return SCAN_OK;
    ABI_GUARD_END
}

static void drop_marks(Ctx *c);

void scan_ctx_destroy(scan_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    drop_marks(c);
    if (c->own_stream && c->stream) {
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
    }
    delete c;
}

uint64_t scan_ctx_device_bytes(const scan_ctx *c) { return c ? c->used : 0; }
uint64_t scan_ctx_kernel_launches(const scan_ctx *c) { return c ? c->launches : 0; }

scan_status scan_ctx_sync(scan_ctx *c) {
    if (!c) { set_error("ctx is NULL"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(c->device));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    return SCAN_OK;
}

static void drop_marks(Ctx *c) {
    for (auto &m : c->marks) {
        cudaEventDestroy(m.start);
        cudaEventDestroy(m.stop);
    }
    c->marks.clear();
}

scan_status scan_ctx_profile(scan_ctx *c, int32_t enable) {
    if (!c) { set_error("ctx is NULL"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(c->device));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    drop_marks(c);
    for (int s = 0; s < SCAN_STAGE_COUNT; ++s) { c->stage_ms[s] = 0; c->stage_n[s] = 0; }
    c->profiling = enable != 0;
    return SCAN_OK;
}

scan_status scan_ctx_set_loop_limit(scan_ctx *c, uint32_t limit) {
    if (!c) { set_error("ctx is NULL"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(c->device));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));  // queries already queued keep the cap they were launched with
    c->loop_limit = limit;
    return SCAN_OK;
}

scan_status scan_ctx_stage_time(scan_ctx *c, int32_t stage, double *total_ms, int64_t *intervals) {
    if (!c || !total_ms || stage < 0 || stage >= SCAN_STAGE_COUNT) { set_error("bad arguments"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(c->device));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &m : c->marks) {
        float ms = 0;
        SCAN_CUDA(cudaEventElapsedTime(&ms, m.start, m.stop));
        c->stage_ms[m.stage] += ms;
        c->stage_n[m.stage] += 1;
    }
    drop_marks(c);
    *total_ms = c->stage_ms[stage];
    if (intervals) *intervals = c->stage_n[stage];
    return SCAN_OK;
}

}  // extern "C"

namespace scan {

scan_status graph_create(Ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz, bool on_dev,
                         Graph **out, const std::function<scan_status(Graph *)> &fill) {
    *out = nullptr;
    if (n < 0 || nnz < 0 || (!fill && ((n > 0 && !offsets) || (nnz > 0 && !adj)))) {
        set_error("bad sizes or NULL arrays");
        return SCAN_EINVAL;
    }
    if (nnz % 2 != 0) { set_error("nnz must be even for a symmetric graph"); return SCAN_EINVAL; }
    if (n == 0 && nnz != 0) { set_error("an empty graph has nnz = 0"); return SCAN_EINVAL; }
    if ((uint64_t)nnz >= (1ull << 32)) {
        set_error("a resident graph needs nnz < 2^32 (use SCAN_LOAD_PINNED_BORROW)");
        return SCAN_EINVAL;
    }
    if (!fill && !on_dev && n > 0) {  // cheap host-side check before any copy
        if (offsets[0] != 0 || offsets[n] != nnz) {
            set_error("offsets[0] must be 0 and offsets[n] must equal nnz");
            return SCAN_EINVAL;
        }
    }
    SCAN_CUDA(cudaSetDevice(ctx->device));
    scan_graph *g = new scan_graph();
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    auto fail = [&](scan_status s) {
        graph_release(g);
        delete g;
        return s;
    };
    const size_t N1 = (size_t)n + 1, E = (size_t)(nnz > 0 ? nnz : 1), M = (size_t)(g->m > 0 ? g->m : 1);
    struct { DevBuf *b; size_t bytes; } plan[] = {
        {&g->off, 8 * N1}, {&g->adj, 4 * E}, {&g->src, 4 * E}, {&g->rev, 4 * E}, {&g->deg, 4 * N1},
        {&g->oe, 4 * M}, {&g->simo, (M + 15) & ~(size_t)15}, {&g->nsim, 4 * N1}, {&g->hst, 4 * N1},
        {&g->mslots, 8}, {&g->core, N1}, {&g->cid, 4 * N1}, {&g->parent, 4 * N1},
        {&g->label, N1}, {&g->cnt, 4 * N1}, {&g->cnt_off, 8 * N1}, {&g->ucnt, 4 * N1}, {&g->pair_off, 8 * N1},
        {&g->raw, 4 * E}, {&g->pairs, 8 * E}, {&g->npairs, 8}, {&g->err, 4}};
    for (auto &p : plan) {
        scan_status s = dev_alloc(ctx, *p.b, p.bytes);
        if (s != SCAN_OK) return fail(s);
    }
    cudaError_t e = cudaMallocHost(&g->h_npairs, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_err, sizeof(uint32_t));
    if (e != cudaSuccess) return fail(cuda_fail(e, "pinned staging"));
    if (fill) {
        const scan_status fs = fill(g);
        if (fs != SCAN_OK) return fail(fs);
    } else {
        const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = n > 0 ? cudaMemcpyAsync(g->off.ptr, offsets, 8 * N1, kind, ctx->stream)
                  : cudaMemsetAsync(g->off.ptr, 0, 8, ctx->stream);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(g->adj.ptr, adj, 4 * (size_t)nnz, kind, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g->err.ptr, 0, 4, ctx->stream);
    // the flags are read 16 at a time: the padding after the last edge stays zero
    if (e == cudaSuccess) e = cudaMemsetAsync(g->simo.ptr, 0, g->simo.bytes, ctx->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "graph upload"));
    scan_status s = graph_prepare(g);
    if (s != SCAN_OK) return fail(s);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "graph prepare"));
    *out = g;
    return SCAN_OK;
}

void graph_destroy(Graph *g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    if (g->part) part_release(g);
    graph_release(g);
    delete static_cast<scan_graph *>(g);
}

// Pinned host blocks for query results and staging, reused from one use to
// the next: page-locking and unlocking memory costs far more than the copies
// into it. Blocks are sized in powers of two; up to kPoolCap bytes of free
// blocks are kept (the rest is released); the pool lives until the process
// exits.
namespace {
std::mutex g_pool_mu;
std::multimap<size_t, void *> g_pool;
size_t g_pool_bytes = 0;
constexpr size_t kPoolCap = size_t(2) << 30;

size_t pool_size(size_t bytes) {
    size_t s = 4096;
    while (s < bytes) s <<= 1;
    return s;
}
}  // namespace

void *pinned_get(size_t bytes, size_t *cap) {
    const size_t sz = pool_size(bytes);
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        auto it = g_pool.find(sz);
        if (it != g_pool.end()) {
            void *p = it->second;
            g_pool.erase(it);
            g_pool_bytes -= sz;
            *cap = sz;
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *cap = sz;
    return p;
}

void pinned_put(void *p, size_t cap) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (g_pool_bytes + cap <= kPoolCap) {
            g_pool.emplace(cap, p);
            g_pool_bytes += cap;
            return;
        }
    }
    cudaFreeHost(p);
}

scan_result *result_new(int32_t n, int64_t k, bool pinned) {
    scan_result *r = new scan_result();
    r->n = n;
    r->k = k;
    r->pinned = pinned;
    const size_t bn = (size_t)n + 1, bk = 8 * (size_t)k + 8;
    if (pinned) {
        r->core = (uint8_t *)pinned_get(bn, &r->cap[0]);
        r->cid = (int32_t *)pinned_get(4 * bn, &r->cap[1]);
        r->label = (uint8_t *)pinned_get(bn, &r->cap[2]);
        r->pairs = (int32_t *)pinned_get(bk, &r->cap[3]);
        if (!r->core || !r->cid || !r->label || !r->pairs) {
            scan_result_free(r);
            return nullptr;
        }
    } else {
        r->core = (uint8_t *)malloc(bn);
        r->cid = (int32_t *)malloc(4 * bn);
        r->label = (uint8_t *)malloc(bn);
        r->pairs = (int32_t *)malloc(bk);
        if (!r->core || !r->cid || !r->label || !r->pairs) {
            scan_result_free(r);
            return nullptr;
        }
    }
    return r;
}

bool result_set_pairs(scan_result *r, int64_t k) {
    const size_t bk = 8 * (size_t)k + 8;
    if (r->pinned) {
        if (bk > r->cap[3]) {
            pinned_put(r->pairs, r->cap[3]);
            r->pairs = (int32_t *)pinned_get(bk, &r->cap[3]);
        }
    } else {
        void *p = realloc(r->pairs, bk);
        if (p) r->pairs = (int32_t *)p;
        else return false;
    }
    if (!r->pairs) return false;
    r->k = k;
    return true;
}

}  // namespace scan

extern "C" {

scan_status scan_graph_load(scan_ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                            uint32_t flags, scan_graph **out) {
    ABI_GUARD_BEGIN
    if (!ctx || !out) { set_error("ctx or out is NULL"); return SCAN_EINVAL; }
    *out = nullptr;
    Graph *g = nullptr;
    if (flags & SCAN_LOAD_PINNED_BORROW) {
        if (flags & SCAN_LOAD_DEVICE_PTRS) { set_error("a partitioned graph takes host arrays"); return SCAN_EINVAL; }
        SCAN_TRY(part_create(ctx, n, offsets, adj, nnz, &g, 0));
    } else {
        SCAN_TRY(graph_create(ctx, n, offsets, adj, nnz, (flags & SCAN_LOAD_DEVICE_PTRS) != 0, &g));
    }
    *out = static_cast<scan_graph *>(g);
    return SCAN_OK;
    ABI_GUARD_END
}

scan_status scan_graph_load_partitioned(scan_ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj,
                                        int64_t nnz, int64_t block_slots, scan_graph **out) {
    ABI_GUARD_BEGIN
    if (!ctx || !out) { set_error("ctx or out is NULL"); return SCAN_EINVAL; }
    *out = nullptr;
    if (block_slots < 0) { set_error("block_slots must be >= 0"); return SCAN_EINVAL; }
    Graph *g = nullptr;
    SCAN_TRY(part_create(ctx, n, offsets, adj, nnz, &g, block_slots));
    *out = static_cast<scan_graph *>(g);
    return SCAN_OK;
    ABI_GUARD_END
}

int32_t scan_graph_blocks(const scan_graph *g) {
    return g && g->part ? part_block_count(g) : 0;
}

uint64_t scan_graph_transfer_bytes(const scan_graph *g) { return g && g->part ? part_transfer_bytes(g) : 0; }

// The checks of a host CSR that the planners need: sizes, offsets, ids in range.
static scan_status check_host_csr(int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz) {
    if (n < 0 || nnz < 0 || (n > 0 && !offsets) || (nnz > 0 && !adj)) {
        set_error("bad sizes or NULL arrays");
        return SCAN_EINVAL;
    }
    if (n > 0 && (offsets[0] != 0 || offsets[n] != nnz)) {
        set_error("offsets[0] must be 0 and offsets[n] must equal nnz");
        return SCAN_EINVAL;
    }
    for (int32_t v = 0; v < n; ++v)
        if (offsets[v + 1] < offsets[v]) {
            set_error("invalid CSR offsets at index " + std::to_string(v + 1));
            return SCAN_EINVAL;
        }
    for (int64_t s = 0; s < nnz; ++s)
        if (adj[s] < 0 || adj[s] >= n) {
            set_error("id out of range at slot " + std::to_string(s));
            return SCAN_EINVAL;
        }
    return SCAN_OK;
}

scan_status scan_plan_edge_extended(int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                                    uint64_t device_bytes, int64_t *subgraphs, uint64_t *bytes) {
    ABI_GUARD_BEGIN
    if (!subgraphs || !bytes) {
        set_error("NULL output");
        return SCAN_EINVAL;
    }
    SCAN_TRY(check_host_csr(n, offsets, adj, nnz));
    return plan_edge_extended(n, offsets, adj, nnz, device_bytes, subgraphs, bytes);
    ABI_GUARD_END
}

scan_status scan_plan_triangle_blocks(int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                                      uint64_t device_bytes, int32_t *blocks, int64_t *pairs, uint64_t *bytes) {
    ABI_GUARD_BEGIN
    if (!blocks || !pairs || !bytes) {
        set_error("NULL output");
        return SCAN_EINVAL;
    }
    SCAN_TRY(check_host_csr(n, offsets, adj, nnz));
    return plan_triangle_blocks(n, offsets, adj, nnz, device_bytes, blocks, pairs, bytes);
    ABI_GUARD_END
}

scan_status scan_graph_set_zero_copy(scan_graph *g, int32_t enable) {
    ABI_GUARD_BEGIN
    if (!g) { set_error("graph is NULL"); return SCAN_EINVAL; }
    if (!g->part) { set_error("only a partitioned graph streams its CSR"); return SCAN_EINVAL; }
    return part_set_zero_copy(g, enable != 0);
    ABI_GUARD_END
}

void scan_graph_free(scan_graph *g) { graph_destroy(g); }

int32_t scan_graph_n(const scan_graph *g) { return g ? g->n : 0; }
int64_t scan_graph_nnz(const scan_graph *g) { return g ? g->nnz : 0; }

uint64_t scan_graph_device_bytes(const scan_graph *g) {
    if (!g) return 0;
    uint64_t s = 0;
    const_cast<scan_graph *>(g)->for_each_buf([&s](DevBuf &b) { s += b.bytes; });
    return s;
}

scan_status scan_graph_drop_cache(scan_graph *g) {
    if (!g) { set_error("graph is NULL"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(g->ctx->device));
    SCAN_CUDA(cudaStreamSynchronize(g->ctx->stream));
    query_graph_drop(g);
    cache_free(g);
    return SCAN_OK;
}

int32_t scan_graph_has_cache(const scan_graph *g) { return g && g->cache_valid ? 1 : 0; }

scan_status scan_graph_set_strategy(scan_graph *g, int32_t strategy) {
    if (!g) { set_error("graph is NULL"); return SCAN_EINVAL; }
    if (g->part) { set_error("not available for a partitioned graph"); return SCAN_EINVAL; }
    if (strategy != SCAN_STRATEGY_FORWARD && strategy != SCAN_STRATEGY_OWNER && strategy != SCAN_STRATEGY_BSEARCH &&
        strategy != SCAN_STRATEGY_FORWARD_LEAN && strategy != SCAN_STRATEGY_PROGRESSIVE) {
        set_error("unknown strategy " + std::to_string(strategy));
        return SCAN_EINVAL;
    }
    if (g->strategy != strategy) query_graph_drop(g);
    g->strategy = strategy;
    return SCAN_OK;
}

int32_t scan_graph_strategy(const scan_graph *g) { return g ? g->strategy : -1; }

scan_status scan_graph_copy_counts(scan_graph *g, int32_t *out) {
    if (!g || !out) { set_error("graph or out is NULL"); return SCAN_EINVAL; }
    if (g->part || !g->cache_valid) { set_error("graph has no common-count cache"); return SCAN_EINVAL; }
    SCAN_CUDA(cudaSetDevice(g->ctx->device));
    if (g->nnz > 0) {
        // the cache is kept per oriented edge; the border scratch receives it per slot
        SCAN_TRY(cache_to_slots(g, (int32_t *)g->raw.ptr));
        SCAN_CUDA(cudaMemcpyAsync(out, g->raw.ptr, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost,
                                  g->ctx->stream));
    }
    SCAN_CUDA(cudaStreamSynchronize(g->ctx->stream));
    return SCAN_OK;
}

scan_status scan_query_device(scan_graph *g, const scan_params *params, uint32_t mode, const scan_device_out *o) {
    ABI_GUARD_BEGIN
    if (!g || !o) { set_error("graph or out is NULL"); return SCAN_EINVAL; }
    SCAN_TRY(check_params(params));
    if (g->part) { set_error("a partitioned graph answers through scan_query / scan_query_ex"); return SCAN_EINVAL; }
    if (g->n > 0 && (!o->core || !o->cid || !o->label)) { set_error("NULL output array"); return SCAN_EINVAL; }
    if (!o->npairs || (o->pairs_cap > 0 && !o->pairs) || o->pairs_cap < 0) {
        set_error("bad pairs output");
        return SCAN_EINVAL;
    }
    SCAN_CUDA(cudaSetDevice(g->ctx->device));
    return query_pipeline(g, uniform_params(*params), mode, o->core, o->cid, o->label, o->pairs, o->pairs_cap, o->npairs);
    ABI_GUARD_END
}

scan_status scan_query_ex(scan_graph *g, const scan_params *params, uint32_t mode, scan_result **out) {
    ABI_GUARD_BEGIN
    if (!g || !out) { set_error("graph or out is NULL"); return SCAN_EINVAL; }
    *out = nullptr;
    SCAN_TRY(check_params(params));
    Ctx *c = g->ctx;
    SCAN_CUDA(cudaSetDevice(c->device));
    if (g->part) return part_query(g, *params, out);  // every mode is a full recompute out of core
    auto *core = (uint8_t *)g->core.ptr;
    auto *cid = (int32_t *)g->cid.ptr;
    auto *label = (uint8_t *)g->label.ptr;
    auto *pairs = (int32_t *)g->pairs.ptr;
    auto *np = (int64_t *)g->npairs.ptr;
    SCAN_TRY(query_pipeline(g, uniform_params(*params), mode, core, cid, label, pairs, g->nnz, np));
    SCAN_CUDA(cudaMemcpyAsync(g->h_npairs, np, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    SCAN_TRY(take_device_error(g));  // synchronises
    const size_t n = (size_t)g->n, k = (size_t)*g->h_npairs;
    scan_result *r = result_new(g->n, (int64_t)k, true);
    if (!r) { set_error("pinned result allocation failed"); return SCAN_ENOMEM; }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(r->core, core, n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(r->cid, cid, 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(r->label, label, n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && k) e = cudaMemcpyAsync(r->pairs, pairs, 8 * k, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        scan_result_free(r);
        return cuda_fail(e, "result download");
    }
    *out = r;
    return SCAN_OK;
    ABI_GUARD_END
}

scan_status scan_query(scan_graph *g, uint32_t eps_num, uint32_t eps_den, uint32_t mu, scan_result **out) {
    scan_params p{eps_num, eps_den, mu};
    return scan_query_ex(g, &p, SCAN_Q_AUTO, out);
}

int32_t scan_result_n(const scan_result *r) { return r ? r->n : 0; }
const uint8_t *scan_result_core(const scan_result *r) { return r ? r->core : nullptr; }
const int32_t *scan_result_cluster(const scan_result *r) { return r ? r->cid : nullptr; }
const uint8_t *scan_result_label(const scan_result *r) { return r ? r->label : nullptr; }
int64_t scan_result_border_count(const scan_result *r) { return r ? r->k : 0; }
const int32_t *scan_result_border_pairs(const scan_result *r) { return r ? r->pairs : nullptr; }

void scan_result_free(scan_result *r) {
    if (!r) return;
    void *bufs[] = {r->core, r->cid, r->label, r->pairs};
    for (int i = 0; i < 4; ++i) {
        if (!bufs[i]) continue;
        if (r->pinned) pinned_put(bufs[i], r->cap[i]);
        else free(bufs[i]);
    }
    delete r;
}

}  // extern "C"

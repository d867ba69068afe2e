// batch.cu -- many graphs clustered together.
//
// A batch stores its k graphs as one resident disjoint union (vertex ids and
// slots shifted by per-graph bases) plus a graph index per vertex. SCAN
// never joins vertices of different graphs -- no edge crosses them -- so one
// query over the union, with each vertex reading its own graph's (eps, mu)
// through the graph index, answers all k queries at once: every pipeline
// stage is a single launch over all graphs, and the owner schedule of the
// union is the work queue over (graph, owner, slot range) items. Results are
// split per graph on the host, with ids shifted back.
#include <algorithm>
#include <cstring>
#include <atomic>
#include <thread>
#include <vector>

#include "scan_internal.cuh"

using namespace scan;

struct scan_batch {
    Ctx *ctx = nullptr;
    Graph *g = nullptr;  // the union
    int32_t k = 0;
    std::vector<int64_t> vbase, ebase;  // k+1 each
    DevBuf gid, gpp, gqq, gmu;
    uint64_t *h_pp = nullptr, *h_qq = nullptr;  // pinned parameter staging
    uint32_t *h_mu = nullptr;
    // pinned download staging for the union result
    uint8_t *h_core = nullptr, *h_label = nullptr;
    int32_t *h_cid = nullptr, *h_pairs = nullptr;
    int64_t h_pairs_cap = 0;
    size_t cap[7] = {0, 0, 0, 0, 0, 0, 0};  // pinned pool block sizes of the seven staging arrays
    // the device query (parameter copies + pipeline), replayed as a CUDA graph
    cudaGraphExec_t exec = nullptr;
    uint64_t key = 0;
    uint64_t launches = 0;  // kernels in the captured graph
    bool graph_off = false;
};

namespace scan {
namespace {

__global__ void k_graph_index(const int64_t *__restrict__ vbase, int32_t k, int32_t n, int32_t *__restrict__ gid) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t lo = 0, hi = k;  // last j with vbase[j] <= v
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (vbase[mid] <= v) lo = mid;
        else hi = mid;
    }
    gid[v] = lo;
}

// Union assembly: each graph's rows were copied into place with local ids
// and offsets; shift them by the graph's vertex and slot bases.
__global__ void k_union_offsets(int64_t *__restrict__ off, int32_t n, const int32_t *__restrict__ gid,
                                const int64_t *__restrict__ ebase) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) off[v] += ebase[gid[v]];
}

// per slot: its graph j (the last with ebase[j] <= s), the id range check
// against that graph's n, and the shift by its vertex base
__global__ void k_union_ids(int32_t *__restrict__ adj, int64_t nnz, const int64_t *__restrict__ vbase,
                            const int64_t *__restrict__ ebase, int32_t k, unsigned long long *bad) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = k;  // ebase[lo] <= s < ebase[hi]
        for (int it = 0; it < 40 && hi - lo > 1; ++it) {
            const int32_t mid = (lo + hi) >> 1;
            if (ebase[mid] <= s) lo = mid;
            else hi = mid;
        }
        const int32_t a = adj[s];
        if (a < 0 || (int64_t)a >= vbase[lo + 1] - vbase[lo]) atomicMin(bad, (unsigned long long)s);
        else adj[s] = a + (int32_t)vbase[lo];
    }
}

// Host-to-device upload of many pageable arrays that are contiguous on the
// device: packed into pinned blocks by a few host threads (two blocks, so the
// next is packed while the previous one is copied), one copy per block.
struct Piece {
    const char *src;
    size_t bytes;
};

scan_status upload_concat(Ctx *ctx, const std::vector<Piece> &pieces, char *dst) {
    constexpr size_t kBlock = size_t(128) << 20;
    std::vector<size_t> start(pieces.size() + 1, 0);
    for (size_t i = 0; i < pieces.size(); ++i) start[i + 1] = start[i] + pieces[i].bytes;
    const size_t total = start.back();
    if (total == 0) return SCAN_OK;
    char *buf[2] = {nullptr, nullptr};
    size_t cap[2] = {0, 0};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    scan_status st = SCAN_OK;
    for (int i = 0; i < 2 && st == SCAN_OK; ++i) {
        buf[i] = (char *)pinned_get(std::min(kBlock, total), &cap[i]);
        if (!buf[i]) st = SCAN_ENOMEM;
        else if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) st = SCAN_ENOMEM;
    }
    const int nt = (int)std::min<unsigned>(8, std::max(1u, std::thread::hardware_concurrency()));
    // copies [a, b) of the concatenation into out
    auto pack = [&](size_t a, size_t b, char *out) {
        size_t i = (size_t)(std::upper_bound(start.begin(), start.end(), a) - start.begin()) - 1;
        for (size_t pos = a; pos < b; ++i) {
            const size_t lo = pos - start[i], n = std::min(start[i + 1], b) - pos;
            if (n) memcpy(out + (pos - a), pieces[i].src + lo, n);
            pos += n;
        }
    };
    int cur = 0;
    for (size_t off = 0; off < total && st == SCAN_OK; off += kBlock, cur ^= 1) {
        const size_t len = std::min(kBlock, total - off);
        if (cudaEventSynchronize(ev[cur]) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "batch upload"); break; }
        std::vector<std::thread> pool;
        const size_t share = (len + nt - 1) / nt;
        for (int t = 1; t < nt; ++t) {
            const size_t a = std::min(len, share * t), b2 = std::min(len, share * (t + 1));
            if (a < b2) pool.emplace_back(pack, off + a, off + b2, buf[cur] + a);
        }
        pack(off, off + std::min(len, share), buf[cur]);
        for (auto &th : pool) th.join();
        cudaError_t e = cudaMemcpyAsync(dst + off, buf[cur], len, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[cur], ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch upload");
    }
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < 2; ++i) {
        if (ev[i]) cudaEventDestroy(ev[i]);
        pinned_put(buf[i], cap[i]);
    }
    if (st == SCAN_ENOMEM) set_error("pinned staging allocation failed");
    return st;
}

void batch_release(scan_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->g) graph_destroy(b->g);
    b->g = nullptr;
    DevBuf *bufs[] = {&b->gid, &b->gpp, &b->gqq, &b->gmu};
    for (DevBuf *d : bufs) dev_free(b->ctx, *d);
    void *pin[] = {b->h_pp, b->h_qq, b->h_mu, b->h_core, b->h_label, b->h_cid, b->h_pairs};
    for (int i = 0; i < 7; ++i) pinned_put(pin[i], b->cap[i]);
    delete b;
}

scan_status batch_query_to_device(scan_batch *b, const scan_params *params, uint32_t mode, uint8_t *core,
                                  int32_t *cid, uint8_t *label, int32_t *pairs, int64_t pairs_cap, int64_t *npairs) {
    Ctx *c = b->ctx;
    for (int32_t j = 0; j < b->k; ++j) SCAN_TRY(check_params(params + j));
    // a replay still in flight may not have read the staged parameters yet
    if (b->exec) SCAN_CUDA(cudaStreamSynchronize(c->stream));
    for (int32_t j = 0; j < b->k; ++j) {
        b->h_pp[j] = (uint64_t)params[j].eps_num * params[j].eps_num;
        b->h_qq[j] = (uint64_t)params[j].eps_den * params[j].eps_den;
        b->h_mu[j] = params[j].mu;
    }
    QParams qp;
    qp.gid = (const int32_t *)b->gid.ptr;
    qp.gpp = (const uint64_t *)b->gpp.ptr;
    qp.gqq = (const uint64_t *)b->gqq.ptr;
    qp.gmu = (const uint32_t *)b->gmu.ptr;
    auto run = [&]() -> scan_status {
        SCAN_CUDA(cudaMemcpyAsync(b->gpp.ptr, b->h_pp, 8 * (size_t)b->k, cudaMemcpyHostToDevice, c->stream));
        SCAN_CUDA(cudaMemcpyAsync(b->gqq.ptr, b->h_qq, 8 * (size_t)b->k, cudaMemcpyHostToDevice, c->stream));
        SCAN_CUDA(cudaMemcpyAsync(b->gmu.ptr, b->h_mu, 4 * (size_t)b->k, cudaMemcpyHostToDevice, c->stream));
        return query_pipeline(b->g, qp, mode, core, cid, label, pairs, pairs_cap, npairs);
    };
    const bool replayable = !(mode & SCAN_Q_BUILD_CACHE) && !c->profiling && !b->graph_off && !c->loop_limit;
    const uint64_t key = replay_key(mode | (b->g->cache_valid ? 0x100u : 0u), core, cid, label, pairs, pairs_cap,
                                    npairs);
    if (replayable && b->exec && b->key == key) {
        SCAN_CUDA(cudaGraphLaunch(b->exec, c->stream));
        c->launches += b->launches;
        return SCAN_OK;
    }
    SCAN_TRY(run());
    if (!replayable) return SCAN_OK;
    // capture the same sequence for the next query with these buffers
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGraph_t graph = nullptr;
    const uint64_t launches0 = c->launches;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    scan_status s = SCAN_OK;
    if (e == cudaSuccess) {
        s = run();
        const cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && s == SCAN_OK && graph) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || s != SCAN_OK || !b->exec) {
        cudaGetLastError();
        c->launches = launches0;
        b->exec = nullptr;
        b->graph_off = true;  // not capturable here: run directly from now on
        set_error("");
        return SCAN_OK;
    }
    b->key = key;
    b->launches = c->launches - launches0;  // capture launched nothing; these run at each replay
    c->launches = launches0;
    return SCAN_OK;
}

}  // namespace

scan_status batch_create(Ctx *ctx, int32_t k, const int32_t *ns, const int64_t *const *offsets,
                         const int32_t *const *adjs, scan_batch **out) {
    *out = nullptr;
    if (k < 1 || !ns || !offsets || !adjs) {
        set_error("a batch needs k >= 1 graphs");
        return SCAN_EINVAL;
    }
    scan_batch *b = new scan_batch();
    b->ctx = ctx;
    b->k = k;
    b->vbase.assign((size_t)k + 1, 0);
    b->ebase.assign((size_t)k + 1, 0);
    auto fail = [&](scan_status s) {
        batch_release(b);
        return s;
    };
    for (int32_t j = 0; j < k; ++j) {
        if (ns[j] < 0 || (ns[j] > 0 && (!offsets[j] || offsets[j][0] != 0))) {
            set_error("graph " + std::to_string(j) + " of the batch has bad offsets");
            return fail(SCAN_EINVAL);
        }
        const int64_t nnz = ns[j] > 0 ? offsets[j][ns[j]] : 0;
        if (nnz > 0 && !adjs[j]) {
            set_error("graph " + std::to_string(j) + " of the batch has no adjacency");
            return fail(SCAN_EINVAL);
        }
        b->vbase[j + 1] = b->vbase[j] + ns[j];
        b->ebase[j + 1] = b->ebase[j] + nnz;
    }
    const int64_t n = b->vbase[k], nnz = b->ebase[k];
    if (n >= (1ll << 31) - 1 || (uint64_t)nnz >= (1ull << 32)) {
        set_error("the batch union exceeds 2^31 vertices or 2^32 slots");
        return fail(SCAN_EINVAL);
    }
    // the union CSR, assembled on the device: every graph's arrays are copied
    // into place as they are, then ids and offsets are shifted by the graph's
    // bases (ids checked against the graph's own n there)
    DevBuf dvb, deb, dbad;
    scan_status s = dev_alloc(ctx, dvb, 8 * ((size_t)k + 1));
    if (s == SCAN_OK) s = dev_alloc(ctx, deb, 8 * ((size_t)k + 1));
    if (s == SCAN_OK) s = dev_alloc(ctx, dbad, sizeof(unsigned long long));
    if (s == SCAN_OK) s = dev_alloc(ctx, b->gid, 4 * ((size_t)n + 1));
    if (s == SCAN_OK) s = dev_alloc(ctx, b->gpp, 8 * (size_t)k);
    if (s == SCAN_OK) s = dev_alloc(ctx, b->gqq, 8 * (size_t)k);
    if (s == SCAN_OK) s = dev_alloc(ctx, b->gmu, 4 * (size_t)k);
    auto free_tmp = [&]() {
        dev_free(ctx, dvb);
        dev_free(ctx, deb);
        dev_free(ctx, dbad);
    };
    if (s != SCAN_OK) {
        free_tmp();
        return fail(s);
    }
    auto fill = [&](Graph *g) -> scan_status {
        cudaStream_t st = ctx->stream;
        auto *doff = (int64_t *)g->off.ptr;
        auto *dadj = (int32_t *)g->adj.ptr;
        const unsigned long long none = ~0ull;
        cudaError_t e = cudaMemcpyAsync(dvb.ptr, b->vbase.data(), 8 * ((size_t)k + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(deb.ptr, b->ebase.data(), 8 * ((size_t)k + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dbad.ptr, &none, sizeof(none), cudaMemcpyHostToDevice, st);
        // the graphs' offset arrays (without their last entry) and adjacency
        // arrays, concatenated, are exactly the union's before the shift
        if (e == cudaSuccess) {
            std::vector<Piece> offp, adjp;
            for (int32_t j = 0; j < k; ++j) {
                offp.push_back({(const char *)offsets[j], 8 * (size_t)ns[j]});
                adjp.push_back({(const char *)adjs[j], 4 * (size_t)(b->ebase[j + 1] - b->ebase[j])});
            }
            const scan_status us = upload_concat(ctx, offp, (char *)doff);
            if (us != SCAN_OK) return us;
            const scan_status ua = upload_concat(ctx, adjp, (char *)dadj);
            if (ua != SCAN_OK) return ua;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(doff + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch upload");
        if (n > 0) {
            k_graph_index<<<grid_for(n, 256), 256, 0, st>>>((const int64_t *)dvb.ptr, k, (int32_t)n,
                                                            (int32_t *)b->gid.ptr);
            k_union_offsets<<<grid_for(n, 256), 256, 0, st>>>(doff, (int32_t)n, (const int32_t *)b->gid.ptr,
                                                              (const int64_t *)deb.ptr);
            ctx->launches += 2;
        }
        if (nnz > 0) {
            k_union_ids<<<grid_for(nnz, 256, ctx->num_sms * 32), 256, 0, st>>>(
                dadj, nnz, (const int64_t *)dvb.ptr, (const int64_t *)deb.ptr, k, (unsigned long long *)dbad.ptr);
            ctx->launches++;
        }
        unsigned long long hbad = none;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, dbad.ptr, sizeof(hbad), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batch union");
        if (hbad != none) {
            const int32_t j = (int32_t)(std::upper_bound(b->ebase.begin(), b->ebase.end(), (int64_t)hbad) -
                                        b->ebase.begin()) - 1;
            set_error("graph " + std::to_string(j) + " of the batch: id out of range at slot " +
                      std::to_string((int64_t)hbad - b->ebase[(size_t)j]));
            return SCAN_EINVAL;
        }
        return SCAN_OK;
    };
    {
        const scan_status gs = graph_create(ctx, (int32_t)n, nullptr, nullptr, nnz, false, &b->g, fill);
        free_tmp();
        if (gs != SCAN_OK) return fail(gs);
        // a union of many small graphs holds mostly small owners: one
        // persistent launch over the work queue counts it (the autotuner may
        // still choose otherwise)
        b->g->fwd_queue = true;
    }
    // parameter and result staging from the pinned pool (reused by the next batch)
    b->h_pp = (uint64_t *)pinned_get(8 * (size_t)k, &b->cap[0]);
    b->h_qq = (uint64_t *)pinned_get(8 * (size_t)k, &b->cap[1]);
    b->h_mu = (uint32_t *)pinned_get(4 * (size_t)k, &b->cap[2]);
    b->h_core = (uint8_t *)pinned_get((size_t)n + 1, &b->cap[3]);
    b->h_label = (uint8_t *)pinned_get((size_t)n + 1, &b->cap[4]);
    b->h_cid = (int32_t *)pinned_get(4 * ((size_t)n + 1), &b->cap[5]);
    if (!b->h_pp || !b->h_qq || !b->h_mu || !b->h_core || !b->h_label || !b->h_cid) {
        set_error("pinned staging allocation failed");
        return fail(SCAN_ENOMEM);
    }
    *out = b;
    return SCAN_OK;
}

}  // namespace scan

extern "C" {

scan_status scan_batch_load(scan_ctx *ctx, int32_t k, const int32_t *n, const int64_t *const *offsets,
                            const int32_t *const *adj, uint32_t flags, scan_batch **out) {
    try {
        if (!ctx || !out) { set_error("ctx or out is NULL"); return SCAN_EINVAL; }
        *out = nullptr;
        if (flags != 0) { set_error("scan_batch_load takes host arrays only (flags must be 0)"); return SCAN_EINVAL; }
        SCAN_CUDA(cudaSetDevice(((Ctx *)ctx)->device));
        return batch_create((Ctx *)ctx, k, n, offsets, adj, out);
    } catch (...) {
        set_error("host allocation failed");
        return SCAN_ENOMEM;
    }
}

int32_t scan_batch_size(const scan_batch *b) { return b ? b->k : 0; }

scan_graph *scan_batch_union(scan_batch *b) { return b ? (scan_graph *)b->g : nullptr; }

void scan_batch_free(scan_batch *b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    batch_release(b);
}

scan_status scan_batch_query_device(scan_batch *b, const scan_params *params, uint32_t mode,
                                    const scan_device_out *o) {
    try {
        if (!b || !params || !o) { set_error("NULL argument"); return SCAN_EINVAL; }
        if (!o->npairs || (!o->core && b->g->n > 0)) { set_error("bad device outputs"); return SCAN_EINVAL; }
        SCAN_CUDA(cudaSetDevice(b->ctx->device));
        return batch_query_to_device(b, params, mode, o->core, o->cid, o->label, o->pairs, o->pairs_cap, o->npairs);
    } catch (...) {
        set_error("internal error");
        return SCAN_EINVAL;
    }
}

scan_status scan_batch_query(scan_batch *b, const scan_params *params, uint32_t mode, scan_result **outs) {
    try {
        if (!b || !params || !outs) { set_error("NULL argument"); return SCAN_EINVAL; }
        for (int32_t j = 0; j < b->k; ++j) outs[j] = nullptr;
        Ctx *c = b->ctx;
        Graph *g = b->g;
        SCAN_CUDA(cudaSetDevice(c->device));
        SCAN_TRY(batch_query_to_device(b, params, mode, (uint8_t *)g->core.ptr, (int32_t *)g->cid.ptr,
                                       (uint8_t *)g->label.ptr, (int32_t *)g->pairs.ptr, g->nnz,
                                       (int64_t *)g->npairs.ptr));
        SCAN_CUDA(cudaMemcpyAsync(g->h_npairs, g->npairs.ptr, 8, cudaMemcpyDeviceToHost, c->stream));
        SCAN_TRY(take_device_error(g));
        const int64_t kp = *g->h_npairs, n = g->n;
        if (kp > b->h_pairs_cap) {
            pinned_put(b->h_pairs, b->cap[6]);
            b->h_pairs_cap = 0;
            b->h_pairs = (int32_t *)pinned_get(8 * (size_t)kp + 8, &b->cap[6]);
            if (!b->h_pairs) {
                set_error("pinned staging allocation failed");
                return SCAN_ENOMEM;
            }
            b->h_pairs_cap = kp;
        }
        if (n > 0) {
            SCAN_CUDA(cudaMemcpyAsync(b->h_core, g->core.ptr, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
            SCAN_CUDA(cudaMemcpyAsync(b->h_cid, g->cid.ptr, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
            SCAN_CUDA(cudaMemcpyAsync(b->h_label, g->label.ptr, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
        }
        if (kp > 0)
            SCAN_CUDA(cudaMemcpyAsync(b->h_pairs, g->pairs.ptr, 8 * (size_t)kp, cudaMemcpyDeviceToHost, c->stream));
        SCAN_CUDA(cudaStreamSynchronize(c->stream));
        // split: pairs are sorted by vertex, so each graph owns a contiguous
        // run; the graphs are shared out over a few host threads
        const int32_t k = b->k;
        std::vector<int64_t> pstart((size_t)k + 1);
        for (int32_t j = 0; j <= k; ++j) {
            const int64_t vb = j < k ? b->vbase[j] : n;
            int64_t lo = 0, hi = kp;  // first pair whose vertex is >= vb
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (b->h_pairs[2 * mid] < vb) lo = mid + 1;
                else hi = mid;
            }
            pstart[(size_t)j] = lo;
        }
        std::atomic<bool> oom{false};
        auto split = [&](int32_t j0, int32_t j1) {
            for (int32_t j = j0; j < j1 && !oom.load(std::memory_order_relaxed); ++j) {
                const int64_t vb = b->vbase[j], ve = b->vbase[j + 1];
                const int64_t p0 = pstart[(size_t)j], p1 = pstart[(size_t)j + 1];
                scan_result *r = result_new((int32_t)(ve - vb), p1 - p0, false);
                if (!r) {
                    oom = true;
                    return;
                }
                for (int64_t v = vb; v < ve; ++v) {
                    r->core[v - vb] = b->h_core[v];
                    r->label[v - vb] = b->h_label[v];
                    const int32_t x = b->h_cid[v];
                    r->cid[v - vb] = x >= 0 ? x - (int32_t)vb : -1;
                }
                for (int64_t i = p0; i < p1; ++i) {
                    r->pairs[2 * (i - p0)] = b->h_pairs[2 * i] - (int32_t)vb;
                    r->pairs[2 * (i - p0) + 1] = b->h_pairs[2 * i + 1] - (int32_t)vb;
                }
                outs[j] = r;
            }
        };
        const int32_t nt = (int32_t)std::min<int64_t>({8, std::max(1u, std::thread::hardware_concurrency()), k});
        std::vector<std::thread> pool;
        for (int32_t t = 1; t < nt; ++t) pool.emplace_back(split, (int32_t)((int64_t)k * t / nt),
                                                           (int32_t)((int64_t)k * (t + 1) / nt));
        split(0, (int32_t)((int64_t)k / nt));
        for (auto &th : pool) th.join();
        if (oom) {
            for (int32_t j = 0; j < k; ++j) { scan_result_free(outs[j]); outs[j] = nullptr; }
            set_error("result allocation failed");
            return SCAN_ENOMEM;
        }
        return SCAN_OK;
    } catch (...) {
        set_error("host allocation failed");
        return SCAN_ENOMEM;
    }
}

scan_status scan_batch_query_packed(scan_batch *b, const scan_params *params, uint32_t mode, scan_result **out,
                                    int64_t *vertex_offsets, int64_t *pair_offsets) {
    try {
        if (!b || !params || !out || !vertex_offsets || !pair_offsets) {
            set_error("NULL argument");
            return SCAN_EINVAL;
        }
        *out = nullptr;
        Ctx *c = b->ctx;
        Graph *g = b->g;
        SCAN_CUDA(cudaSetDevice(c->device));
        SCAN_TRY(batch_query_to_device(b, params, mode, (uint8_t *)g->core.ptr, (int32_t *)g->cid.ptr,
                                       (uint8_t *)g->label.ptr, (int32_t *)g->pairs.ptr, g->nnz,
                                       (int64_t *)g->npairs.ptr));
        SCAN_CUDA(cudaMemcpyAsync(g->h_npairs, g->npairs.ptr, 8, cudaMemcpyDeviceToHost, c->stream));
        SCAN_TRY(take_device_error(g));
        const int64_t kp = *g->h_npairs, n = g->n;
        // the union's arrays straight into one pinned result
        scan_result *r = result_new(g->n, kp, true);
        if (!r) {
            set_error("pinned result allocation failed");
            return SCAN_ENOMEM;
        }
        cudaError_t e = cudaSuccess;
        if (n > 0) {
            e = cudaMemcpyAsync(r->core, g->core.ptr, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->cid, g->cid.ptr, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->label, g->label.ptr, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
        }
        if (e == cudaSuccess && kp > 0)
            e = cudaMemcpyAsync(r->pairs, g->pairs.ptr, 8 * (size_t)kp, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            scan_result_free(r);
            return cuda_fail(e, "batch result download");
        }
        // pairs are sorted by union vertex, so each graph owns a contiguous run
        const int32_t k = b->k;
        for (int32_t j = 0; j <= k; ++j) {
            const int64_t vb = j < k ? b->vbase[j] : n;
            int64_t lo = 0, hi = kp;  // first pair whose vertex is >= vb
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (r->pairs[2 * mid] < vb) lo = mid + 1;
                else hi = mid;
            }
            pair_offsets[j] = lo;
            vertex_offsets[j] = vb;
        }
        // union ids to each graph's own ids, the graphs shared out over a few host threads
        auto local = [&](int32_t j0, int32_t j1) {
            for (int32_t j = j0; j < j1; ++j) {
                const int32_t vb = (int32_t)b->vbase[j], ve = (int32_t)b->vbase[j + 1];
                for (int32_t v = vb; v < ve; ++v)
                    if (r->cid[v] >= 0) r->cid[v] -= vb;
                for (int64_t i = pair_offsets[j]; i < pair_offsets[j + 1]; ++i) {
                    r->pairs[2 * i] -= vb;
                    r->pairs[2 * i + 1] -= vb;
                }
            }
        };
        const int32_t nt = (int32_t)std::min<int64_t>({8, std::max(1u, std::thread::hardware_concurrency()), k});
        std::vector<std::thread> pool;
        for (int32_t t = 1; t < nt; ++t)
            pool.emplace_back(local, (int32_t)((int64_t)k * t / nt), (int32_t)((int64_t)k * (t + 1) / nt));
        local(0, (int32_t)((int64_t)k / nt));
        for (auto &th : pool) th.join();
        *out = r;
        return SCAN_OK;
    } catch (...) {
        set_error("host allocation failed");
        return SCAN_ENOMEM;
    }
}

scan_status scan_query_batch(scan_graph *const *gs, const scan_params *params, int32_t k, scan_result **outs) {
    try {
        if (!gs || !params || !outs || k < 1 || !gs[0]) { set_error("bad arguments"); return SCAN_EINVAL; }
        Ctx *c = gs[0]->ctx;
        for (int32_t j = 0; j < k; ++j) {
            if (!gs[j] || gs[j]->ctx != c) { set_error("all graphs of a batch must share one context"); return SCAN_EINVAL; }
            if (gs[j]->part) { set_error("a partitioned graph cannot join a batch"); return SCAN_EINVAL; }
        }
        SCAN_CUDA(cudaSetDevice(c->device));
        // bring every graph's CSR back to the host and build the union
        std::vector<std::vector<int64_t>> offs((size_t)k);
        std::vector<std::vector<int32_t>> adjs((size_t)k);
        std::vector<int32_t> ns((size_t)k);
        std::vector<const int64_t *> po((size_t)k);
        std::vector<const int32_t *> pa((size_t)k);
        for (int32_t j = 0; j < k; ++j) {
            Graph *g = gs[j];
            ns[j] = g->n;
            offs[j].resize((size_t)g->n + 1);
            adjs[j].resize((size_t)std::max<int64_t>(g->nnz, 1));
            SCAN_CUDA(cudaMemcpyAsync(offs[j].data(), g->off.ptr, 8 * ((size_t)g->n + 1), cudaMemcpyDeviceToHost,
                                      c->stream));
            if (g->nnz > 0)
                SCAN_CUDA(cudaMemcpyAsync(adjs[j].data(), g->adj.ptr, 4 * (size_t)g->nnz, cudaMemcpyDeviceToHost,
                                          c->stream));
            po[j] = offs[j].data();
            pa[j] = adjs[j].data();
        }
        SCAN_CUDA(cudaStreamSynchronize(c->stream));
        scan_batch *b = nullptr;
        SCAN_TRY(batch_create(c, k, ns.data(), po.data(), pa.data(), &b));
        scan_status s = scan_batch_query(b, params, SCAN_Q_RECOMPUTE, outs);
        scan_batch_free(b);
        return s;
    } catch (...) {
        set_error("host allocation failed");
        return SCAN_ENOMEM;
    }
}

}  // extern "C"

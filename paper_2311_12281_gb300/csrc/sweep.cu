// Parameter sweep over one resident graph: k (eps, mu) queries answered in
// order, each result's copy to the host overlapped with the next query.
//
// Choosing eps and mu means clustering the same graph many times (the
// parameter study of Section 6); every answer is the one a single query gives
// (Definitions 2.1-2.6). The queries alternate between two device output
// sets: while query j writes one set on the context's stream, the copies of
// query j-1's result leave the other set on the graph's sweep stream, and a
// set is written again only after its copies have finished.
#include "scan_internal.cuh"

namespace scan {

void sweep_release(Graph *g) {
    if (g->sweep_stream) {
        cudaStreamSynchronize(g->sweep_stream);
        cudaStreamDestroy(g->sweep_stream);
    }
    g->sweep_stream = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (g->sweep_done[i]) cudaEventDestroy(g->sweep_done[i]);
        if (g->sweep_copied[i]) cudaEventDestroy(g->sweep_copied[i]);
        g->sweep_done[i] = nullptr;
        g->sweep_copied[i] = nullptr;
    }
    if (g->h_sweep_np) cudaFreeHost(g->h_sweep_np);
    g->h_sweep_np = nullptr;
}

namespace {

struct OutSet {
    uint8_t *core;
    int32_t *cid;
    uint8_t *label;
    int32_t *pairs;
    int64_t *np;
};

OutSet out_set(Graph *g, int s) {
    if (s == 0)
        return {(uint8_t *)g->core.ptr, (int32_t *)g->cid.ptr, (uint8_t *)g->label.ptr, (int32_t *)g->pairs.ptr,
                (int64_t *)g->npairs.ptr};
    return {(uint8_t *)g->core2.ptr, (int32_t *)g->cid2.ptr, (uint8_t *)g->label2.ptr, (int32_t *)g->pairs2.ptr,
            (int64_t *)g->npairs2.ptr};
}

// The second output set (6(n+1) + 8 nnz bytes, kept with the graph), the copy
// stream and the events. *ok is false when the set does not fit the device or
// the budget: the sweep then answers one query at a time.
scan_status sweep_setup(Graph *g, bool *ok) {
    *ok = false;
    Ctx *c = g->ctx;
    if (!g->core2.ptr) {
        const size_t N1 = (size_t)g->n + 1, E = (size_t)(g->nnz > 0 ? g->nnz : 1);
        struct {
            DevBuf *b;
            size_t bytes;
        } plan[] = {{&g->core2, N1}, {&g->cid2, 4 * N1}, {&g->label2, N1}, {&g->pairs2, 8 * E}, {&g->npairs2, 8}};
        for (auto &p : plan) {
            if (dev_alloc(c, *p.b, p.bytes) != SCAN_OK) {
                for (auto &q : plan) dev_free(c, *q.b);
                set_error("");
                return SCAN_OK;
            }
        }
    }
    if (!g->sweep_stream) SCAN_CUDA(cudaStreamCreateWithFlags(&g->sweep_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        if (!g->sweep_done[i]) SCAN_CUDA(cudaEventCreateWithFlags(&g->sweep_done[i], cudaEventDisableTiming));
        if (!g->sweep_copied[i]) SCAN_CUDA(cudaEventCreateWithFlags(&g->sweep_copied[i], cudaEventDisableTiming));
    }
    if (!g->h_sweep_np) SCAN_CUDA(cudaMallocHost(&g->h_sweep_np, 2 * sizeof(int64_t)));
    *ok = true;
    return SCAN_OK;
}

// Once set s's query has finished: a pinned result of the right size, and
// its copies enqueued on the sweep stream (recorded by sweep_copied[s]).
scan_status sweep_collect(Graph *g, int s, scan_result **out) {
    SCAN_CUDA(cudaEventSynchronize(g->sweep_done[s]));
    const OutSet o = out_set(g, s);
    const size_t n = (size_t)g->n, k = (size_t)g->h_sweep_np[s];
    scan_result *r = result_new(g->n, (int64_t)k, true);
    if (!r) {
        set_error("pinned result allocation failed");
        return SCAN_ENOMEM;
    }
    *out = r;
    cudaStream_t cs = g->sweep_stream;
    SCAN_CUDA(cudaStreamWaitEvent(cs, g->sweep_done[s], 0));
    if (n) {
        SCAN_CUDA(cudaMemcpyAsync(r->core, o.core, n, cudaMemcpyDeviceToHost, cs));
        SCAN_CUDA(cudaMemcpyAsync(r->cid, o.cid, 4 * n, cudaMemcpyDeviceToHost, cs));
        SCAN_CUDA(cudaMemcpyAsync(r->label, o.label, n, cudaMemcpyDeviceToHost, cs));
    }
    if (k) SCAN_CUDA(cudaMemcpyAsync(r->pairs, o.pairs, 8 * k, cudaMemcpyDeviceToHost, cs));
    SCAN_CUDA(cudaEventRecord(g->sweep_copied[s], cs));
    return SCAN_OK;
}

scan_status sweep_run(Graph *g, const scan_params *params, int32_t k, uint32_t mode, scan_result **outs) {
    Ctx *c = g->ctx;
    bool ok = false;
    SCAN_TRY(sweep_setup(g, &ok));
    if (!ok) {
        for (int32_t j = 0; j < k; ++j)
            SCAN_TRY(scan_query_ex(static_cast<scan_graph *>(g), &params[j], mode, &outs[j]));
        return SCAN_OK;
    }
    cudaStream_t st = c->stream;
    for (int32_t j = 0; j < k; ++j) {
        const int s = j & 1;
        // set s held query j-2's result: its copies must have left it
        if (j >= 2) SCAN_CUDA(cudaStreamWaitEvent(st, g->sweep_copied[s], 0));
        const OutSet o = out_set(g, s);
        SCAN_TRY(query_pipeline(g, uniform_params(params[j]), mode, o.core, o.cid, o.label, o.pairs, g->nnz, o.np));
        SCAN_CUDA(cudaMemcpyAsync(g->h_sweep_np + s, o.np, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SCAN_CUDA(cudaEventRecord(g->sweep_done[s], st));
        // query j is queued: collect query j-1 while it runs
        if (j >= 1) SCAN_TRY(sweep_collect(g, s ^ 1, &outs[j - 1]));
    }
    SCAN_TRY(sweep_collect(g, (k - 1) & 1, &outs[k - 1]));
    SCAN_CUDA(cudaStreamSynchronize(g->sweep_stream));
    return take_device_error(g);  // a bounded loop that gave up in any query fails the sweep
}

}  // namespace
}  // namespace scan

using namespace scan;

extern "C" {

scan_status scan_query_sweep(scan_graph *g, const scan_params *params, int32_t k, uint32_t mode,
                             scan_result **outs) {
    try {
        if (!g || !params || !outs || k < 1) {
            set_error("bad arguments");
            return SCAN_EINVAL;
        }
        for (int32_t j = 0; j < k; ++j) outs[j] = nullptr;
        for (int32_t j = 0; j < k; ++j) SCAN_TRY(check_params(&params[j]));
        SCAN_CUDA(cudaSetDevice(g->ctx->device));
        scan_status s = SCAN_OK;
        if (g->part || k == 1) {
            for (int32_t j = 0; j < k && s == SCAN_OK; ++j) s = scan_query_ex(g, &params[j], mode, &outs[j]);
        } else {
            s = sweep_run(g, params, k, mode, outs);
        }
        if (s != SCAN_OK) {
            // no copy may still be writing into a result that is freed
            if (g->sweep_stream) cudaStreamSynchronize(g->sweep_stream);
            cudaStreamSynchronize(g->ctx->stream);
            for (int32_t j = 0; j < k; ++j) {
                scan_result_free(outs[j]);
                outs[j] = nullptr;
            }
        }
        return s;
    } catch (...) {
        set_error("host allocation failed");
        return SCAN_ENOMEM;
    }
}

}  // extern "C"

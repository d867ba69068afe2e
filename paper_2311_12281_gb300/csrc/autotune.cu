// autotune.cu -- choose the similarity kernel family, the forward
// schedule's work sizes and its launch form (one launch per item class, or
// one persistent launch over a work queue) by timing them on the graph, and
// remember the choice per graph shape in a plain text file (one line per
// choice: "fwd2", key, strategy, warp-owner work bound, CTA item work, queue,
// milliseconds).
//
// A graph's shape key is (floor log2 n, floor log2 nnz, floor log2 max
// degree): graphs with the same key reuse a stored choice without timing.
#include <cstdio>
#include <string>
#include <vector>

#include "scan_internal.cuh"

namespace scan {
namespace {

__global__ void k_max_deg(const int32_t *__restrict__ deg, int32_t n, int *out) {
    int best = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        best = max(best, deg[v]);
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

struct Choice {
    int strategy = SCAN_STRATEGY_FORWARD;
    int64_t small_work = 1 << 15;
    int64_t item_work = 1 << 20;
    int queue = 0;
    double ms = 0;
};

int ilog2(uint64_t x) { return x ? 63 - __builtin_clzll(x) : -1; }

void reset_forward_schedule(Graph *g) {
    Ctx *c = g->ctx;
    dev_free(c, g->fwd_owners);
    dev_free(c, g->fwd_items[0]);
    dev_free(c, g->fwd_items[1]);
    dev_free(c, g->fwd_items[2]);
    g->fwd_items_n[0] = g->fwd_items_n[1] = g->fwd_items_n[2] = 0;
    dev_free(c, g->fwd_ebase);
    dev_free(c, g->fwd_elen);
    dev_free(c, g->fwd_efin);
    g->fwd_entries = false;
    g->fwd_entries_tried = false;
    g->fwd_small = 0;
    g->fwd_ready = false;
}

scan_status apply(Graph *g, const Choice &ch) {
    query_graph_drop(g);
    g->strategy = ch.strategy;
    g->fwd_queue = ch.queue != 0;
    if (ch.strategy == SCAN_STRATEGY_FORWARD &&
        (g->fwd_small_work != ch.small_work || g->fwd_item_work != ch.item_work)) {
        g->fwd_small_work = ch.small_work;
        g->fwd_item_work = ch.item_work;
        reset_forward_schedule(g);
    }
    if (ch.strategy == SCAN_STRATEGY_FORWARD) return fwd_prepare(g);
    return SCAN_OK;
}

// One full count with the graph's current choice, timed with events.
scan_status time_count(Graph *g, float *ms) {
    Ctx *c = g->ctx;
    cudaEvent_t a, b;
    SCAN_CUDA(cudaEventCreate(&a));
    SCAN_CUDA(cudaEventCreate(&b));
    SCAN_CUDA(cudaEventRecord(a, c->stream));
    scan_status s = build_count_cache(g);
    cudaEventRecord(b, c->stream);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != SCAN_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    return SCAN_OK;
}

bool load_choice(const char *path, const std::string &key, Choice *out) {
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512], tag[16], k[128];
    int strat, queue;
    long long sw, iw;
    double ms;
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        // lines of another format are skipped
        if (sscanf(line, "%15s %127s %d %lld %lld %d %lf", tag, k, &strat, &sw, &iw, &queue, &ms) != 7) continue;
        if (std::string(tag) == "fwd2" && key == k) {
            out->strategy = strat;
            out->small_work = sw;
            out->item_work = iw;
            out->queue = queue;
            out->ms = ms;
            found = true;  // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

void store_choice(const char *path, const std::string &key, const Choice &ch) {
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "fwd2 %s %d %lld %lld %d %.9g\n", key.c_str(), ch.strategy, (long long)ch.small_work,
            (long long)ch.item_work, ch.queue, ch.ms);
    fclose(f);
}

}  // namespace
}  // namespace scan

using namespace scan;

extern "C" scan_status scan_graph_autotune(scan_graph *g, const char *cache_path, int32_t *strategy_out,
                                           double *ms_out) {
    try {
        if (!g) { set_error("graph is NULL"); return SCAN_EINVAL; }
        if (g->part) { set_error("not available for a partitioned graph"); return SCAN_EINVAL; }
        Ctx *c = g->ctx;
        SCAN_CUDA(cudaSetDevice(c->device));
        if (g->m == 0) {
            if (strategy_out) *strategy_out = g->strategy;
            if (ms_out) *ms_out = 0;
            return SCAN_OK;
        }
        // shape key
        DevBuf mx;
        SCAN_TRY(dev_alloc(c, mx, sizeof(int)));
        int hmax = 0;
        SCAN_CUDA(cudaMemsetAsync(mx.ptr, 0, sizeof(int), c->stream));
        k_max_deg<<<grid_for(g->n, 256, c->num_sms * 8), 256, 0, c->stream>>>((const int32_t *)g->deg.ptr, g->n,
                                                                            (int *)mx.ptr);
        c->launches++;
        SCAN_CUDA(cudaMemcpyAsync(&hmax, mx.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        SCAN_CUDA(cudaStreamSynchronize(c->stream));
        dev_free(c, mx);
        char key[128];
        snprintf(key, sizeof(key), "n%d_e%d_d%d", ilog2((uint64_t)g->n), ilog2((uint64_t)g->nnz),
                 ilog2((uint64_t)hmax + 1));

        Choice best;
        if (load_choice(cache_path, key, &best)) {
            SCAN_TRY(apply(g, best));
        } else {
            const bool had_cache = g->cache_valid;
            std::vector<Choice> cands;
            for (int64_t iw : {int64_t(1) << 18, int64_t(1) << 20, int64_t(1) << 22})
                for (int64_t sw : {int64_t(1) << 12, int64_t(1) << 15})
                    for (int queue : {0, 1}) {
                        Choice ch;
                        ch.strategy = SCAN_STRATEGY_FORWARD;
                        ch.item_work = iw;
                        ch.small_work = sw;
                        ch.queue = queue;
                        cands.push_back(ch);
                    }
            Choice own;
            own.strategy = SCAN_STRATEGY_OWNER;
            cands.push_back(own);
            Choice bs;
            bs.strategy = SCAN_STRATEGY_BSEARCH;
            cands.push_back(bs);
            best.ms = -1;
            for (Choice ch : cands) {
                SCAN_TRY(apply(g, ch));
                float warm = 0, t = 0;
                SCAN_TRY(time_count(g, &warm));
                // a family far slower than the best so far is not timed again
                if (best.ms > 0 && warm > 8 * best.ms) continue;
                SCAN_TRY(time_count(g, &t));
                ch.ms = t;
                if (best.ms < 0 || t < best.ms) best = ch;
            }
            SCAN_TRY(apply(g, best));
            if (!had_cache) cache_free(g);
            store_choice(cache_path, key, best);
        }
        if (strategy_out) *strategy_out = best.strategy;
        if (ms_out) *ms_out = best.ms;
        return SCAN_OK;
    } catch (...) {
        set_error("autotune failed");
        return SCAN_EINVAL;
    }
}

// server.cu -- a SCAN query server with continuous batching and cached counts.
//
// Graphs are registered once (host CSR kept in pinned memory) and kept
// resident on the device while memory allows. The first query on a graph
// computes every edge's closed common count and keeps it (the count cache),
// so later (eps, mu) queries on that graph skip the intersection and run the
// eps-test, cores, union-find, borders and labels only.
//
// One worker thread owns every CUDA call. Requests queue as they arrive; the
// worker admits them into a fixed number of slots, each with its own stream,
// as slots and device memory free up, so queries on different graphs run
// concurrently on the device (queries on one graph share its scratch and
// are serialised). Admission is by device memory against the context's
// budget: idle graphs' count caches are evicted first (least recently used),
// then idle graphs themselves, which reload from their pinned host copy on
// their next request. A request that can never fit fails with SCAN_EBUSY.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "scan_internal.cuh"

using namespace scan;

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvGraph {
    int32_t n = 0;
    int64_t nnz = 0;
    int64_t *h_off = nullptr;  // pinned, server-owned
    int32_t *h_adj = nullptr;
    Graph *g = nullptr;        // resident device graph, or null
    bool busy = false;
    uint64_t last_use = 0;
};

struct Request {
    uint64_t ticket = 0;
    int32_t gid = -1;
    scan_params p{};
    double t_arrive = 0;
};

struct Done {
    scan_result *r = nullptr;
    scan_status st = SCAN_OK;
    std::string err;
    double latency_ms = 0;
};

// Graphs up to this many slots are served on high-priority streams: their
// short kernels then take SMs as soon as the long kernels of a big graph's
// query release them, instead of queueing behind them.
constexpr int64_t kSmallGraphSlots = int64_t(1) << 24;

struct Slot {
    cudaStream_t stream = nullptr;  // the stream of the request in flight: hi or lo
    cudaStream_t hi = nullptr, lo = nullptr;
    cudaEvent_t ev = nullptr;
    int state = 0;  // 0 idle, 1 arrays in flight, 2 border pairs in flight
    Request req;
    scan_result *res = nullptr;  // the answer, copied from the device straight into its pinned blocks
    int64_t *h_np = nullptr;
    uint32_t *h_err = nullptr;
};

// Points the context's launch stream at `s` for the lifetime of the guard
// (the server's worker is the only thread using the context).
struct StreamScope {
    Ctx *c;
    cudaStream_t saved;
    StreamScope(Ctx *ctx, cudaStream_t s) : c(ctx), saved(ctx->stream) { c->stream = s; }
    ~StreamScope() { c->stream = saved; }
};

}  // namespace

struct scan_server {
    Ctx *ctx = nullptr;
    scan_server_opts opts{};
    std::vector<SrvGraph> graphs;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request> incoming;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::deque<Request> pending;  // worker only
    cudaStream_t load_stream = nullptr;
    std::thread worker;
    std::atomic<bool> stop{false};
    uint64_t tick = 0;
    // statistics (guarded by mu)
    std::vector<double> latencies;
    uint64_t rejected = 0, cache_builds = 0, cache_evictions = 0, graph_loads = 0, graph_evictions = 0;
    double t_first_arrive = -1, t_last_done = 0;
    int32_t inflight = 0, max_inflight_seen = 0;

    void finish(const Request &rq, scan_result *r, scan_status st, const std::string &err) {
        const double t = now_ms();
        std::lock_guard<std::mutex> lock(mu);
        Done d;
        d.r = r;
        d.st = st;
        d.err = err;
        d.latency_ms = t - rq.t_arrive;
        done[rq.ticket] = std::move(d);
        if (st == SCAN_OK) latencies.push_back(t - rq.t_arrive);
        else ++rejected;
        t_last_done = t;
        cv_done.notify_all();
    }

    // Evict one idle victim (cache first, then graph). Returns false if none.
    bool evict_one(const SrvGraph *keep) {
        SrvGraph *best = nullptr;
        for (auto &sg : graphs)
            if (&sg != keep && sg.g && !sg.busy && sg.g->cache_valid && (!best || sg.last_use < best->last_use))
                best = &sg;
        if (best) {
            query_graph_drop(best->g);
            cache_free(best->g);
            std::lock_guard<std::mutex> lock(mu);
            ++cache_evictions;
            return true;
        }
        for (auto &sg : graphs)
            if (&sg != keep && sg.g && !sg.busy && (!best || sg.last_use < best->last_use)) best = &sg;
        if (best) {
            graph_destroy(best->g);
            best->g = nullptr;
            std::lock_guard<std::mutex> lock(mu);
            ++graph_evictions;
            return true;
        }
        return false;
    }

    // Make the graph resident (evicting idle ones as needed). SCAN_EBUDGET
    // means "not now" while anything is in flight, else "never".
    scan_status ensure_resident(SrvGraph &sg) {
        if (sg.g) return SCAN_OK;
        for (int attempt = 0; attempt < 1 << 20; ++attempt) {
            StreamScope scope(ctx, load_stream);
            Graph *g = nullptr;
            scan_status s = graph_create(ctx, sg.n, sg.h_off, sg.h_adj, sg.nnz, false, &g);
            if (s == SCAN_OK) s = fwd_prepare(g);
            // the slots' streams read what the load stream wrote: finish it here
            if (s == SCAN_OK) {
                const cudaError_t e = cudaStreamSynchronize(load_stream);
                if (e != cudaSuccess) s = cuda_fail(e, "graph load");
            }
            if (s == SCAN_OK) {
                sg.g = g;
                std::lock_guard<std::mutex> lock(mu);
                ++graph_loads;
                return SCAN_OK;
            }
            if (g) graph_destroy(g);
            if (s != SCAN_EBUDGET && s != SCAN_ENOMEM) return s;
            if (!evict_one(&sg)) return SCAN_EBUDGET;
        }
        return SCAN_EBUDGET;
    }

    // Launch one request on a free slot. Returns false if it must wait.
    bool admit(const Request &rq, Slot &sl) {
        SrvGraph &sg = graphs[(size_t)rq.gid];
        scan_status s = ensure_resident(sg);
        if (s == SCAN_EBUDGET && inflight > 0) return false;  // wait for memory
        if (s != SCAN_OK) {
            finish(rq, nullptr, s == SCAN_EBUDGET ? SCAN_EBUSY : s,
                   s == SCAN_EBUDGET ? "graph can never fit the device budget" : "graph load failed");
            return true;
        }
        Graph *g = sg.g;
        sl.stream = g->nnz <= kSmallGraphSlots ? sl.hi : sl.lo;
        uint32_t mode = opts.use_cache == 2 ? SCAN_Q_PLAIN : SCAN_Q_RECOMPUTE;
        if (opts.use_cache == 1) {
            if (g->cache_valid) {
                mode = SCAN_Q_AUTO;
            } else {
                // reserve the cache up front; without room the query recomputes
                bool ok = false;
                for (int attempt = 0; attempt < 1 << 20 && !ok; ++attempt) {
                    scan_status a = cache_reserve(g);
                    if (a == SCAN_OK) ok = true;
                    else if (!evict_one(&sg)) break;
                }
                if (ok) {
                    mode = SCAN_Q_BUILD_CACHE;
                    std::lock_guard<std::mutex> lock(mu);
                    ++cache_builds;
                }
            }
        }
        // the result's arrays come from the pinned block pool, so the device
        // writes them directly and the worker never copies a result on the host
        sl.res = result_new(g->n, 0, true);
        if (!sl.res) {
            finish(rq, nullptr, SCAN_ENOMEM, "pinned result allocation failed");
            return true;
        }
        {
            StreamScope scope(ctx, sl.stream);
            s = query_replay(g, rq.p, mode, (uint8_t *)g->core.ptr, (int32_t *)g->cid.ptr,
                               (uint8_t *)g->label.ptr, (int32_t *)g->pairs.ptr, g->nnz, (int64_t *)g->npairs.ptr);
            cudaError_t e = cudaSuccess;
            if (s == SCAN_OK) e = cudaMemcpyAsync(sl.h_np, g->npairs.ptr, 8, cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_err, g->err.ptr, 4, cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess && g->n > 0) {
                scan_result *r = sl.res;
                e = cudaMemcpyAsync(r->core, g->core.ptr, (size_t)g->n, cudaMemcpyDeviceToHost, sl.stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(r->cid, g->cid.ptr, 4 * (size_t)g->n, cudaMemcpyDeviceToHost, sl.stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(r->label, g->label.ptr, (size_t)g->n, cudaMemcpyDeviceToHost, sl.stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
            if (s == SCAN_OK && e != cudaSuccess) s = cuda_fail(e, "server launch");
        }
        if (s != SCAN_OK) {
            cudaStreamSynchronize(sl.stream);  // copies into the result may be queued
            scan_result_free(sl.res);
            sl.res = nullptr;
            finish(rq, nullptr, s, "query launch failed");
            return true;
        }
        sg.busy = true;
        sg.last_use = ++tick;
        sl.req = rq;
        sl.state = 1;
        std::lock_guard<std::mutex> lock(mu);
        ++inflight;
        max_inflight_seen = std::max(max_inflight_seen, inflight);
        return true;
    }

    void release_slot(Slot &sl) {
        graphs[(size_t)sl.req.gid].busy = false;
        scan_result_free(sl.res);  // null once handed to the caller
        sl.res = nullptr;
        sl.state = 0;
        std::lock_guard<std::mutex> lock(mu);
        --inflight;
    }

    // Advance a slot whose event completed.
    void advance(Slot &sl) {
        SrvGraph &sg = graphs[(size_t)sl.req.gid];
        Graph *g = sg.g;
        if (sl.state == 1) {
            if (*sl.h_err) {
                cudaMemsetAsync(g->err.ptr, 0, 4, sl.stream);
                cudaStreamSynchronize(sl.stream);
                finish(sl.req, nullptr, SCAN_ETIMEOUT, "a bounded device loop gave up");
                release_slot(sl);
                return;
            }
            if (g->cache_valid == false && g->cn_cache.ptr) g->cache_valid = true;
            const int64_t k = *sl.h_np;
            if (k > 0) {
                if (!result_set_pairs(sl.res, k)) {
                    finish(sl.req, nullptr, SCAN_ENOMEM, "pinned result allocation failed");
                    release_slot(sl);
                    return;
                }
                cudaMemcpyAsync(sl.res->pairs, g->pairs.ptr, 8 * (size_t)k, cudaMemcpyDeviceToHost, sl.stream);
                cudaEventRecord(sl.ev, sl.stream);
                sl.state = 2;
                return;
            }
        }
        scan_result *r = sl.res;
        sl.res = nullptr;
        finish(sl.req, r, SCAN_OK, "");
        release_slot(sl);
    }

    void run() {
        cudaSetDevice(ctx->device);
        for (;;) {
            bool progressed = false;
            {
                std::unique_lock<std::mutex> lock(mu);
                while (!incoming.empty()) {
                    pending.push_back(incoming.front());
                    incoming.pop_front();
                    progressed = true;
                }
                if (stop && pending.empty() && inflight == 0) return;
            }
            for (auto &sl : slots) {
                if (sl.state == 0) continue;
                const cudaError_t q = cudaEventQuery(sl.ev);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) {
                    finish(sl.req, nullptr, SCAN_ECUDA, cudaGetErrorString(q));
                    release_slot(sl);
                } else {
                    advance(sl);
                }
                progressed = true;
            }
            for (auto &sl : slots) {
                if (sl.state != 0 || pending.empty()) continue;
                // first pending request whose graph is idle
                auto it = std::find_if(pending.begin(), pending.end(),
                                       [&](const Request &r) { return !graphs[(size_t)r.gid].busy; });
                if (it == pending.end()) break;
                const Request rq = *it;
                if (!admit(rq, sl)) break;  // must wait for memory
                pending.erase(std::find_if(pending.begin(), pending.end(),
                                           [&](const Request &r) { return r.ticket == rq.ticket; }));
                progressed = true;
            }
            if (!progressed) {
                std::unique_lock<std::mutex> lock(mu);
                if (incoming.empty()) {
                    if (inflight == 0 && pending.empty())
                        cv_submit.wait_for(lock, std::chrono::milliseconds(2));
                    else
                        cv_submit.wait_for(lock, std::chrono::microseconds(20));
                }
            }
        }
    }
};

extern "C" {

scan_status scan_server_create(scan_ctx *ctx, const scan_server_opts *opts, scan_server **out) {
    try {
        if (!ctx || !out) { set_error("ctx or out is NULL"); return SCAN_EINVAL; }
        *out = nullptr;
        scan_server *s = new scan_server();
        s->ctx = ctx;
        s->opts.max_inflight = opts ? opts->max_inflight : 8;
        s->opts.use_cache = opts ? opts->use_cache : 1;
        if (s->opts.max_inflight < 1 || s->opts.max_inflight > 256) {
            delete s;
            set_error("max_inflight must be in [1, 256]");
            return SCAN_EINVAL;
        }
        SCAN_CUDA(cudaSetDevice(ctx->device));
        s->slots.resize((size_t)s->opts.max_inflight);
        int prio_lo = 0, prio_hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->load_stream, cudaStreamNonBlocking);
        for (auto &sl : s->slots) {
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.hi, cudaStreamNonBlocking, prio_hi);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.lo, cudaStreamNonBlocking, prio_lo);
            sl.stream = sl.lo;
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h_np, 8);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h_err, 4);
        }
        if (e != cudaSuccess) {
            scan_server_destroy(s);
            return cuda_fail(e, "server setup");
        }
        s->worker = std::thread([s] { s->run(); });
        *out = s;
        return SCAN_OK;
    } catch (...) {
        set_error("server creation failed");
        return SCAN_ENOMEM;
    }
}

scan_status scan_server_add_graph(scan_server *s, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                                  int32_t *graph_id) {
    if (!s || !graph_id || n < 0 || nnz < 0 || (n > 0 && !offsets) || (nnz > 0 && !adj)) {
        set_error("bad arguments");
        return SCAN_EINVAL;
    }
    if (n > 0 && (offsets[0] != 0 || offsets[n] != nnz)) {
        set_error("offsets[0] must be 0 and offsets[n] must equal nnz");
        return SCAN_EINVAL;
    }
    SrvGraph sg;
    sg.n = n;
    sg.nnz = nnz;
    cudaError_t e = cudaMallocHost(&sg.h_off, 8 * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMallocHost(&sg.h_adj, 4 * (size_t)(nnz > 0 ? nnz : 1));
    if (e != cudaSuccess) {
        if (sg.h_off) cudaFreeHost(sg.h_off);
        return cuda_fail(e, "pinned graph copy");
    }
    if (n > 0) memcpy(sg.h_off, offsets, 8 * ((size_t)n + 1));
    else sg.h_off[0] = 0;
    if (nnz > 0) memcpy(sg.h_adj, adj, 4 * (size_t)nnz);
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->pending.empty() || !s->incoming.empty() || s->inflight > 0) {
        cudaFreeHost(sg.h_off);
        cudaFreeHost(sg.h_adj);
        set_error("graphs must be added while the server is idle");
        return SCAN_EBUSY;
    }
    *graph_id = (int32_t)s->graphs.size();
    s->graphs.push_back(sg);
    return SCAN_OK;
}

scan_status scan_server_submit(scan_server *s, int32_t graph_id, const scan_params *params, uint64_t *ticket) {
    if (!s || !ticket || !params) { set_error("NULL argument"); return SCAN_EINVAL; }
    SCAN_TRY(check_params(params));
    std::lock_guard<std::mutex> lock(s->mu);
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) { set_error("unknown graph id"); return SCAN_EINVAL; }
    if (s->stop) { set_error("server is shutting down"); return SCAN_EBUSY; }
    Request rq;
    rq.ticket = s->next_ticket++;
    rq.gid = graph_id;
    rq.p = *params;
    rq.t_arrive = now_ms();
    if (s->t_first_arrive < 0) s->t_first_arrive = rq.t_arrive;
    s->incoming.push_back(rq);
    *ticket = rq.ticket;
    s->cv_submit.notify_one();
    return SCAN_OK;
}

static scan_status take_done(scan_server *s, uint64_t ticket, scan_result **out, double *latency_ms) {
    auto it = s->done.find(ticket);
    Done d = std::move(it->second);
    s->done.erase(it);
    if (latency_ms) *latency_ms = d.latency_ms;
    if (d.st != SCAN_OK) {
        set_error(d.err);
        return d.st;
    }
    *out = d.r;
    return SCAN_OK;
}

scan_status scan_server_wait(scan_server *s, uint64_t ticket, scan_result **out, double *latency_ms) {
    if (!s || !out) { set_error("NULL argument"); return SCAN_EINVAL; }
    *out = nullptr;
    std::unique_lock<std::mutex> lock(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) { set_error("unknown ticket"); return SCAN_EINVAL; }
    for (int it = 0; it < (1 << 30) && s->done.find(ticket) == s->done.end(); ++it)
        s->cv_done.wait_for(lock, std::chrono::milliseconds(50));
    if (s->done.find(ticket) == s->done.end()) { set_error("ticket already taken"); return SCAN_EINVAL; }
    return take_done(s, ticket, out, latency_ms);
}

scan_status scan_server_poll(scan_server *s, uint64_t ticket, scan_result **out, double *latency_ms, int32_t *ready) {
    if (!s || !out || !ready) { set_error("NULL argument"); return SCAN_EINVAL; }
    *out = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->done.find(ticket) == s->done.end()) {
        *ready = 0;
        return SCAN_OK;
    }
    *ready = 1;
    return take_done(s, ticket, out, latency_ms);
}

scan_status scan_server_stats(scan_server *s, scan_server_report *st) {
    if (!s || !st) { set_error("NULL argument"); return SCAN_EINVAL; }
    std::lock_guard<std::mutex> lock(s->mu);
    memset(st, 0, sizeof(*st));
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    st->completed = l.size();
    st->rejected = s->rejected;
    auto pct = [&](double q) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(q * (double)l.size()))]; };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : l) sum += x;
    st->mean_ms = l.empty() ? 0.0 : sum / (double)l.size();
    const double span = s->t_last_done - s->t_first_arrive;
    st->throughput_rps = (span > 0 && !l.empty()) ? 1e3 * (double)l.size() / span : 0.0;
    st->cache_builds = s->cache_builds;
    st->cache_evictions = s->cache_evictions;
    st->graph_loads = s->graph_loads;
    st->graph_evictions = s->graph_evictions;
    st->max_inflight = s->max_inflight_seen;
    st->device_bytes = s->ctx->used;
    return SCAN_OK;
}

scan_status scan_server_reset_stats(scan_server *s) {
    if (!s) { set_error("NULL argument"); return SCAN_EINVAL; }
    std::lock_guard<std::mutex> lock(s->mu);
    s->latencies.clear();
    s->rejected = s->cache_builds = s->cache_evictions = s->graph_loads = s->graph_evictions = 0;
    s->t_first_arrive = -1;
    s->t_last_done = 0;
    s->max_inflight_seen = s->inflight;
    return SCAN_OK;
}

void scan_server_destroy(scan_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_submit.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx->device);
    for (auto &kv : s->done) scan_result_free(kv.second.r);
    for (auto &sg : s->graphs) {
        if (sg.g) graph_destroy(sg.g);
        if (sg.h_off) cudaFreeHost(sg.h_off);
        if (sg.h_adj) cudaFreeHost(sg.h_adj);
    }
    for (auto &sl : s->slots) {
        for (cudaStream_t st : {sl.hi, sl.lo})
            if (st) cudaStreamSynchronize(st), cudaStreamDestroy(st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        scan_result_free(sl.res);
        void *pin[] = {sl.h_np, sl.h_err};
        for (void *p : pin)
            if (p) cudaFreeHost(p);
    }
    if (s->load_stream) cudaStreamDestroy(s->load_stream);
    delete s;
}

}  // extern "C"

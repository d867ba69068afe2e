/*
 * scan.h -- C ABI of libscan.so: exact structural graph clustering (SCAN)
 * on one NVIDIA GB300 (sm_103a).
 *
 * The operation (GPUSCAN++, Section 2.1, Definitions 2.1-2.3, Core,
 * Structural Reachability, Cluster, Hub and Outlier): for an undirected
 * simple graph and eps = eps_num/eps_den, mu, compute
 *   sigma(u,v) = |N[u] cap N[v]| / sqrt(|N[u]| |N[v]|) over closed
 *   neighbourhoods for every edge, the eps-test (exact: cn^2 q^2 >= p^2
 *   |N[u]| |N[v]| in 128-bit integers), the cores (|N_eps[u]| >= mu), the
 *   clusters (connected components of cores through eps-similar core-core
 *   edges; each cluster is named by its smallest core id), every
 *   (vertex, cluster) membership of non-core vertices, and the hub/outlier
 *   label of every vertex in no cluster (hub iff its neighbours' memberships
 *   span >= 2 clusters).
 *
 * Conventions for every call:
 *   - Return value: scan_status (SCAN_OK = 0). On failure nothing is
 *     returned through out-parameters and scan_last_error() (thread-local)
 *     describes the failure. No call aborts, exits or throws across the ABI.
 *   - Vertex ids are int32 in [0, n); CSR offsets are int64[n + 1].
 *   - Host pointers stay owned by the caller unless stated otherwise.
 *   - Objects (ctx, graph, result, server) are owned by the library and
 *     released with their *_free / *_destroy call. A graph must be freed
 *     before its context is destroyed.
 *   - A context is not thread-safe: calls on one context (and its graphs)
 *     must be serialised by the caller. Distinct contexts are independent.
 */
#ifndef SCAN_H
#define SCAN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SCAN_API __attribute__((visibility("default")))
#else
#define SCAN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum scan_status {
    SCAN_OK = 0,
    SCAN_EINVAL = 1,   /* bad argument or malformed graph (detail names the first bad index) */
    SCAN_ENOMEM = 2,   /* a host or device allocation failed */
    SCAN_EBUDGET = 3,  /* the request does not fit the context's device-memory budget */
    SCAN_ECUDA = 4,    /* a CUDA runtime error (detail has the CUDA error string) */
    SCAN_ETIMEOUT = 5, /* a bounded device loop ran out of iterations (kernel returned early) */
    SCAN_EBUSY = 6     /* a server request can never be admitted, or the server is shutting down */
} scan_status;

/* Vertex labels of a result. */
enum { SCAN_CORE = 0, SCAN_BORDER = 1, SCAN_HUB = 2, SCAN_OUTLIER = 3 };

typedef struct scan_ctx scan_ctx;
typedef struct scan_graph scan_graph;
typedef struct scan_result scan_result;

/* Thread-local description of the last failure on this thread ("" if none).
 * The pointer stays valid until the next failing call on this thread. */
SCAN_API const char *scan_last_error(void);

/* ------------------------------------------------------------- context */
typedef struct scan_ctx_opts {
    int32_t device;        /* CUDA device ordinal */
    uint64_t budget_bytes; /* cap on device memory this context may hold; 0 = no cap */
    void *stream;          /* cudaStream_t to launch on; NULL = a stream the context creates */
} scan_ctx_opts;

/* Create a context on opts->device (opts may be NULL: device 0, no cap, own
 * stream). Errors: SCAN_EINVAL (bad device), SCAN_ECUDA, SCAN_ENOMEM. */
SCAN_API scan_status scan_ctx_create(const scan_ctx_opts *opts, scan_ctx **out);
SCAN_API void scan_ctx_destroy(scan_ctx *ctx);
/* Device bytes the context currently holds (graphs, caches, scratch). */
SCAN_API uint64_t scan_ctx_device_bytes(const scan_ctx *ctx);
/* Number of CUDA kernels this context has launched so far. */
SCAN_API uint64_t scan_ctx_kernel_launches(const scan_ctx *ctx);
/* Synchronise the context's stream. */
SCAN_API scan_status scan_ctx_sync(scan_ctx *ctx);

/* Per-stage device timing with CUDA events recorded on the context's stream
 * around each stage of every query (the paper reports per-phase times in its
 * Table 3; these are the same phases, split finer). */
enum {
    SCAN_STAGE_SIMILARITY = 0, /* common counts + eps-test (Algorithm 2's checkSim work) */
    SCAN_STAGE_CORE = 1,       /* |N_eps| >= mu */
    SCAN_STAGE_CLUSTER = 2,    /* union-find over core-core similar edges */
    SCAN_STAGE_BORDER = 3,     /* border memberships */
    SCAN_STAGE_LABEL = 4,      /* hub / outlier */
    SCAN_STAGE_COUNT = 5
};
/* enable != 0 turns recording on and clears the totals; 0 turns it off. */
SCAN_API scan_status scan_ctx_profile(scan_ctx *ctx, int32_t enable);
/* Synchronises, then returns the summed milliseconds and number of timed
 * intervals of a stage since profiling was (re)enabled. */
SCAN_API scan_status scan_ctx_stage_time(scan_ctx *ctx, int32_t stage, double *total_ms, int64_t *intervals);
/*
 * Iteration cap of the union-find loops (Algorithm 3's root walks and hook
 * retries; every device loop of this library is bounded) for the context's
 * later queries, resident and out of core: limit = 0 restores the compiled
 * bound (2^22 iterations, never reached by a correct run); a smaller value
 * lowers it. A query whose loops run out returns SCAN_ETIMEOUT with no
 * result; the context and its graphs stay usable. This exists to exercise
 * that error path (a diagnostic: limits far below a graph's union-find
 * depth make queries fail). While a cap is set, queries run their kernels
 * directly instead of replaying a captured CUDA graph. Synchronises the
 * context's stream first.
 */
SCAN_API scan_status scan_ctx_set_loop_limit(scan_ctx *ctx, uint32_t limit);

/* ---------------------------------------------------------------- graph */
/* Load flags. */
#define SCAN_LOAD_DEVICE_PTRS 0x1u   /* offsets/adj are device pointers (copied device-to-device) */
#define SCAN_LOAD_PINNED_BORROW 0x2u /* partitioned mode: keep the CSR in the caller's host memory
                                        (registered as pinned; the caller keeps it alive and
                                        unmodified until scan_graph_free) and stream slices */

/*
 * Load an undirected simple graph given as CSR: offsets int64[n + 1] with
 * offsets[0] = 0 and offsets[n] = nnz, adj int32[nnz] (nnz = 2m directed
 * slots). The CSR layout is the vertex array / adjacency array of the
 * paper's CSR-enhanced layout (Section 4.1).
 *
 * Requirements (checked on the device; nothing is repaired): each row sorted
 * strictly ascending (so no duplicates), ids in [0, n), no self-loops, and
 * symmetric (v in row u <=> u in row v). Violations: SCAN_EINVAL with the
 * first bad slot in scan_last_error(); when every slot pointing to a higher
 * id has its reverse and the graph is still not symmetric, the numbers of
 * slots pointing to higher and to lower ids instead. n = 0 is valid.
 *
 * Without SCAN_LOAD_PINNED_BORROW the library copies the arrays to the
 * device and the caller may release them on return. If the graph's device
 * footprint exceeds the budget: SCAN_EBUDGET (pass SCAN_LOAD_PINNED_BORROW
 * to cluster it out of core). With SCAN_LOAD_PINNED_BORROW the host arrays
 * must stay valid until scan_graph_free.
 */
SCAN_API scan_status scan_graph_load(scan_ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj,
                            int64_t nnz, uint32_t flags, scan_graph **out);
SCAN_API void scan_graph_free(scan_graph *g);
/*
 * Out of core (the paper's Section 5 setting: vertices fit on the device,
 * edges do not): the CSR stays in the caller's host memory -- pinned by the
 * library if it is not already, and kept alive and unmodified by the caller
 * until scan_graph_free -- and every query streams it in contiguous row
 * blocks of at most block_slots slots (0: sized from the context's budget
 * left after the per-vertex state). Lemma 5.1 makes the result equal the
 * resident one: an edge's similarity needs only its two endpoints' rows.
 * Validation as scan_graph_load (symmetry found missing during a query is
 * reported then). Queries: scan_query / scan_query_ex (every mode is a full
 * recompute); the cache, strategy and device-output calls return SCAN_EINVAL.
 * scan_graph_load with SCAN_LOAD_PINNED_BORROW is this call with block_slots 0.
 */
SCAN_API scan_status scan_graph_load_partitioned(scan_ctx *ctx, int32_t n, const int64_t *offsets,
                                                 const int32_t *adj, int64_t nnz, int64_t block_slots,
                                                 scan_graph **out);
/* Number of row blocks of a partitioned graph (0 for a resident one). */
SCAN_API int32_t scan_graph_blocks(const scan_graph *g);
/* Host-to-device bytes a partitioned graph's blocks have been copied in, in
 * total since it was loaded (validation and every query; Section 5's
 * transfer volume); 0 for a resident graph. */
SCAN_API uint64_t scan_graph_transfer_bytes(const scan_graph *g);
/*
 * Zero-copy reading of a partitioned graph (enable != 0; 0 returns to
 * copied blocks): the kernels read the streamed partner blocks of the
 * similarity pass, and the blocks of the later passes, in place from the
 * caller's pinned host CSR through the host link (NVLink-C2C on GB300),
 * instead of copying each block into device memory first; the held block of
 * each pass-1 row of pairs is still copied. The paper's Section 6.3 sets
 * its partitioned design against a unified-memory version; this is that
 * comparison's counterpart here. Results are identical either way (Lemma
 * 5.1). SCAN_EINVAL for a resident graph; SCAN_ECUDA when the host arrays
 * are not mapped for device access. Synchronises the context's stream.
 */
SCAN_API scan_status scan_graph_set_zero_copy(scan_graph *g, int32_t enable);
/*
 * The paper's own out-of-core partition (Section 5, Algorithm 5's CPU part,
 * Definition "Edge Extended Subgraph"), planned on the host for comparison
 * with the row-block pairs above: undirected edges (u, v), u < v, are taken
 * in CSR order into the current subgraph with every edge incident to them;
 * when Memof(G_s) + Memof(G'_s) + 15 |V(G)| would exceed device_bytes the
 * subgraph is closed. Memof(G) = 25 |E(G)| + 4 |V(G)|. Returns the number of
 * subgraphs and the bytes loading each of them once moves (the sum of their
 * Memof). offsets int64[n+1] and adj int32[nnz] are host arrays, read only;
 * no device work. SCAN_EINVAL on malformed offsets or ids out of range.
 */
SCAN_API scan_status scan_plan_edge_extended(int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                                             uint64_t device_bytes, int64_t *subgraphs, uint64_t *bytes);
/*
 * Plan (host only, no device work) of counting by degree-oriented triangle
 * enumeration (Section 4.1's orientation) over pairs of vertex blocks, for a
 * graph whose CSR stays in host memory. A triangle a < b < c in (deg, id)
 * rank is found at b, and its three counts lie in out(a) and out(b), so the
 * pair (block of a, block of b) needs only those two blocks; blocks are cut
 * in rank order, so only pairs i <= j carry work. The device keeps 19 B per
 * vertex and a bit per slot; three block slots share 90 % of the rest, a
 * block holding whole out-lists at 8 B per oriented edge and 12 B per row.
 * Returns the blocks, the pairs with at least one oriented edge from block i
 * to block j, and the bytes moved when each block is loaded (12 B per row
 * and 8 B per oriented edge in) and unloaded (4 B per oriented edge out) once
 * as the resident block and once per later pair that streams it.
 * SCAN_EINVAL on malformed offsets or ids out of range; SCAN_EBUDGET when
 * device_bytes cannot hold the per-vertex state or one out-list, or would
 * need more than 8192 blocks.
 */
SCAN_API scan_status scan_plan_triangle_blocks(int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz,
                                               uint64_t device_bytes, int32_t *blocks, int64_t *pairs,
                                               uint64_t *bytes);
SCAN_API int32_t scan_graph_n(const scan_graph *g);
SCAN_API int64_t scan_graph_nnz(const scan_graph *g);
/* Device bytes held by this graph (including its count cache). */
SCAN_API uint64_t scan_graph_device_bytes(const scan_graph *g);
/* Release the per-edge common-count cache, if any. */
SCAN_API scan_status scan_graph_drop_cache(scan_graph *g);
/* 1 if the graph holds a valid per-edge common-count cache. */
SCAN_API int32_t scan_graph_has_cache(const scan_graph *g);
/* Copy the cached closed common counts |N[u] cap N[v]| (the numerator of
 * Definition 2.2's sigma, Eq. 1) to host memory out[nnz], slot-aligned with
 * adj. Requires a cache (a query with SCAN_Q_BUILD_CACHE), else SCAN_EINVAL.
 * The cache keeps 12 bytes per undirected edge (the count and the product of
 * the closed degrees); this call writes both slots of every edge.
 * Synchronous. */
SCAN_API scan_status scan_graph_copy_counts(scan_graph *g, int32_t *out);

/* --------------------------------------------------------------- query */
typedef struct scan_params {
    uint32_t eps_num; /* eps = eps_num / eps_den, 0 < eps <= 1 (Definition 2.3) */
    uint32_t eps_den;
    uint32_t mu;      /* mu >= 2 (Definition Core) */
} scan_params;

/* Kernel family of the similarity stage (common counts). Every family gives
 * the same result; they differ in speed by graph shape. */
#define SCAN_STRATEGY_FORWARD 0 /* degree-oriented triangle enumeration: each triangle found once at its
                                   middle vertex through a shared-memory table (the default) */
#define SCAN_STRATEGY_OWNER 1   /* per edge: the higher-degree endpoint's row in a shared-memory hash,
                                   the lower one streamed; skips edges the degrees decide */
#define SCAN_STRATEGY_BSEARCH 2 /* per edge: binary search of the smaller row in the larger (checkSim
                                   of Algorithm 2); skips edges the degrees decide */
#define SCAN_STRATEGY_FORWARD_LEAN 3 /* FORWARD without its precomputed per-item entry lists (12 bytes
                                        per oriented edge): derived round by round, slower; FORWARD
                                        falls back to it when the lists do not fit the budget */
#define SCAN_STRATEGY_PROGRESSIVE 4 /* per edge, BSEARCH's intersection with the paper's progressive
                                       role-based skipping (Algorithms 2-3): an edge whose two endpoints'
                                       core roles the bounds already fix is not intersected during core
                                       detection; afterwards only core-core edges not yet in one
                                       union-find tree and core-non-core edges are; non-core pairs never.
                                       Queries only (no count cache): SCAN_Q_BUILD_CACHE counts with
                                       BSEARCH */
/* Select the similarity kernel family used by SCAN_Q_RECOMPUTE and
 * SCAN_Q_BUILD_CACHE on this graph (SCAN_Q_PLAIN always uses BSEARCH without
 * pruning). SCAN_EINVAL for an unknown value. */
SCAN_API scan_status scan_graph_set_strategy(scan_graph *g, int32_t strategy);
SCAN_API int32_t scan_graph_strategy(const scan_graph *g);
/* Autotuner: times one full count of this graph with every kernel family
 * and a few work-item sizes of the forward schedule, keeps the fastest, and
 * appends the choice to the text file cache_path (NULL: not stored) under a
 * key of the graph's shape (log2 of n, nnz and the maximum degree). A later
 * call on a graph with the same key takes the stored choice without timing.
 * *strategy_out / *ms_out (may be NULL) receive the choice and its time.
 * Leaves no count cache behind unless the graph had one. Synchronous. */
SCAN_API scan_status scan_graph_autotune(scan_graph *g, const char *cache_path, int32_t *strategy_out,
                                         double *ms_out);

/* Query modes. */
#define SCAN_Q_AUTO 0x0u        /* use the count cache if present, else full recompute */
#define SCAN_Q_RECOMPUTE 0x1u   /* full recompute with degree pruning; ignore any cache */
#define SCAN_Q_PLAIN 0x2u       /* comparator path: per-edge binary-search intersection of every
                                   edge, no pruning, no cache (Algorithm 2's checkSim, exact) */
#define SCAN_Q_BUILD_CACHE 0x4u /* compute every edge's common count, keep it on the graph,
                                   then answer from it */

/*
 * One SCAN query. Requires 0 < eps_num <= eps_den and mu >= 2, else
 * SCAN_EINVAL. The result lives in library-owned host memory until
 * scan_result_free. Synchronous: returns when the result is on the host.
 */
SCAN_API scan_status scan_query(scan_graph *g, uint32_t eps_num, uint32_t eps_den, uint32_t mu, scan_result **out);
SCAN_API scan_status scan_query_ex(scan_graph *g, const scan_params *params, uint32_t mode, scan_result **out);

/*
 * Parameter sweep: k >= 1 queries (params[0..k-1], one mode for all) on one
 * graph, answered in order; outs[j] receives what scan_query_ex(g,
 * &params[j], mode, ...) would return (Definitions 2.1-2.6 at each (eps,
 * mu); the parameter study of Section 6 runs such sweeps). Each result's copy
 * to the host overlaps the next query's computation: the queries alternate
 * between the graph's output buffers and a second set of 6(n+1) + 8 nnz
 * bytes, allocated by the first sweep on the graph and kept (counted in
 * scan_graph_device_bytes) until scan_graph_free. When that set does not fit
 * the device or the budget, and for a partitioned graph, the queries run one
 * at a time. Every params[j] is checked first (SCAN_EINVAL, nothing run);
 * on any failure every result is freed and every outs[j] is NULL. The
 * results are the caller's (scan_result_free each). Synchronous; not to be
 * called concurrently with another query on the same graph.
 */
SCAN_API scan_status scan_query_sweep(scan_graph *g, const scan_params *params, int32_t k, uint32_t mode,
                                      scan_result **outs);

SCAN_API int32_t scan_result_n(const scan_result *r);
SCAN_API const uint8_t *scan_result_core(const scan_result *r);     /* [n] 1 = core */
SCAN_API const int32_t *scan_result_cluster(const scan_result *r);  /* [n] cluster id for cores, -1 otherwise */
SCAN_API const uint8_t *scan_result_label(const scan_result *r);    /* [n] SCAN_CORE/BORDER/HUB/OUTLIER */
SCAN_API int64_t scan_result_border_count(const scan_result *r);    /* k */
SCAN_API const int32_t *scan_result_border_pairs(const scan_result *r); /* [2k] (v, c) ascending by (v, c) */
/* Releases a result. Results of resident queries and of the server live in
 * page-locked host blocks that the library pools (up to 2 GiB of free blocks
 * are kept for reuse); freeing a result promptly returns its blocks. */
SCAN_API void scan_result_free(scan_result *r);

/*
 * Device-resident query: writes into caller-provided device buffers on the
 * context's stream and does not synchronise. Buffers: core uint8[n],
 * cid int32[n], label uint8[n], pairs int32[2 * pairs_cap], npairs int64[1]
 * (device). pairs_cap >= nnz always suffices (a non-core has fewer than mu-1
 * similar neighbours, so k <= nnz). If k > pairs_cap only the first
 * pairs_cap pairs are written and *npairs still holds k.
 */
typedef struct scan_device_out {
    uint8_t *core;
    int32_t *cid;
    uint8_t *label;
    int32_t *pairs;
    int64_t pairs_cap;
    int64_t *npairs;
} scan_device_out;

SCAN_API scan_status scan_query_device(scan_graph *g, const scan_params *params, uint32_t mode, const scan_device_out *out);

/* --------------------------------------------------------------- batch */
/*
 * Many independent graphs clustered together (each with its own eps, mu).
 * The k graphs are kept on the device as one disjoint union; since no edge
 * joins two graphs, one pass over the union answers all k queries, every
 * pipeline stage being a single launch over all of them. Each result equals
 * the single-graph result (ids local to its graph). Not in the paper: its
 * algorithms take one graph at a time (Algorithm 1).
 */
typedef struct scan_batch scan_batch;

/* Host CSRs of k graphs (n[j], offsets[j] int64[n[j]+1], adj[j] int32[...]),
 * each under scan_graph_load's contract; flags must be 0. The union must stay
 * below 2^31 vertices and 2^32 slots. Errors as scan_graph_load. */
SCAN_API scan_status scan_batch_load(scan_ctx *ctx, int32_t k, const int32_t *n, const int64_t *const *offsets,
                                     const int32_t *const *adj, uint32_t flags, scan_batch **out);
SCAN_API int32_t scan_batch_size(const scan_batch *b);
/* The resident union as a graph handle (owned by the batch; do not free). */
SCAN_API scan_graph *scan_batch_union(scan_batch *b);
/* params[k]: graph j's eps, mu. outs[k] receive one result per graph (each
 * freed with scan_result_free). On failure no result is returned. */
SCAN_API scan_status scan_batch_query(scan_batch *b, const scan_params *params, uint32_t mode, scan_result **outs);
/* The same answers as scan_batch_query, as ONE result over the k graphs in
 * batch order, with no per-graph host objects. Graph j owns the vertex range
 * [vertex_offsets[j], vertex_offsets[j+1]) of core, cluster and label (its
 * cluster ids are its own: the smallest core id of the cluster within graph
 * j, -1 for a non-core) and the pair range [pair_offsets[j],
 * pair_offsets[j+1]) of the border pairs (its own vertex and cluster ids,
 * sorted). vertex_offsets and pair_offsets are caller arrays of k + 1
 * entries. The result is the caller's (scan_result_free). */
SCAN_API scan_status scan_batch_query_packed(scan_batch *b, const scan_params *params, uint32_t mode,
                                             scan_result **out, int64_t *vertex_offsets, int64_t *pair_offsets);
/* Device-resident form: writes the union's result (union ids) into device
 * buffers sized for the union, on the context's stream, without syncing. */
SCAN_API scan_status scan_batch_query_device(scan_batch *b, const scan_params *params, uint32_t mode,
                                             const scan_device_out *out);
SCAN_API void scan_batch_free(scan_batch *b);
/* One-call form over graphs loaded separately in one context: builds a
 * temporary union, answers all k queries (full recompute) and frees it. */
SCAN_API scan_status scan_query_batch(scan_graph *const *gs, const scan_params *params, int32_t k, scan_result **outs);

/* ------------------------------------------------------------- serving */
/*
 * A query server over many resident graphs with continuous batching. Not in
 * the paper (it clusters one graph per run); its cached counts are the
 * numerators of Eq. 1 kept per edge across queries.
 *
 * Graphs are registered once (the server keeps a pinned host copy) and kept
 * on the device while memory allows. The first query on a graph computes
 * and keeps every edge's closed common count; later queries on it skip the
 * intersection. One worker thread owns the GPU: requests queue as they
 * arrive and are admitted into max_inflight slots (each with its own CUDA
 * stream) as slots and device memory free up, so queries on different
 * graphs overlap on the device; queries on one graph run one at a time.
 * Admission is by the context's device budget: idle graphs' count caches are
 * evicted first (least recently used), then idle graphs, which reload from
 * their host copy when next asked for. A request that can never fit fails
 * with SCAN_EBUSY. Every result equals the single-query result.
 *
 * While a server lives it owns its context: make no other calls on that
 * context or its graphs. submit / wait / poll / stats are thread-safe.
 */
typedef struct scan_server scan_server;
typedef struct scan_server_opts {
    int32_t max_inflight; /* concurrent requests on the device, 1..256 */
    int32_t use_cache;    /* 1: keep per-edge counts after a graph's first query; 0: recompute every query
                             with the graph's kernel family; 2: every query by the plain comparator path
                             (SCAN_Q_PLAIN: binary-search counts of every edge, no pruning, no cache) */
} scan_server_opts;
typedef struct scan_server_report {
    uint64_t completed, rejected;
    double p50_ms, p99_ms, mean_ms; /* latency = completion - submission (queueing included) */
    double throughput_rps;          /* completed / (last completion - first submission) */
    uint64_t cache_builds, cache_evictions, graph_loads, graph_evictions;
    int32_t max_inflight;           /* most requests seen in flight at once */
    uint64_t device_bytes;          /* context bytes in use */
} scan_server_report;

SCAN_API scan_status scan_server_create(scan_ctx *ctx, const scan_server_opts *opts, scan_server **out);
/* Register a host CSR (copied; same contract as scan_graph_load, validated
 * on its first load). Only while the server is idle; returns its id. */
SCAN_API scan_status scan_server_add_graph(scan_server *srv, int32_t n, const int64_t *offsets, const int32_t *adj,
                                           int64_t nnz, int32_t *graph_id);
/* Queue one query; returns at once with a ticket. SCAN_EINVAL for bad
 * parameters or an unknown graph id. */
SCAN_API scan_status scan_server_submit(scan_server *srv, int32_t graph_id, const scan_params *params,
                                        uint64_t *ticket);
/* Block until the ticket's query finishes; its status is returned and, on
 * success, its result (free with scan_result_free). latency_ms may be NULL.
 * Each ticket can be taken once. */
SCAN_API scan_status scan_server_wait(scan_server *srv, uint64_t ticket, scan_result **out, double *latency_ms);
/* Non-blocking: *ready = 0 if still running, else as scan_server_wait. */
SCAN_API scan_status scan_server_poll(scan_server *srv, uint64_t ticket, scan_result **out, double *latency_ms,
                                      int32_t *ready);
SCAN_API scan_status scan_server_stats(scan_server *srv, scan_server_report *stats);
SCAN_API scan_status scan_server_reset_stats(scan_server *srv);
/* Finishes queued and running requests, then frees everything it holds. */
SCAN_API void scan_server_destroy(scan_server *srv);

/* ----------------------------------------------- no-allocation counting */
/*
 * Closed common counts |N[u] cap N[v]| for every slot of a caller's device
 * CSR, with no memory allocation of any kind. The paper has no counterpart;
 * this exists for callers that cannot allocate device memory -- code that
 * runs inside another framework's memory pool or under a hard memory budget,
 * or at a point where a cudaMalloc/cudaFree (which can synchronise the whole
 * device) is not allowed.
 *
 * offsets int64[n+1], adj int32[nnz] and cn int32[nnz] are device pointers
 * owned by the caller; the CSR must meet scan_graph_load's contract (checked;
 * SCAN_EINVAL names the first bad slot). cn[s] receives the count of the
 * slot s, as scan_graph_copy_counts would return it. Runs on `stream` (a
 * cudaStream_t, NULL = legacy default stream) on the current device and
 * returns when the counts are written (it synchronises that stream).
 *
 * Working memory is one fixed 64 MiB __device__ array inside the library
 * (held by every GPU that loads it until the process exits): graphs need
 * 4(n+1) + 8 nnz bytes plus alignment of it, about n + 2 nnz <= 16.7M
 * entries; larger graphs get SCAN_EINVAL before any device work. Every call
 * looks up that array's device address on the current device (no state is
 * cached across calls, so a device reset leaves nothing stale). The call
 * synchronises `stream` and copies an error word to the host, so it must
 * never be called while that stream is being captured into a CUDA graph.
 * The array lies outside any context's budget_bytes accounting. All calls
 * share the one array and it keeps the last call's contents, so calls that
 * overlap on the GPU (other threads, other streams) race: serialise them.
 */
SCAN_API scan_status scan_common_counts_static(const int64_t *offsets, const int32_t *adj, int32_t n, int64_t nnz,
                                               int32_t *cn, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SCAN_H */

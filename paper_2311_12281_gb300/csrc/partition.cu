// partition.cu -- SCAN of a graph larger than the device budget (Section 5's
// out-of-core setting): the CSR stays in the caller's pinned host memory and
// is streamed in contiguous row blocks; only per-vertex state and one
// similarity bit per slot stay on the device.
//
// By Lemma 5.1 the similarity of an edge needs only the rows of its two
// endpoints, so every edge (u, v), u < v, is decided while the blocks of u
// and v are resident: the blocks are visited in pairs (i <= j), block i held
// while the blocks j stream past it (the next one copied on a side stream
// while the current pair computes). Then three more streams over the blocks
// form clusters (union-find over core-core similar edges), border
// memberships, and hub / outlier labels. The paper's own design streams
// edge-extended subgraphs built by a CPU partitioner (Algorithm 5); row
// blocks need no preprocessing and are read sequentially.
#include <algorithm>
#include <cstring>
#include <vector>

#include "scan_internal.cuh"

namespace scan {

struct Block {
    int32_t v0, v1;  // vertex range
    int64_t e0, e1;  // slot range
};

struct Part {
    const int64_t *h_off = nullptr;
    const int32_t *h_adj = nullptr;
    bool reg_off = false, reg_adj = false;
    std::vector<Block> blocks;
    int32_t max_rows = 0;
    int64_t max_slots = 0;
    // device state (all vertices)
    DevBuf ecnt, core, parent, cid, mfirst, mmulti, sbits, err;
    // block slots: [0] holds block i, [1], [2] alternate for block j
    DevBuf boff[3], badj[3];
    int loaded[3] = {-1, -1, -1};
    bool pending[3] = {false, false, false};  // copied on the side stream; compute has not waited yet
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copied[3] = {nullptr, nullptr, nullptr};
    uint64_t h2d_bytes = 0;  // block copies issued since the load
    // zero-copy mode: block slots 1 and 2 (the streamed partner and single
    // blocks) are read by the kernels straight from the pinned host CSR
    // through these device-side addresses, with no copy
    bool zero_copy = false;
    const int64_t *d_hoff = nullptr;
    const int32_t *d_hadj = nullptr;
};

namespace {

constexpr int kChunkEdges = 64;     // edges per chunk of a light row
constexpr int kChunkWork = 4096;    // a row of degree d gets chunks of max(1, kChunkWork / d) edges

__device__ __forceinline__ int32_t chunk_edges(int32_t du) {
    return max(1, min(kChunkEdges, kChunkWork / max(du, 1)));
}
constexpr int kUfLimitP = 1 << 22;

inline __device__ bool sbit(const uint32_t *bits, int64_t s) { return (bits[s >> 5] >> (s & 31)) & 1u; }
inline __device__ void sbit_set(uint32_t *bits, int64_t s) { atomicOr(bits + (s >> 5), 1u << (s & 31)); }

// ------------------------------------------------------------ validation
// thread per row of a block: ascending, in range, no self-loop; counts the
// entries above and below their row (equal totals + mirror lookups = symmetric)
__global__ void k_p_check(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t v0, int32_t rows,
                          int64_t e0, int32_t n, unsigned long long *updown, unsigned long long *bad) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t u = v0 + (int32_t)r;
    unsigned long long up = 0, down = 0;
    for (int64_t s = off[r]; s < off[r + 1]; ++s) {
        const int32_t v = adj[s - e0];
        bool ok = v >= 0 && v < n && v != u;
        if (ok && s > off[r]) ok = adj[s - 1 - e0] < v;
        if (!ok) atomicMin(bad, (unsigned long long)s);
        if (v > u) ++up;
        else ++down;
    }
    atomicAdd(updown + 0, up);
    atomicAdd(updown + 1, down);
}

// ------------------------------------------------------------ pass 1
// per row of block i: the chunks of edges (u, v) with v in block j and v > u
__global__ void k_p_range(const int64_t *__restrict__ offi, const int32_t *__restrict__ adji, int32_t v0i,
                          int32_t rows_i, int64_t e0i, int32_t v0j, int32_t v1j, int32_t *__restrict__ nchunks,
                          int32_t *__restrict__ ra, int32_t *__restrict__ rb) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows_i) return;
    const int32_t u = v0i + (int32_t)r;
    const int32_t *row = adji + (offi[r] - e0i);
    const int32_t len = (int32_t)(offi[r + 1] - offi[r]);
    const int32_t lo = max(v0j, u + 1);
    int32_t l = 0, h = len;
    for (int it = 0; it < 40 && l < h; ++it) {  // first id >= lo
        const int32_t mid = (l + h) >> 1;
        if (row[mid] < lo) l = mid + 1;
        else h = mid;
    }
    const int32_t a = l;
    h = len;
    for (int it = 0; it < 40 && l < h; ++it) {  // first id >= v1j
        const int32_t mid = (l + h) >> 1;
        if (row[mid] < v1j) l = mid + 1;
        else h = mid;
    }
    const int32_t b = max(a, l);
    ra[r] = a;
    rb[r] = b;
    const int32_t ce = chunk_edges(len);
    nchunks[r] = (b - a + ce - 1) / ce;
}

struct Chunk {
    int32_t r, a, b;
};

__global__ void k_p_chunks(const int64_t *__restrict__ offi, const int32_t *__restrict__ ra,
                           const int32_t *__restrict__ rb, const int64_t *__restrict__ pos, int32_t rows_i,
                           Chunk *__restrict__ chunks) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows_i) return;
    int64_t p = pos[r];
    const int32_t ce = chunk_edges((int32_t)(offi[r + 1] - offi[r]));
    for (int32_t a = ra[r]; a < rb[r]; a += ce) chunks[p++] = Chunk{(int32_t)r, a, min(rb[r], a + ce)};
}

// warp per chunk: closed common count of each edge, exact eps-test, both
// slots' similarity bits and both endpoints' eps-degrees
__global__ void __launch_bounds__(256) k_p_similar(const Chunk *__restrict__ chunks,
                                                   const int64_t *__restrict__ nchunks_dev,
                                                   const int64_t *__restrict__ offi, const int32_t *__restrict__ adji,
                                                   int32_t v0i, int64_t e0i, const int64_t *__restrict__ offj,
                                                   const int32_t *__restrict__ adjj, int32_t v0j, int64_t e0j,
                                                   uint64_t pp, uint64_t qq, uint32_t *__restrict__ bits,
                                                   int32_t *__restrict__ ecnt, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t nchunks = *nchunks_dev;
    for (int64_t ci = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ci < nchunks; ci += warps) {
        const Chunk ch = chunks[ci];
        const int32_t u = v0i + ch.r;
        const int32_t *ru = adji + (offi[ch.r] - e0i);
        const int32_t du = (int32_t)(offi[ch.r + 1] - offi[ch.r]);
        for (int32_t k = ch.a; k < ch.b; ++k) {
            const int32_t v = ru[k];
            const int32_t rv_i = v - v0j;
            const int32_t *rv = adjj + (offj[rv_i] - e0j);
            const int32_t dv = (int32_t)(offj[rv_i + 1] - offj[rv_i]);
            // degree-only outcomes first: no intersection when they decide
            const uint64_t a1 = (uint64_t)du + 1, b1 = (uint64_t)dv + 1;
            const bool never = dev::prune_dissimilar(a1 < b1 ? a1 : b1, a1 < b1 ? b1 : a1, pp, qq);
            const bool always = !never && dev::prune_similar(a1, b1, pp, qq);
            int c = 0;
            if (!never && !always)  // rows of similar length merged, else the shorter probed in the longer
                c = dev::warp_common(ru, du, rv, dv) + 2;
            // mirror slot: position of u in row v, looked up for every edge (its
            // absence means an asymmetric input). The warp narrows the range 32
            // pivots at a time, then checks the last 32 positions at once.
            int32_t lo = 0, hi = dv;
            for (int it = 0; it < 8 && hi - lo > kWarp; ++it) {
                const int32_t step = (hi - lo + kWarp - 1) / kWarp;
                const int32_t p = lo + lane * step;
                const unsigned le = __ballot_sync(0xffffffffu, p < hi && rv[p] <= u);
                if (le == 0) {
                    hi = lo;  // u below the row's first id
                    break;
                }
                lo += (31 - __clz(le)) * step;
                hi = min(hi, lo + step);
            }
            const unsigned em = __ballot_sync(0xffffffffu, lo + lane < hi && rv[lo + lane] == u);
            const int32_t pos = em ? lo + __ffs(em) - 1 : -1;
            if (lane == 0) {
                if (pos < 0) {
                    atomicOr(err, ERR_LOOP_LIMIT);
                } else if (!never && (always || dev::eps_similar((uint64_t)c, a1, b1, pp, qq))) {
                    sbit_set(bits, offi[ch.r] + k);
                    sbit_set(bits, offj[rv_i] + pos);
                    atomicAdd(ecnt + u, 1);
                    atomicAdd(ecnt + v, 1);
                }
            }
        }
    }
}

__global__ void k_p_core(const int32_t *__restrict__ ecnt, int32_t n, uint32_t mu, uint8_t *__restrict__ core,
                         int32_t *__restrict__ parent) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const bool c = (uint32_t)ecnt[v] + 1u >= mu;  // u itself: sigma(u, u) = 1
    core[v] = c;
    parent[v] = c ? (int32_t)v : -1;
}

// ------------------------------------------------------------ pass 2
__device__ int32_t p_find(int32_t *parent, int32_t x, uint32_t *err, int limit) {
    for (int it = 0; it < limit; ++it) {
        const int32_t p = ((volatile int32_t *)parent)[x];
        if (p == x) return x;
        const int32_t gp = ((volatile int32_t *)parent)[p];
        if (gp != p) ((volatile int32_t *)parent)[x] = gp;
        x = gp;
    }
    atomicOr(err, ERR_FIND_LIMIT);
    return x;
}

__device__ void p_unite(int32_t *parent, int32_t a, int32_t b, uint32_t *err, int limit) {
    for (int it = 0; it < limit; ++it) {
        a = p_find(parent, a, err, limit);
        b = p_find(parent, b, err, limit);
        if (a == b) return;
        if (a > b) { const int32_t t = a; a = b; b = t; }
        if (atomicCAS(parent + b, b, a) == b) return;
    }
    atomicOr(err, ERR_UF_LIMIT);
}

// warp per row of the block: core-core similar edges with v > u join
__global__ void k_p_hook(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t v0, int32_t rows,
                         int64_t e0, const uint32_t *__restrict__ bits, const uint8_t *__restrict__ core,
                         int32_t *parent, uint32_t *err, int limit) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int32_t u = v0 + (int32_t)r;
    if (!core[u]) return;
    for (int64_t s = off[r] + lane; s < off[r + 1]; s += 32) {
        const int32_t v = adj[s - e0];
        if (v > u && sbit(bits, s) && core[v]) p_unite(parent, u, v, err, limit);
    }
}

// cid into its own array: writing roots back into parent would race with the
// path halving of concurrent finds (which may store a non-root ancestor over
// a root written a moment earlier)
__global__ void k_p_final(const uint8_t *__restrict__ core, int32_t n, int32_t *parent, int32_t *__restrict__ cid,
                          uint32_t *err, int limit) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    cid[v] = core[v] ? p_find(parent, (int32_t)v, err, limit) : -1;
}

// ------------------------------------------------------------ pass 3
// warp per non-core row: sorted unique clusters of its similar core
// neighbours (< mu - 1 of them), first id + "more than one" flag, and the
// (v, c) pairs into the block's output at pos[r]
__global__ void k_p_border_count(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t v0,
                                 int32_t rows, int64_t e0, const uint32_t *__restrict__ bits,
                                 const uint8_t *__restrict__ core, int32_t *__restrict__ cnt) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int32_t v = v0 + (int32_t)r;
    int c = 0;
    if (!core[v])
        for (int64_t s = off[r] + lane; s < off[r + 1]; s += 32) c += (sbit(bits, s) && core[adj[s - e0]]) ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[r] = c;
}

__global__ void k_p_border_fill(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t v0,
                                int32_t rows, int64_t e0, const uint32_t *__restrict__ bits,
                                const uint8_t *__restrict__ core, const int32_t *__restrict__ cid,
                                const int64_t *__restrict__ pos, int32_t *__restrict__ raw, int32_t *__restrict__ ucnt,
                                int32_t *__restrict__ mfirst, uint8_t *__restrict__ mmulti) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int32_t v = v0 + (int32_t)r;
    const int64_t base = pos[r], k = pos[r + 1] - base;
    if (k == 0) {
        if (lane == 0) { ucnt[r] = 0; mfirst[v] = -1; mmulti[v] = 0; }
        return;
    }
    int64_t w = base;
    for (int64_t s0 = off[r]; s0 < off[r + 1]; s0 += 32) {
        const int64_t s = s0 + lane;
        bool f = false;
        int32_t x = -1;
        if (s < off[r + 1] && sbit(bits, s)) {
            const int32_t u = adj[s - e0];
            if (core[u]) { f = true; x = cid[u]; }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, f);
        if (f) raw[w + __popc(mask & ((1u << lane) - 1u))] = x;
        w += __popc(mask);
    }
    __syncwarp();
    if (lane == 0) {
        int32_t *a = raw + base;
        for (int64_t i = 1; i < k; ++i) {
            const int32_t t = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > t) { a[j + 1] = a[j]; --j; }
            a[j + 1] = t;
        }
        int64_t uq = 1;
        for (int64_t i = 1; i < k; ++i)
            if (a[i] != a[uq - 1]) a[uq++] = a[i];
        ucnt[r] = (int32_t)uq;
        mfirst[v] = a[0];
        mmulti[v] = uq > 1;
    }
}

__global__ void k_p_border_emit(const int64_t *__restrict__ pos, const int32_t *__restrict__ raw,
                                const int32_t *__restrict__ ucnt, const int64_t *__restrict__ ppos, int32_t v0,
                                int32_t rows, int32_t *__restrict__ pairs) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int32_t i = 0; i < ucnt[r]; ++i) {
        pairs[2 * (ppos[r] + i)] = v0 + (int32_t)r;
        pairs[2 * (ppos[r] + i) + 1] = raw[pos[r] + i];
    }
}

__global__ void k_p_label(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t v0, int32_t rows,
                          int64_t e0, const uint8_t *__restrict__ core, const int32_t *__restrict__ cid,
                          const int32_t *__restrict__ mfirst, const uint8_t *__restrict__ mmulti,
                          uint8_t *__restrict__ label) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int32_t u = v0 + (int32_t)r;
    if (core[u]) { if (lane == 0) label[u] = SCAN_CORE; return; }
    if (mfirst[u] >= 0) { if (lane == 0) label[u] = SCAN_BORDER; return; }
    int32_t lo = INT32_MAX, hi = -1;
    bool multi = false;
    for (int64_t s0 = off[r]; s0 < off[r + 1]; s0 += 32) {
        const int64_t s = s0 + lane;
        if (s < off[r + 1]) {
            const int32_t w = adj[s - e0];
            int32_t id = -1;
            if (core[w]) id = cid[w];
            else if (mfirst[w] >= 0) { id = mfirst[w]; multi |= mmulti[w] != 0; }
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

// ------------------------------------------------------------ host driver
// Copies block bi into a slot. async: on the side stream, after the slot's
// previous user (the event recorded on the compute stream after its last
// kernel) -- the compute stream waits for the copy only when it first uses
// the slot (use_block), so the copy overlaps the kernels issued in between.
static scan_status load_block(Graph *g, int slot, int bi, bool async) {
    Part *P = g->part;
    Ctx *c = g->ctx;
    if (P->loaded[slot] == bi) return SCAN_OK;
    if (P->zero_copy && slot != 0) {  // read in place through the host link
        P->loaded[slot] = bi;
        P->pending[slot] = false;
        return SCAN_OK;
    }
    const Block &B = P->blocks[(size_t)bi];
    const int32_t rows = B.v1 - B.v0;
    cudaStream_t st = async ? P->copy_stream : c->stream;
    if (async) SCAN_CUDA(cudaStreamWaitEvent(P->copy_stream, P->copied[slot], 0));  // previous user finished
    SCAN_CUDA(cudaMemcpyAsync(P->boff[slot].ptr, P->h_off + B.v0, 8 * ((size_t)rows + 1), cudaMemcpyHostToDevice, st));
    if (B.e1 > B.e0)
        SCAN_CUDA(cudaMemcpyAsync(P->badj[slot].ptr, P->h_adj + B.e0, 4 * (size_t)(B.e1 - B.e0),
                                  cudaMemcpyHostToDevice, st));
    P->h2d_bytes += 8 * ((uint64_t)rows + 1) + 4 * (uint64_t)(B.e1 - B.e0);
    SCAN_CUDA(cudaEventRecord(P->copied[slot], st));
    P->loaded[slot] = bi;
    P->pending[slot] = async;
    return SCAN_OK;
}

// Makes block bi resident in the slot for the compute stream.
static scan_status use_block(Graph *g, int slot, int bi) {
    Part *P = g->part;
    SCAN_TRY(load_block(g, slot, bi, true));
    if (P->pending[slot]) {
        SCAN_CUDA(cudaStreamWaitEvent(g->ctx->stream, P->copied[slot], 0));
        P->pending[slot] = false;
    }
    return SCAN_OK;
}

// The offsets and ids of the block in a slot, as the kernels address them
// (offsets global, ids from the block's first slot): the slot's device copy,
// or in zero-copy mode the host CSR itself.
static const int64_t *slot_off(const Part *P, int slot) {
    if (P->zero_copy && slot != 0) return P->d_hoff + P->blocks[(size_t)P->loaded[slot]].v0;
    return (const int64_t *)P->boff[slot].ptr;
}

static const int32_t *slot_adj(const Part *P, int slot) {
    if (P->zero_copy && slot != 0) return P->d_hadj + P->blocks[(size_t)P->loaded[slot]].e0;
    return (const int32_t *)P->badj[slot].ptr;
}

// Marks the end of the compute stream's use of a slot.
static scan_status release_slot(Graph *g, int slot) {
    SCAN_CUDA(cudaEventRecord(g->part->copied[slot], g->ctx->stream));
    return SCAN_OK;
}

int32_t part_block_count(const Graph *g) { return g->part ? (int32_t)g->part->blocks.size() : 0; }

uint64_t part_transfer_bytes(const Graph *g) { return g->part ? g->part->h2d_bytes : 0; }

// ------------------------------------------------------------ the paper's partitioner
// Section 5's edge extended subgraphs, planned on the host as Algorithm 5
// does (its CPU part): the undirected edges (u, v), u < v, are taken in CSR
// order into the current subgraph G_s together with every edge incident to
// them (the rows of u and v); when Memof(G_s) + Memof(G'_s) + 15 |V(G)| would
// exceed the device memory, G_s is closed and a new one started. Memof(G) =
// 25 |E(G)| + 4 |V(G)| (the paper's CSR-enhanced layout). The subgraph's
// edges are the union of the rows of the endpoints taken (`inrow`), its
// vertices those rows' endpoints (`touched`); both are cleared through the
// lists of what was marked, so a subgraph costs only what it holds.
scan_status plan_edge_extended(int32_t n, const int64_t *off, const int32_t *adj, int64_t nnz, uint64_t mem,
                               int64_t *subgraphs, uint64_t *bytes) {
    std::vector<uint8_t> inrow((size_t)n, 0), touched((size_t)n, 0);
    std::vector<int32_t> rows, verts;
    const double fixed = 15.0 * (double)n;
    double es = 0, vs = 0;  // edges and vertices of the current subgraph
    int64_t k = 0;
    double total = 0;
    auto close = [&]() {
        if (es == 0 && vs == 0) return;
        total += 25.0 * es + 4.0 * vs;
        ++k;
        for (int32_t x : rows) inrow[(size_t)x] = 0;
        for (int32_t x : verts) touched[(size_t)x] = 0;
        rows.clear();
        verts.clear();
        es = vs = 0;
    };
    auto take = [&](int32_t x) {
        if (inrow[(size_t)x]) return;
        for (int64_t s = off[x]; s < off[x + 1]; ++s) {
            const int32_t y = adj[s];
            if (!inrow[(size_t)y]) es += 1;
            if (!touched[(size_t)y]) {
                touched[(size_t)y] = 1;
                verts.push_back(y);
                vs += 1;
            }
        }
        if (!touched[(size_t)x]) {
            touched[(size_t)x] = 1;
            verts.push_back(x);
            vs += 1;
        }
        inrow[(size_t)x] = 1;
        rows.push_back(x);
    };
    for (int32_t u = 0; u < n; ++u) {
        for (int64_t s = off[u]; s < off[u + 1]; ++s) {
            const int32_t v = adj[s];
            if (v <= u) continue;
            if (inrow[(size_t)u] && inrow[(size_t)v]) continue;
            // G'_s: take both rows, and if the subgraph no longer fits, undo
            // them, close it, and take them into a new one
            const size_t nr = rows.size(), nv = verts.size();
            const double es0 = es, vs0 = vs;
            take(u);
            take(v);
            const bool grew = es > es0 || vs > vs0;  // nothing new: the subgraph already holds G'_s
            if (grew && 25.0 * es + 4.0 * vs + fixed > (double)mem && (es0 > 0 || vs0 > 0)) {
                for (size_t i = nr; i < rows.size(); ++i) inrow[(size_t)rows[i]] = 0;
                for (size_t i = nv; i < verts.size(); ++i) touched[(size_t)verts[i]] = 0;
                rows.resize(nr);
                verts.resize(nv);
                es = es0;
                vs = vs0;
                close();
                take(u);
                take(v);
            }
        }
    }
    close();
    (void)nnz;
    *subgraphs = k;
    *bytes = (uint64_t)total;
    return SCAN_OK;
}

// Plan of triangle enumeration over block pairs out of core (host only).
// For a triangle a < b < c in (deg, id) rank, found at its middle vertex b,
// the three counts lie in out(a) and out(b) (Section 4.1's degree-oriented
// lists), so the pair (block of a, block of b) needs only those two blocks'
// out-lists and counts; with blocks cut in rank order a < b puts block(a) <=
// block(b). The device keeps the per-vertex state (19 B per vertex, as the
// row-block driver) and one similarity bit per slot; three block slots (the
// resident block, the streamed one and its prefetch) share 90 % of the rest.
// A block holds whole out-lists: 8 B per oriented edge (id, count) and 12 B
// per row. The bytes are those of each block loaded (ids and counts in) and
// unloaded (counts out) once as the resident block and once for every later
// pair (i < j) that holds an oriented edge from block i to block j.
scan_status plan_triangle_blocks(int32_t n, const int64_t *off, const int32_t *adj, int64_t nnz, uint64_t mem,
                                 int32_t *blocks, int64_t *pairs, uint64_t *bytes) {
    *blocks = 0;
    *pairs = 0;
    *bytes = 0;
    if (n == 0) return SCAN_OK;
    const uint64_t state = 19ull * ((uint64_t)n + 1) + (uint64_t)nnz / 8 + 16;
    if (mem <= state) {
        set_error("device_bytes does not hold the per-vertex state");
        return SCAN_EBUDGET;
    }
    const double cap = 0.9 * (double)(mem - state) / 3.0;
    // rank order (deg, id): a counting sort by degree keeps ids ascending within a degree
    std::vector<int64_t> start((size_t)n + 2, 0);
    // degrees are at most n - 1 in a simple graph; larger ones share the last bucket
    for (int32_t v = 0; v < n; ++v) ++start[(size_t)std::min<int64_t>(off[v + 1] - off[v], n) + 1];
    for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
    std::vector<int32_t> order((size_t)n);
    {
        std::vector<int64_t> cur(start.begin(), start.end() - 1);
        for (int32_t v = 0; v < n; ++v) {
            const size_t d = (size_t)std::min<int64_t>(off[v + 1] - off[v], n);
            order[(size_t)cur[d]++] = v;
        }
    }
    auto above = [&](int32_t x, int32_t y) {  // y ranks above x
        const int64_t dx = off[x + 1] - off[x], dy = off[y + 1] - off[y];
        return dy > dx || (dy == dx && y > x);
    };
    std::vector<int32_t> blk((size_t)n, 0);
    std::vector<int64_t> bedges, brows;
    double used = 0;
    int64_t e_cur = 0, r_cur = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t v = order[(size_t)i];
        int64_t dp = 0;
        for (int64_t s = off[v]; s < off[v + 1]; ++s) dp += above(v, adj[s]) ? 1 : 0;
        const double row = 12.0 + 8.0 * (double)dp;
        if (row > cap) {
            set_error("an out-list of " + std::to_string(dp) + " ids does not fit a block slot");
            return SCAN_EBUDGET;
        }
        if (used + row > cap && r_cur > 0) {
            bedges.push_back(e_cur);
            brows.push_back(r_cur);
            used = 0;
            e_cur = r_cur = 0;
        }
        blk[(size_t)v] = (int32_t)bedges.size();
        used += row;
        e_cur += dp;
        ++r_cur;
    }
    bedges.push_back(e_cur);
    brows.push_back(r_cur);
    const int64_t P = (int64_t)bedges.size();
    if (P > 8192) {
        set_error("more than 8192 blocks: device_bytes is too small for this graph");
        return SCAN_EBUDGET;
    }
    std::vector<uint8_t> work((size_t)(P * P), 0);
    for (int32_t a = 0; a < n; ++a)
        for (int64_t s = off[a]; s < off[a + 1]; ++s)
            if (above(a, adj[s])) work[(size_t)(blk[(size_t)a] * P + blk[(size_t)adj[s]])] = 1;
    auto moved = [&](int64_t j) { return 12ull * (uint64_t)brows[(size_t)j] + 12ull * (uint64_t)bedges[(size_t)j]; };
    uint64_t total = 0;
    int64_t np = 0;
    for (int64_t i = 0; i < P; ++i) {
        total += moved(i);
        for (int64_t j = i; j < P; ++j) {
            if (!work[(size_t)(i * P + j)]) continue;
            ++np;
            if (j > i) total += moved(j);
        }
    }
    *blocks = (int32_t)P;
    *pairs = np;
    *bytes = total;
    return SCAN_OK;
}

scan_status part_set_zero_copy(Graph *g, bool on) {
    Part *P = g->part;
    Ctx *c = g->ctx;
    SCAN_CUDA(cudaSetDevice(c->device));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    SCAN_CUDA(cudaStreamSynchronize(P->copy_stream));
    if (on && g->n > 0 && !P->d_hoff) {
        void *po = nullptr, *pa = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&po, (void *)P->h_off, 0);
        if (e == cudaSuccess && g->nnz > 0) e = cudaHostGetDevicePointer(&pa, (void *)P->h_adj, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("the host CSR is not mapped for device access (pinned, mapped memory is needed)");
            return SCAN_ECUDA;
        }
        P->d_hoff = (const int64_t *)po;
        P->d_hadj = (const int32_t *)pa;
    }
    P->zero_copy = on && g->n > 0;
    for (int k = 1; k < 3; ++k) {  // nothing is resident in the streamed slots any more
        P->loaded[k] = -1;
        P->pending[k] = false;
    }
    return SCAN_OK;
}

void part_release(Graph *g) {
    Part *P = g->part;
    if (!P) return;
    Ctx *c = g->ctx;
    DevBuf *bufs[] = {&P->ecnt, &P->core, &P->parent, &P->cid, &P->mfirst, &P->mmulti, &P->sbits, &P->err,
                      &P->boff[0], &P->boff[1], &P->boff[2], &P->badj[0], &P->badj[1], &P->badj[2]};
    for (DevBuf *b : bufs) dev_free(c, *b);
    if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
    for (auto &e : P->copied)
        if (e) cudaEventDestroy(e);
    if (P->reg_off) cudaHostUnregister((void *)P->h_off);
    if (P->reg_adj) cudaHostUnregister((void *)P->h_adj);
    delete P;
    g->part = nullptr;
}

scan_status part_create(Ctx *ctx, int32_t n, const int64_t *offsets, const int32_t *adj, int64_t nnz, Graph **out,
                        int64_t block_slots_hint) {
    *out = nullptr;
    if (n < 0 || nnz < 0 || (n > 0 && !offsets) || (nnz > 0 && !adj) || nnz % 2) {
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
    SCAN_CUDA(cudaSetDevice(ctx->device));
    scan_graph *sg = new scan_graph();
    Graph *g = sg;
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    g->part = new Part();
    Part *P = g->part;
    P->h_off = offsets;
    P->h_adj = adj;
    auto fail = [&](scan_status s) {
        part_release(g);
        delete sg;
        return s;
    };
    // pin the caller's arrays unless they already are; where the driver
    // refuses (e.g. a range sharing pages with another registration) the
    // copies still work from pageable memory, only without overlap
    auto pin = [](const void *p, size_t bytes) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) return false;
        cudaGetLastError();
        if (cudaHostRegister((void *)p, bytes, cudaHostRegisterReadOnly | cudaHostRegisterMapped) == cudaSuccess)
            return true;
        cudaGetLastError();
        if (cudaHostRegister((void *)p, bytes, cudaHostRegisterMapped) == cudaSuccess) return true;
        cudaGetLastError();
        if (cudaHostRegister((void *)p, bytes, cudaHostRegisterDefault) == cudaSuccess) return true;
        cudaGetLastError();
        return false;
    };
    if (n > 0) P->reg_off = pin(offsets, 8 * ((size_t)n + 1));
    if (nnz > 0) P->reg_adj = pin(adj, 4 * (size_t)nnz);
    // device-resident per-vertex state: eps-degree, core flag, union-find
    // parent, cluster id, first membership, "more than one membership" flag
    // and the label (20 B per vertex); one similarity bit per slot
    const size_t N1 = (size_t)n + 1;
    scan_status s = dev_alloc(ctx, P->ecnt, 4 * N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->core, N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->parent, 4 * N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->cid, 4 * N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->mfirst, 4 * N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->mmulti, N1);
    if (s == SCAN_OK) s = dev_alloc(ctx, P->sbits, 4 * ((size_t)nnz / 32 + 1));
    if (s == SCAN_OK) s = dev_alloc(ctx, P->err, 16);
    if (s == SCAN_OK) s = dev_alloc(ctx, g->label, N1);
    if (s != SCAN_OK) return fail(s);
    // Blocks from what is left of the budget. The block-sized device memory
    // is three block slots (8 B per row offset, 4 B per slot), the per-row
    // scratch (24 B), the pass-1 chunks (12 B per row and per slot) and the
    // border candidates and pairs of pass 3 (12 B per slot): 60 B per row and
    // 36 B per slot of the largest block. Rows go into a block while it stays
    // within 90 % of that; the plan shrinks until the largest block's rows
    // and slots together fit (a single row longer than that forms a block
    // alone, and its load fails with SCAN_EBUDGET if it cannot fit at all).
    const uint64_t avail = ctx->budget ? (ctx->budget > ctx->used ? ctx->budget - ctx->used : 0)
                                       : (uint64_t)4 << 30;
    auto plan = [&](double cap_bytes, int64_t cap_slots) {
        P->blocks.clear();
        P->max_rows = 0;
        P->max_slots = 0;
        for (int32_t v = 0; v < n;) {
            Block B;
            B.v0 = v;
            B.e0 = offsets[v];
            int32_t w = v;
            while (w < n) {
                const int64_t rows = (int64_t)w + 1 - v, slots = offsets[w + 1] - B.e0;
                const bool fits = cap_slots > 0 ? slots <= cap_slots : 60.0 * rows + 36.0 * slots <= cap_bytes;
                if (!fits && w > v) break;
                ++w;
            }
            B.v1 = w;
            B.e1 = offsets[w];
            P->blocks.push_back(B);
            P->max_rows = std::max(P->max_rows, B.v1 - B.v0);
            P->max_slots = std::max(P->max_slots, B.e1 - B.e0);
            v = w;
        }
    };
    if (block_slots_hint > 0) {
        plan(0.0, block_slots_hint);
    } else {
        double cap = 0.9 * (double)avail;
        for (int attempt = 0; attempt < 16; ++attempt) {
            plan(cap, 0);
            if (60.0 * (double)P->max_rows + 36.0 * (double)P->max_slots <= 0.95 * (double)avail) break;
            cap *= 0.85;
        }
    }
    for (int k = 0; k < 3 && s == SCAN_OK; ++k) {
        s = dev_alloc(ctx, P->boff[k], 8 * ((size_t)P->max_rows + 1));
        if (s == SCAN_OK) s = dev_alloc(ctx, P->badj[k], 4 * (size_t)std::max<int64_t>(P->max_slots, 1));
    }
    // per-block scratch on the graph's ordinary query buffers
    const size_t R1 = (size_t)P->max_rows + 1;
    if (s == SCAN_OK) s = dev_alloc(ctx, g->cnt, 4 * R1);       // chunk counts / border counts
    if (s == SCAN_OK) s = dev_alloc(ctx, g->cnt_off, 8 * R1);   // their offsets
    if (s == SCAN_OK) s = dev_alloc(ctx, g->ucnt, 4 * R1);      // row range starts / unique counts
    if (s == SCAN_OK) s = dev_alloc(ctx, g->pair_off, 8 * R1);  // row range ends (int32 view) / pair offsets
    // chunks: at most one per row plus one per kChunkEdges slots of light rows,
    // or per slot of the heaviest rows
    if (s == SCAN_OK) s = dev_alloc(ctx, g->src, sizeof(Chunk) * ((size_t)P->max_rows + P->max_slots + 2));
    if (s == SCAN_OK) s = dev_alloc(ctx, g->npairs, 8);
    if (s != SCAN_OK) return fail(s);
    if (cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "copy stream"));
    for (auto &e : P->copied)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "copy events"));
    cudaStream_t st = ctx->stream;
    // validation, one stream over the blocks
    DevBuf chk;
    if (dev_alloc(ctx, chk, 32) != SCAN_OK) return fail(SCAN_EBUDGET);
    unsigned long long init[4] = {0, 0, ~0ull, 0};
    SCAN_CUDA(cudaMemcpyAsync(chk.ptr, init, sizeof(init), cudaMemcpyHostToDevice, st));
    auto *ud = (unsigned long long *)chk.ptr;
    for (size_t bi = 0; bi < P->blocks.size(); ++bi) {
        const Block &B = P->blocks[bi];
        if (load_block(g, 1, (int)bi, false) != SCAN_OK) { dev_free(ctx, chk); return fail(SCAN_ECUDA); }
        const int32_t rows = B.v1 - B.v0;
        if (rows > 0)
            k_p_check<<<grid_for(rows, 256), 256, 0, st>>>((const int64_t *)P->boff[1].ptr,
                                                          (const int32_t *)P->badj[1].ptr, B.v0, rows, B.e0, n, ud,
                                                          ud + 2);
        ctx->launches++;
    }
    unsigned long long res[4];
    cudaError_t e = cudaMemcpyAsync(res, chk.ptr, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(ctx, chk);
    P->loaded[1] = -1;
    if (e != cudaSuccess) return fail(cuda_fail(e, "partition validation"));
    if (res[2] != ~0ull) {
        set_error("invalid CSR at slot " + std::to_string(res[2]) +
                  " (rows must be strictly ascending, ids in [0, n), no self-loops)");
        return fail(SCAN_EINVAL);
    }
    if (res[0] != res[1]) {
        set_error("the CSR is not symmetric");
        return fail(SCAN_EINVAL);
    }
    *out = g;
    return SCAN_OK;
}

scan_status part_query(Graph *g, const scan_params &prm, scan_result **out) {
    Part *P = g->part;
    Ctx *c = g->ctx;
    cudaStream_t st = c->stream;
    const int32_t n = g->n;
    const uint64_t pp = (uint64_t)prm.eps_num * prm.eps_num, qq = (uint64_t)prm.eps_den * prm.eps_den;
    auto *ecnt = (int32_t *)P->ecnt.ptr;
    auto *core = (uint8_t *)P->core.ptr;
    auto *parent = (int32_t *)P->parent.ptr;
    auto *cid = (int32_t *)P->cid.ptr;
    auto *mfirst = (int32_t *)P->mfirst.ptr;
    auto *mmulti = (uint8_t *)P->mmulti.ptr;
    auto *bits = (uint32_t *)P->sbits.ptr;
    auto *err = (uint32_t *)P->err.ptr;
    auto *label = (uint8_t *)g->label.ptr;
    SCAN_CUDA(cudaMemsetAsync(ecnt, 0, 4 * ((size_t)n + 1), st));
    SCAN_CUDA(cudaMemsetAsync(bits, 0, P->sbits.bytes, st));
    SCAN_CUDA(cudaMemsetAsync(err, 0, 4, st));
    const int nb = (int)P->blocks.size();
    // ---- pass 1: every block pair i <= j. Block i sits in slot 0; the
    // blocks j > i alternate between slots 1 and 2, block j + 1 copied on
    // the side stream while pair (i, j) computes. No host synchronisation:
    // the similarity kernel reads the pair's chunk total on the device.
    const int sim_blocks = c->num_sms * 16;
    for (int i = 0; i < nb; ++i) {
        SCAN_TRY(load_block(g, 0, i, false));
        const Block &Bi = P->blocks[(size_t)i];
        const int32_t rows_i = Bi.v1 - Bi.v0;
        if (i + 1 < nb) SCAN_TRY(load_block(g, 1, i + 1, true));
        for (int j = i, t = 0; j < nb; ++j, ++t) {
            int sj = 0;
            if (j != i) {
                sj = 1 + ((t - 1) & 1);
                SCAN_TRY(use_block(g, sj, j));
                if (j + 1 < nb) SCAN_TRY(load_block(g, 1 + (t & 1), j + 1, true));
            }
            const Block &Bj = P->blocks[(size_t)j];
            if (rows_i > 0) {
                auto *offi = (const int64_t *)P->boff[0].ptr;
                auto *adji = (const int32_t *)P->badj[0].ptr;
                int32_t *nch = (int32_t *)g->cnt.ptr;
                int32_t *ra = (int32_t *)g->ucnt.ptr;
                int32_t *rb = (int32_t *)g->pair_off.ptr;
                int64_t *pos = (int64_t *)g->cnt_off.ptr;
                k_p_range<<<grid_for(rows_i, 256), 256, 0, st>>>(offi, adji, Bi.v0, rows_i, Bi.e0, Bj.v0, Bj.v1, nch,
                                                                ra, rb);
                SCAN_TRY(launch_exclusive_scan_i32_to_i64(c, nch, pos, rows_i, g->scan_tmp));
                k_p_chunks<<<grid_for(rows_i, 256), 256, 0, st>>>(offi, ra, rb, pos, rows_i, (Chunk *)g->src.ptr);
                // at most one chunk per row plus one per slot of block i
                const int64_t bound = (int64_t)rows_i + (Bi.e1 - Bi.e0) + 1;
                k_p_similar<<<grid_for(bound * 32, 256, sim_blocks), 256, 0, st>>>(
                    (const Chunk *)g->src.ptr, pos + rows_i, offi, adji, Bi.v0, Bi.e0,
                    slot_off(P, sj), slot_adj(P, sj), Bj.v0, Bj.e0, pp, qq, bits,
                    ecnt, err);
                c->launches += 3;
            }
            if (j != i) SCAN_TRY(release_slot(g, sj));
        }
    }
    const int uf_limit = c->loop_limit ? (int)std::min<uint32_t>(c->loop_limit, kUfLimitP) : kUfLimitP;
    k_p_core<<<grid_for(n, 256), 256, 0, st>>>(ecnt, n, prm.mu, core, parent);
    c->launches++;
    // ---- pass 2: union-find, one block at a time
    for (int i = 0; i < nb; ++i) {
        const int slot = 1 + (i & 1);
        SCAN_TRY(use_block(g, slot, i));
        if (i + 1 < nb) SCAN_TRY(load_block(g, 1 + ((i + 1) & 1), i + 1, true));
        const Block &B = P->blocks[(size_t)i];
        const int32_t rows = B.v1 - B.v0;
        if (rows > 0) {
            k_p_hook<<<grid_for((int64_t)rows * 32, 256), 256, 0, st>>>(
                slot_off(P, slot), slot_adj(P, slot), B.v0, rows, B.e0, bits, core,
                parent, err, uf_limit);
            c->launches++;
        }
        SCAN_TRY(release_slot(g, slot));
    }
    k_p_final<<<grid_for(n, 256), 256, 0, st>>>(core, n, parent, cid, err, uf_limit);
    c->launches++;
    // ---- pass 3a: border memberships, block by block, pairs to the host.
    // A non-core vertex has at most mu - 2 similar neighbours besides itself.
    std::vector<int32_t> host_pairs;
    const int64_t mu2 = prm.mu > 2 ? (int64_t)prm.mu - 2 : 0;
    int64_t per_block_pairs_cap = P->max_slots;
    if (mu2 == 0) per_block_pairs_cap = 0;
    else if ((int64_t)P->max_rows <= P->max_slots / mu2) per_block_pairs_cap = (int64_t)P->max_rows * mu2;
    per_block_pairs_cap = std::min<int64_t>(per_block_pairs_cap, P->max_slots) + 1;
    DevBuf raw, dpairs;
    SCAN_TRY(dev_alloc(c, raw, 4 * (size_t)per_block_pairs_cap));
    {
        scan_status s = dev_alloc(c, dpairs, 8 * (size_t)per_block_pairs_cap);
        if (s != SCAN_OK) { dev_free(c, raw); return s; }
    }
    for (int i = 0; i < nb; ++i) {
        const int slot = 1 + (i & 1);
        scan_status s = use_block(g, slot, i);
        if (s == SCAN_OK && i + 1 < nb) s = load_block(g, 1 + ((i + 1) & 1), i + 1, true);
        if (s != SCAN_OK) { dev_free(c, raw); dev_free(c, dpairs); return s; }
        const Block &B = P->blocks[(size_t)i];
        const int32_t rows = B.v1 - B.v0;
        if (rows == 0) {
            release_slot(g, slot);
            continue;
        }
        auto *offb = slot_off(P, slot);
        auto *adjb = slot_adj(P, slot);
        int32_t *cnt = (int32_t *)g->cnt.ptr;
        int64_t *pos = (int64_t *)g->cnt_off.ptr;
        int32_t *ucnt = (int32_t *)g->ucnt.ptr;
        int64_t *ppos = (int64_t *)g->pair_off.ptr;
        k_p_border_count<<<grid_for((int64_t)rows * 32, 256), 256, 0, st>>>(offb, adjb, B.v0, rows, B.e0, bits, core,
                                                                           cnt);
        s = launch_exclusive_scan_i32_to_i64(c, cnt, pos, rows, g->scan_tmp);
        if (s != SCAN_OK) { dev_free(c, raw); dev_free(c, dpairs); return s; }
        k_p_border_fill<<<grid_for((int64_t)rows * 32, 256), 256, 0, st>>>(offb, adjb, B.v0, rows, B.e0, bits, core,
                                                                          cid, pos, (int32_t *)raw.ptr, ucnt,
                                                                          mfirst, mmulti);
        s = launch_exclusive_scan_i32_to_i64(c, ucnt, ppos, rows, g->scan_tmp);
        if (s != SCAN_OK) { dev_free(c, raw); dev_free(c, dpairs); return s; }
        k_p_border_emit<<<grid_for(rows, 256), 256, 0, st>>>(pos, (const int32_t *)raw.ptr, ucnt, ppos, B.v0, rows,
                                                            (int32_t *)dpairs.ptr);
        c->launches += 3;
        release_slot(g, slot);
        int64_t k = 0;
        cudaError_t e = cudaMemcpyAsync(&k, ppos + rows, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && k > 0) {
            const size_t at = host_pairs.size();
            host_pairs.resize(at + 2 * (size_t)k);
            e = cudaMemcpyAsync(host_pairs.data() + at, dpairs.ptr, 8 * (size_t)k, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) { dev_free(c, raw); dev_free(c, dpairs); return cuda_fail(e, "border pairs"); }
    }
    dev_free(c, raw);
    dev_free(c, dpairs);
    // ---- pass 3b: hub / outlier labels
    for (int i = 0; i < nb; ++i) {
        const int slot = 1 + (i & 1);
        SCAN_TRY(use_block(g, slot, i));
        if (i + 1 < nb) SCAN_TRY(load_block(g, 1 + ((i + 1) & 1), i + 1, true));
        const Block &B = P->blocks[(size_t)i];
        const int32_t rows = B.v1 - B.v0;
        if (rows > 0) {
            k_p_label<<<grid_for((int64_t)rows * 32, 256), 256, 0, st>>>(
                slot_off(P, slot), slot_adj(P, slot), B.v0, rows, B.e0, core,
                cid, mfirst, mmulti, label);
            c->launches++;
        }
        SCAN_TRY(release_slot(g, slot));
    }
    // ---- results
    uint32_t herr = 0;
    SCAN_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    SCAN_CUDA(cudaStreamSynchronize(st));
    if (herr & ERR_LOOP_LIMIT) {
        set_error("the CSR is not symmetric (a mirror entry is missing)");
        return SCAN_EINVAL;
    }
    if (herr) {
        set_error("a bounded device loop gave up (error bits " + std::to_string(herr) + ")");
        return SCAN_ETIMEOUT;
    }
    const int64_t k = (int64_t)host_pairs.size() / 2;
    scan_result *r = result_new(n, k, true);
    if (!r) { set_error("result allocation failed"); return SCAN_ENOMEM; }
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(r->core, core, (size_t)n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->label, label, (size_t)n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->cid, cid, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        scan_result_free(r);
        return cuda_fail(e, "result download");
    }
    if (k > 0) memcpy(r->pairs, host_pairs.data(), 8 * (size_t)k);
    *out = r;
    return SCAN_OK;
}

}  // namespace scan

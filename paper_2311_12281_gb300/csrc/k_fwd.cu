// k_fwd.cu -- closed common counts of every edge by degree-oriented triangle
// enumeration.
//
// Orient every edge from its lower to its higher (deg, id) endpoint (the
// degree-oriented edge array of Section 4.1); out(x) is x's list of higher
// neighbours, ascending by id. For an edge the open common count
// |nbr(u) cap nbr(v)| is the number of triangles through it, and each
// triangle a < b < c (in that order) is found exactly once: at its middle
// vertex b, when the row out(a) of an in-neighbour a is streamed through a
// shared-memory table of out(b). A hit c then adds one to each of the three
// edges: (a, b) through a per-in-edge counter, (b, c) through a per-owner
// counter in shared memory, and (a, c) by an atomic add at the streamed
// position of c in out(a). In a degree orientation out-degrees stay below
// sqrt(2m), so the tables are small and sparse (load <= 1/4), and the work is
// the sum over oriented edges (a, b) of |out(a)| instead of the
// sum over edges of min(deg) that a per-edge intersection pays.
//
// closed count of an edge = triangles through it + 2 (Definition 2.2 with
// closed neighbourhoods: both endpoints are in both N[.]).
#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr int kFwdSmallOut = 64;         // warp-level owners: out-degree bound
constexpr int64_t kFwdSmallWork = 1 << 15;  // ... and probe bound
constexpr int kFwdSmallTable = 256;      // slots per warp table
constexpr int kFwdChunk = 4096;          // max out(b) elements per CTA table
constexpr int64_t kFwdItemWork = 1 << 20;  // target probes per CTA item
constexpr int kFwdPiece = 256;
constexpr int kFwdUnroll = 8;
constexpr unsigned long long kSlotEmpty = ~0ull;

struct FItem {
    int32_t v, chunk, sb, se;
};

__device__ __forceinline__ uint32_t fhash(int32_t x, int logc) { return ((uint32_t)x * 0x9E3779B1u) >> (32 - logc); }

// table slot = (index << 32) | key; empty = all ones
__device__ __forceinline__ void ftab_insert(unsigned long long *t, int logc, int32_t key, int32_t idx) {
    const uint32_t mask = (1u << logc) - 1u;
    const unsigned long long item = ((unsigned long long)(uint32_t)idx << 32) | (uint32_t)key;
    uint32_t h = fhash(key, logc);
    for (uint32_t it = 0; it <= mask; ++it) {
        const unsigned long long old = atomicCAS(t + h, kSlotEmpty, item);
        if (old == kSlotEmpty) return;
        h = (h + 1) & mask;
    }
}

// index of key in the table, or -1
__device__ __forceinline__ int32_t ftab_find(const unsigned long long *t, int logc, int32_t key) {
    const uint32_t mask = (1u << logc) - 1u;
    uint32_t h = fhash(key, logc);
    for (uint32_t it = 0; it <= mask; ++it) {
        const unsigned long long y = t[h];
        if (y == kSlotEmpty) return -1;
        if ((int32_t)(uint32_t)y == key) return (int32_t)(y >> 32);
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ int fceil_log2(int x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

__device__ __forceinline__ int32_t lower_bound_row(const int32_t *__restrict__ r, int32_t len, int32_t x) {
    int32_t lo = 0, hi = len;
    for (int it = 0; it < 40 && lo < hi; ++it) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(r + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Probe elements out(a)[start + k], k in [k0, k1) stepping by `step`, against
// the owner table; returns the hits and records the (a, c) and (b, c) counts.
template <int UNROLL>
__device__ __forceinline__ int probe_run(const int32_t *__restrict__ row, int32_t *__restrict__ cnt_row, int32_t k0,
                                         int32_t k1, int32_t step, const unsigned long long *t, int logc,
                                         int32_t *ocnt) {
    int c = 0;
    for (int32_t kb = k0; kb < k1; kb += step * UNROLL) {
        int32_t x[UNROLL];
#pragma unroll
        for (int j = 0; j < UNROLL; ++j) {
            const int32_t k = kb + j * step;
            x[j] = k < k1 ? __ldg(row + k) : -1;
        }
#pragma unroll
        for (int j = 0; j < UNROLL; ++j) {
            const int32_t k = kb + j * step;
            if (k < k1) {
                const int32_t idx = ftab_find(t, logc, x[j]);
                if (idx >= 0) {
                    ++c;
                    atomicAdd(cnt_row + k, 1);
                    atomicAdd(ocnt + idx, 1);
                }
            }
        }
    }
    return c;
}

// ------------------------------------------------------------ warp owners
__global__ void __launch_bounds__(256) k_fwd_small(const int32_t *__restrict__ owners, int32_t nown,
                                                   const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                   const int32_t *__restrict__ deg, const int64_t *__restrict__ foff,
                                                   const int32_t *__restrict__ fadj, const uint32_t *__restrict__ fin,
                                                   int32_t *__restrict__ fcnt) {
    __shared__ unsigned long long tables[8][kFwdSmallTable];
    __shared__ int32_t ocnts[8][kFwdSmallOut];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *t = tables[wid];
    int32_t *ocnt = ocnts[wid];
    const int warps_total = gridDim.x * 8;
    for (int32_t i = blockIdx.x * 8 + wid; i < nown; i += warps_total) {
        const int32_t b = owners[i];
        const int64_t fb = foff[b];
        const int32_t db = deg[b], ob = (int32_t)(foff[b + 1] - fb);
        const int logc = max(5, fceil_log2(4 * ob));
        for (int k = lane; k < (1 << logc); k += kWarp) t[k] = kSlotEmpty;
        for (int k = lane; k < kFwdSmallOut; k += kWarp) ocnt[k] = 0;
        __syncwarp();
        for (int k = lane; k < ob; k += kWarp) ftab_insert(t, logc, fadj[fb + k], k);
        __syncwarp();
        const int64_t rb = off[b];
        for (int32_t g0 = 0; g0 < db; g0 += kWarp) {
            const int64_t s = rb + g0 + lane;
            int32_t a = -1, oa = 0;
            int64_t fa = 0;
            if (g0 + lane < db) {
                a = adj[s];
                const int32_t da = deg[a];
                if (dev::rank_less(da, a, db, b)) {
                    fa = foff[a];
                    oa = (int32_t)(foff[a + 1] - fa);
                }
            }
            int mine = 0;
            if (oa > 0 && oa < 16) mine = probe_run<4>(fadj + fa, fcnt + fa, 0, oa, 1, t, logc, ocnt);
            unsigned longs = __ballot_sync(0xffffffffu, oa >= 16);
            while (longs) {
                const int src = __ffs(longs) - 1;
                longs &= longs - 1;
                const int64_t fas = __shfl_sync(0xffffffffu, fa, src);
                const int32_t oas = __shfl_sync(0xffffffffu, oa, src);
                int c = probe_run<kFwdUnroll>(fadj + fas, fcnt + fas, lane, oas, kWarp, t, logc, ocnt);
                c = __reduce_add_sync(0xffffffffu, c);
                if (lane == src) mine = c;
            }
            if (oa > 0 && mine) atomicAdd(fcnt + fin[s], mine);
        }
        __syncwarp();
        for (int k = lane; k < ob; k += kWarp)
            if (ocnt[k]) atomicAdd(fcnt + fb + k, ocnt[k]);
        __syncwarp();
    }
}

// ------------------------------------------------------------ CTA owners
template <int BLOCK, typename T>
__device__ __forceinline__ T fblock_scan(T x, T *total, T *wsum) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = lane < BLOCK / 32 ? wsum[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < BLOCK / 32) wsum[lane] = si - s;
        if (lane == BLOCK / 32 - 1) wsum[BLOCK / 32] = si;
    }
    __syncthreads();
    const T ex = inc - x + wsum[wid];
    *total = wsum[BLOCK / 32];
    __syncthreads();
    return ex;
}

// One CTA per item (owner b, value chunk of out(b), slot range of b's row).
// Dynamic shared memory: the table (cap 64-bit slots) then the per-owner
// counters (kFwdChunk ints).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_fwd_cta(const FItem *__restrict__ items, const int64_t *__restrict__ off,
                                                   const int32_t *__restrict__ adj, const int32_t *__restrict__ deg,
                                                   const int64_t *__restrict__ foff, const int32_t *__restrict__ fadj,
                                                   const uint32_t *__restrict__ fin, int32_t *__restrict__ fcnt,
                                                   int cap_log) {
    extern __shared__ unsigned long long t[];
    int32_t *ocnt = (int32_t *)(t + (1 << cap_log));
    __shared__ int32_t w_s[BLOCK], w_start[BLOCK], w_len[BLOCK], w_cnt[BLOCK];
    __shared__ int64_t w_fa[BLOCK];
    __shared__ int32_t l_idx[BLOCK], l_poff[BLOCK + 1], s_idx[BLOCK];
    __shared__ long long wsum64[BLOCK / 32 + 1];
    __shared__ int32_t wsum32[BLOCK / 32 + 1];
    __shared__ int32_t piece_ctr, short_ctr;

    const FItem it = items[blockIdx.x];
    const int32_t b = it.v;
    const int64_t rb = off[b], fb = foff[b];
    const int32_t db = (int32_t)(off[b + 1] - rb), ob = (int32_t)(foff[b + 1] - fb);
    const int32_t tb = it.chunk * kFwdChunk, te = min(tb + kFwdChunk, ob), tlen = te - tb;
    const bool chunked = ob > kFwdChunk;
    const int32_t lo = tb == 0 ? INT32_MIN : fadj[fb + tb];
    const int32_t hi = te == ob ? INT32_MAX : fadj[fb + te];
    const int logc = min(cap_log, max(5, fceil_log2(4 * tlen)));
    for (int k = threadIdx.x; k < (1 << logc); k += BLOCK) t[k] = kSlotEmpty;
    for (int k = threadIdx.x; k < tlen; k += BLOCK) ocnt[k] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < tlen; k += BLOCK) ftab_insert(t, logc, fadj[fb + tb + k], k);
    const int lane = threadIdx.x & 31;

    for (int32_t r0 = it.sb; r0 < it.se; r0 += BLOCK) {
        const int32_t rel = r0 + threadIdx.x;
        bool work = false;
        int32_t start = 0, len = 0, s32 = 0;
        int64_t fa = 0;
        if (rel < it.se) {
            const int64_t s = rb + rel;
            const int32_t a = adj[s], da = deg[a];
            if (dev::rank_less(da, a, db, b)) {
                fa = foff[a];
                len = (int32_t)(foff[a + 1] - fa);
                if (chunked && len > 0) {
                    const int32_t *row = fadj + fa;
                    start = lo == INT32_MIN ? 0 : lower_bound_row(row, len, lo);
                    const int32_t end = hi == INT32_MAX ? len : lower_bound_row(row, len, hi);
                    len = end - start;
                }
                work = len > 0;
                s32 = rel;
            }
        }
        const bool is_long = work && len >= kWarp;
        const bool is_short = work && len < kWarp;
        const long long flags = (long long)work | ((long long)is_long << 21) | ((long long)is_short << 42);
        long long tot;
        const long long ex = fblock_scan<BLOCK, long long>(flags, &tot, wsum64);
        int32_t tot_pieces;
        const int32_t pex = fblock_scan<BLOCK, int32_t>(is_long ? (len + kFwdPiece - 1) / kFwdPiece : 0, &tot_pieces,
                                                        wsum32);
        const int32_t n_work = (int32_t)(tot & 0x1FFFFF);
        const int32_t n_long = (int32_t)((tot >> 21) & 0x1FFFFF);
        const int32_t n_short = (int32_t)((tot >> 42) & 0x1FFFFF);
        if (work) {
            const int32_t e = (int32_t)(ex & 0x1FFFFF);
            w_s[e] = s32;
            w_fa[e] = fa;
            w_start[e] = start;
            w_len[e] = len;
            w_cnt[e] = 0;
            if (is_long) {
                const int32_t l = (int32_t)((ex >> 21) & 0x1FFFFF);
                l_idx[l] = e;
                l_poff[l] = pex;
            }
            if (is_short) s_idx[(ex >> 42) & 0x1FFFFF] = e;
        }
        if (threadIdx.x == 0) {
            l_poff[n_long] = tot_pieces;
            piece_ctr = 0;
            short_ctr = 0;
        }
        __syncthreads();
        for (int guard = 0; guard < (1 << 30); ++guard) {
            int32_t p = 0;
            if (lane == 0) p = atomicAdd(&piece_ctr, 1);
            p = __shfl_sync(0xffffffffu, p, 0);
            if (p >= tot_pieces) break;
            int32_t li = 0, hi_i = n_long;
            while (hi_i - li > 1) {
                const int32_t mid = (li + hi_i) >> 1;
                if (l_poff[mid] <= p) li = mid;
                else hi_i = mid;
            }
            const int32_t e = l_idx[li];
            const int32_t o = w_start[e] + (p - l_poff[li]) * kFwdPiece;
            const int32_t pend = min(o + kFwdPiece, w_start[e] + w_len[e]);
            const int64_t fa = w_fa[e];
            int c = probe_run<kFwdUnroll>(fadj + fa, fcnt + fa, o + lane, pend, kWarp, t, logc, ocnt);
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0 && c) atomicAdd(&w_cnt[e], c);
        }
        for (int guard = 0; guard < (1 << 30); ++guard) {
            int32_t q = 0;
            if (lane == 0) q = atomicAdd(&short_ctr, kWarp);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= n_short) break;
            const int32_t k = q + lane;
            if (k < n_short) {
                const int32_t e = s_idx[k];
                const int64_t fa = w_fa[e];
                w_cnt[e] = probe_run<4>(fadj + fa, fcnt + fa, w_start[e], w_start[e] + w_len[e], 1, t, logc, ocnt);
            }
        }
        __syncthreads();
        if (threadIdx.x < n_work) {
            const int32_t e = threadIdx.x;
            if (w_cnt[e]) atomicAdd(fcnt + fin[rb + w_s[e]], w_cnt[e]);
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < tlen; k += BLOCK)
        if (ocnt[k]) atomicAdd(fcnt + fb + tb + k, ocnt[k]);
}

// per forward edge: closed count, mirrored to both slots; optional eps-test
template <bool WRITE_SIM, bool WRITE_CN>
__global__ void k_fwd_finish(const uint32_t *__restrict__ oe, int64_t m, const int32_t *__restrict__ fcnt,
                             const int32_t *__restrict__ src, const int32_t *__restrict__ adj,
                             const uint32_t *__restrict__ rev, const int32_t *__restrict__ deg, QParams qp,
                             uint8_t *__restrict__ sim, int32_t *__restrict__ cn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = oe[i];
        const uint32_t r = rev[e];
        const int32_t c = fcnt[i] + 2;
        if (WRITE_CN) { cn[e] = c; cn[r] = c; }
        if (WRITE_SIM) {
            const int32_t u = src[e], v = adj[e];
            uint64_t pp, qq;
            qp.eps(u, pp, qq);
            if (dev::eps_similar((uint64_t)c, (uint64_t)deg[u] + 1, (uint64_t)deg[v] + 1, pp, qq)) {
                sim[e] = 1;
                sim[r] = 1;
            }
        }
    }
}

// ------------------------------------------------------------ load time
__global__ void k_fwd_adj(const uint32_t *__restrict__ oe, int64_t m, const int32_t *__restrict__ adj,
                          const uint32_t *__restrict__ rev, int32_t *__restrict__ fadj, uint32_t *__restrict__ fin) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = oe[i];
        fadj[i] = adj[e];
        fin[rev[e]] = (uint32_t)i;
    }
}

// warp per vertex: work as a middle vertex and the number of items
__global__ void __launch_bounds__(256) k_fwd_sched_count(const int64_t *__restrict__ off,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ deg,
                                                         const int64_t *__restrict__ foff, int32_t n,
                                                         int32_t *__restrict__ nranges,
                                                         unsigned long long *counts) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (b >= n) return;
    const int32_t ob = (int32_t)(foff[b + 1] - foff[b]);
    if (lane == 0) nranges[b] = 0;
    if (ob == 0) return;  // no higher neighbour: never a middle vertex
    const int32_t db = deg[b];
    const int64_t rb = off[b];
    unsigned long long w = 0;
    for (int32_t k = lane; k < db; k += kWarp) {
        const int32_t a = adj[rb + k], da = deg[a];
        if (dev::rank_less(da, a, db, (int32_t)b)) w += (unsigned long long)(foff[a + 1] - foff[a]);
    }
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane != 0 || w == 0) return;
    if (ob <= kFwdSmallOut && (int64_t)w <= kFwdSmallWork) {
        nranges[b] = -1;  // warp owner
        atomicAdd(counts + 0, 1ull);
        return;
    }
    const int64_t nchunks = (ob + kFwdChunk - 1) / kFwdChunk;
    int64_t nr = (int64_t)((w + kFwdItemWork - 1) / kFwdItemWork);
    nr = max((int64_t)1, min(nr, (int64_t)(db + 255) / 256));
    nranges[b] = (int32_t)nr;
    atomicAdd(counts + (ob <= 1024 ? 1 : 2), (unsigned long long)(nchunks * nr));
}

__global__ void k_fwd_sched_write(const int32_t *__restrict__ deg, const int64_t *__restrict__ foff, int32_t n,
                                  const int32_t *__restrict__ nranges, unsigned long long *cursor,
                                  int32_t *__restrict__ small, FItem *__restrict__ i1, FItem *__restrict__ i2) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int32_t nr = nranges[b];
    if (nr == 0) return;
    if (nr < 0) {
        small[atomicAdd(cursor + 0, 1ull)] = (int32_t)b;
        return;
    }
    const int32_t ob = (int32_t)(foff[b + 1] - foff[b]), db = deg[b];
    const int32_t nchunks = (ob + kFwdChunk - 1) / kFwdChunk;
    const int32_t len = (db + nr - 1) / nr;
    const int cls = ob <= 1024 ? 1 : 2;
    FItem *dst = cls == 1 ? i1 : i2;
    unsigned long long p = atomicAdd(cursor + cls, (unsigned long long)(nchunks * nr));
    for (int32_t c = 0; c < nchunks; ++c)
        for (int32_t r = 0; r < nr; ++r) dst[p++] = FItem{(int32_t)b, c, r * len, min(db, (r + 1) * len)};
}

}  // namespace

scan_status fwd_prepare(Graph *g) {
    Ctx *c = g->ctx;
    const int32_t n = g->n;
    const int64_t m = g->m;
    if (g->fwd_ready) return SCAN_OK;
    if (n == 0 || m == 0) {
        g->fwd_ready = true;
        return SCAN_OK;
    }
    SCAN_TRY(dev_alloc(c, g->fadj, 4 * (size_t)m));
    SCAN_TRY(dev_alloc(c, g->fin, 4 * (size_t)g->nnz));
    SCAN_TRY(dev_alloc(c, g->fcnt, 4 * (size_t)m));
    // foff (built at load) already holds the out-degree offsets
    k_fwd_adj<<<grid_for(m, 256, c->num_sms * 32), 256, 0, c->stream>>>(
        (const uint32_t *)g->oe.ptr, m, (const int32_t *)g->adj.ptr, (const uint32_t *)g->rev.ptr,
        (int32_t *)g->fadj.ptr, (uint32_t *)g->fin.ptr);
    c->launches++;
    // schedule
    DevBuf cnts;
    SCAN_TRY(dev_alloc(c, cnts, 4 * sizeof(unsigned long long)));
    auto *counts = (unsigned long long *)cnts.ptr;
    SCAN_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), c->stream));
    int32_t *nranges = (int32_t *)g->ucnt.ptr;  // scratch int32[n+1]
    k_fwd_sched_count<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(
        (const int64_t *)g->off.ptr, (const int32_t *)g->adj.ptr, (const int32_t *)g->deg.ptr,
        (const int64_t *)g->foff.ptr, n, nranges, counts);
    c->launches++;
    unsigned long long h[4];
    SCAN_CUDA(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    g->fwd_small = (int32_t)h[0];
    g->fwd_items_n[1] = (int64_t)h[1];
    g->fwd_items_n[2] = (int64_t)h[2];
    scan_status s = dev_alloc(c, g->fwd_owners, 4 * (size_t)(h[0] + 1));
    if (s == SCAN_OK) s = dev_alloc(c, g->fwd_items[1], sizeof(FItem) * (size_t)(h[1] + 1));
    if (s == SCAN_OK) s = dev_alloc(c, g->fwd_items[2], sizeof(FItem) * (size_t)(h[2] + 1));
    if (s != SCAN_OK) {
        dev_free(c, cnts);
        return s;
    }
    SCAN_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), c->stream));
    k_fwd_sched_write<<<grid_for(n, 256), 256, 0, c->stream>>>(
        (const int32_t *)g->deg.ptr, (const int64_t *)g->foff.ptr, n, nranges, counts,
        (int32_t *)g->fwd_owners.ptr, (FItem *)g->fwd_items[1].ptr, (FItem *)g->fwd_items[2].ptr);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, cnts);
    if (e != cudaSuccess) return cuda_fail(e, "forward schedule");
    g->fwd_ready = true;
    return SCAN_OK;
}

scan_status launch_fwd_counts(Graph *g, bool write_sim, bool write_cn, const QParams &qp, int32_t *cn) {
    Ctx *c = g->ctx;
    if (g->m == 0) return SCAN_OK;
    SCAN_TRY(fwd_prepare(g));
    cudaStream_t st = c->stream;
    auto *off = (const int64_t *)g->off.ptr;
    auto *adj = (const int32_t *)g->adj.ptr;
    auto *deg = (const int32_t *)g->deg.ptr;
    auto *foff = (const int64_t *)g->foff.ptr;
    auto *fadj = (const int32_t *)g->fadj.ptr;
    auto *fin = (const uint32_t *)g->fin.ptr;
    auto *fcnt = (int32_t *)g->fcnt.ptr;
    SCAN_CUDA(cudaMemsetAsync(fcnt, 0, 4 * (size_t)g->m, st));
    if (g->fwd_items_n[2] > 0) {  // out-degree > 1024: 16384-slot tables
        const int cap_log = 14;
        const size_t smem = (8u << cap_log) + 4 * kFwdChunk;
        auto kern = k_fwd_cta<512>;
        SCAN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)g->fwd_items_n[2], 512, smem, st>>>((const FItem *)g->fwd_items[2].ptr, off, adj, deg, foff,
                                                           fadj, fin, fcnt, cap_log);
        c->launches++;
    }
    if (g->fwd_items_n[1] > 0) {  // out-degree <= 1024: 4096-slot tables
        const int cap_log = 12;
        const size_t smem = (8u << cap_log) + 4 * 1024;
        auto kern = k_fwd_cta<512>;
        SCAN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)g->fwd_items_n[1], 512, smem, st>>>((const FItem *)g->fwd_items[1].ptr, off, adj, deg, foff,
                                                           fadj, fin, fcnt, cap_log);
        c->launches++;
    }
    if (g->fwd_small > 0) {
        k_fwd_small<<<grid_for((int64_t)g->fwd_small * kWarp, 256, c->num_sms * 16), 256, 0, st>>>(
            (const int32_t *)g->fwd_owners.ptr, g->fwd_small, off, adj, deg, foff, fadj, fin, fcnt);
        c->launches++;
    }
    const unsigned gf = grid_for(g->m, 256, c->num_sms * 32);
    auto *oe = (const uint32_t *)g->oe.ptr;
    auto *src = (const int32_t *)g->src.ptr;
    auto *rev = (const uint32_t *)g->rev.ptr;
    auto *sim = (uint8_t *)g->sim.ptr;
    if (write_sim && write_cn)
        k_fwd_finish<true, true><<<gf, 256, 0, st>>>(oe, g->m, fcnt, src, adj, rev, deg, qp, sim, cn);
    else if (write_cn)
        k_fwd_finish<false, true><<<gf, 256, 0, st>>>(oe, g->m, fcnt, src, adj, rev, deg, qp, sim, cn);
    else
        k_fwd_finish<true, false><<<gf, 256, 0, st>>>(oe, g->m, fcnt, src, adj, rev, deg, qp, sim, cn);
    c->launches++;
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

}  // namespace scan

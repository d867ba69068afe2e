// k_isect_owner.cu -- closed common counts by owner-staged shared-memory hashing.
//
// Every undirected edge (u, v) is owned by its higher (deg, id) endpoint v --
// the degree orientation of Section 4.1 read from the other side, so the
// lower-degree row drives the work as in checkSim (Algorithm 2). An owner's
// row nbr(v) is inserted once into a shared-memory hash table; each owned
// neighbour u then streams nbr(u) and probes it, so an edge costs deg(u)
// probes and nbr(v) is read once per work item instead of once per edge.
//
//   small owners  deg(v) <= 128: one warp per owner, a 256-slot table per warp
//   big owners    deg(v) > 128: one CTA per work item (owner, chunk, slot
//                 range); items split an owner's row so that each carries a
//                 bounded number of probes, in three table-size classes
//   hubs          deg(v) > kChunk: the table holds one value-chunk of nbr(v)
//                 at a time; chunks add partial counts into acc[] and a
//                 finishing pass applies the eps-test
//
// Inside a work item a warp takes 32 consecutive slots of the owner's row,
// one per lane. Owned neighbours with short rows are probed by their own
// lane; long rows are probed by the whole warp, lanes striding the row.
#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr int kSmallMax = 128;      // warp-level owners
constexpr int kSmallTable = 256;    // slots per warp table
constexpr int kChunk = 16384;       // max table elements per CTA (hubs are chunked)
constexpr int kShortRow = 16;       // rows below this are probed by one lane
constexpr int64_t kItemWork = 1 << 21;  // target probes per work item
constexpr int kEmpty = -1;

struct Item {
    int32_t v;       // owner
    int32_t chunk;   // value-chunk of nbr(v) in the table
    int32_t sb, se;  // slot range of the owner's row, relative to off[v]
};

__device__ __forceinline__ uint32_t hslot(int32_t x, int logc) {
    return ((uint32_t)x * 0x9E3779B1u) >> (32 - logc);
}

__device__ __forceinline__ void table_insert(int32_t *t, int logc, int32_t x) {
    const uint32_t mask = (1u << logc) - 1u;
    uint32_t h = hslot(x, logc);
    for (uint32_t it = 0; it <= mask; ++it) {
        int32_t old = atomicCAS(t + h, kEmpty, x);
        if (old == kEmpty || old == x) return;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int table_has(const int32_t *t, int logc, int32_t x) {
    const uint32_t mask = (1u << logc) - 1u;
    uint32_t h = hslot(x, logc);
    for (uint32_t it = 0; it <= mask; ++it) {
        const int32_t y = t[h];
        if (y == x) return 1;
        if (y == kEmpty) return 0;
        h = (h + 1) & mask;
    }
    return 0;
}

__device__ __forceinline__ int ceil_log2(int x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// What an owner decides for one owned slot before any probing.
struct SlotPlan {
    int32_t u, du;
    bool work;     // needs the intersection
};

template <bool PRUNE>
__device__ __forceinline__ SlotPlan plan_slot(int64_t s, bool valid, int32_t v, int32_t dv,
                                              const int32_t *__restrict__ adj, const int32_t *__restrict__ deg,
                                              const uint32_t *__restrict__ rev, uint64_t pp, uint64_t qq,
                                              uint8_t *__restrict__ sim, bool write_sure) {
    SlotPlan pl{-1, 0, false};
    if (!valid) return pl;
    pl.u = adj[s];
    pl.du = deg[pl.u];
    if (!dev::rank_less(pl.du, pl.u, dv, v)) return pl;  // owned by the other endpoint
    if (PRUNE) {
        if (dev::prune_dissimilar((uint64_t)pl.du + 1, (uint64_t)dv + 1, pp, qq)) return pl;
        if (dev::prune_similar((uint64_t)pl.du + 1, (uint64_t)dv + 1, pp, qq)) {
            if (write_sure) { sim[s] = 1; sim[rev[s]] = 1; }
            return pl;
        }
    }
    pl.work = true;
    return pl;
}

// Final decision for one owned edge from its closed count c.
template <bool WRITE_SIM, bool WRITE_CN>
__device__ __forceinline__ void emit(int64_t s, int32_t c, int32_t du, int32_t dv, const uint32_t *__restrict__ rev,
                                     uint64_t pp, uint64_t qq, uint8_t *__restrict__ sim, int32_t *__restrict__ cn) {
    const uint32_t r = rev[s];
    if (WRITE_CN) { cn[s] = c; cn[r] = c; }
    if (WRITE_SIM && dev::eps_similar((uint64_t)c, (uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) {
        sim[s] = 1;
        sim[r] = 1;
    }
}

// Probe the owned slots of one 32-slot group of an owner's row against the
// table t; values outside [lo, hi) are not in this chunk and are skipped.
// Returns per lane the count of its own slot (full counts, not closed).
template <bool CHUNKED>
__device__ __forceinline__ int32_t probe_group(const SlotPlan &pl, const int64_t *__restrict__ off,
                                               const int32_t *__restrict__ adj, const int32_t *t, int logc,
                                               int32_t lo, int32_t hi) {
    const int lane = threadIdx.x & 31;
    int32_t mine = 0;
    // short rows: each lane its own
    if (pl.work && pl.du < kShortRow) {
        const int32_t *ru = adj + off[pl.u];
        for (int k = 0; k < pl.du; ++k) {
            const int32_t x = __ldg(ru + k);
            if (CHUNKED && (x < lo || x >= hi)) continue;
            mine += table_has(t, logc, x);
        }
    }
    // long rows: the whole warp per row
    unsigned longs = __ballot_sync(0xffffffffu, pl.work && pl.du >= kShortRow);
    while (longs) {
        const int src = __ffs(longs) - 1;
        longs &= longs - 1;
        const int32_t u = __shfl_sync(0xffffffffu, pl.u, src);
        const int32_t du = __shfl_sync(0xffffffffu, pl.du, src);
        const int32_t *ru = adj + off[u];
        int c = 0;
        for (int32_t k = lane; k < du; k += kWarp) {
            const int32_t x = __ldg(ru + k);
            if (CHUNKED && (x < lo || x >= hi)) continue;
            c += table_has(t, logc, x);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == src) mine = c;
    }
    return mine;
}

// ------------------------------------------------------------ small owners
template <bool PRUNE, bool WRITE_SIM, bool WRITE_CN>
__global__ void __launch_bounds__(256) k_owner_small(
    const int32_t *__restrict__ owners, int32_t nown, const int64_t *__restrict__ off,
    const int32_t *__restrict__ adj, const int32_t *__restrict__ deg, const uint32_t *__restrict__ rev, QParams qp,
    uint8_t *__restrict__ sim, int32_t *__restrict__ cn) {
    __shared__ int32_t tables[256 / kWarp][kSmallTable];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *t = tables[wid];
    const int warps_total = gridDim.x * (blockDim.x / kWarp);
    for (int32_t i = blockIdx.x * (blockDim.x / kWarp) + wid; i < nown; i += warps_total) {
        const int32_t v = owners[i];
        uint64_t pp, qq;
        qp.eps(v, pp, qq);
        const int64_t b = off[v];
        const int32_t dv = (int32_t)(off[v + 1] - b);
        const int logc = max(5, ceil_log2(2 * dv));
        const int cap = 1 << logc;
        for (int k = lane; k < cap; k += kWarp) t[k] = kEmpty;
        __syncwarp();
        for (int k = lane; k < dv; k += kWarp) table_insert(t, logc, adj[b + k]);
        __syncwarp();
        for (int32_t g0 = 0; g0 < dv; g0 += kWarp) {
            const int64_t s = b + g0 + lane;
            const SlotPlan pl = plan_slot<PRUNE>(s, g0 + lane < dv, v, dv, adj, deg, rev, pp, qq, sim, true);
            const int32_t c = probe_group<false>(pl, off, adj, t, logc, 0, 0);
            if (pl.work) emit<WRITE_SIM, WRITE_CN>(s, c + 2, pl.du, dv, rev, pp, qq, sim, cn);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ big owners
constexpr int kPiece = 256;  // elements of a long row one warp probes per grab
constexpr int kUnroll = 8;   // independent loads per lane issued before probing

// First index of row r[0, len) holding a value >= x (bounded binary search).
__device__ __forceinline__ int32_t row_lower_bound(const int32_t *__restrict__ r, int32_t len, int32_t x) {
    int32_t lo = 0, hi = len;
    for (int it = 0; it < 40 && lo < hi; ++it) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(r + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Exclusive block-wide prefix sum; every thread gets the total.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_scan(T x, T *total, T *wsum) {
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

// One CTA per work item (owner v, value-chunk of nbr(v), slot range). The
// item's slots are taken BLOCK at a time ("rounds"): every thread plans one
// slot, the owned edges that need counting are compacted in shared memory,
// long rows are cut into kPiece-element pieces that warps grab from a
// shared counter (so no warp waits on another's row), and short rows are
// probed one lane each. Every lane issues kUnroll independent loads before
// it probes, to keep loads in flight.
template <int BLOCK, bool PRUNE, bool WRITE_SIM, bool WRITE_CN>
__global__ void __launch_bounds__(BLOCK) k_owner_cta(const Item *__restrict__ items, const int64_t *__restrict__ off,
                                                     const int32_t *__restrict__ adj, const int32_t *__restrict__ deg,
                                                     const uint32_t *__restrict__ rev, QParams qp,
                                                     uint8_t *__restrict__ sim, int32_t *__restrict__ cn,
                                                     int32_t *__restrict__ acc) {
    extern __shared__ int32_t t[];
    __shared__ int32_t w_rel[BLOCK], w_u[BLOCK], w_du[BLOCK], w_start[BLOCK], w_len[BLOCK], w_cnt[BLOCK];
    __shared__ int32_t l_idx[BLOCK], l_poff[BLOCK + 1], s_idx[BLOCK];
    __shared__ long long wsum64[BLOCK / 32 + 1];
    __shared__ int32_t wsum32[BLOCK / 32 + 1];
    __shared__ int32_t piece_ctr, short_ctr;

    const Item it = items[blockIdx.x];
    const int32_t v = it.v;
    const int64_t b = off[v];
    const int32_t dv = (int32_t)(off[v + 1] - b);
    uint64_t pp, qq;
    qp.eps(v, pp, qq);
    const int32_t *rv = adj + b;
    const int32_t tb = it.chunk * kChunk;
    const int32_t te = min(tb + kChunk, dv);
    const bool chunked = dv > kChunk;
    const int32_t lo = tb == 0 ? INT32_MIN : rv[tb];
    const int32_t hi = te == dv ? INT32_MAX : rv[te];
    const int logc = max(5, ceil_log2(2 * (te - tb)));
    const int cap = 1 << logc;
    for (int k = threadIdx.x; k < cap; k += BLOCK) t[k] = kEmpty;
    __syncthreads();
    for (int k = tb + threadIdx.x; k < te; k += BLOCK) table_insert(t, logc, rv[k]);
    const int lane = threadIdx.x & 31;

    for (int32_t r0 = it.sb; r0 < it.se; r0 += BLOCK) {
        // ---- plan one slot per thread
        const int32_t rel = r0 + threadIdx.x;
        bool work = false;
        int32_t u = -1, du = 0, start = 0, len = 0;
        if (rel < it.se) {
            const int64_t s = b + rel;
            u = adj[s];
            du = deg[u];
            if (dev::rank_less(du, u, dv, v)) {
                work = true;
                if (PRUNE) {
                    if (dev::prune_dissimilar((uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) {
                        work = false;
                    } else if (dev::prune_similar((uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) {
                        if (it.chunk == 0) { sim[s] = 1; sim[rev[s]] = 1; }
                        work = false;
                    }
                }
                if (work) {
                    len = du;
                    if (chunked) {
                        const int32_t *ru = adj + off[u];
                        start = lo == INT32_MIN ? 0 : row_lower_bound(ru, du, lo);
                        const int32_t end = hi == INT32_MAX ? du : row_lower_bound(ru, du, hi);
                        len = end - start;
                    }
                }
            }
        }
        const bool is_long = work && len >= kWarp;
        const bool is_short = work && len > 0 && len < kWarp;
        // packed counts: work | long << 21 | short << 42
        const long long flags = (long long)work | ((long long)is_long << 21) | ((long long)is_short << 42);
        long long tot;
        const long long ex = block_scan<BLOCK, long long>(flags, &tot, wsum64);
        const int32_t npieces_mine = is_long ? (len + kPiece - 1) / kPiece : 0;
        int32_t tot_pieces;
        const int32_t pex = block_scan<BLOCK, int32_t>(npieces_mine, &tot_pieces, wsum32);
        const int32_t n_work = (int32_t)(tot & 0x1FFFFF);
        const int32_t n_long = (int32_t)((tot >> 21) & 0x1FFFFF);
        const int32_t n_short = (int32_t)((tot >> 42) & 0x1FFFFF);
        if (work) {
            const int32_t e = (int32_t)(ex & 0x1FFFFF);
            w_rel[e] = rel;
            w_u[e] = u;
            w_du[e] = du;
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

        // ---- long rows: warps grab pieces
        for (int guard = 0; guard < (1 << 30); ++guard) {
            int32_t p = 0;
            if (lane == 0) p = atomicAdd(&piece_ctr, 1);
            p = __shfl_sync(0xffffffffu, p, 0);
            if (p >= tot_pieces) break;
            int32_t lo_i = 0, hi_i = n_long;  // last l with l_poff[l] <= p
            while (hi_i - lo_i > 1) {
                const int32_t mid = (lo_i + hi_i) >> 1;
                if (l_poff[mid] <= p) lo_i = mid;
                else hi_i = mid;
            }
            const int32_t e = l_idx[lo_i];
            const int32_t o = (p - l_poff[lo_i]) * kPiece;
            const int32_t plen = min(kPiece, w_len[e] - o);
            const int32_t *src_row = adj + off[w_u[e]] + w_start[e] + o;
            int32_t x[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                const int k = lane + j * kWarp;
                x[j] = k < plen ? __ldg(src_row + k) : 0;
            }
            int c = 0;
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if (lane + j * kWarp < plen) c += table_has(t, logc, x[j]);
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0 && c) atomicAdd(&w_cnt[e], c);
        }
        // ---- short rows: one lane each, 32 per grab
        for (int guard = 0; guard < (1 << 30); ++guard) {
            int32_t q = 0;
            if (lane == 0) q = atomicAdd(&short_ctr, kWarp);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= n_short) break;
            const int32_t k = q + lane;
            if (k < n_short) {
                const int32_t e = s_idx[k];
                const int32_t *src_row = adj + off[w_u[e]] + w_start[e];
                const int32_t L = w_len[e];
                int c = 0;
                for (int32_t j0 = 0; j0 < L; j0 += kUnroll) {
                    int32_t x[kUnroll];
#pragma unroll
                    for (int j = 0; j < kUnroll; ++j) x[j] = j0 + j < L ? __ldg(src_row + j0 + j) : 0;
#pragma unroll
                    for (int j = 0; j < kUnroll; ++j)
                        if (j0 + j < L) c += table_has(t, logc, x[j]);
                }
                w_cnt[e] = c;
            }
        }
        __syncthreads();
        // ---- emit one owned edge per thread
        if (threadIdx.x < n_work) {
            const int32_t e = threadIdx.x;
            const int64_t s = b + w_rel[e];
            if (chunked) {
                if (w_cnt[e]) atomicAdd(acc + s, w_cnt[e]);
            } else {
                emit<WRITE_SIM, WRITE_CN>(s, w_cnt[e] + 2, w_du[e], dv, rev, pp, qq, sim, cn);
            }
        }
        __syncthreads();
    }
}

// Chunked owners: closed count = accumulated partial counts + 2; resets acc.
template <bool PRUNE, bool WRITE_SIM, bool WRITE_CN>
__global__ void __launch_bounds__(256) k_owner_finish(const int32_t *__restrict__ owners, int32_t nown,
                                                      const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                      const int32_t *__restrict__ deg, const uint32_t *__restrict__ rev,
                                                      QParams qp, uint8_t *__restrict__ sim,
                                                      int32_t *__restrict__ cn, int32_t *__restrict__ acc) {
    const int32_t v = owners[blockIdx.x];
    const int64_t b = off[v];
    const int32_t dv = (int32_t)(off[v + 1] - b);
    uint64_t pp, qq;
    qp.eps(v, pp, qq);
    for (int32_t k = threadIdx.x; k < dv; k += blockDim.x) {
        const int64_t s = b + k;
        const int32_t u = adj[s], du = deg[u];
        if (!dev::rank_less(du, u, dv, v)) continue;
        const int32_t a = acc[s];
        acc[s] = 0;
        if (PRUNE && dev::prune_dissimilar((uint64_t)du + 1, (uint64_t)dv + 1, pp, qq)) continue;
        emit<WRITE_SIM, WRITE_CN>(s, a + 2, du, dv, rev, pp, qq, sim, cn);
    }
}

// ------------------------------------------------------------ schedule
__device__ __forceinline__ int owner_class(int32_t d) {
    return d <= kSmallMax ? 0 : d <= 1024 ? 1 : d <= 8192 ? 2 : 3;
}

// Warp per vertex: owned work (probes) and the number of work items.
__global__ void __launch_bounds__(256) k_sched_count(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                     const int32_t *__restrict__ deg, int32_t n,
                                                     int32_t *__restrict__ nranges, unsigned long long *counts) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const int32_t dv = deg[v];
    if (dv == 0) return;
    const int cls = owner_class(dv);
    if (cls == 0) {
        if (lane == 0) { nranges[v] = 1; atomicAdd(counts + 0, 1ull); }
        return;
    }
    const int64_t b = off[v];
    unsigned long long w = 0;
    for (int32_t k = lane; k < dv; k += kWarp) {
        const int32_t u = adj[b + k], du = deg[u];
        if (dev::rank_less(du, u, dv, (int32_t)v)) w += (unsigned long long)du;
    }
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
        const int64_t nchunks = (dv + kChunk - 1) / kChunk;
        int64_t nr = (int64_t)((w + kItemWork - 1) / kItemWork);
        nr = max((int64_t)1, min(nr, (int64_t)(dv + 255) / 256));
        nranges[v] = (int32_t)nr;
        atomicAdd(counts + cls, (unsigned long long)(nchunks * nr));
        if (nchunks > 1) atomicAdd(counts + 4, 1ull);
    }
}

__global__ void k_sched_write(const int32_t *__restrict__ deg, int32_t n, const int32_t *__restrict__ nranges,
                              unsigned long long *cursor, int32_t *__restrict__ small, Item *__restrict__ i1,
                              Item *__restrict__ i2, Item *__restrict__ i3, int32_t *__restrict__ chunked) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t dv = deg[v];
    if (dv == 0) return;
    const int cls = owner_class(dv);
    if (cls == 0) {
        small[atomicAdd(cursor + 0, 1ull)] = (int32_t)v;
        return;
    }
    const int32_t nchunks = (dv + kChunk - 1) / kChunk;
    const int32_t nr = nranges[v];
    const int32_t len = (dv + nr - 1) / nr;
    Item *dst = cls == 1 ? i1 : cls == 2 ? i2 : i3;
    unsigned long long p = atomicAdd(cursor + cls, (unsigned long long)(nchunks * nr));
    for (int32_t c = 0; c < nchunks; ++c)
        for (int32_t r = 0; r < nr; ++r) {
            Item it;
            it.v = (int32_t)v;
            it.chunk = c;
            it.sb = r * len;
            it.se = min(dv, (r + 1) * len);
            dst[p++] = it;
        }
    if (nchunks > 1) chunked[atomicAdd(cursor + 4, 1ull)] = (int32_t)v;
}

}  // namespace

// Class table sizes (ints) and block sizes.
static const int kClassCap[4] = {0, 2048, 16384, 2 * kChunk};

scan_status owner_schedule_build(Graph *g) {
    Ctx *c = g->ctx;
    const int32_t n = g->n;
    if (n == 0 || g->nnz == 0) return SCAN_OK;
    DevBuf cnts;
    SCAN_TRY(dev_alloc(c, cnts, 8 * sizeof(unsigned long long)));
    auto *counts = (unsigned long long *)cnts.ptr;
    SCAN_CUDA(cudaMemsetAsync(counts, 0, 8 * sizeof(unsigned long long), c->stream));
    int32_t *nranges = (int32_t *)g->cnt.ptr;  // scratch int32[n+1]
    k_sched_count<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(
        (const int64_t *)g->off.ptr, (const int32_t *)g->adj.ptr, (const int32_t *)g->deg.ptr, n, nranges, counts);
    c->launches++;
    unsigned long long h[8];
    SCAN_CUDA(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    g->n_small = (int32_t)h[0];
    for (int k = 1; k < 4; ++k) g->n_items[k] = (int64_t)h[k];
    g->n_chunked = (int32_t)h[4];
    auto fail = [&](scan_status s) { dev_free(c, cnts); return s; };
    scan_status s = dev_alloc(c, g->owners_small, sizeof(int32_t) * (size_t)(h[0] + 1));
    for (int k = 1; k < 4 && s == SCAN_OK; ++k) s = dev_alloc(c, g->items[k], sizeof(Item) * (size_t)(h[k] + 1));
    if (s == SCAN_OK) s = dev_alloc(c, g->owners_chunked, sizeof(int32_t) * (size_t)(h[4] + 1));
    if (s == SCAN_OK && h[4] > 0) {
        s = dev_alloc(c, g->acc, sizeof(int32_t) * (size_t)g->nnz);
        if (s == SCAN_OK && cudaMemsetAsync(g->acc.ptr, 0, sizeof(int32_t) * (size_t)g->nnz, c->stream) != cudaSuccess)
            s = SCAN_ECUDA;
    }
    if (s != SCAN_OK) return fail(s);
    if (cudaMemsetAsync(counts, 0, 8 * sizeof(unsigned long long), c->stream) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "schedule reset"));
    k_sched_write<<<grid_for(n, 256), 256, 0, c->stream>>>(
        (const int32_t *)g->deg.ptr, n, nranges, counts, (int32_t *)g->owners_small.ptr, (Item *)g->items[1].ptr,
        (Item *)g->items[2].ptr, (Item *)g->items[3].ptr, (int32_t *)g->owners_chunked.ptr);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "schedule write"));
    dev_free(c, cnts);
    return SCAN_OK;
}

template <bool PRUNE, bool WRITE_SIM, bool WRITE_CN>
static scan_status launch_owner_t(Graph *g, const QParams &qp, int32_t *cn) {
    Ctx *c = g->ctx;
    auto *off = (const int64_t *)g->off.ptr;
    auto *adj = (const int32_t *)g->adj.ptr;
    auto *deg = (const int32_t *)g->deg.ptr;
    auto *rev = (const uint32_t *)g->rev.ptr;
    auto *sim = (uint8_t *)g->sim.ptr;
    auto *acc = (int32_t *)g->acc.ptr;
    // biggest tables first so the long items start early
    for (int cls = 3; cls >= 1; --cls) {
        const int64_t ni = g->n_items[cls];
        if (ni == 0) continue;
        const size_t smem = sizeof(int32_t) * (size_t)kClassCap[cls];
        const Item *items = (const Item *)g->items[cls].ptr;
        if (cls == 3) {
            auto kern = k_owner_cta<1024, PRUNE, WRITE_SIM, WRITE_CN>;
            SCAN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<(unsigned)ni, 1024, smem, c->stream>>>(items, off, adj, deg, rev, qp, sim, cn, acc);
        } else if (cls == 2) {
            auto kern = k_owner_cta<512, PRUNE, WRITE_SIM, WRITE_CN>;
            SCAN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<(unsigned)ni, 512, smem, c->stream>>>(items, off, adj, deg, rev, qp, sim, cn, acc);
        } else {
            k_owner_cta<256, PRUNE, WRITE_SIM, WRITE_CN><<<(unsigned)ni, 256, smem, c->stream>>>(
                items, off, adj, deg, rev, qp, sim, cn, acc);
        }
        c->launches++;
    }
    if (g->n_small > 0) {
        k_owner_small<PRUNE, WRITE_SIM, WRITE_CN><<<grid_for((int64_t)g->n_small * kWarp, 256, c->num_sms * 16), 256, 0,
                                                    c->stream>>>((const int32_t *)g->owners_small.ptr, g->n_small, off,
                                                                 adj, deg, rev, qp, sim, cn);
        c->launches++;
    }
    if (g->n_chunked > 0) {
        k_owner_finish<PRUNE, WRITE_SIM, WRITE_CN><<<(unsigned)g->n_chunked, 256, 0, c->stream>>>(
            (const int32_t *)g->owners_chunked.ptr, g->n_chunked, off, adj, deg, rev, qp, sim, cn, acc);
        c->launches++;
    }
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status launch_owner_isect(Graph *g, bool prune, bool write_sim, bool write_cn, const QParams &qp, int32_t *cn) {
    if (g->m == 0) return SCAN_OK;
    if (!g->owner_ready) {
        SCAN_TRY(owner_schedule_build(g));
        g->owner_ready = true;
    }
    if (prune) return launch_owner_t<true, true, false>(g, qp, cn);
    if (write_cn && !write_sim) return launch_owner_t<false, false, true>(g, qp, cn);
    return launch_owner_t<false, true, false>(g, qp, cn);
}

}  // namespace scan

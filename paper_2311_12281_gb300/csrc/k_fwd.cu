// k_fwd.cu -- closed common counts of every edge by degree-oriented triangle
// enumeration.
//
// Orient every edge from its lower to its higher (deg, id) endpoint (the
// degree-oriented edge array of Section 4.1); out(x) is x's list of higher
// neighbours, ordered by (deg, id) rank when no list exceeds kSortMax (else
// by id). For an edge the open common count |nbr(u) cap nbr(v)| is the number
// of triangles through it, and each triangle a < b < c (in that order) is
// found exactly once: at its middle vertex b, when out(a) of an in-neighbour
// a -- with rank-ordered lists only its suffix after b -- is streamed through
// a shared-memory table of out(b). A hit c then adds one to each of the three
// edges: (a, b) through the entry's sum, (b, c) through a per-owner counter
// in shared memory, and (a, c) by an atomic add at the streamed position of
// c in out(a). In a degree orientation out-degrees stay below sqrt(2m), so
// the tables are small, and the work is the sum over a of d+(a)(d+(a)-1)/2
// instead of the sum over edges of min(deg) that a per-edge intersection pays.
//
// Kernels: k_fwd_small (warp per small owner), k_fwd_ent (CTA per work item,
// streaming precomputed entry lists; the default), k_fwd_cta (CTA per work
// item deriving the entries round by round: the lean family and the fallback
// when the lists do not fit), k_fwd_finish (closed counts, eps-test, mirror).
//
// closed count of an edge = triangles through it + 2 (Definition 2.2 with
// closed neighbourhoods: both endpoints are in both N[.]).
#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr int kFwdSmallOut = 64;         // warp-level owners: out-degree bound
constexpr int kFwdSmallTable = 256;      // slots per warp table
constexpr int kFwdChunk = 4096;          // max out(b) elements per CTA table
// (the warp-owner probe bound and the probes per CTA item are per-graph
// schedule parameters: Graph::fwd_small_work, Graph::fwd_item_work)
constexpr int kFwdUnroll = 8;
constexpr unsigned long long kSlotEmpty = ~0ull;

// CTA item classes by the owner's out-degree: 0 up to 256 (128-thread CTAs,
// 8 KB tables), 1 up to 1024 (256 threads, hash tables up to 32 KB), 2 above
// (512 threads, tables of 4096-key chunks, 128 KB)
__host__ __device__ __forceinline__ int fwd_class(int32_t ob) { return ob <= 256 ? 0 : (ob <= 1024 ? 1 : 2); }

// log2 of the hash slots of a class's tables (8 bytes per slot: 8, 32 and
// 128 KB); a bitmap table must fit the same shared memory
__host__ __device__ __forceinline__ int fwd_cap_logs(int cls) { return cls == 0 ? 10 : (cls == 1 ? 12 : 14); }

// hash slots per key, as a shift: 2^3 in class 1 (load <= 1/8 up to 512
// keys), 2^2 in classes 0 and 2
__host__ __device__ __forceinline__ int fwd_load_shift(int cls) { return cls == 1 ? 3 : 2; }

// A CTA work item: owner v, value chunk of out(v), slot range [sb, se) of
// v's row; with precomputed entry lists, the item's entries start at e0 (the
// nlong long ones first, then the short ones). hspan > 0: the owner's table
// is a bitmap over the dense ids [hlo, hlo + hspan) (else a hash table).
struct FItem {
    int32_t v, chunk, sb, se;
    int64_t e0;
    int32_t nlong, nent;
    int32_t hlo, hspan;
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

// Membership filter in front of the table: one bit per hashed id (a
// different hash from the table's), about 32 bits per element, so most
// probes of absent ids end after one shared-memory load.
__device__ __forceinline__ uint32_t fbit(int32_t x, int logb) { return ((uint32_t)x * 0x85EBCA6Bu) >> (32 - logb); }

__device__ __forceinline__ void fbits_set(uint32_t *bm, int logb, int32_t x) {
    const uint32_t h = fbit(x, logb);
    atomicOr(bm + (h >> 5), 1u << (h & 31));
}

__device__ __forceinline__ bool fbits_has(const uint32_t *bm, int logb, int32_t x) {
    const uint32_t h = fbit(x, logb);
    return (bm[h >> 5] >> (h & 31)) & 1u;
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

__device__ __forceinline__ unsigned long long rank_key(const int32_t *__restrict__ deg, int32_t x) {
    return ((unsigned long long)(uint32_t)deg[x] << 32) | (uint32_t)x;
}

// first index of a rank-sorted row whose (deg, id) key is >= key
__device__ __forceinline__ int32_t rank_lower_bound(const int32_t *__restrict__ r, int32_t len,
                                                    const int32_t *__restrict__ deg, unsigned long long key) {
    int32_t lo = 0, hi = len;
    for (int it = 0; it < 40 && lo < hi; ++it) {
        const int32_t mid = (lo + hi) >> 1;
        if (rank_key(deg, __ldg(r + mid)) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

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
                                         const uint32_t *bm, int logb, int32_t *ocnt) {
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
            if (k < k1 && fbits_has(bm, logb, x[j])) {
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
// One warp-level owner b (out-degree <= 64): a linear-probing hash table of
// out(b) with a membership filter in front, in the warp's own shared memory
// (t: kFwdSmallTable slots, bm: 64 words, ocnt: kFwdSmallOut counts); every
// in-neighbour a below b streams its part of out(a) through it.
__device__ __forceinline__ void fwd_small_owner(int32_t b, unsigned long long *t, uint32_t *bm, int32_t *ocnt,
                                                const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                const int32_t *__restrict__ deg, const int64_t *__restrict__ foff,
                                                const int32_t *__restrict__ fadj, const uint32_t *__restrict__ fin,
                                                int32_t *__restrict__ fcnt, int rank_sorted) {
    const int lane = threadIdx.x & 31;
    const int64_t fb = foff[b];
    const int32_t db = deg[b], ob = (int32_t)(foff[b + 1] - fb);
    const int logc = max(5, fceil_log2(4 * ob));
    const int logb = max(5, fceil_log2(32 * ob));  // <= 2048 bits
    for (int k = lane; k < (1 << logc); k += kWarp) t[k] = kSlotEmpty;
    for (int k = lane; k < (1 << (logb - 5)); k += kWarp) bm[k] = 0u;
    for (int k = lane; k < kFwdSmallOut; k += kWarp) ocnt[k] = 0;
    __syncwarp();
    for (int k = lane; k < ob; k += kWarp) {
        const int32_t x = fadj[fb + k];
        ftab_insert(t, logc, x, k);
        fbits_set(bm, logb, x);
    }
    __syncwarp();
    const int64_t rb = off[b];
    for (int32_t g0 = 0; g0 < db; g0 += kWarp) {
        const int64_t s = rb + g0 + lane;
        int32_t oa = 0, st = 0;
        int64_t fa = 0;
        if (g0 + lane < db) {
            const int32_t a = adj[s];
            const int32_t da = deg[a];
            if (dev::rank_less(da, a, db, b)) {
                fa = foff[a];
                oa = (int32_t)(foff[a + 1] - fa);
                // a rank-sorted out(a) holds b's common neighbours above b only
                if (rank_sorted) st = (int32_t)((int64_t)fin[s] - fa) + 1;
            }
        }
        const int32_t len = oa - st;
        int mine = 0;
        if (len > 0 && len < 16) mine = probe_run<4>(fadj + fa, fcnt + fa, st, oa, 1, t, logc, bm, logb, ocnt);
        unsigned longs = __ballot_sync(0xffffffffu, len >= 16);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t fas = __shfl_sync(0xffffffffu, fa, src);
            const int32_t oas = __shfl_sync(0xffffffffu, oa, src);
            const int32_t sts = __shfl_sync(0xffffffffu, st, src);
            int c = probe_run<kFwdUnroll>(fadj + fas, fcnt + fas, sts + lane, oas, kWarp, t, logc, bm, logb, ocnt);
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

// shared memory of one warp-level owner: table, filter, counts (in 32-bit words)
constexpr int kSmallWarpWords = 2 * kFwdSmallTable + 64 + kFwdSmallOut;

__global__ void __launch_bounds__(256) k_fwd_small(const int32_t *__restrict__ owners, int32_t nown,
                                                   const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                   const int32_t *__restrict__ deg, const int64_t *__restrict__ foff,
                                                   const int32_t *__restrict__ fadj, const uint32_t *__restrict__ fin,
                                                   int32_t *__restrict__ fcnt, int rank_sorted) {
    __shared__ unsigned long long tables[8][kFwdSmallTable];
    __shared__ uint32_t bitmaps[8][64];
    __shared__ int32_t ocnts[8][kFwdSmallOut];
    const int wid = threadIdx.x >> 5;
    const int warps_total = gridDim.x * 8;
    for (int32_t i = blockIdx.x * 8 + wid; i < nown; i += warps_total)
        fwd_small_owner(owners[i], tables[wid], bitmaps[wid], ocnts[wid], off, adj, deg, foff, fadj, fin, fcnt,
                        rank_sorted);
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

// Table of the CTA owners: buckets of two (key, count) pairs, 16 bytes, so
// one 128-bit shared-memory load answers most lookups. A key goes to the
// first bucket, from its hash on, with a free pair; a bucket whose second
// key is empty never overflowed, which ends a lookup. Empty key: -1.
__device__ __forceinline__ void btab_insert(int4 *tab, int lognb, int32_t key) {
    const uint32_t mask = (1u << lognb) - 1u;
    uint32_t h = fhash(key, lognb);
    for (uint32_t it = 0; it <= mask; ++it) {
        int *w = (int *)(tab + h);
        if (atomicCAS(w + 0, -1, key) == -1) return;
        if (atomicCAS(w + 2, -1, key) == -1) return;
        h = (h + 1) & mask;
    }
}

// index (in ints) of key's count word, or -1
__device__ __forceinline__ int32_t btab_find(const int4 *tab, int lognb, int32_t key) {
    const uint32_t mask = (1u << lognb) - 1u;
    uint32_t h = fhash(key, lognb);
    for (uint32_t it = 0; it <= mask; ++it) {
        const int4 b = tab[h];
        if (b.x == key) return (int32_t)(4 * h + 1);
        if (b.z == key) return (int32_t)(4 * h + 3);
        if (b.z == -1) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

constexpr int kStepsPerGroup = 4;  // 32-position steps whose loads are issued together

// One CTA per item (owner b, value chunk of out(b), slot range of b's row).
// The rows of b are taken BLOCK at a time. Each in-neighbour a of such a
// round with something to stream contributes an entry: the part of out(a)
// that can close a triangle a < b < c. The entries are compacted and their
// lengths prefix-summed into one flat range of probe positions, which the
// warps split evenly. A warp walks its share 32 consecutive positions per
// step, lane l on position q0 + l: the entries starting inside the step are
// found with one shared-memory load per lane and a warp-wide OR of their
// offsets, so the walk is uniform however short or long the entries are.
// A hit c adds one to (b, c) in the table, to (a, c) at the streamed slot in
// global memory, and to (a, b) through the entry's shared counter.
// Dynamic shared memory: 2^cap_lognb buckets.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_fwd_cta(const FItem *__restrict__ items, const int64_t *__restrict__ off,
                                                   const int32_t *__restrict__ adj, const int32_t *__restrict__ deg,
                                                   const int64_t *__restrict__ foff, const int32_t *__restrict__ fadj,
                                                   const uint32_t *__restrict__ fin, int32_t *__restrict__ fcnt,
                                                   int cap_lognb, int load_shift, int rank_sorted) {
    extern __shared__ int4 btab[];
    int *tword = (int *)btab;
    __shared__ int32_t c_pos[BLOCK + 1];   // flat start of each compacted entry; c_pos[nwork] = total
    __shared__ int32_t c_base[BLOCK + 1];  // fadj index of an entry's first id, minus its flat start
    __shared__ uint32_t c_fin[BLOCK];      // fcnt index of the entry's edge (a, b)
    __shared__ int32_t e_cnt[BLOCK];       // triangles found per entry
    __shared__ long long wsum[BLOCK / 32 + 1];

    const FItem it = items[blockIdx.x];
    const int32_t b = it.v;
    const int64_t rb = off[b], fb = foff[b];
    const int32_t db = (int32_t)(off[b + 1] - rb), ob = (int32_t)(foff[b + 1] - fb);
    const int32_t tb = it.chunk * kFwdChunk, te = min(tb + kFwdChunk, ob), tlen = te - tb;
    const bool chunked = ob > kFwdChunk;
    // the chunk's bounds, as ids (id-sorted lists) or as rank keys (rank-sorted)
    const int32_t lo = tb == 0 ? INT32_MIN : fadj[fb + tb];
    const int32_t hi = te == ob ? INT32_MAX : fadj[fb + te];
    const unsigned long long lo_key = tb == 0 ? 0ull : rank_key(deg, lo);
    const unsigned long long hi_key = te == ob ? ~0ull : rank_key(deg, hi);
    // buckets: 2^load_shift per key (two pairs each), at most 2^cap_lognb
    const int lognb = min(cap_lognb, max(4, fceil_log2(tlen << load_shift)));
    for (int k = threadIdx.x; k < (1 << lognb); k += BLOCK) btab[k] = make_int4(-1, 0, -1, 0);
    __syncthreads();
    for (int k = threadIdx.x; k < tlen; k += BLOCK) btab_insert(btab, lognb, fadj[fb + tb + k]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned le_mask = 0xffffffffu >> (31 - lane);  // lanes 0..lane
    constexpr long long kIdx = 1ll << 40;

    for (int32_t r0 = it.sb; r0 < it.se; r0 += BLOCK) {
        const int32_t rel = r0 + threadIdx.x;
        bool work = false;
        int32_t start = 0, len = 0;
        int64_t fa = 0;
        uint32_t fab = 0;
        if (rel < it.se) {
            const int64_t s = rb + rel;
            const int32_t a = adj[s], da = deg[a];
            if (dev::rank_less(da, a, db, b)) {
                fa = foff[a];
                const int32_t oa = (int32_t)(foff[a + 1] - fa);
                const int32_t *row = fadj + fa;
                int32_t end = oa;
                fab = fin[s];
                if (rank_sorted) {
                    // common neighbours of a and b rank above b: the suffix after b
                    start = (int32_t)((int64_t)fab - fa) + 1;
                    if (chunked) {
                        start = max(start, rank_lower_bound(row, oa, deg, lo_key));
                        end = hi_key == ~0ull ? oa : rank_lower_bound(row, oa, deg, hi_key);
                    }
                } else if (chunked && oa > 0) {
                    start = lo == INT32_MIN ? 0 : lower_bound_row(row, oa, lo);
                    end = hi == INT32_MAX ? oa : lower_bound_row(row, oa, hi);
                }
                len = max(end - start, 0);
                work = len > 0;
            }
        }
        // one scan: compacted index in the high bits, flat position in the low 40
        long long tot;
        const long long ex = fblock_scan<BLOCK, long long>(work ? kIdx + len : 0ll, &tot, wsum);
        const int32_t nwork = (int32_t)(tot >> 40), total = (int32_t)(tot & (kIdx - 1));
        if (work) {
            const int32_t k = (int32_t)(ex >> 40), pos = (int32_t)(ex & (kIdx - 1));
            c_pos[k] = pos;
            c_base[k] = (int32_t)(fa + start - pos);  // fadj indices are < m < 2^31
            c_fin[k] = fab;
            e_cnt[k] = 0;
        }
        if (threadIdx.x == 0) {
            c_pos[nwork] = total;
            c_base[nwork] = 0;
        }
        __syncthreads();
        // this warp's share of [0, total), in whole steps
        const int32_t share = (((total + BLOCK / 32 - 1) / (BLOCK / 32)) + 31) & ~31;
        const int32_t q_begin = warp * share, q_end = min(total, q_begin + share);
        if (q_begin < q_end) {
            // entry holding q_begin: the last e with c_pos[e] <= q_begin
            int32_t el = 0, eh = nwork;
            while (eh - el > 1) {
                const int32_t mid = (el + eh) >> 1;
                if (c_pos[mid] <= q_begin) el = mid;
                else eh = mid;
            }
            int32_t e0 = el;  // entry of the current step's first position
            for (int32_t g0 = q_begin; g0 < q_end; g0 += 32 * kStepsPerGroup) {
                int32_t aj[kStepsPerGroup], ej[kStepsPerGroup];
                unsigned mj[kStepsPerGroup];
#pragma unroll
                for (int u = 0; u < kStepsPerGroup; ++u) {
                    const int32_t qs = g0 + 32 * u;
                    // entries starting inside this step (offsets 1..31) or at the next one (32)
                    const int32_t bk = c_pos[min(e0 + 1 + lane, nwork)];
                    const int32_t d = bk - qs;
                    const unsigned m = __reduce_or_sync(0xffffffffu, (d > 0 && d < 32) ? (1u << d) : 0u);
                    const int32_t e = e0 + __popc(m & le_mask);
                    const int32_t q = qs + lane;
                    ej[u] = e;
                    mj[u] = m;
                    aj[u] = q < q_end ? c_base[e] + q : -1;
                    e0 += __popc(m) + (__any_sync(0xffffffffu, d == 32) ? 1 : 0);
                }
                int32_t xj[kStepsPerGroup];
#pragma unroll
                for (int u = 0; u < kStepsPerGroup; ++u) xj[u] = aj[u] >= 0 ? __ldg(fadj + aj[u]) : -1;
#pragma unroll
                for (int u = 0; u < kStepsPerGroup; ++u) {
                    bool hit = false;
                    if (aj[u] >= 0) {
                        const int32_t w = btab_find(btab, lognb, xj[u]);
                        if (w >= 0) {
                            hit = true;
                            atomicAdd(tword + w, 1);       // edge (b, c)
                            atomicAdd(fcnt + aj[u], 1);    // edge (a, c)
                        }
                    }
                    // edge (a, b): one add per step when the step lies in one entry
                    const unsigned hm = __ballot_sync(0xffffffffu, hit);
                    if (mj[u] == 0) {
                        if (lane == 0 && hm) atomicAdd(&e_cnt[ej[u]], __popc(hm));
                    } else if (hit) {
                        atomicAdd(&e_cnt[ej[u]], 1);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < nwork && e_cnt[threadIdx.x]) atomicAdd(fcnt + c_fin[threadIdx.x], e_cnt[threadIdx.x]);
        __syncthreads();
    }
    for (int k = threadIdx.x; k < tlen; k += BLOCK) {
        const int32_t w = btab_find(btab, lognb, fadj[fb + tb + k]);
        if (w >= 0 && tword[w]) atomicAdd(fcnt + fb + tb + k, tword[w]);
    }
}

// ------------------------------------------------------------ precomputed entries
// The entries of a work item (one per in-neighbour a of its owner b with a
// non-empty stretch of out(a) to stream) depend on the graph only, so they
// are built once, sorted by length -- long ones (>= kLongEntry ids, coarse
// descending) first, then short ones (exact descending) -- and every count
// just streams them.
constexpr int kLongEntry = 32;  // entries this long are streamed by a whole warp
constexpr int kEntBuckets = 58; // 27 long (by log2 length) + 31 short (by length)

__device__ __forceinline__ int ent_bucket(int32_t len) {
    if (len >= kLongEntry) return 26 - (31 - __clz(len) - 5);  // log2 5..31 -> 26..0
    return 27 + (31 - len);                                    // 31..1 -> 27..57
}

// Chunk bounds of an item, as ids (id-sorted lists) or rank keys.
struct ItemBounds {
    int32_t lo, hi;
    unsigned long long lo_key, hi_key;
    bool chunked;
};

__device__ __forceinline__ ItemBounds item_bounds(const FItem &it, const int32_t *__restrict__ deg,
                                                  const int32_t *__restrict__ fadj, int64_t fb, int32_t ob) {
    ItemBounds r;
    const int32_t tb = it.chunk * kFwdChunk, te = min(tb + kFwdChunk, ob);
    r.chunked = ob > kFwdChunk;
    r.lo = tb == 0 ? INT32_MIN : fadj[fb + tb];
    r.hi = te == ob ? INT32_MAX : fadj[fb + te];
    r.lo_key = tb == 0 ? 0ull : rank_key(deg, r.lo);
    r.hi_key = te == ob ? ~0ull : rank_key(deg, r.hi);
    return r;
}

// Entry of row slot s of owner b: stretch [fa + start, fa + start + len) of
// out(a) and the fcnt index of (a, b); len = 0 when there is none.
__device__ __forceinline__ int32_t item_entry(int64_t s, int32_t b, int32_t db, const ItemBounds &ib,
                                              const int32_t *__restrict__ adj, const int32_t *__restrict__ deg,
                                              const int64_t *__restrict__ foff, const int32_t *__restrict__ fadj,
                                              const uint32_t *__restrict__ fin, int rank_sorted, int32_t *base,
                                              uint32_t *fab) {
    const int32_t a = adj[s], da = deg[a];
    if (!dev::rank_less(da, a, db, b)) return 0;
    const int64_t fa = foff[a];
    const int32_t oa = (int32_t)(foff[a + 1] - fa);
    const int32_t *row = fadj + fa;
    int32_t start = 0, end = oa;
    *fab = fin[s];
    if (rank_sorted) {
        // common neighbours of a and b rank above b: the suffix after b
        start = (int32_t)((int64_t)*fab - fa) + 1;
        if (ib.chunked) {
            start = max(start, rank_lower_bound(row, oa, deg, ib.lo_key));
            end = ib.hi_key == ~0ull ? oa : rank_lower_bound(row, oa, deg, ib.hi_key);
        }
    } else if (ib.chunked && oa > 0) {
        start = ib.lo == INT32_MIN ? 0 : lower_bound_row(row, oa, ib.lo);
        end = ib.hi == INT32_MAX ? oa : lower_bound_row(row, oa, ib.hi);
    }
    *base = (int32_t)(fa + start);  // fadj indices are < m < 2^31
    return max(end - start, 0);
}

// CTA per item: number of entries
__global__ void __launch_bounds__(256) k_fwd_ent_count(const FItem *__restrict__ items, int64_t nitems,
                                                       const int64_t *__restrict__ off,
                                                       const int32_t *__restrict__ adj,
                                                       const int32_t *__restrict__ deg,
                                                       const int64_t *__restrict__ foff,
                                                       const int32_t *__restrict__ fadj,
                                                       const uint32_t *__restrict__ fin, int rank_sorted,
                                                       int32_t *__restrict__ nent) {
    __shared__ int32_t wsum[256 / 32 + 1];
    const FItem it = items[blockIdx.x];
    const int32_t b = it.v;
    const int64_t rb = off[b], fb = foff[b];
    const int32_t db = (int32_t)(off[b + 1] - rb), ob = (int32_t)(foff[b + 1] - fb);
    const ItemBounds ib = item_bounds(it, deg, fadj, fb, ob);
    int32_t cnt = 0;
    for (int32_t rel = it.sb + threadIdx.x; rel < it.se; rel += 256) {
        int32_t base;
        uint32_t fab;
        cnt += item_entry(rb + rel, b, db, ib, adj, deg, foff, fadj, fin, rank_sorted, &base, &fab) > 0;
    }
    int32_t total;
    fblock_scan<256, int32_t>(cnt, &total, wsum);
    if (threadIdx.x == 0) nent[blockIdx.x] = total;
}

// CTA per item: the entries, bucketed by length, from eoff[item] on
__global__ void __launch_bounds__(256) k_fwd_ent_write(FItem *__restrict__ items, int64_t nitems,
                                                       const int64_t *__restrict__ eoff, int64_t ebase_shift,
                                                       const int64_t *__restrict__ off,
                                                       const int32_t *__restrict__ adj,
                                                       const int32_t *__restrict__ deg,
                                                       const int64_t *__restrict__ foff,
                                                       const int32_t *__restrict__ fadj,
                                                       const uint32_t *__restrict__ fin, int rank_sorted,
                                                       int32_t *__restrict__ e_base, int32_t *__restrict__ e_len,
                                                       uint32_t *__restrict__ e_fin,
                                                       const int32_t *__restrict__ fhid, int32_t cap_words,
                                                       int cap_logs, int load_shift, int32_t *need_words) {
    __shared__ int32_t hist[kEntBuckets], boff[kEntBuckets];
    __shared__ int32_t hmin, hmax;
    FItem it = items[blockIdx.x];
    const int32_t b = it.v;
    const int64_t rb = off[b], fb = foff[b];
    const int32_t db = (int32_t)(off[b + 1] - rb), ob = (int32_t)(foff[b + 1] - fb);
    const ItemBounds ib = item_bounds(it, deg, fadj, fb, ob);
    for (int k = threadIdx.x; k < kEntBuckets; k += 256) hist[k] = 0;
    if (threadIdx.x == 0) {
        hmin = INT32_MAX;
        hmax = -1;
    }
    __syncthreads();
    // dense-id span of the item's part of out(b): its bitmap table's extent
    const int32_t tb = it.chunk * kFwdChunk, tlen = min(tb + kFwdChunk, ob) - tb;
    if (fhid != nullptr) {
        int32_t lo = INT32_MAX, hi = -1, bad = 0;
        for (int32_t k = threadIdx.x; k < tlen; k += 256) {
            const int32_t h = fhid[fb + tb + k];
            bad |= h < 0;
            lo = min(lo, h);
            hi = max(hi, h);
        }
        if (bad) hi = INT32_MAX;  // an element without a dense id: no bitmap
        atomicMin(&hmin, lo);
        atomicMax(&hmax, hi);
    }
    for (int32_t rel = it.sb + threadIdx.x; rel < it.se; rel += 256) {
        int32_t base;
        uint32_t fab;
        const int32_t len = item_entry(rb + rel, b, db, ib, adj, deg, foff, fadj, fin, rank_sorted, &base, &fab);
        if (len > 0) atomicAdd(&hist[ent_bucket(len)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0, nlong = 0;
        for (int k = 0; k < kEntBuckets; ++k) {
            boff[k] = acc;
            acc += hist[k];
            if (k == 26) nlong = acc;
            hist[k] = 0;
        }
        it.e0 = ebase_shift + eoff[blockIdx.x];
        it.nlong = nlong;
        it.nent = acc;
        // 16 ids per 32-bit word (the high half holds the word's prefix
        // count) through the word of id span, then one count per element of
        // the part of out(b)
        it.hlo = 0;
        it.hspan = 0;
        int32_t words = 2 << min(cap_logs, max(5, fceil_log2(tlen << load_shift)));  // hash: keys and counts
        if (fhid != nullptr && hmax >= hmin && hmax != INT32_MAX) {
            const int64_t span = (int64_t)hmax - hmin + 1;
            if (span / 16 + 1 + tlen <= (int64_t)cap_words) {
                it.hlo = hmin;
                it.hspan = (int32_t)span;
                words = (int32_t)(span / 16 + 1 + tlen);
            }
        }
        atomicMax(need_words, words);
        items[blockIdx.x] = it;
    }
    __syncthreads();
    const int64_t e0 = ebase_shift + eoff[blockIdx.x];
    for (int32_t rel = it.sb + threadIdx.x; rel < it.se; rel += 256) {
        int32_t base;
        uint32_t fab;
        const int32_t len = item_entry(rb + rel, b, db, ib, adj, deg, foff, fadj, fin, rank_sorted, &base, &fab);
        if (len > 0) {
            const int k = ent_bucket(len);
            const int64_t e = e0 + boff[k] + atomicAdd(&hist[k], 1);
            e_base[e] = base;
            e_len[e] = len;
            e_fin[e] = fab;
        }
    }
}

// Table of the streaming kernel: 32-bit keys (empty: -1) and a count per
// slot. Two-choice cuckoo hashing: a key sits at one of its two hashed slots,
// so a lookup is two independent shared-memory loads and no loop, and the
// lanes of a warp never wait on one another's collision chains (with linear
// probing at load 1/8 almost every warp had a lane on a second probe). Keys
// are placed by eviction chains; a table with a chain longer than
// kCuckooKicks is rebuilt with linear probing and looked up that way (a
// CTA-wide choice, so no lane diverges on it).
struct FTable {
    int *keys;  // 2^logs keys
    int *cnt;   // 2^logs counts
    int logs;
};

constexpr int kCuckooKicks = 64;

// second slot: differs from the first in at least the lowest bit
__device__ __forceinline__ uint32_t fhash_alt(int32_t x, uint32_t h1, int logc) {
    return h1 ^ ((((uint32_t)x * 0x85EBCA77u) >> (32 - logc)) | 1u);
}

// true when placed; false when the chain ran out (a key is then missing)
__device__ __forceinline__ bool ck_insert(const FTable &t, int32_t key) {
    uint32_t h = fhash(key, t.logs);
    for (int it = 0; it < kCuckooKicks; ++it) {
        const int old = atomicExch(t.keys + h, key);
        if (old == -1) return true;
        key = old;  // evicted: it moves to its other slot
        const uint32_t h1 = fhash(key, t.logs);
        h = h == h1 ? fhash_alt(key, h1, t.logs) : h1;
    }
    return false;
}

// slot of key (>= 0), or -1; a key of -2 finds nothing
__device__ __forceinline__ int32_t ck_find(const FTable &t, int32_t key) {
    const uint32_t h1 = fhash(key, t.logs), h2 = fhash_alt(key, h1, t.logs);
    const int y1 = t.keys[h1], y2 = t.keys[h2];
    return y1 == key ? (int32_t)h1 : (y2 == key ? (int32_t)h2 : -1);
}

__device__ __forceinline__ void lp_insert(const FTable &t, int32_t key) {
    const uint32_t mask = (1u << t.logs) - 1u;
    uint32_t h = fhash(key, t.logs);
    for (uint32_t it = 0; it <= mask; ++it) {
        const int old = atomicCAS(t.keys + h, -1, key);
        if (old == -1 || old == key) return;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int32_t lp_find(const FTable &t, int32_t key) {
    const uint32_t mask = (1u << t.logs) - 1u;
    uint32_t h = fhash(key, t.logs);
    int32_t y = t.keys[h];
    if (y == key) return (int32_t)h;
    for (uint32_t it = 1; it <= mask && y != -1; ++it) {
        h = (h + 1) & mask;
        y = t.keys[h];
        if (y == key) return (int32_t)h;
    }
    return -1;
}

template <bool LP>
__device__ __forceinline__ int32_t tab_find(const FTable &t, int32_t key) {
    return LP ? lp_find(t, key) : ck_find(t, key);
}

// Hash table of an owner, as the streaming loop sees it: count slot of an id.
template <bool LP>
struct HashTab {
    FTable t;
    __device__ __forceinline__ int32_t find(int32_t x) const { return tab_find<LP>(t, x); }
    __device__ __forceinline__ int *counts() const { return t.cnt; }
};

// Bitmap table over dense ids. Every vertex has a dense id, given in order of
// degree level (floor(log2 deg)), highest level first, then by id; an owner b
// and every element it meets (its out-neighbours, and the streamed suffix
// elements, all ranked above b) have degree >= deg(b), so the ids an owner
// meets stay below the count of vertices of its level and above. Each 32-bit
// word holds 16 ids in its low half and, in its high half, the number of
// the owner's elements in the words below it, so one load answers a probe:
// a set bit, and the element's count slot = prefix + set bits below it.
struct BitTab {
    uint32_t *w;
    int *cnt;
    int32_t lo;
    uint32_t span;
    __device__ __forceinline__ int32_t find(int32_t x) const {
        // -2 padding and ids below lo wrap above span; every id at or past the
        // span reads the zero word after the bitmap, so no branch is needed
        const uint32_t r = min((uint32_t)(x - lo), span);
        const uint32_t y = w[r >> 4], bit = 1u << (r & 15u);
        return (y & bit) ? (int32_t)((y >> 16) + __popc(y & (bit - 1u))) : -1;
    }
    __device__ __forceinline__ int *counts() const { return cnt; }
};

constexpr int kEntUnroll = 4;
constexpr int kEntBatch = 8;  // long entries a warp takes at a time

// Streams the item's entries: long ones one per warp (taken in turn, lanes on
// consecutive ids), then short ones 32 at a time, one per lane (neighbours in
// the sorted order have about the same length, so the lanes stay busy).
// Positions past an entry's end read as -2, which no lookup finds. `xs` is
// what the table is keyed by, position for position with fadj: the vertex
// ids for a hash table, the dense ids for a bitmap.
template <class TAB>
__device__ __forceinline__ void ent_stream(const FItem &it, const TAB &t, const int32_t *__restrict__ xs,
                                           const int32_t *__restrict__ e_base, const int32_t *__restrict__ e_len,
                                           const uint32_t *__restrict__ e_fin, int32_t *__restrict__ fcnt,
                                           int32_t *next_long, int32_t *next_short) {
    const int lane = threadIdx.x & 31;
    int *tc = t.counts();
    const int32_t nlong = it.nlong, nshort = it.nent - it.nlong;
    // Long entries, kEntBatch at a time per warp: lane l holds the descriptor
    // of the batch's entry l (one load per array for the whole batch), and
    // the warp streams the batch's entries one after the other.
    for (int32_t guard = 0; guard <= nlong; guard += kEntBatch) {
        int32_t k0 = 0;
        if (lane == 0) k0 = atomicAdd(next_long, kEntBatch);
        k0 = __shfl_sync(0xffffffffu, k0, 0);
        if (k0 >= nlong) break;
        const int nb = min(kEntBatch, nlong - k0);
        int32_t deb = 0, del = 0;
        uint32_t def = 0;
        if (lane < nb) {
            const int64_t e = it.e0 + k0 + lane;
            deb = e_base[e];
            del = e_len[e];
            def = e_fin[e];
        }
        for (int i = 0; i < nb; ++i) {
            const int32_t eb = __shfl_sync(0xffffffffu, deb, i), el = __shfl_sync(0xffffffffu, del, i);
            int c = 0;
            // whole groups of kEntUnroll * 32 ids: every lane busy, no bounds checks
            int32_t j0 = 0;
            for (; j0 + kWarp * kEntUnroll <= el; j0 += kWarp * kEntUnroll) {
                int32_t x[kEntUnroll];
#pragma unroll
                for (int u = 0; u < kEntUnroll; ++u) x[u] = __ldg(xs + eb + j0 + u * kWarp + lane);
#pragma unroll
                for (int u = 0; u < kEntUnroll; ++u) {
                    const int32_t r = t.find(x[u]);
                    if (r >= 0) {
                        ++c;
                        atomicAdd(tc + r, 1);                                // edge (b, c)
                        atomicAdd(fcnt + (eb + j0 + u * kWarp + lane), 1);  // edge (a, c)
                    }
                }
            }
            // the tail (fewer than kEntUnroll * 32 ids): its loads issued together
            if (j0 < el) {
                int32_t x[kEntUnroll];
#pragma unroll
                for (int u = 0; u < kEntUnroll; ++u) {
                    const int32_t j = j0 + u * kWarp + lane;
                    x[u] = j < el ? __ldg(xs + eb + j) : -2;
                }
#pragma unroll
                for (int u = 0; u < kEntUnroll; ++u) {
                    if (j0 + u * kWarp >= el) break;  // warp-uniform: no lane has work left
                    const int32_t r = t.find(x[u]);
                    if (r >= 0) {
                        ++c;
                        atomicAdd(tc + r, 1);
                        atomicAdd(fcnt + (eb + j0 + u * kWarp + lane), 1);
                    }
                }
            }
            c = __reduce_add_sync(0xffffffffu, c);
            const uint32_t ef = __shfl_sync(0xffffffffu, def, i);
            if (lane == 0 && c) atomicAdd(fcnt + ef, c);  // edge (a, b)
        }
    }
    for (int32_t guard = 0; guard <= nshort; guard += kWarp) {
        int32_t k0 = 0;
        if (lane == 0) k0 = atomicAdd(next_short, kWarp);
        k0 = __shfl_sync(0xffffffffu, k0, 0);
        if (k0 >= nshort) break;
        const int32_t k = k0 + lane;
        if (k < nshort) {
            const int64_t e = it.e0 + nlong + k;
            const int32_t eb = e_base[e], el = e_len[e];
            int c = 0;
            for (int32_t j0 = 0; j0 < el; j0 += 4) {
                int32_t x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = j0 + u < el ? __ldg(xs + eb + j0 + u) : -2;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t r = t.find(x[u]);
                    if (r >= 0) {
                        ++c;
                        atomicAdd(tc + r, 1);
                        atomicAdd(fcnt + (eb + j0 + u), 1);
                    }
                }
            }
            if (c) atomicAdd(fcnt + e_fin[e], c);
        }
    }
}

// A team of threads that builds and streams one owner table: the whole CTA,
// or a quarter of it in the persistent kernel, synchronised by its own
// named barrier (1 + id; barrier 0 is __syncthreads).
template <int SIZE, bool WHOLE>
struct Team {
    static constexpr int size = SIZE;
    int tid, id;
    __device__ __forceinline__ void sync() const {
        if (WHOLE) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(1 + id), "r"(SIZE) : "memory");
    }
};

// Shared counters of a team: long and short entries taken, a failed cuckoo
// chain, and the per-warp totals of the bitmap prefix counts.
struct TeamVars {
    int32_t next_long, next_short, failed;
    int32_t wtot[16];
};

// the owner's counts, added to its out-edges (b, c)
template <class TEAM, class TAB>
__device__ __forceinline__ void ent_flush(const TEAM &tm, const TAB &t, const int32_t *__restrict__ xs, int64_t base,
                                          int32_t tlen, int32_t *__restrict__ fcnt) {
    const int *tc = t.counts();
    for (int k = tm.tid; k < tlen; k += tm.size) {
        const int32_t r = t.find(xs[base + k]);
        if (r >= 0 && tc[r]) atomicAdd(fcnt + base + k, tc[r]);
    }
}

// Bitmap table of the item's part of out(b) (dense ids xs[base, base+tlen)):
// clear, set the bits, then each word's prefix count, by warps walking
// consecutive words (lane l on word w0 + 32j + l: no bank conflicts).
template <class TEAM>
__device__ __forceinline__ void bit_build(const TEAM &tm, const BitTab &t, const int32_t *__restrict__ xs,
                                          int64_t base, int32_t tlen, int32_t *wtot) {
    const int lane = tm.tid & 31, wid = tm.tid >> 5;
    constexpr int nwarps = TEAM::size >> 5;
    const int32_t nw = (int32_t)(t.span >> 4) + 1;  // through the word of id span (no member: zero)
    for (int k = tm.tid; k < nw; k += tm.size) t.w[k] = 0u;
    for (int k = tm.tid; k < tlen; k += tm.size) t.cnt[k] = 0;
    tm.sync();
    for (int k = tm.tid; k < tlen; k += tm.size) {
        const uint32_t r = (uint32_t)(xs[base + k] - t.lo);
        atomicOr(t.w + (r >> 4), 1u << (r & 15u));
    }
    tm.sync();
    const int32_t per = ((nw + nwarps - 1) / nwarps + 31) & ~31;
    const int32_t w0 = min(nw, wid * per), w1 = min(nw, w0 + per);
    int tot = 0;
    for (int32_t k = w0 + lane; k < w1; k += kWarp) tot += __popc(t.w[k]);
    tot = __reduce_add_sync(0xffffffffu, tot);
    if (lane == 0) wtot[wid] = tot;
    tm.sync();
    int acc = 0;
    for (int j = 0; j < wid; ++j) acc += wtot[j];
    for (int32_t k0 = w0; k0 < w1; k0 += kWarp) {
        const int32_t k = k0 + lane;
        const uint32_t y = k < w1 ? t.w[k] : 0u;
        const int c = __popc(y);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += z;
        }
        if (k < w1) t.w[k] = y | ((uint32_t)(acc + inc - c) << 16);
        acc += __shfl_sync(0xffffffffu, inc, 31);
    }
    tm.sync();
}

// One CTA item (owner b, a chunk of out(b), a slot range of b's row) done by
// a team: the owner's table in `tsm` (a bitmap when the item has a dense-id
// span, else a cuckoo hash table, rebuilt with linear probing when an
// eviction chain runs out), its entries streamed, its counts flushed. A hit
// c adds one to (b, c) in the table, to (a, c) at the streamed slot in global
// memory, and -- summed over the entry -- to (a, b). Ends synchronised, so the
// team may reuse `tsm` and `tv` for its next item.
template <class TEAM>
__device__ __forceinline__ void fwd_item(const TEAM &tm, const FItem &it, int *tsm, TeamVars &tv, int cap_logs,
                                         int load_shift, const int64_t *__restrict__ foff,
                                         const int32_t *__restrict__ fadj, const int32_t *__restrict__ fhid,
                                         const int32_t *__restrict__ e_base, const int32_t *__restrict__ e_len,
                                         const uint32_t *__restrict__ e_fin, int32_t *__restrict__ fcnt) {
    const int32_t b = it.v;
    const int64_t fb = foff[b];
    const int32_t ob = (int32_t)(foff[b + 1] - fb);
    const int32_t tb = it.chunk * kFwdChunk, te = min(tb + kFwdChunk, ob), tlen = te - tb;
    if (tm.tid == 0) {
        tv.next_long = 0;
        tv.next_short = 0;
        tv.failed = 0;
    }
    if (it.hspan > 0) {
        BitTab t;
        t.w = (uint32_t *)tsm;
        t.lo = it.hlo;
        t.span = (uint32_t)it.hspan;
        t.cnt = tsm + (t.span >> 4) + 1;
        bit_build(tm, t, fhid, fb + tb, tlen, tv.wtot);
        ent_stream(it, t, fhid, e_base, e_len, e_fin, fcnt, &tv.next_long, &tv.next_short);
        tm.sync();
        ent_flush(tm, t, fhid, fb + tb, tlen, fcnt);
        tm.sync();
        return;
    }
    FTable t;
    t.logs = min(cap_logs, max(5, fceil_log2(tlen << load_shift)));
    t.keys = tsm;
    t.cnt = tsm + (1 << t.logs);
    for (int k = tm.tid; k < (1 << t.logs); k += tm.size) {
        t.keys[k] = -1;
        t.cnt[k] = 0;
    }
    tm.sync();
    for (int k = tm.tid; k < tlen; k += tm.size)
        if (!ck_insert(t, fadj[fb + tb + k])) tv.failed = 1;
    tm.sync();
    if (tv.failed) {  // an eviction chain ran out: linear probing for this table
        for (int k = tm.tid; k < (1 << t.logs); k += tm.size) t.keys[k] = -1;
        tm.sync();
        for (int k = tm.tid; k < tlen; k += tm.size) lp_insert(t, fadj[fb + tb + k]);
        tm.sync();
        const HashTab<true> h{t};
        ent_stream(it, h, fadj, e_base, e_len, e_fin, fcnt, &tv.next_long, &tv.next_short);
        tm.sync();
        ent_flush(tm, h, fadj, fb + tb, tlen, fcnt);
    } else {
        const HashTab<false> h{t};
        ent_stream(it, h, fadj, e_base, e_len, e_fin, fcnt, &tv.next_long, &tv.next_short);
        tm.sync();
        ent_flush(tm, h, fadj, fb + tb, tlen, fcnt);
    }
    tm.sync();
}

// One CTA per item, streaming its precomputed entries (fwd_item). Dynamic
// shared memory: the table (2^logs keys, then 2^logs counts, logs <=
// cap_logs; or, for a bitmap item, the bitmap words, then one count per
// element), sized for the class's largest table.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_fwd_ent(const FItem *__restrict__ items, const int64_t *__restrict__ foff,
                                                   const int32_t *__restrict__ fadj,
                                                   const int32_t *__restrict__ fhid,
                                                   const int32_t *__restrict__ e_base,
                                                   const int32_t *__restrict__ e_len,
                                                   const uint32_t *__restrict__ e_fin, int32_t *__restrict__ fcnt,
                                                   int cap_logs, int load_shift) {
    extern __shared__ int tsm[];
    __shared__ TeamVars tv;
    const Team<BLOCK, true> tm{(int)threadIdx.x, 0};
    fwd_item(tm, items[blockIdx.x], tsm, tv, cap_logs, load_shift, foff, fadj, fhid, e_base, e_len, e_fin, fcnt);
}

// The whole counting stage as one persistent launch: every CTA takes work
// from one device queue until it is empty. First the CTA items of classes 2
// and 1 (a whole 512-thread CTA per item, heaviest first), then the class-0
// items (each quarter of the CTA, 128 threads under its own named barrier, a
// team per item, in its quarter of the shared memory), then the warp-level
// owners (one warp each, in its team's memory). queue[0..2] are the take
// counters of the three parts, zero at launch; every loop is bounded by the
// count of its part. Dynamic shared memory: max(the largest class-1/2
// table, 4 x team_words) 32-bit words.
constexpr int kQueueBlock = 512;
constexpr int kQueueTeams = 4;
constexpr int32_t kQueueMaxWords = 14336;  // 56 KB: class-2 tables above this get their own launch

__global__ void __launch_bounds__(kQueueBlock, 3) k_fwd_queue(
    const FItem *__restrict__ items2, int64_t n2, const FItem *__restrict__ items1, int64_t n1,
    const FItem *__restrict__ items0, int64_t n0, const int32_t *__restrict__ small, int32_t nsmall,
    unsigned long long *queue, int team_words, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
    const int32_t *__restrict__ deg, const int64_t *__restrict__ foff, const int32_t *__restrict__ fadj,
    const int32_t *__restrict__ fhid, const uint32_t *__restrict__ fin, const int32_t *__restrict__ e_base,
    const int32_t *__restrict__ e_len, const uint32_t *__restrict__ e_fin, int32_t *__restrict__ fcnt,
    int rank_sorted) {
    extern __shared__ int tsm[];
    __shared__ TeamVars tv[kQueueTeams];
    __shared__ int64_t pick[kQueueTeams];
    // classes 2 and 1: the whole CTA per item
    const Team<kQueueBlock, true> all{(int)threadIdx.x, 0};
    for (int64_t guard = 0; guard <= n2 + n1; ++guard) {
        if (threadIdx.x == 0) pick[0] = (int64_t)atomicAdd(queue + 0, 1ull);
        __syncthreads();
        const int64_t i = pick[0];
        __syncthreads();
        if (i >= n2 + n1) break;
        const int cls = i < n2 ? 2 : 1;
        fwd_item(all, i < n2 ? items2[i] : items1[i - n2], tsm, tv[0], fwd_cap_logs(cls), fwd_load_shift(cls), foff,
                 fadj, fhid, e_base, e_len, e_fin, fcnt);
    }
    // class 0: a team of 128 threads per item
    const Team<kQueueBlock / kQueueTeams, false> tm{(int)(threadIdx.x % (kQueueBlock / kQueueTeams)),
                                                   (int)(threadIdx.x / (kQueueBlock / kQueueTeams))};
    int *tsm_t = tsm + (size_t)tm.id * team_words;
    for (int64_t guard = 0; guard <= n0; ++guard) {
        if (tm.tid == 0) pick[tm.id] = (int64_t)atomicAdd(queue + 1, 1ull);
        tm.sync();
        const int64_t i = pick[tm.id];
        tm.sync();
        if (i >= n0) break;
        fwd_item(tm, items0[i], tsm_t, tv[tm.id], fwd_cap_logs(0), fwd_load_shift(0), foff, fadj, fhid, e_base, e_len,
                 e_fin, fcnt);
    }
    // warp-level owners, each warp in its own part of its team's memory
    const int lane = threadIdx.x & 31, wq = (tm.tid >> 5);
    int *wmem = tsm_t + wq * kSmallWarpWords;
    for (int32_t guard = 0; guard <= nsmall; ++guard) {
        int32_t i = 0;
        if (lane == 0) i = (int32_t)atomicAdd(queue + 2, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= nsmall) break;
        fwd_small_owner(small[i], reinterpret_cast<unsigned long long *>(wmem), (uint32_t *)(wmem + 2 * kFwdSmallTable),
                        wmem + 2 * kFwdSmallTable + 64, off, adj, deg, foff, fadj, fin, fcnt, rank_sorted);
    }
}

// per forward edge: closed count and either the count cache (count and
// closed-degree product) or the eps-test (a flag per oriented edge and the
// endpoints' eps-degrees)
template <bool WRITE_SIM, bool WRITE_CN>
__global__ void k_fwd_finish(int64_t m, const int32_t *__restrict__ fcnt, const int32_t *__restrict__ fsrc,
                             const int32_t *__restrict__ fadj, const int32_t *__restrict__ deg, QParams qp,
                             uint8_t *__restrict__ simo, int32_t *__restrict__ nsim, int32_t *__restrict__ cn,
                             uint64_t *__restrict__ dd) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = fcnt[i] + 2;
        const int32_t u = fsrc[i], v = fadj[i];
        if (WRITE_CN) {
            cn[i] = c;
            dd[i] = ((uint64_t)deg[u] + 1) * ((uint64_t)deg[v] + 1);
        }
        if (WRITE_SIM) {
            uint64_t pp, qq;
            qp.eps(u, pp, qq);
            const bool s = dev::eps_similar((uint64_t)c, (uint64_t)deg[u] + 1, (uint64_t)deg[v] + 1, pp, qq);
            simo[i] = s ? 1 : 0;
            if (s) {
                atomicAdd(nsim + u, 1);
                atomicAdd(nsim + v, 1);
            }
        }
    }
}

// ------------------------------------------------------------ load time
// Rank order inside every out-list: key (deg, id), carried with the slot id.
constexpr int kSortMax = 4096;  // longest out-list sorted by rank (longer: all lists stay in id order)

// warp per vertex with out-degree <= 32: bitonic sort in registers
__global__ void k_fwd_sort_warp(const int64_t *__restrict__ foff, int32_t n, const int32_t *__restrict__ deg,
                                int32_t *__restrict__ fadj, uint32_t *__restrict__ oe) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & 31;
    if (a >= n) return;
    const int64_t b = foff[a];
    const int32_t len = (int32_t)(foff[a + 1] - b);
    if (len < 2 || len > kWarp) return;
    unsigned long long key = ~0ull;
    uint32_t pay = 0;
    if (lane < len) {
        key = rank_key(deg, fadj[b + lane]);
        pay = oe[b + lane];
    }
    for (int k = 2; k <= kWarp; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, j);
            const uint32_t op = __shfl_xor_sync(0xffffffffu, pay, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            const bool take = lower == up ? ok < key : ok > key;
            if (take) { key = ok; pay = op; }
        }
    if (lane < len) {
        fadj[b + lane] = (int32_t)(uint32_t)key;
        oe[b + lane] = pay;
    }
}

// CTA per vertex with an out-list of up to CAP (> 32) ids: bitonic sort in
// shared memory. Three sizes (CAP 256, 1024, kSortMax on 128, 256 and 1024
// threads), so short lists do not hold a 1024-thread CTA at its barriers.
template <int BLOCK, int CAP>
__global__ void __launch_bounds__(BLOCK) k_fwd_sort_cta(const int32_t *__restrict__ verts,
                                                        const int64_t *__restrict__ foff,
                                                        const int32_t *__restrict__ deg, int32_t *__restrict__ fadj,
                                                        uint32_t *__restrict__ oe) {
    __shared__ unsigned long long key[CAP];
    __shared__ uint32_t pay[CAP];
    const int32_t a = verts[blockIdx.x];
    const int64_t b = foff[a];
    const int32_t len = (int32_t)(foff[a + 1] - b);
    int size = 64;
    while (size < len) size <<= 1;
    for (int i = threadIdx.x; i < size; i += BLOCK) {
        key[i] = i < len ? rank_key(deg, fadj[b + i]) : ~0ull;
        pay[i] = i < len ? oe[b + i] : 0u;
    }
    __syncthreads();
    for (int k = 2; k <= size; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < size; i += BLOCK) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    if ((key[i] > key[p]) == up) {
                        const unsigned long long tk = key[i];
                        key[i] = key[p];
                        key[p] = tk;
                        const uint32_t tp = pay[i];
                        pay[i] = pay[p];
                        pay[p] = tp;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += BLOCK) {
        fadj[b + i] = (int32_t)(uint32_t)key[i];
        oe[b + i] = pay[i];
    }
}

__global__ void k_fwd_fin(const uint32_t *__restrict__ oe, int64_t m, const uint32_t *__restrict__ rev,
                          uint32_t *__restrict__ fin) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        fin[rev[oe[i]]] = (uint32_t)i;
}

// vertices whose out-list needs the CTA sort; flags a list too long to sort
// out-lists above a warp, by sort size: up to 256 (v256), 1024 (v1024) and
// kSortMax (vmax); counts[3] = lists above kSortMax
__global__ void k_fwd_sort_pick(const int64_t *__restrict__ foff, int32_t n, int32_t *__restrict__ v256,
                                int32_t *__restrict__ v1024, int32_t *__restrict__ vmax, unsigned long long *counts) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int64_t len = foff[a + 1] - foff[a];
    if (len > kSortMax) atomicAdd(counts + 3, 1ull);
    else if (len > 1024) vmax[atomicAdd(counts + 2, 1ull)] = (int32_t)a;
    else if (len > 256) v1024[atomicAdd(counts + 1, 1ull)] = (int32_t)a;
    else if (len > kWarp) v256[atomicAdd(counts + 0, 1ull)] = (int32_t)a;
}

__global__ void k_fwd_adj(const uint32_t *__restrict__ oe, int64_t m, const int32_t *__restrict__ adj,
                          const uint32_t *__restrict__ rev, int32_t *__restrict__ fadj, uint32_t *__restrict__ fin) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = oe[i];
        fadj[i] = adj[e];
        fin[rev[e]] = (uint32_t)i;
    }
}

// lower endpoint of every oriented edge, in fadj order (once the lists are final)
__global__ void k_fwd_src(const uint32_t *__restrict__ oe, int64_t m, const int32_t *__restrict__ src,
                          int32_t *__restrict__ fsrc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        fsrc[i] = src[oe[i]];
}

// Dense ids of the bitmap tables: vertices ordered by degree level
// (floor(log2 deg)), highest level first, then by id (isolated vertices get
// none). A stable partition by level over tiles of kHidTile ids: per-tile
// level counts, one exclusive scan over them laid out level-major (highest
// level first), then each vertex's place among its tile's vertices of the
// same level.
constexpr int kHidTile = 256;

__device__ __forceinline__ int deg_level(int32_t d) { return 31 - __clz(d); }  // d >= 1

__global__ void __launch_bounds__(kHidTile) k_hid_count(const int32_t *__restrict__ deg, int32_t n, int64_t ntiles,
                                                         int32_t *__restrict__ tcnt) {
    __shared__ int32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kHidTile + threadIdx.x;
    const int32_t d = v < n ? deg[v] : 0;
    if (d > 0) atomicAdd(&h[deg_level(d)], 1);
    __syncthreads();
    if (threadIdx.x < 32) tcnt[(int64_t)(31 - threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kHidTile) k_hid_assign(const int32_t *__restrict__ deg, int32_t n, int64_t ntiles,
                                                          const int64_t *__restrict__ toff,
                                                          int32_t *__restrict__ vhid) {
    __shared__ int32_t wc[kHidTile / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kHidTile; k += kHidTile) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kHidTile + threadIdx.x;
    const int32_t d = v < n ? deg[v] : 0;
    const int L = d > 0 ? deg_level(d) : 32;  // 32: no dense id
    const unsigned same = __match_any_sync(0xffffffffu, L);
    const int below = __popc(same & ((1u << lane) - 1u));
    if (L < 32 && below == 0) wc[wid][L] = __popc(same);
    __syncthreads();
    if (v >= n) return;
    if (L == 32) {
        vhid[v] = -1;
        return;
    }
    int32_t before = 0;
    for (int j = 0; j < wid; ++j) before += wc[j][L];
    vhid[v] = (int32_t)(toff[(int64_t)(31 - L) * ntiles + blockIdx.x] + before + below);
}

__global__ void k_fwd_hid(const int32_t *__restrict__ fadj, int64_t m, const int32_t *__restrict__ vhid,
                          int32_t *__restrict__ fhid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        fhid[i] = vhid[fadj[i]];
}



// warp per vertex: work as a middle vertex and the number of items
__global__ void __launch_bounds__(256) k_fwd_sched_count(const int64_t *__restrict__ off,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ deg,
                                                         const int64_t *__restrict__ foff, int32_t n,
                                                         int32_t *__restrict__ nranges,
                                                         unsigned long long *counts, int64_t small_work,
                                                         int64_t item_work) {
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
    if (ob <= kFwdSmallOut && (int64_t)w <= small_work) {
        nranges[b] = -1;  // warp owner
        atomicAdd(counts + 0, 1ull);
        return;
    }
    const int64_t nchunks = (ob + kFwdChunk - 1) / kFwdChunk;
    int64_t nr = (int64_t)((w + item_work - 1) / item_work);
    nr = max((int64_t)1, min(nr, (int64_t)(db + 255) / 256));
    nranges[b] = (int32_t)nr;
    atomicAdd(counts + 1 + fwd_class(ob), (unsigned long long)(nchunks * nr));
}

__global__ void k_fwd_sched_write(const int32_t *__restrict__ deg, const int64_t *__restrict__ foff, int32_t n,
                                  const int32_t *__restrict__ nranges, unsigned long long *cursor,
                                  int32_t *__restrict__ small, FItem *__restrict__ i0, FItem *__restrict__ i1,
                                  FItem *__restrict__ i2) {
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
    const int cls = fwd_class(ob);
    FItem *dst = cls == 0 ? i0 : (cls == 1 ? i1 : i2);
    unsigned long long p = atomicAdd(cursor + 1 + cls, (unsigned long long)(nchunks * nr));
    for (int32_t c = 0; c < nchunks; ++c)
        for (int32_t r = 0; r < nr; ++r) dst[p++] = FItem{(int32_t)b, c, r * len, min(db, (r + 1) * len), 0, 0, 0, 0, 0};
}

}  // namespace

// Items in descending order of their owner's degree (a counting sort over
// degrees, capped at kDegBuckets - 1): owners of similar rank run at the same
// time, and the tails of the out-lists they stream stay in L2.
constexpr int kDegBuckets = 1 << 16;

__global__ void k_item_deg_hist(const FItem *__restrict__ items, int64_t ni, const int32_t *__restrict__ deg,
                                int32_t *__restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ni) return;
    const int32_t d = min(deg[items[i].v], kDegBuckets - 1);
    atomicAdd(hist + (kDegBuckets - 1 - d), 1);
}

__global__ void k_item_scatter(const FItem *__restrict__ items, int64_t ni, const int32_t *__restrict__ deg,
                               const int64_t *__restrict__ boff, int32_t *__restrict__ cur, FItem *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ni) return;
    const FItem it = items[i];
    const int k = kDegBuckets - 1 - min(deg[it.v], kDegBuckets - 1);
    out[boff[k] + atomicAdd(cur + k, 1)] = it;
}

static scan_status fwd_order_items(Graph *g) {
    Ctx *c = g->ctx;
    const int64_t nmax = std::max(g->fwd_items_n[0], std::max(g->fwd_items_n[1], g->fwd_items_n[2]));
    if (nmax == 0) return SCAN_OK;
    DevBuf hist, boff, tmp;
    auto done = [&](scan_status s) {
        dev_free(c, hist);
        dev_free(c, boff);
        dev_free(c, tmp);
        return s;
    };
    if (dev_alloc(c, hist, 4 * (size_t)kDegBuckets) != SCAN_OK ||
        dev_alloc(c, boff, 8 * ((size_t)kDegBuckets + 1)) != SCAN_OK ||
        dev_alloc(c, tmp, sizeof(FItem) * (size_t)nmax) != SCAN_OK) {
        set_error("");
        return done(SCAN_OK);  // no room: items stay in schedule order
    }
    auto *deg = (const int32_t *)g->deg.ptr;
    for (int cls = 0; cls < 3; ++cls) {
        const int64_t ni = g->fwd_items_n[cls];
        if (ni < 2) continue;
        auto *items = (FItem *)g->fwd_items[cls].ptr;
        SCAN_CUDA(cudaMemsetAsync(hist.ptr, 0, hist.bytes, c->stream));
        k_item_deg_hist<<<grid_for(ni, 256), 256, 0, c->stream>>>(items, ni, deg, (int32_t *)hist.ptr);
        scan_status s = launch_exclusive_scan_i32_to_i64(c, (const int32_t *)hist.ptr, (int64_t *)boff.ptr,
                                                         kDegBuckets, g->scan_tmp);
        if (s != SCAN_OK) return done(s);
        SCAN_CUDA(cudaMemsetAsync(hist.ptr, 0, hist.bytes, c->stream));
        k_item_scatter<<<grid_for(ni, 256), 256, 0, c->stream>>>(items, ni, deg, (const int64_t *)boff.ptr,
                                                                 (int32_t *)hist.ptr, (FItem *)tmp.ptr);
        SCAN_CUDA(cudaMemcpyAsync(items, tmp.ptr, sizeof(FItem) * (size_t)ni, cudaMemcpyDeviceToDevice, c->stream));
        c->launches += 2;
    }
    SCAN_CUDA(cudaGetLastError());
    return done(SCAN_OK);
}

// Entry lists of every CTA item (12 bytes per entry, at most one entry per
// oriented edge and chunk). Without room for them under the budget the
// counting kernel derives the entries itself, round by round.
static scan_status fwd_build_entries(Graph *g) {
    Ctx *c = g->ctx;
    g->fwd_entries = false;
    const int64_t nmax = std::max(g->fwd_items_n[0], std::max(g->fwd_items_n[1], g->fwd_items_n[2]));
    if (nmax == 0) return SCAN_OK;
    const int rs = g->fwd_rank_sorted ? 1 : 0;
    auto *off = (const int64_t *)g->off.ptr;
    auto *adj = (const int32_t *)g->adj.ptr;
    auto *deg = (const int32_t *)g->deg.ptr;
    auto *foff = (const int64_t *)g->foff.ptr;
    auto *fadj = (const int32_t *)g->fadj.ptr;
    auto *fin = (const uint32_t *)g->fin.ptr;
    DevBuf nent, eoff[3];
    int64_t total[3] = {0, 0, 0};
    auto cleanup = [&]() {
        dev_free(c, nent);
        for (auto &b : eoff) dev_free(c, b);
    };
    SCAN_TRY(dev_alloc(c, nent, 4 * (size_t)std::max<int64_t>(nmax, 3)));
    for (int cls = 0; cls < 3; ++cls) {
        const int64_t ni = g->fwd_items_n[cls];
        if (ni == 0) continue;
        scan_status s = dev_alloc(c, eoff[cls], 8 * ((size_t)ni + 1));
        if (s != SCAN_OK) {
            cleanup();
            return SCAN_OK;  // no room: per-round entries
        }
        k_fwd_ent_count<<<(unsigned)ni, 256, 0, c->stream>>>((const FItem *)g->fwd_items[cls].ptr, ni, off, adj, deg,
                                                            foff, fadj, fin, rs, (int32_t *)nent.ptr);
        c->launches++;
        s = launch_exclusive_scan_i32_to_i64(c, (const int32_t *)nent.ptr, (int64_t *)eoff[cls].ptr, ni, g->scan_tmp);
        if (s != SCAN_OK) {
            cleanup();
            return s;
        }
        cudaError_t e = cudaMemcpyAsync(&total[cls], (int64_t *)eoff[cls].ptr + ni, 8, cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "forward entry counts");
        }
    }
    const size_t E = (size_t)std::max<int64_t>(total[0] + total[1] + total[2], 1);
    if (dev_alloc(c, g->fwd_ebase, 4 * E) != SCAN_OK || dev_alloc(c, g->fwd_elen, 4 * E) != SCAN_OK ||
        dev_alloc(c, g->fwd_efin, 4 * E) != SCAN_OK) {
        dev_free(c, g->fwd_ebase);
        dev_free(c, g->fwd_elen);
        dev_free(c, g->fwd_efin);
        cleanup();
        set_error("");
        return SCAN_OK;  // no room: per-round entries
    }
    // the largest table of each class, so each launch takes only the shared
    // memory it needs (the rest stays L1 cache for the streamed lists)
    int32_t *need = (int32_t *)nent.ptr;  // the entry counts are no longer needed
    SCAN_CUDA(cudaMemsetAsync(need, 0, 3 * sizeof(int32_t), c->stream));
    for (int cls = 0; cls < 3; ++cls) {
        const int64_t ni = g->fwd_items_n[cls];
        const int64_t first = cls == 0 ? 0 : (cls == 1 ? total[0] : total[0] + total[1]);
        if (ni == 0) continue;
        k_fwd_ent_write<<<(unsigned)ni, 256, 0, c->stream>>>(
            (FItem *)g->fwd_items[cls].ptr, ni, (const int64_t *)eoff[cls].ptr, first, off, adj,
            deg, foff, fadj, fin, rs, (int32_t *)g->fwd_ebase.ptr, (int32_t *)g->fwd_elen.ptr,
            (uint32_t *)g->fwd_efin.ptr, (const int32_t *)g->fhid.ptr, 2 << fwd_cap_logs(cls), fwd_cap_logs(cls),
            fwd_load_shift(cls), need + cls);
        c->launches++;
    }
    int32_t hneed[3] = {0, 0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hneed, need, sizeof(hneed), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    for (int cls = 0; cls < 3; ++cls) g->fwd_smem_words[cls] = hneed[cls];
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "forward entries");
    g->fwd_entries = true;
    return SCAN_OK;
}

// Dense ids of the out-list elements (Graph::fhid) for the bitmap tables.
// Without room for them under the budget every owner keeps a hash table.
static scan_status fwd_build_hid(Graph *g) {
    Ctx *c = g->ctx;
    const int32_t n = g->n;
    const int64_t m = g->m;
    if (dev_alloc(c, g->fhid, 4 * (size_t)m) != SCAN_OK) {
        set_error("");
        return SCAN_OK;
    }
    const int64_t ntiles = ((int64_t)n + kHidTile - 1) / kHidTile;
    DevBuf tcnt, toff;
    if (dev_alloc(c, tcnt, 4 * (size_t)(32 * ntiles)) != SCAN_OK ||
        dev_alloc(c, toff, 8 * (size_t)(32 * ntiles + 1)) != SCAN_OK) {
        dev_free(c, tcnt);
        dev_free(c, toff);
        dev_free(c, g->fhid);
        set_error("");
        return SCAN_OK;
    }
    auto *deg = (const int32_t *)g->deg.ptr;
    int32_t *vhid = (int32_t *)g->parent.ptr;  // scratch int32[n+1] (free until the query's later stages)
    k_hid_count<<<(unsigned)ntiles, kHidTile, 0, c->stream>>>(deg, n, ntiles, (int32_t *)tcnt.ptr);
    c->launches++;
    scan_status s = launch_exclusive_scan_i32_to_i64(c, (const int32_t *)tcnt.ptr, (int64_t *)toff.ptr, 32 * ntiles,
                                                     g->scan_tmp);
    if (s == SCAN_OK) {
        k_hid_assign<<<(unsigned)ntiles, kHidTile, 0, c->stream>>>(deg, n, ntiles, (const int64_t *)toff.ptr, vhid);
        k_fwd_hid<<<grid_for(m, 256, c->num_sms * 32), 256, 0, c->stream>>>((const int32_t *)g->fadj.ptr, m, vhid,
                                                                             (int32_t *)g->fhid.ptr);
        c->launches += 2;
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "dense ids");
    }
    dev_free(c, tcnt);
    dev_free(c, toff);
    if (s != SCAN_OK) dev_free(c, g->fhid);
    return s;
}

scan_status fwd_prepare(Graph *g) {
    Ctx *c = g->ctx;
    const int32_t n = g->n;
    const int64_t m = g->m;
    if (g->fwd_ready) return SCAN_OK;
    if (n == 0 || m == 0) {
        g->fwd_ready = true;
        return SCAN_OK;
    }
    DevBuf cnts;
    SCAN_TRY(dev_alloc(c, cnts, 4 * sizeof(unsigned long long)));
    auto *counts = (unsigned long long *)cnts.ptr;
    if (!g->fadj.ptr) {
        scan_status s = dev_alloc(c, g->fadj, 4 * (size_t)m);
        if (s == SCAN_OK) s = dev_alloc(c, g->fin, 4 * (size_t)g->nnz);
        if (s == SCAN_OK) s = dev_alloc(c, g->fcnt, 4 * (size_t)m);
        if (s == SCAN_OK) s = dev_alloc(c, g->fsrc, 4 * (size_t)m);
        if (s != SCAN_OK) {
            dev_free(c, g->fadj);
            dev_free(c, g->fin);
            dev_free(c, g->fcnt);
            dev_free(c, g->fsrc);
            dev_free(c, cnts);
            return s;
        }
        // foff (built at load) already holds the out-degree offsets
        k_fwd_adj<<<grid_for(m, 256, c->num_sms * 32), 256, 0, c->stream>>>(
            (const uint32_t *)g->oe.ptr, m, (const int32_t *)g->adj.ptr, (const uint32_t *)g->rev.ptr,
            (int32_t *)g->fadj.ptr, (uint32_t *)g->fin.ptr);
        c->launches++;
        // order every out-list by rank, carrying the slot ids, then re-index fin
        SCAN_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), c->stream));
        // scratch int32[n+1] lists (free until the query's later stages)
        int32_t *v256 = (int32_t *)g->cnt.ptr, *v1024 = (int32_t *)g->ucnt.ptr, *vmax = (int32_t *)g->parent.ptr;
        k_fwd_sort_pick<<<grid_for(n, 256), 256, 0, c->stream>>>((const int64_t *)g->foff.ptr, n, v256, v1024, vmax,
                                                                 counts);
        unsigned long long h4[4];
        SCAN_CUDA(cudaMemcpyAsync(h4, counts, sizeof(h4), cudaMemcpyDeviceToHost, c->stream));
        SCAN_CUDA(cudaStreamSynchronize(c->stream));
        c->launches++;
        g->fwd_rank_sorted = h4[3] == 0;
        if (g->fwd_rank_sorted) {
            auto *foff = (const int64_t *)g->foff.ptr;
            auto *deg = (const int32_t *)g->deg.ptr;
            auto *fadj = (int32_t *)g->fadj.ptr;
            auto *oe = (uint32_t *)g->oe.ptr;
            k_fwd_sort_warp<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(foff, n, deg, fadj, oe);
            c->launches++;
            if (h4[0] > 0) {
                k_fwd_sort_cta<128, 256><<<(unsigned)h4[0], 128, 0, c->stream>>>(v256, foff, deg, fadj, oe);
                c->launches++;
            }
            if (h4[1] > 0) {
                k_fwd_sort_cta<256, 1024><<<(unsigned)h4[1], 256, 0, c->stream>>>(v1024, foff, deg, fadj, oe);
                c->launches++;
            }
            if (h4[2] > 0) {
                k_fwd_sort_cta<1024, kSortMax><<<(unsigned)h4[2], 1024, 0, c->stream>>>(vmax, foff, deg, fadj, oe);
                c->launches++;
            }
            k_fwd_fin<<<grid_for(m, 256, c->num_sms * 32), 256, 0, c->stream>>>(
                (const uint32_t *)g->oe.ptr, m, (const uint32_t *)g->rev.ptr, (uint32_t *)g->fin.ptr);
            c->launches++;
        }
        k_fwd_src<<<grid_for(m, 256, c->num_sms * 32), 256, 0, c->stream>>>(
            (const uint32_t *)g->oe.ptr, m, (const int32_t *)g->src.ptr, (int32_t *)g->fsrc.ptr);
        c->launches++;
        const scan_status hs = fwd_build_hid(g);
        if (hs != SCAN_OK) {
            dev_free(c, cnts);
            return hs;
        }
    }
    // schedule (rebuilt alone when the autotuner changes its parameters)
    SCAN_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), c->stream));
    int32_t *nranges = (int32_t *)g->ucnt.ptr;  // scratch int32[n+1]
    k_fwd_sched_count<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(
        (const int64_t *)g->off.ptr, (const int32_t *)g->adj.ptr, (const int32_t *)g->deg.ptr,
        (const int64_t *)g->foff.ptr, n, nranges, counts, g->fwd_small_work, g->fwd_item_work);
    c->launches++;
    unsigned long long h[4];
    SCAN_CUDA(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    SCAN_CUDA(cudaStreamSynchronize(c->stream));
    g->fwd_small = (int32_t)h[0];
    for (int cls = 0; cls < 3; ++cls) g->fwd_items_n[cls] = (int64_t)h[1 + cls];
    scan_status s = dev_alloc(c, g->fwd_owners, 4 * (size_t)(h[0] + 1));
    for (int cls = 0; cls < 3 && s == SCAN_OK; ++cls)
        s = dev_alloc(c, g->fwd_items[cls], sizeof(FItem) * (size_t)(h[1 + cls] + 1));
    if (s != SCAN_OK) {
        dev_free(c, cnts);
        return s;
    }
    SCAN_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), c->stream));
    k_fwd_sched_write<<<grid_for(n, 256), 256, 0, c->stream>>>(
        (const int32_t *)g->deg.ptr, (const int64_t *)g->foff.ptr, n, nranges, counts,
        (int32_t *)g->fwd_owners.ptr, (FItem *)g->fwd_items[0].ptr, (FItem *)g->fwd_items[1].ptr,
        (FItem *)g->fwd_items[2].ptr);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, cnts);
    if (e != cudaSuccess) return cuda_fail(e, "forward schedule");
    SCAN_TRY(fwd_order_items(g));
    g->fwd_ready = true;
    return SCAN_OK;
}

void fwd_release(Graph *g) {
    if (g->fwd_side) cudaStreamDestroy(g->fwd_side);
    if (g->fwd_fork) cudaEventDestroy(g->fwd_fork);
    if (g->fwd_join) cudaEventDestroy(g->fwd_join);
    g->fwd_side = nullptr;
    g->fwd_fork = nullptr;
    g->fwd_join = nullptr;
}

// The side stream of the per-class launches, when the query's stream has the
// default priority (a prioritised stream, as the server's, keeps every launch
// on itself). Null: no fork.
static cudaStream_t fwd_side_stream(Graph *g, cudaStream_t st) {
    int prio = 0;
    if (cudaStreamGetPriority(st, &prio) != cudaSuccess || prio != 0) {
        cudaGetLastError();
        return nullptr;
    }
    if (!g->fwd_side) {
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (s) cudaStreamDestroy(s);
            if (a) cudaEventDestroy(a);
            return nullptr;
        }
        g->fwd_side = s;
        g->fwd_fork = a;
        g->fwd_join = b;
    }
    return g->fwd_side;
}

scan_status launch_fwd_counts(Graph *g, bool write_sim, bool write_cn, const QParams &qp, int32_t *cn,
                              uint64_t *dd) {
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
    auto *fhid = (const int32_t *)g->fhid.ptr;
    // entry lists: built on the first count of the default family (not for
    // the lean one, and not again after they did not fit the budget)
    const bool lean = g->strategy == SCAN_STRATEGY_FORWARD_LEAN;
    if (!lean && !g->fwd_entries && !g->fwd_entries_tried) {
        g->fwd_entries_tried = true;
        SCAN_TRY(fwd_build_entries(g));
    }
    const bool use_entries = !lean && g->fwd_entries;
    SCAN_CUDA(cudaMemsetAsync(fcnt, 0, 4 * (size_t)g->m, st));
    const int rs = g->fwd_rank_sorted ? 1 : 0;
    bool small_done = false;
    if (use_entries && g->fwd_queue) {
        // one persistent launch over the work queue (class-2 items whose
        // tables do not fit its CTAs run first in their own launch)
        const int64_t n2 = g->fwd_items_n[2], n1 = g->fwd_items_n[1], n0 = g->fwd_items_n[0];
        auto *eb = (const int32_t *)g->fwd_ebase.ptr;
        auto *el = (const int32_t *)g->fwd_elen.ptr;
        auto *ef = (const uint32_t *)g->fwd_efin.ptr;
        const int32_t team_words = std::max(n0 ? g->fwd_smem_words[0] : 0, (kQueueBlock / kQueueTeams / 32) * kSmallWarpWords);
        const bool sep2 = n2 > 0 && g->fwd_smem_words[2] > kQueueMaxWords;
        int32_t words = kQueueTeams * team_words;
        if (n1) words = std::max(words, g->fwd_smem_words[1]);
        if (n2 && !sep2) words = std::max(words, g->fwd_smem_words[2]);
        if (sep2) {
            const size_t smem = 4 * (size_t)g->fwd_smem_words[2];
            SCAN_CUDA(cudaFuncSetAttribute(k_fwd_ent<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_fwd_ent<512><<<(unsigned)n2, 512, smem, st>>>((const FItem *)g->fwd_items[2].ptr, foff, fadj, fhid, eb, el,
                                                            ef, fcnt, fwd_cap_logs(2), fwd_load_shift(2));
            c->launches++;
        }
        if (!g->fwd_qctr.ptr) SCAN_TRY(dev_alloc(c, g->fwd_qctr, 4 * sizeof(unsigned long long)));
        SCAN_CUDA(cudaMemsetAsync(g->fwd_qctr.ptr, 0, 4 * sizeof(unsigned long long), st));
        const size_t smem = 4 * (size_t)words;
        SCAN_CUDA(cudaFuncSetAttribute(k_fwd_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SCAN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_queue, kQueueBlock, smem));
        const int64_t work = (sep2 ? 0 : n2) + n1 + (n0 + kQueueTeams - 1) / kQueueTeams +
                             (g->fwd_small + kQueueBlock / 32 - 1) / (kQueueBlock / 32);
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * c->num_sms, work));
        k_fwd_queue<<<grid, kQueueBlock, smem, st>>>(
            (const FItem *)g->fwd_items[2].ptr, sep2 ? 0 : n2, (const FItem *)g->fwd_items[1].ptr, n1,
            (const FItem *)g->fwd_items[0].ptr, n0, (const int32_t *)g->fwd_owners.ptr, g->fwd_small,
            (unsigned long long *)g->fwd_qctr.ptr, team_words, off, adj, deg, foff, fadj, fhid, fin, eb, el, ef, fcnt,
            rs);
        c->launches++;
        small_done = true;
    } else if (use_entries) {
        // Class 2 (a few large owners: at scale 22, six CTAs for 0.2 ms) and
        // then the warp owners run on the side stream while classes 1 and 0
        // run on the query's: the class-2 CTAs would otherwise hold a handful
        // of SMs while the rest idle. The counts are atomic, so the launches
        // may overlap; the finish waits for both streams.
        cudaStream_t side = fwd_side_stream(g, st);
        if (side) {
            SCAN_CUDA(cudaEventRecord(g->fwd_fork, st));
            SCAN_CUDA(cudaStreamWaitEvent(side, g->fwd_fork, 0));
        }
        for (int cls = 2; cls >= 0; --cls) {
            const int64_t ni = g->fwd_items_n[cls];
            if (ni == 0) continue;
            const cudaStream_t cs = (side && cls == 2) ? side : st;
            // Hash tables take 8 bytes per slot (key + count). Class 0: four
            // slots per key, 8 KB, 128-thread CTAs (sixteen per SM: these owners
            // hold little work, and small CTAs wait less at their barriers).
            // Class 1: eight slots per key up to 512 keys, four above, 32 KB;
            // its items mostly take bitmaps of a few KB, on 256-thread CTAs
            // (eight per SM: 1.3 % faster than four 512-thread ones). Class 2:
            // four per key, 128 KB, 512-thread CTAs. The launch takes only the
            // shared memory of the class's largest table.
            const int cap_logs = fwd_cap_logs(cls), load_shift = fwd_load_shift(cls);
            const size_t full = (size_t)(2 * sizeof(int)) << cap_logs;
            const size_t smem = g->fwd_smem_words[cls] > 0 ? std::min(full, 4 * (size_t)g->fwd_smem_words[cls]) : full;
            auto *items = (const FItem *)g->fwd_items[cls].ptr;
            auto *eb = (const int32_t *)g->fwd_ebase.ptr;
            auto *el = (const int32_t *)g->fwd_elen.ptr;
            auto *ef = (const uint32_t *)g->fwd_efin.ptr;
            if (cls == 0) {
                SCAN_CUDA(cudaFuncSetAttribute(k_fwd_ent<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_fwd_ent<128><<<(unsigned)ni, 128, smem, cs>>>(items, foff, fadj, fhid, eb, el, ef, fcnt,
                                                                cap_logs, load_shift);
            } else if (cls == 1) {
                SCAN_CUDA(cudaFuncSetAttribute(k_fwd_ent<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_fwd_ent<256><<<(unsigned)ni, 256, smem, cs>>>(items, foff, fadj, fhid, eb, el, ef, fcnt,
                                                                cap_logs, load_shift);
            } else {
                SCAN_CUDA(cudaFuncSetAttribute(k_fwd_ent<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_fwd_ent<512><<<(unsigned)ni, 512, smem, cs>>>(items, foff, fadj, fhid, eb, el, ef, fcnt,
                                                                cap_logs, load_shift);
            }
            c->launches++;
        }
        if (side) {
            if (g->fwd_small > 0) {
                k_fwd_small<<<grid_for((int64_t)g->fwd_small * kWarp, 256, c->num_sms * 16), 256, 0, side>>>(
                    (const int32_t *)g->fwd_owners.ptr, g->fwd_small, off, adj, deg, foff, fadj, fin, fcnt, rs);
                c->launches++;
            }
            small_done = true;
            SCAN_CUDA(cudaEventRecord(g->fwd_join, side));
            SCAN_CUDA(cudaStreamWaitEvent(st, g->fwd_join, 0));
        }
    }
    auto kern = k_fwd_cta<512>;
    for (int cls = 2; cls >= 0 && !use_entries; --cls) {
        if (g->fwd_items_n[cls] == 0) continue;
        // classes 0 and 1 (out-degree <= 1024): 4 buckets per key, up to 4096
        // (64 KB); class 2 (chunks of up to 4096 keys): 2 buckets per key, up
        // to 8192 (128 KB); the kernel's table is 2^cap_lognb int4 buckets
        const int cap_lognb = cls == 2 ? 13 : 12, load_shift = cls == 2 ? 1 : 2;
        const size_t smem = sizeof(int4) << cap_lognb;
        SCAN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)g->fwd_items_n[cls], 512, smem, st>>>((const FItem *)g->fwd_items[cls].ptr, off, adj, deg,
                                                             foff, fadj, fin, fcnt, cap_lognb, load_shift, rs);
        c->launches++;
    }
    if (g->fwd_small > 0 && !small_done) {
        k_fwd_small<<<grid_for((int64_t)g->fwd_small * kWarp, 256, c->num_sms * 16), 256, 0, st>>>(
            (const int32_t *)g->fwd_owners.ptr, g->fwd_small, off, adj, deg, foff, fadj, fin, fcnt, rs);
        c->launches++;
    }
    const unsigned gf = grid_for(g->m, 256, c->num_sms * 32);
    auto *fsrc = (const int32_t *)g->fsrc.ptr;
    auto *simo = (uint8_t *)g->simo.ptr;
    auto *nsim = (int32_t *)g->nsim.ptr;
    if (write_sim && write_cn)
        k_fwd_finish<true, true><<<gf, 256, 0, st>>>(g->m, fcnt, fsrc, fadj, deg, qp, simo, nsim, cn, dd);
    else if (write_cn)
        k_fwd_finish<false, true><<<gf, 256, 0, st>>>(g->m, fcnt, fsrc, fadj, deg, qp, simo, nsim, cn, dd);
    else
        k_fwd_finish<true, false><<<gf, 256, 0, st>>>(g->m, fcnt, fsrc, fadj, deg, qp, simo, nsim, cn, dd);
    c->launches++;
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

}  // namespace scan

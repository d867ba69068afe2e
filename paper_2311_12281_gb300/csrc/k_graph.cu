// k_graph.cu -- load-time preparation of a resident graph.
//
// Validates the CSR contract (offsets monotone, rows strictly ascending, ids
// in range, no self-loops, symmetric), then derives deg, src (row of each
// slot), rev (slot of the reverse direction; the Eid role of the paper's
// CSR-enhanced layout, Section 4.1) and oe, the degree-oriented edge list:
// every undirected edge once, as the slot in the row of its lower (deg, id)
// endpoint (Section 4.1's degree-oriented edge array).
#include <limits>

#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr unsigned long long kNoBad = std::numeric_limits<unsigned long long>::max();

__global__ void k_check_offsets(const int64_t *__restrict__ off, int32_t n, int64_t nnz,
                                unsigned long long *bad) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    int64_t o = off[u];
    bool ok = (u == 0) ? (o == 0) : (o >= off[u - 1]);
    if (u == n) ok = ok && (o == nnz);
    if (!ok) atomicMin(bad, (unsigned long long)u | (1ull << 62));  // tag: an offsets index
}

// warp per vertex: deg and the row id of every slot
__global__ void k_deg_src(const int64_t *__restrict__ off, int32_t n, int32_t *__restrict__ deg,
                          int32_t *__restrict__ src) {
    int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & 31;
    if (u >= n) return;
    int64_t b = off[u], e = off[u + 1];
    if (lane == 0) deg[u] = (int32_t)(e - b);
    for (int64_t s = b + lane; s < e; s += kWarp) src[s] = (int32_t)u;
}

// Slot checks, and for each slot (u, v) with u < v the position of u in row
// v by binary search: the reverse slot of both. Each such slot finds a
// distinct partner with a smaller id, so once every one has found it and the
// two kinds are equally many (counted in `up`), every slot is matched.
__global__ void k_check_rev(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            const int32_t *__restrict__ src, int32_t n, int64_t nnz, uint32_t *__restrict__ rev,
                            unsigned long long *bad, unsigned long long *up) {
    __shared__ unsigned int block_up;
    if (threadIdx.x == 0) block_up = 0;
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nnz) {
        const int32_t u = src[s], v = adj[s];
        bool ok = v >= 0 && v < n && v != u;
        if (ok && s > off[u]) ok = adj[s - 1] < v;
        if (ok && v > u) {
            atomicAdd(&block_up, 1u);
            int64_t lo = off[v], hi = off[v + 1];
            int64_t found = -1;
            for (int it = 0; it < 64 && lo < hi; ++it) {
                const int64_t mid = lo + ((hi - lo) >> 1);
                const int32_t x = adj[mid];
                if (x < u) lo = mid + 1;
                else if (x > u) hi = mid;
                else { found = mid; break; }
            }
            if (found < 0) {
                ok = false;
            } else {
                rev[s] = (uint32_t)found;
                rev[found] = (uint32_t)s;
            }
        }
        if (!ok) atomicMin(bad, (unsigned long long)s);
    }
    __syncthreads();
    if (threadIdx.x == 0 && block_up) atomicAdd(up, (unsigned long long)block_up);
}

// per vertex: number of slots whose neighbour ranks above it
__global__ void k_count_oriented(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                 const int32_t *__restrict__ deg, int32_t n, int32_t *__restrict__ cnt) {
    int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & 31;
    if (u >= n) return;
    int64_t b = off[u], e = off[u + 1];
    int32_t du = deg[u];
    int c = 0;
    for (int64_t s = b + lane; s < e; s += kWarp) {
        int32_t v = adj[s];
        c += dev::rank_less(du, (int32_t)u, deg[v], v);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[u] = c;
}

__global__ void k_write_oriented(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                 const int32_t *__restrict__ deg, int32_t n, const int64_t *__restrict__ pos,
                                 uint32_t *__restrict__ oe) {
    int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & 31;
    if (u >= n) return;
    int64_t b = off[u], e = off[u + 1];
    int32_t du = deg[u];
    int64_t w = pos[u];
    for (int64_t s0 = b; s0 < e; s0 += kWarp) {
        int64_t s = s0 + lane;
        bool f = false;
        if (s < e) {
            int32_t v = adj[s];
            f = dev::rank_less(du, (int32_t)u, deg[v], v);
        }
        unsigned mask = __ballot_sync(0xffffffffu, f);
        if (f) oe[w + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)s;
        w += __popc(mask);
    }
}

}  // namespace

scan_status graph_prepare(Graph *g) {
    Ctx *c = g->ctx;
    const int32_t n = g->n;
    const int64_t nnz = g->nnz;
    DevBuf badb;
    SCAN_TRY(dev_alloc(c, badb, 2 * sizeof(unsigned long long)));
    unsigned long long *bad = (unsigned long long *)badb.ptr, *up = bad + 1;
    unsigned long long hbad = kNoBad, hup = 0;
    auto fail = [&](scan_status s) { dev_free(c, badb); return s; };
    cudaError_t e = cudaMemcpyAsync(bad, &hbad, sizeof(hbad), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(up, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "upload bad flag"));

    const int64_t *off = (const int64_t *)g->off.ptr;
    const int32_t *adj = (const int32_t *)g->adj.ptr;
    k_check_offsets<<<grid_for((int64_t)n + 1, 256), 256, 0, c->stream>>>(off, n, nnz, bad);
    c->launches++;
    e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "offsets check"));
    if (hbad != kNoBad) {
        set_error("invalid CSR offsets at index " + std::to_string(hbad & ~(1ull << 62)) +
                  " (need offsets[0] = 0, non-decreasing, offsets[n] = nnz)");
        return fail(SCAN_EINVAL);
    }

    int32_t *deg = (int32_t *)g->deg.ptr;
    int32_t *src = (int32_t *)g->src.ptr;
    uint32_t *rev = (uint32_t *)g->rev.ptr;
    if (n > 0) {
        k_deg_src<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(off, n, deg, src);
        c->launches++;
    }
    if (nnz > 0) {
        k_check_rev<<<grid_for(nnz, 256), 256, 0, c->stream>>>(off, adj, src, n, nnz, rev, bad, up);
        c->launches++;
    }
    e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hup, up, sizeof(hup), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "slot checks"));
    if (hbad != kNoBad) {
        set_error("invalid CSR at slot " + std::to_string(hbad) +
                  " (rows must be strictly ascending, ids in [0, n), no self-loops, symmetric)");
        return fail(SCAN_EINVAL);
    }
    if (2 * hup != (unsigned long long)nnz) {
        set_error("invalid CSR: not symmetric (" + std::to_string(hup) + " slots point to a higher id, " +
                  std::to_string((unsigned long long)nnz - hup) + " to a lower one)");
        return fail(SCAN_EINVAL);
    }
    dev_free(c, badb);

    // degree-oriented edge list, grouped by the lower endpoint (offsets kept in foff)
    int32_t *cnt = (int32_t *)g->cnt.ptr;
    SCAN_TRY(dev_alloc(c, g->foff, 8 * ((size_t)n + 1)));
    int64_t *pos = (int64_t *)g->foff.ptr;
    if (n > 0) {
        k_count_oriented<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(off, adj, deg, n, cnt);
        c->launches++;
    }
    SCAN_TRY(launch_exclusive_scan_i32_to_i64(c, cnt, pos, n, g->scan_tmp));
    if (n > 0) {
        k_write_oriented<<<grid_for((int64_t)n * kWarp, 256), 256, 0, c->stream>>>(off, adj, deg, n, pos,
                                                                                 (uint32_t *)g->oe.ptr);
        c->launches++;
    }
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;  // the kernel families build their schedules on first use
}

}  // namespace scan

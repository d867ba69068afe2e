// static_counts.cu -- closed common counts for a caller's device CSR with no
// allocation at all.
//
// For callers that cannot allocate device memory: code running inside
// another library's memory pool or under a strict memory budget, a process
// whose allocator is owned by someone else, or a context where a
// cudaMalloc/cudaFree would synchronise the device at a bad moment. The
// caller passes the CSR and the output array; the working arrays (degree,
// row of each slot, reverse slot, an error word) live in one file-scope
// __device__ array of fixed size that every GPU loading this library holds
// until the process exits.
//
// The kernel is the per-edge binary-search count (the library's plain
// comparator kernel) with its scratch moved into that array.
#include "scan_internal.cuh"

namespace {

constexpr size_t kStaticBytes = 64ull << 20;  // 64 MiB of device scratch

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_st_check_offsets(const int64_t *__restrict__ off, int32_t n, int64_t nnz,
                                   unsigned long long *bad) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    const int64_t o = off[u];
    bool ok = (u == 0) ? (o == 0) : (o >= off[u - 1]);
    if (u == n) ok = ok && (o == nnz);
    if (!ok) atomicMin(bad, 0ull);  // slot 0 stands for "bad offsets"
}

__global__ void k_st_deg_src(const int64_t *__restrict__ off, int32_t n, int32_t *__restrict__ deg,
                             int32_t *__restrict__ src) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const int64_t b = off[u], e = off[u + 1];
    if (lane == 0) deg[u] = (int32_t)(e - b);
    for (int64_t s = b + lane; s < e; s += 32) src[s] = (int32_t)u;
}

__global__ void k_st_rev(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                         const int32_t *__restrict__ src, int32_t n, int64_t nnz, uint32_t *__restrict__ rev,
                         unsigned long long *bad) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    const int32_t u = src[s], v = adj[s];
    bool ok = v >= 0 && v < n && v != u;
    if (ok && s > off[u]) ok = adj[s - 1] < v;
    if (ok) {
        int64_t lo = off[v], hi = off[v + 1], found = -1;
        for (int it = 0; it < 64 && lo < hi; ++it) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            const int32_t x = adj[mid];
            if (x < u) lo = mid + 1;
            else if (x > u) hi = mid;
            else { found = mid; break; }
        }
        if (found < 0) ok = false;
        else rev[s] = (uint32_t)found;
    }
    if (!ok) atomicMin(bad, (unsigned long long)s + 1);
}

// warp per slot; the lower (deg, id) endpoint's slot counts the edge
__global__ void __launch_bounds__(256) k_st_counts(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                   const int32_t *__restrict__ src, const uint32_t *__restrict__ rev,
                                                   const int32_t *__restrict__ deg, int64_t nnz,
                                                   int32_t *__restrict__ cn) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; s < nnz; s += warps) {
        const int32_t u = src[s], v = adj[s];
        const int32_t du = deg[u], dv = deg[v];
        if (!scan::dev::rank_less(du, u, dv, v)) continue;
        const int32_t *ru = adj + off[u];
        const int32_t *rv = adj + off[v];
        int c = 0;
        for (int32_t k = lane; k < du; k += 32) {
            const int32_t x = ru[k];
            int32_t lo = 0, hi = dv;
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                const int32_t y = rv[mid];
                if (y < x) lo = mid + 1;
                else if (y > x) hi = mid;
                else { ++c; break; }
            }
        }
        c = __reduce_add_sync(0xffffffffu, c) + 2;
        if (lane == 0) {
            cn[s] = c;
            cn[rev[s]] = c;
        }
    }
}

}  // namespace

extern "C" scan_status scan_common_counts_static(const int64_t *offsets, const int32_t *adj, int32_t n, int64_t nnz,
                                                 int32_t *cn, void *stream) {
    using scan::set_error;
    if (n < 0 || nnz < 0 || (n > 0 && !offsets) || (nnz > 0 && (!adj || !cn)) || nnz % 2 != 0) {
        set_error("bad sizes or NULL arrays");
        return SCAN_EINVAL;
    }
    if (n == 0 && nnz != 0) {
        set_error("an empty graph has nnz = 0");
        return SCAN_EINVAL;
    }
    const size_t need = 256 + align256(4 * ((size_t)n + 1)) + align256(4 * (size_t)nnz) * 2;
    if (need > kStaticBytes || (uint64_t)nnz >= (1ull << 32)) {
        set_error("graph too large for the fixed scratch: needs " + std::to_string(need) + " bytes of the " +
                  std::to_string(kStaticBytes) + " available (about n + 2*nnz <= 16.7M entries)");
        return SCAN_EINVAL;
    }
    // The host-side symbol is only a stand-in; the array's device address on
    // the current device comes from the runtime. It is looked up on every
    // call (a host-side table lookup once the module is loaded), so a device
    // or context reset, which reloads the module at a new address, can never
    // leave a stale address behind.
    unsigned char *base = nullptr;
    {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return scan::cuda_fail(e, "cudaGetSymbolAddress");
        base = (unsigned char *)p;
    }
    cudaStream_t st = (cudaStream_t)stream;
    auto *bad = (unsigned long long *)base;
    auto *deg = (int32_t *)(base + 256);
    auto *src = (int32_t *)(base + 256 + align256(4 * ((size_t)n + 1)));
    auto *rev = (uint32_t *)((unsigned char *)src + align256(4 * (size_t)nnz));
    // the error word must start at "no error" (all ones) on every call
    SCAN_CUDA(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st));
    unsigned long long hbad = 0;
    if (n > 0) {
        k_st_check_offsets<<<scan::grid_for((int64_t)n + 1, 256), 256, 0, st>>>(offsets, n, nnz, bad);
        SCAN_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
        SCAN_CUDA(cudaStreamSynchronize(st));
        if (hbad != ~0ull) {
            set_error("invalid CSR offsets (need offsets[0] = 0, non-decreasing, offsets[n] = nnz)");
            return SCAN_EINVAL;
        }
        k_st_deg_src<<<scan::grid_for((int64_t)n * 32, 256), 256, 0, st>>>(offsets, n, deg, src);
    }
    if (nnz > 0) {
        k_st_rev<<<scan::grid_for(nnz, 256), 256, 0, st>>>(offsets, adj, src, n, nnz, rev, bad);
        SCAN_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
        SCAN_CUDA(cudaStreamSynchronize(st));
        if (hbad != ~0ull) {
            set_error("invalid CSR at slot " + std::to_string(hbad - 1) +
                      " (rows must be strictly ascending, ids in [0, n), no self-loops, symmetric)");
            return SCAN_EINVAL;
        }
        k_st_counts<<<scan::grid_for(nnz * 32, 256, 1 << 16), 256, 0, st>>>(offsets, adj, src, rev, deg, nnz, cn);
    }
    SCAN_CUDA(cudaGetLastError());
    SCAN_CUDA(cudaStreamSynchronize(st));
    return SCAN_OK;
}

// k_util.cu -- device-wide exclusive prefix sum (int32 counts -> int64 offsets).
//
// Three launches: per-tile sums, one block scanning the tile sums, then each
// tile scanned and offset. out has count+1 entries; out[count] = total.
#include "scan_internal.cuh"

namespace scan {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total. Safe to call repeatedly (ends with a barrier).
__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t *total) {
    constexpr int kW = kScanThreads / 32;
    __shared__ int64_t warp_off[kW];
    __shared__ int64_t tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(x);
    if (lane == 31) warp_off[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < kW ? warp_off[lane] : 0;
        int64_t si = warp_incl_scan(s);
        if (lane < kW) warp_off[lane] = si - s;
        if (lane == kW - 1) tot = si;
    }
    __syncthreads();
    int64_t excl = inc - x + warp_off[wid];
    *total = tot;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int32_t *__restrict__ in, int64_t count,
                                                             int64_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < count) s += in[i];
    }
    int64_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *__restrict__ sums, int64_t nsums) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nsums; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        int64_t x = i < nsums ? sums[i] : 0;
        int64_t total;
        int64_t ex = block_excl_scan(x, &total);
        if (i < nsums) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const int32_t *__restrict__ in, int64_t count,
                                                             const int64_t *__restrict__ sums,
                                                             int64_t *__restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < count ? in[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_excl_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < count) out[i] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = sums[blockIdx.x] + total;
}

}  // namespace

scan_status launch_exclusive_scan_i32_to_i64(Ctx *c, const int32_t *in, int64_t *out, int64_t count,
                                             DevBuf &tmp) {
    if (count == 0) {
        SCAN_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
        return SCAN_OK;
    }
    int64_t tiles = (count + kTile - 1) / kTile;
    if (tmp.bytes < (size_t)tiles * sizeof(int64_t)) {
        dev_free(c, tmp);
        SCAN_TRY(dev_alloc(c, tmp, (size_t)tiles * sizeof(int64_t)));
    }
    int64_t *sums = (int64_t *)tmp.ptr;
    k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, count, sums);
    k_scan_sums<<<1, kScanThreads, 0, c->stream>>>(sums, tiles);
    k_tile_scan<<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, count, sums, out);
    c->launches += 3;
    SCAN_CUDA(cudaGetLastError());
    return SCAN_OK;
}

}  // namespace scan

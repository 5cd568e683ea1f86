// scan.cu -- device-wide exclusive scan of int32 counts into int64 offsets.
//
// out[0] = base, out[i+1] = base + in[0] + ... + in[i]  (count+1 outputs).
// Three passes: per-tile sums, a single-block scan of the tile sums, and a
// per-tile rescan that adds the tile's prefix.
#include "internal.cuh"

namespace im {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;                      // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total, int64_t *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan<int64_t>(v, lane);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < (kScanThreads / 32) ? sh[lane] : 0;
        int64_t si = warp_incl_scan<int64_t>(s, lane);
        if (lane < kScanThreads / 32) sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    int64_t r = sh[warp] + incl - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int32_t *in, int64_t count,
                                                            int64_t *sums) {
    __shared__ int64_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < count) s += in[idx];
    }
    int64_t total;
    block_excl_scan(s, &total, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *sums, int64_t ntiles,
                                                            const int64_t *base, int64_t *grand) {
    __shared__ int64_t sh[33];
    int64_t carry = base ? *base : 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        int64_t idx = b0 + threadIdx.x;
        int64_t v = idx < ntiles ? sums[idx] : 0;
        int64_t total;
        int64_t ex = block_excl_scan(v, &total, sh);
        if (idx < ntiles) sums[idx] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const int32_t *in, int64_t count,
                                                            const int64_t *prefix, int64_t *out,
                                                            const int64_t *grand) {
    __shared__ int64_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    // each thread owns kScanItems consecutive items
    int32_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = idx < count ? in[idx] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t run = prefix[blockIdx.x] + block_excl_scan(s, &total, sh);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < count) out[idx] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[count] = *grand;
}

}  // namespace

size_t scan_tmp_bytes(int64_t count) {
    int64_t ntiles = (count + kScanTile - 1) / kScanTile;
    return (size_t)(ntiles + 2) * sizeof(int64_t);
}

im_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t count,
                                    const int64_t *base, void *tmp, size_t tmp_bytes,
                                    cudaStream_t st) {
    int64_t ntiles = (count + kScanTile - 1) / kScanTile;
    if (tmp_bytes < scan_tmp_bytes(count)) return IM_ERR_INVALID_ARG;
    int64_t *sums = (int64_t *)tmp;
    int64_t *grand = sums + ntiles + 1;
    if (count == 0) {
        // out[0] = base
        {
            KernelTimer kt(st, "scan");
            k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, 0, base, grand);
        }
        IM_CUDA(cudaMemcpyAsync(out, grand, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        return IM_OK;
    }
    {
        KernelTimer kt(st, "scan");
        k_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, count, sums);
    }
    {
        KernelTimer kt(st, "scan");
        k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, ntiles, base, grand);
    }
    {
        KernelTimer kt(st, "scan");
        k_tile_scan<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, count, sums, out, grand);
    }
    IM_CUDA(cudaGetLastError());
    return IM_OK;
}

}  // namespace im

// index.cu -- covering subsets S(v) (Sec. 3.2) and the RandGreedi partition
// structures (Alg. 3).
//
// S(v) is the transpose of the RRR CSR: a histogram of member ids, an
// exclusive scan into vtx_off, and a scatter of set ids.  On one GPU this is
// the paper's all-to-all shuffle of covering subsets (Alg. 3), done in place.
// Set ids inside one S(v) land in atomic order; nothing downstream depends on
// that order.
//
// For RandGreedi every vertex gets a Philox label part(v) in [0, P); the
// vertices of each part are listed in ascending id (part_off / part_vtx), and
// loc(v) is v's rank inside its part.
#include <algorithm>

#include "internal.cuh"

namespace im {

namespace {

constexpr int kChunk = 4096;   // vertices per chunk of the stable partition scatter

// Counters are replicated R times (replica of member position t: (t >> 12) % R,
// the same rule in the histogram and the scatter) so that the atomics on a
// hub vertex, which appears in a large share of the sets, spread over R
// addresses instead of queueing on one.
__device__ __forceinline__ int64_t replica_of(int64_t t, int32_t R) { return (t >> 12) % R; }

__global__ void k_vertex_hist(const int32_t *members, int64_t T, int32_t *cnt, int64_t n,
                              int32_t R) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < T;
         base += stride) {
        const int64_t t = base + lane;
        if (t < T) red_add_s32(&cnt[replica_of(t, R) * n + members[t]], 1);
    }
}

// total[v] = sum of v's replica counts; each replica count becomes the
// replica's starting offset inside S(v)
__global__ void k_replica_offsets(int32_t *cnt, int64_t n, int32_t R, int32_t *total) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        for (int32_t r = 0; r < R; ++r) {
            const int32_t x = cnt[r * n + v];
            cnt[r * n + v] = c;
            c += x;
        }
        total[v] = c;
    }
}

__global__ void k_scatter(const int64_t *set_off, const int32_t *members, int64_t theta,
                          const int64_t *vtx_off, int32_t *cursor, int64_t n, int32_t R,
                          int32_t *set_ids) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         i0 < theta; i0 += warps * 32) {
        // the 32 sets' members are contiguous from set_off[i0]; the lane of a
        // position is found among the inclusive set sizes, U positions per
        // lane at a time so that U cursor atomics are in flight
        const int64_t i = i0 + lane;
        int64_t len = 0;
        if (i < theta) len = set_off[i + 1] - set_off[i];
        const int64_t incl = warp_incl_scan<int64_t>(len, lane);
        const int64_t total = __shfl_sync(kFull, incl, 31);
        const int64_t first = set_off[i0];
        constexpr int U = 8;
        for (int64_t base = 0; base < total; base += 32 * U) {
            int32_t sid[U], u[U];
            int64_t t[U], pos[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                t[q] = base + q * 32 + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int64_t c = __shfl_sync(kFull, incl, owner + step - 1);
                    if (c <= t[q]) owner += step;
                }
                sid[q] = (int32_t)(i0 + owner);
                u[q] = t[q] < total ? __ldg(members + first + t[q]) : -1;
            }
#pragma unroll
            for (int q = 0; q < U; ++q)
                pos[q] = u[q] >= 0 ? atomicAdd(&cursor[replica_of(first + t[q], R) * n + u[q]], 1) : 0;
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (u[q] >= 0) set_ids[vtx_off[u[q]] + pos[q]] = sid[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Covering subsets by a stable LSD radix sort of the (vertex, set id) pairs of
// the RRR CSR, digit by digit from the low bits.  Pairs start in set order, so
// every S(v) comes out with its set ids ascending.  A pass over one digit:
//   k_rx_count    per tile of kRxTile pairs, the count of every digit value
//                 (table, digit-major: [digit][tile]);
//   a scan of the table gives every (digit, tile) run its output offset;
//   k_rx_scatter  ranks the tile's pairs by digit in shared memory (stable:
//                 warp by warp, item by item, lanes in order), places them in
//                 digit order there, and writes each digit's run to its offset
//                 (consecutive threads write consecutive positions).
// The first pass reads the members and derives each pair's set id from
// set_off; the last writes the set ids to S(v) and the keys to a buffer from
// which k_rx_bounds counts |S(v)| (start and end of every run of equal keys).
// ---------------------------------------------------------------------------
constexpr int kRxThreads = 512;
constexpr int kRxWarps = kRxThreads / 32;
constexpr int kRxItems = 16;
constexpr int kRxTile = kRxThreads * kRxItems;   // pairs per tile
constexpr int kRxMaxBits = 8;
constexpr int kRxMaxBins = 1 << kRxMaxBits;

// Position of item j of lane `lane` of warp w in tile `tile`: warp w holds the
// tile's w-th run of 32 kRxItems positions, item j its j-th run of 32.
__device__ __forceinline__ int64_t rx_pos(int64_t tile, int w, int j, int lane) {
    return tile * kRxTile + (int64_t)w * (32 * kRxItems) + j * 32 + lane;
}

__global__ void __launch_bounds__(kRxThreads) k_rx_count(const int32_t *keys, int64_t T, int shift,
                                                         int bits, int64_t ntiles, int32_t *table) {
    __shared__ int32_t h[kRxWarps][kRxMaxBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t mask = (1u << bits) - 1u;
    const int bins = 1 << bits;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < kRxWarps * kRxMaxBins; i += kRxThreads) (&h[0][0])[i] = 0;
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < kRxItems; ++j) {
            const int64_t t = rx_pos(tile, w, j, lane);
            if (t < T) atomicAdd(&h[w][((uint32_t)__ldg(keys + t) >> shift) & mask], 1);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < bins; d += kRxThreads) {
            int32_t c = 0;
            for (int q = 0; q < kRxWarps; ++q) c += h[q][d];
            table[(int64_t)d * ntiles + tile] = c;
        }
        __syncthreads();
    }
}

// kFirst: the keys are the members and the values the set ids, found from
// set_off (lane 0 of a warp searches the set of the warp's first position, then
// every lane advances through set_off as its positions grow).
template <bool kFirst>
__global__ void __launch_bounds__(kRxThreads, 2) k_rx_scatter(
    const int32_t *kin, const int32_t *vin, const int64_t *set_off, int64_t theta, int64_t T,
    int shift, int bits, int64_t ntiles, const int64_t *goff, int32_t *kout, int32_t *vout) {
    extern __shared__ int32_t rx_smem[];          // [kRxTile] keys, then [kRxTile] values
    int32_t *skey = rx_smem, *sval = rx_smem + kRxTile;
    __shared__ int32_t wc[kRxWarps][kRxMaxBins];  // per warp and digit: count, then start
    __shared__ int32_t dstart[kRxMaxBins];        // first local index of every digit
    __shared__ int64_t sgo[kRxMaxBins];           // output offset of every digit's run
    __shared__ int32_t wsum[kRxMaxBins / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t mask = (1u << bits) - 1u;
    const int bins = 1 << bits;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < kRxWarps * kRxMaxBins; i += kRxThreads) (&wc[0][0])[i] = 0;
        for (int d = threadIdx.x; d < bins; d += kRxThreads)
            sgo[d] = goff[(int64_t)d * ntiles + tile];
        __syncthreads();
        uint32_t key[kRxItems];
        uint32_t rk[kRxItems / 2];                 // two 16-bit ranks per register
#pragma unroll
        for (int j = 0; j < kRxItems; ++j) {
            const int64_t t = rx_pos(tile, w, j, lane);
            key[j] = t < T ? (uint32_t)__ldg(kin + t) : 0u;
        }
        // rank of every pair among the warp's earlier pairs of its digit
#pragma unroll
        for (int j = 0; j < kRxItems; ++j) {
            const bool ok = rx_pos(tile, w, j, lane) < T;
            const uint32_t d = ok ? (key[j] >> shift) & mask : (uint32_t)(kRxMaxBins + lane);
            const unsigned peers = __match_any_sync(kFull, d);
            int32_t base = 0;
            if (ok) base = wc[w][d];
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wc[w][d] = base + __popc(peers);
            __syncwarp();
            const uint32_t r = (uint32_t)(base + __popc(peers & lt));
            rk[j >> 1] = (j & 1) ? (rk[j >> 1] | (r << 16)) : r;
        }
        __syncthreads();
        // digit-major starts: digit d's run of warp q begins after every
        // smaller digit and after digit d's pairs of warps < q
        int32_t tot = 0;
        if (threadIdx.x < bins) {
            for (int q = 0; q < kRxWarps; ++q) {
                const int32_t c = wc[q][threadIdx.x];
                wc[q][threadIdx.x] = tot;
                tot += c;
            }
        }
        const int32_t incl = warp_incl_scan<int32_t>(tot, lane);
        if (lane == 31 && w < kRxMaxBins / 32) wsum[w] = incl;
        __syncthreads();
        if (threadIdx.x < bins) {
            int32_t before = 0;
            for (int q = 0; q < w; ++q) before += wsum[q];
            const int32_t ds = before + incl - tot;
            dstart[threadIdx.x] = ds;
            for (int q = 0; q < kRxWarps; ++q) wc[q][threadIdx.x] += ds;
        }
        __syncthreads();
        // place every pair at its local sorted index
        int64_t cur = 0;
        if (kFirst) {
            const int64_t t0 = rx_pos(tile, w, 0, 0);
            if (lane == 0 && t0 < T) {
                int64_t lo = 0, hi = theta - 1;       // largest s with set_off[s] <= t0
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(set_off + mid) <= t0) lo = mid;
                    else hi = mid - 1;
                }
                cur = lo;
            }
            cur = __shfl_sync(kFull, cur, 0);
        }
#pragma unroll
        for (int j = 0; j < kRxItems; ++j) {
            const int64_t t = rx_pos(tile, w, j, lane);
            if (t < T) {
                const uint32_t d = (key[j] >> shift) & mask;
                const int32_t idx = wc[w][d] + (int32_t)((rk[j >> 1] >> (16 * (j & 1))) & 0xffffu);
                skey[idx] = (int32_t)key[j];
                if (kFirst) {
                    while (__ldg(set_off + cur + 1) <= t) ++cur;
                    sval[idx] = (int32_t)cur;
                } else {
                    sval[idx] = __ldg(vin + t);
                }
            }
        }
        __syncthreads();
        const int64_t t0 = tile * kRxTile;
        const int32_t tn = (int32_t)min((int64_t)kRxTile, T - t0);
        for (int32_t i = threadIdx.x; i < tn; i += kRxThreads) {
            const uint32_t k = (uint32_t)skey[i];
            const uint32_t d = (k >> shift) & mask;
            const int64_t pos = sgo[d] + (i - dstart[d]);
            vout[pos] = sval[i];
            kout[pos] = (int32_t)k;
        }
        __syncthreads();
    }
}

// |S(v)| from the sorted keys: a run of key v over positions [b, e) adds
// e - b to cnt[v] (as -b at its first position and +e at its last, modulo
// 2^32; the total is below 2^31).
__global__ void k_rx_bounds(const int32_t *keys, int64_t T, uint32_t *cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < T;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = keys[p];
        if (p == 0 || keys[p - 1] != k) atomicAdd(cnt + k, 0u - (uint32_t)p);
        if (p == T - 1 || keys[p + 1] != k) atomicAdd(cnt + k, (uint32_t)(p + 1));
    }
}

__global__ void k_part_labels(int64_t n, uint32_t P, uint64_t pseed, int32_t *part) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        part[v] = vertex_part(pseed, (uint32_t)v, P);
}

// hist[c * P + p] = |{v in chunk c : part(v) = p}|
__global__ void k_part_hist(const int32_t *part, int64_t n, int32_t P, int32_t *hist) {
    extern __shared__ int32_t sh[];
    for (int p = threadIdx.x; p < P; p += blockDim.x) sh[p] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)blockIdx.x * kChunk;
    const int64_t v1 = min(n, v0 + kChunk);
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) atomicAdd(&sh[part[v]], 1);
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) hist[(int64_t)blockIdx.x * P + p] = sh[p];
}

// part_off[p] = vertices in parts < p; hist turns into chunk start offsets
__global__ void k_part_offsets(int32_t *hist, int64_t nchunks, int32_t P, int32_t *part_off) {
    // one thread per part scans its column; then a serial scan of the totals
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int32_t run = 0;
        for (int64_t c = 0; c < nchunks; ++c) {
            const int32_t h = hist[c * P + p];
            hist[c * P + p] = run;
            run += h;
        }
        part_off[p + 1] = run;   // temporarily the size of part p
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        part_off[0] = 0;
        for (int p = 0; p < P; ++p) {
            const int32_t sz = part_off[p + 1];
            part_off[p + 1] = run + sz;
            run += sz;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x)
        for (int64_t c = 0; c < nchunks; ++c) hist[c * P + p] += part_off[p];
}

// One warp per chunk writes its vertices in ascending order into their parts.
__global__ void k_part_scatter(const int32_t *part, int64_t n, int32_t P, const int32_t *hist,
                               const int32_t *part_off, int32_t *part_vtx, int32_t *part_loc) {
    extern __shared__ int32_t run[];   // per-part write cursor of this chunk
    const int lane = threadIdx.x;
    for (int p = lane; p < P; p += 32) run[p] = hist[(int64_t)blockIdx.x * P + p];
    __syncwarp();
    const int64_t v0 = (int64_t)blockIdx.x * kChunk;
    const int64_t v1 = min(n, v0 + kChunk);
    for (int64_t base = v0; base < v1; base += 32) {
        const int64_t v = base + lane;
        const int32_t p = v < v1 ? part[v] : -1 - lane;
        const unsigned peers = __match_any_sync(kFull, p);
        const int rank = __popc(peers & ((1u << lane) - 1));
        int32_t at = 0;
        if (v < v1) at = run[p] + rank;
        __syncwarp();
        if (v < v1 && rank == __popc(peers) - 1) run[p] = at + 1;
        __syncwarp();
        if (v < v1) {
            part_vtx[at] = (int32_t)v;
            part_loc[v] = at - part_off[p];
        }
    }
}

__global__ void k_max_seg(const int64_t *off, int64_t n, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
        m = d > m ? d : m;
    }
    m = warp_max_u64(m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace

im_status max_segment_length(const int64_t *off, int64_t n, int64_t *d_out, cudaStream_t st) {
    IM_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int64_t), st));
    {
        KernelTimer kt(st, "max_subset_size");
        k_max_seg<<<num_sms() * 4, 256, 0, st>>>(off, n, (unsigned long long *)d_out);
    }
    IM_CUDA(cudaGetLastError());
    return IM_OK;
}

im_status launch_partition_labels(int64_t n, int32_t P, uint64_t pseed, int32_t *part,
                                  cudaStream_t st) {
    {
        KernelTimer kt(st, "partition_labels");
        k_part_labels<<<num_sms() * 4, 256, 0, st>>>(n, (uint32_t)P, pseed, part);
    }
    IM_CUDA(cudaGetLastError());
    return IM_OK;
}

im_status build_index_raw(const int64_t *set_off, const int32_t *members, int64_t theta, int64_t T,
                          int64_t n, int64_t *vtx_off, int32_t *set_ids, int32_t *cursor,
                          int32_t replicas, void *tmp, cudaStream_t st) {
    // cursor holds R counter replicas and, when R > 1, a row of totals
    const int32_t R = std::max<int32_t>(1, replicas);
    const size_t rows = (size_t)R * n;
    IM_CUDA(cudaMemsetAsync(cursor, 0, rows * sizeof(int32_t), st));
    if (T > 0) {
        KernelTimer kt(st, "index_hist");
        k_vertex_hist<<<num_sms() * 8, 256, 0, st>>>(members, T, cursor, n, R);
    }
    IM_CUDA(cudaGetLastError());
    int32_t *total = cursor;
    if (R > 1) {
        total = cursor + rows;
        KernelTimer kt(st, "index_hist");
        k_replica_offsets<<<num_sms() * 4, 256, 0, st>>>(cursor, n, R, total);
    }
    IM_CUDA(cudaGetLastError());
    im_status s = exclusive_scan_i32_to_i64(total, vtx_off, n, nullptr, tmp, scan_tmp_bytes(n), st);
    if (s != IM_OK) return s;
    if (R == 1) IM_CUDA(cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), st));
    if (theta > 0) {
        KernelTimer kt(st, "index_scatter");
        k_scatter<<<num_sms() * 8, 256, 0, st>>>(set_off, members, theta, vtx_off, cursor, n, R,
                                                 set_ids);
    }
    IM_CUDA(cudaGetLastError());
    return IM_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t radix_index_bytes(int64_t T, int64_t n) {
    const int64_t ntiles = (T + kRxTile - 1) / kRxTile;
    const int64_t cells = (int64_t)kRxMaxBins * ntiles;
    return 3 * up256((size_t)T * 4) + up256((size_t)cells * 4) + up256((size_t)(cells + 1) * 8) +
           std::max(scan_tmp_bytes(cells), scan_tmp_bytes(n)) + 256;
}

im_status build_index_radix(const int64_t *set_off, const int32_t *members, int64_t theta,
                            int64_t T, int64_t n, int64_t *vtx_off, int32_t *set_ids,
                            int32_t *cnt, void *scratch, cudaStream_t st) {
    const int64_t ntiles = (T + kRxTile - 1) / kRxTile;
    const int64_t cells = (int64_t)kRxMaxBins * ntiles;
    char *b = (char *)scratch;
    auto take = [&](size_t bytes) {
        char *r = b;
        b += up256(bytes);
        return r;
    };
    int32_t *kA = (int32_t *)take((size_t)T * 4), *kB = (int32_t *)take((size_t)T * 4),
            *vB = (int32_t *)take((size_t)T * 4);
    int32_t *table = (int32_t *)take((size_t)cells * 4);
    int64_t *goff = (int64_t *)take((size_t)(cells + 1) * 8);
    void *stmp = take(0);
    const size_t stmp_bytes = std::max(scan_tmp_bytes(cells), scan_tmp_bytes(n));
    // digits: nbits = bit length of n - 1, split evenly over ceil(nbits / 8) passes
    int nbits = 0;
    while (nbits < 63 && ((int64_t)1 << nbits) < n) ++nbits;
    const int passes = std::max(1, (nbits + kRxMaxBits - 1) / kRxMaxBits);
    const int width = (nbits + passes - 1) / passes;
    IM_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * 4, st));
    if (T > 0) {
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms() * 2);
        const size_t smem = (size_t)2 * kRxTile * 4;
        // the scatter's 64 KB of dynamic shared memory (a per-device attribute)
        IM_TRY(raise_dyn_smem((const void *)k_rx_scatter<true>, smem));
        IM_TRY(raise_dyn_smem((const void *)k_rx_scatter<false>, smem));
        const int32_t *kin = members, *vin = nullptr;
        for (int ps = 0; ps < passes; ++ps) {
            const int shift = ps * width;
            const int bits = std::max(0, std::min(width, nbits - shift));
            int32_t *kout = (ps & 1) ? kB : kA;
            int32_t *vout = ((passes - 1 - ps) & 1) ? vB : set_ids;
            {
                KernelTimer kt(st, "index_radix");
                k_rx_count<<<grid, kRxThreads, 0, st>>>(kin, T, shift, bits, ntiles, table);
            }
            IM_CUDA(cudaGetLastError());
            const int64_t used = ((int64_t)1 << bits) * ntiles;
            IM_TRY(exclusive_scan_i32_to_i64(table, goff, used, nullptr, stmp, stmp_bytes, st));
            {
                KernelTimer kt(st, "index_radix");
                if (ps == 0)
                    k_rx_scatter<true><<<grid, kRxThreads, smem, st>>>(
                        kin, vin, set_off, theta, T, shift, bits, ntiles, goff, kout, vout);
                else
                    k_rx_scatter<false><<<grid, kRxThreads, smem, st>>>(
                        kin, vin, set_off, theta, T, shift, bits, ntiles, goff, kout, vout);
            }
            IM_CUDA(cudaGetLastError());
            kin = kout;
            vin = vout;
        }
        {
            KernelTimer kt(st, "index_bounds");
            k_rx_bounds<<<num_sms() * 8, 256, 0, st>>>(kin, T, (uint32_t *)cnt);
        }
        IM_CUDA(cudaGetLastError());
    }
    return exclusive_scan_i32_to_i64(cnt, vtx_off, n, nullptr, stmp, stmp_bytes, st);
}

im_status build_index(im_pool *p, cudaStream_t st) {
    if (p->index_valid) return IM_OK;
    void *tmp = nullptr;
    im_status s = IM_OK;
    const int32_t replicas = (int32_t)tune_value(IM_TUNE_INDEX_REPLICAS);
    if (replicas == 0) {
        // radix sort; with too little device memory for its buffers, the
        // counting transpose below (4 replicas) instead
        s = pool_scratch(p, radix_index_bytes(p->total, p->g->n), &tmp);
        if (s == IM_OK) {
            s = build_index_radix(p->set_off, p->members, p->theta, p->total, p->g->n,
                                  p->vtx_off, p->set_ids, p->vtx_cursor, tmp, st);
            if (s != IM_OK) return s;
            p->index_valid = true;
            return IM_OK;
        }
        if (s != IM_ERR_OOM) return s;
        cudaGetLastError();
    }
    s = pool_scratch(p, scan_tmp_bytes(p->g->n), &tmp);
    if (s != IM_OK) return s;
    s = build_index_raw(p->set_off, p->members, p->theta, p->total, p->g->n, p->vtx_off, p->set_ids,
                        p->vtx_cursor, replicas > 0 ? replicas : 4, tmp, st);
    if (s != IM_OK) return s;
    p->index_valid = true;
    return IM_OK;
}

im_status build_partition(im_pool *p, int32_t P, uint64_t pseed, cudaStream_t st) {
    if (p->part_valid && p->part_P == P && p->part_seed == pseed) return IM_OK;
    const int64_t n = p->g->n;
    p->part_valid = false;   // until this build completes
    if (!p->part) IM_TRY(dev_alloc(&p->part, (size_t)n * 4));
    if (!p->part_vtx) IM_TRY(dev_alloc(&p->part_vtx, (size_t)n * 4));
    if (!p->part_loc) IM_TRY(dev_alloc(&p->part_loc, (size_t)n * 4));
    if (p->part_cap < P) {
        dev_free(p->part_off);
        p->part_off = nullptr;
        p->part_cap = 0;
        IM_TRY(dev_alloc(&p->part_off, (size_t)(P + 1) * 4));
        p->part_cap = P;
    }
    im_status s = launch_partition_labels(n, P, pseed, p->part, st);
    if (s != IM_OK) return s;
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    const size_t hist_bytes = (size_t)nchunks * P * 4;
    void *tmp = nullptr;
    s = pool_scratch(p, hist_bytes, &tmp);
    if (s != IM_OK) return s;
    int32_t *hist = (int32_t *)tmp;
    {
        KernelTimer kt(st, "partition_build");
        k_part_hist<<<(unsigned)nchunks, 256, (size_t)P * 4, st>>>(p->part, n, P, hist);
        k_part_offsets<<<1, 256, 0, st>>>(hist, nchunks, P, p->part_off);
        k_part_scatter<<<(unsigned)nchunks, 32, (size_t)P * 4, st>>>(p->part, n, P, hist,
                                                                      p->part_off, p->part_vtx,
                                                                      p->part_loc);
    }
    IM_CUDA(cudaGetLastError());
    p->part_valid = true;
    p->part_P = P;
    p->part_seed = pseed;
    return IM_OK;
}

}  // namespace im

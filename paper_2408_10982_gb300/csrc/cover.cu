// cover.cu -- max-k-cover over the pool: standard greedy (Sec. 3.2) and
// RandGreedi with streaming aggregation and truncation (Alg. 4, Alg. 5,
// Sec. 3.3.2).
//
// Standard greedy: one cooperative persistent kernel runs all k steps.  A step
// is a grid-wide argmax over the marginal gains counts[v] (packed as
// gain << 32 | ~v so that ties go to the smallest id), a grid barrier, the
// cover of S(v*) (atomicOr on a theta-bit bitmap; every newly covered set
// decrements the gains of its members), and a second barrier.  Barriers wait
// at most kWaitLimitNs and then report IM_ERR_TIMEOUT.
//
// RandGreedi: the paper's m sender machines are m "producer" blocks, each
// running the local greedy of one vertex part V_p with its gains in shared
// memory and its own theta-bit covered bitmap; the receiver's B bucketing
// threads are B "consumer" blocks, one bucket each.  A producer publishes its
// j-th seed (j < ceil(alpha k)) in slot (j, p) of a device array and raises a
// release flag; consumers read the slots in (j, p) order with acquire loads,
// so the buckets see the same stream order in every run.  In the fused mode
// producers and consumers are one cooperative launch (co-resident), so the
// aggregation overlaps the local greedy as in the paper's streaming design.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace im {

namespace {

constexpr int kGreedyThreads = 512;
constexpr int kRGThreads = 512;
constexpr int kBatch = 256;                  // stream slots a consumer reads at once

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max_u64(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
        x = warp_max_u64(x);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    const unsigned long long r = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ long long block_sum_i64(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum<long long>(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ll;
        x = warp_sum<long long>(x);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    const long long r = sh[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// standard greedy
// ---------------------------------------------------------------------------
struct GreedyArgs {
    int64_t n, theta;
    const int64_t *set_off;
    const int32_t *members;
    const int64_t *vtx_off;
    const int32_t *set_ids;
    int32_t k;
    int32_t *counts;                    // [n]
    uint32_t *covered;                  // [ceil(theta/32)]
    unsigned long long *block_best;     // [grid]
    GridBarrier *bar;
    int32_t *seeds;
    int64_t *gains;
    int32_t *nseeds;
    int64_t *coverage;
    int *status;
};

__global__ void __launch_bounds__(kGreedyThreads) k_greedy(GreedyArgs a) {
    __shared__ unsigned long long shm[33];
    const uint32_t nb = gridDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = tid >> 5, nwarps = stride >> 5;
    const int64_t words = (a.theta + 31) / 32;
    for (int64_t v = tid; v < a.n; v += stride) a.counts[v] = (int32_t)(a.vtx_off[v + 1] - a.vtx_off[v]);
    for (int64_t x = tid; x < words; x += stride) a.covered[x] = 0u;
    if (!grid_sync(a.bar, nb, a.status)) return;
    int64_t cov = 0;
    int32_t j = 0;
    for (; j < a.k; ++j) {
        unsigned long long best = 0;
        for (int64_t v = tid; v < a.n; v += stride) {
            const int32_t c = __ldcg(a.counts + v);
            if (c > 0) {
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)c << 32) | (0xffffffffu - (uint32_t)v);
                best = key > best ? key : best;
            }
        }
        best = block_max_u64(best, shm);
        if (threadIdx.x == 0) a.block_best[blockIdx.x] = best;
        if (!grid_sync(a.bar, nb, a.status)) return;
        unsigned long long gbest = 0;
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
            const unsigned long long x = __ldcg(a.block_best + b);
            gbest = x > gbest ? x : gbest;
        }
        gbest = block_max_u64(gbest, shm);
        if (gbest == 0) break;                       // every remaining gain is zero
        const int32_t vs = (int32_t)(0xffffffffu - (uint32_t)(gbest & 0xffffffffu));
        const int64_t gain = (int64_t)(gbest >> 32);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.seeds[j] = vs;
            a.gains[j] = gain;
        }
        cov += gain;
        const int64_t sb = a.vtx_off[vs], se = a.vtx_off[vs + 1];
        for (int64_t base = sb + gwarp * 32; base < se; base += nwarps * 32) {
            const int64_t t = base + lane;
            int32_t i = -1;
            bool fresh = false;
            if (t < se) {
                i = a.set_ids[t];
                const uint32_t bit = 1u << (i & 31);
                fresh = !(atomicOr(&a.covered[i >> 5], bit) & bit);
            }
            unsigned fm = __ballot_sync(kFull, fresh);
            while (fm) {
                const int f = __ffs(fm) - 1;
                fm &= fm - 1;
                const int32_t set = __shfl_sync(kFull, i, f);
                const int64_t so = a.set_off[set], eo = a.set_off[set + 1];
                for (int64_t q = so + lane; q < eo; q += 32) atomicSub(&a.counts[a.members[q]], 1);
            }
        }
        if (!grid_sync(a.bar, nb, a.status)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.nseeds = j;
        *a.coverage = cov;
    }
}

// ---------------------------------------------------------------------------
// RandGreedi
// ---------------------------------------------------------------------------
struct RGArgs {
    int64_t n, theta, words;
    int32_t k, P, trunc, B;
    const int64_t *set_off;
    const uint64_t *pkeys;
    const int64_t *vtx_off;
    const int32_t *set_ids;
    const int32_t *part_off;
    const int32_t *part_vtx;
    uint32_t *covered;        // [P][words] producer bitmaps
    uint32_t *bcovered;       // [B][words] bucket bitmaps
    int32_t *local_seeds;
    int64_t *local_gains;
    int32_t *local_n;
    int64_t *local_cov;
    const int64_t *thr;
    int64_t *bucket_cov;
    int32_t *bucket_n;
    int32_t *bucket_seeds;
    int64_t *bucket_gains;
    uint32_t *flags;          // [trunc][P]: 0 empty, 1 seed ready, 2 no seed
    int32_t *elems;           // [trunc][P]
    int32_t nprod, ncons;     // block roles in this launch
    int32_t first_role;       // 0: blocks start with producers; 1: consumers only
    int *status;
};

// Local greedy of part p (Alg. 4, one sender): gains of V_p live in shared memory.
__device__ void produce(const RGArgs &a, int p, int32_t *cnt, unsigned long long *shm) {
    const int32_t vb = a.part_off[p], np = a.part_off[p + 1] - vb;
    const int32_t *vtx = a.part_vtx + vb;
    uint32_t *cov = a.covered + (size_t)p * (size_t)a.words;
    for (int64_t x = threadIdx.x; x < a.words; x += blockDim.x) cov[x] = 0u;
    for (int32_t l = threadIdx.x; l < np; l += blockDim.x) {
        const int32_t v = vtx[l];
        cnt[l] = (int32_t)(a.vtx_off[v + 1] - a.vtx_off[v]);
    }
    __syncthreads();
    const uint64_t lo_key = (uint64_t)(uint32_t)p << 32, hi_key = (uint64_t)(uint32_t)(p + 1) << 32;
    int64_t total = 0;
    int32_t j = 0;
    for (; j < a.k; ++j) {
        unsigned long long best = 0;
        for (int32_t l = threadIdx.x; l < np; l += blockDim.x) {
            const int32_t c = cnt[l];
            if (c > 0) {
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)c << 32) | (0xffffffffu - (uint32_t)l);
                best = key > best ? key : best;
            }
        }
        best = block_max_u64(best, shm);
        if (best == 0) break;
        const int32_t l = (int32_t)(0xffffffffu - (uint32_t)(best & 0xffffffffu));
        const int32_t v = vtx[l];
        const int64_t gain = (int64_t)(best >> 32);
        if (threadIdx.x == 0) {
            a.local_seeds[(int64_t)p * a.k + j] = v;
            a.local_gains[(int64_t)p * a.k + j] = gain;
            if (j < a.trunc) {
                a.elems[(int64_t)j * a.P + p] = v;
                st_release_u32(&a.flags[(int64_t)j * a.P + p], 1u);
            }
        }
        total += gain;
        const int64_t sb = a.vtx_off[v], se = a.vtx_off[v + 1];
        for (int64_t t = sb + threadIdx.x; t < se; t += blockDim.x) {
            const int32_t i = a.set_ids[t];
            const uint32_t bit = 1u << (i & 31);
            if (atomicOr(&cov[i >> 5], bit) & bit) continue;
            // members of R(i) in V_p: keys in [lo_key, hi_key)
            const int64_t so = a.set_off[i], eo = a.set_off[i + 1];
            if (eo - so <= kSortedKeyCap64) {
                int64_t lo = so, hi = eo;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (a.pkeys[mid] < lo_key) lo = mid + 1;
                    else hi = mid;
                }
                for (int64_t q = lo; q < eo; ++q) {
                    const uint64_t key = a.pkeys[q];
                    if (key >= hi_key) break;
                    atomicSub(&cnt[(uint32_t)key], 1);
                }
            } else {
                for (int64_t q = so; q < eo; ++q) {
                    const uint64_t key = a.pkeys[q];
                    if (key >= lo_key && key < hi_key) atomicSub(&cnt[(uint32_t)key], 1);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.local_n[p] = j;
        a.local_cov[p] = total;
        for (int32_t jj = j; jj < a.trunc; ++jj) st_release_u32(&a.flags[(int64_t)jj * a.P + p], 2u);
    }
    __syncthreads();
}

// Streaming bucket b (Alg. 5): consume the stream in (j, p) order.
__device__ void consume(const RGArgs &a, int b, long long *shs) {
    __shared__ int32_t s_x[kBatch];
    __shared__ int64_t s_off[kBatch];
    __shared__ int64_t s_len[kBatch];
    __shared__ int s_timeout;
    uint32_t *C = a.bcovered + (size_t)b * (size_t)a.words;
    for (int64_t x = threadIdx.x; x < a.words; x += blockDim.x) C[x] = 0u;
    if (threadIdx.x == 0) s_timeout = 0;
    __syncthreads();
    const int64_t T = a.thr[b];
    const int64_t E = (int64_t)a.trunc * a.P;
    int32_t bn = 0;
    int64_t bcov = 0;
    for (int64_t base = 0; base < E && bn < a.k; base += kBatch) {
        const int64_t cntb = min((int64_t)kBatch, E - base);
        if (threadIdx.x < cntb) {
            const int64_t slot = base + threadIdx.x;
            uint32_t f = ld_acquire_u32(a.flags + slot);
            if (f == 0) {
                const uint64_t t0 = global_ns();
                while ((f = ld_acquire_u32(a.flags + slot)) == 0) {
                    if (global_ns() - t0 > kWaitLimitNs) {
                        raise_status(a.status, kDevTimeout);
                        s_timeout = 1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            int32_t x = -1;
            int64_t off = 0, len = 0;
            if (f == 1) {
                x = __ldcg(a.elems + slot);
                off = a.vtx_off[x];
                len = a.vtx_off[x + 1] - off;
            }
            s_x[threadIdx.x] = x;
            s_off[threadIdx.x] = off;
            s_len[threadIdx.x] = len;
        }
        __syncthreads();
        if (s_timeout) break;
        for (int64_t q = 0; q < cntb && bn < a.k; ++q) {
            const int32_t x = s_x[q];
            const int64_t len = s_len[q];
            if (x < 0 || len < T) continue;      // |S(x) \ C_b| <= |S(x)| < threshold
            const int64_t off = s_off[q];
            long long miss = 0;
            for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
                const int32_t i = a.set_ids[off + t];
                miss += !((__ldcg(C + (i >> 5)) >> (i & 31)) & 1u);
            }
            const long long gain = block_sum_i64(miss, shs);
            if (gain >= T) {
                for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
                    const int32_t i = a.set_ids[off + t];
                    atomicOr(&C[i >> 5], 1u << (i & 31));
                }
                if (threadIdx.x == 0) {
                    a.bucket_seeds[(int64_t)b * a.k + bn] = x;
                    a.bucket_gains[(int64_t)b * a.k + bn] = gain;
                }
                ++bn;
                bcov += gain;
                __syncthreads();
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.bucket_n[b] = bn;
        a.bucket_cov[b] = bcov;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kRGThreads) k_randgreedi(RGArgs a) {
    extern __shared__ int32_t cnt[];
    __shared__ unsigned long long shm[33];
    const int r = blockIdx.x;
    if (a.first_role == 0 && r < a.nprod) {
        for (int p = r; p < a.P; p += a.nprod) produce(a, p, cnt, shm);
    } else {
        const int c = a.first_role == 0 ? r - a.nprod : r;
        for (int b = c; b < a.B; b += a.ncons) consume(a, b, (long long *)shm);
    }
}

// Alg. 4's final compare: best bucket (ties: smallest b) against the best
// local solution (ties: smallest p); the bucket wins ties.
__global__ void k_rg_final(RGArgs a, int32_t *seeds, int64_t *gains, int32_t *nseeds,
                           int64_t *coverage, int32_t *chosen) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int bstar = 0;
    for (int b = 1; b < a.B; ++b)
        if (a.bucket_cov[b] > a.bucket_cov[bstar]) bstar = b;
    int pbest = 0;
    for (int p = 1; p < a.P; ++p)
        if (a.local_cov[p] > a.local_cov[pbest]) pbest = p;
    if (a.bucket_cov[bstar] >= a.local_cov[pbest]) {
        *chosen = -1;
        const int32_t m = a.bucket_n[bstar];
        for (int32_t j = 0; j < m; ++j) {
            seeds[j] = a.bucket_seeds[(int64_t)bstar * a.k + j];
            gains[j] = a.bucket_gains[(int64_t)bstar * a.k + j];
        }
        *nseeds = m;
        *coverage = a.bucket_cov[bstar];
    } else {
        *chosen = pbest;
        const int32_t m = a.local_n[pbest];
        for (int32_t j = 0; j < m; ++j) {
            seeds[j] = a.local_seeds[(int64_t)pbest * a.k + j];
            gains[j] = a.local_gains[(int64_t)pbest * a.k + j];
        }
        *nseeds = m;
        *coverage = a.local_cov[pbest];
    }
}

}  // namespace

int32_t num_buckets(int32_t k, double delta) {
    double x = 1.0;
    int32_t b = 0;
    while (x < (double)k) {
        x *= 1.0 + delta;
        ++b;
    }
    return b < 1 ? 1 : b;
}

im_status greedy_plain(im_pool *p, int32_t k, int32_t *d_seeds, int64_t *d_gains,
                       int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st, int *d_status) {
    const int64_t n = p->g->n, theta = p->theta;
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy, kGreedyThreads, 0));
    if (per_sm < 1) return IM_ERR_UNSUPPORTED;
    const int grid = per_sm * num_sms();
    const int64_t words = (theta + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t o_cnt = take((size_t)n * 4), o_cov = take((size_t)std::max<int64_t>(words, 1) * 4),
                 o_best = take((size_t)grid * 8), o_bar = take(sizeof(GridBarrier));
    void *base = nullptr;
    im_status s = pool_scratch(p, off, &base);
    if (s != IM_OK) return s;
    char *B = (char *)base;
    IM_CUDA(cudaMemsetAsync(B + o_bar, 0, sizeof(GridBarrier), st));
    IM_CUDA(cudaMemsetAsync(d_nseeds, 0, sizeof(int32_t), st));
    IM_CUDA(cudaMemsetAsync(d_cov, 0, sizeof(int64_t), st));
    GreedyArgs a;
    a.n = n;
    a.theta = theta;
    a.set_off = p->set_off;
    a.members = p->members;
    a.vtx_off = p->vtx_off;
    a.set_ids = p->set_ids;
    a.k = k;
    a.counts = (int32_t *)(B + o_cnt);
    a.covered = (uint32_t *)(B + o_cov);
    a.block_best = (unsigned long long *)(B + o_best);
    a.bar = (GridBarrier *)(B + o_bar);
    a.seeds = d_seeds;
    a.gains = d_gains;
    a.nseeds = d_nseeds;
    a.coverage = d_cov;
    a.status = d_status;
    void *args[] = {&a};
    KernelTimer kt(st, "greedy");
    IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_greedy, dim3(grid), dim3(kGreedyThreads),
                                        args, 0, st));
    return IM_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

im_status randgreedi(im_pool *p, int32_t k, const im_cover_opts *o, int32_t *d_seeds,
                     int64_t *d_gains, int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st,
                     int *d_status) {
    const int32_t P = o->partitions;
    const int64_t n = p->g->n, theta = p->theta;
    const int64_t words = std::max<int64_t>(1, (theta + 31) / 32);
    const int32_t B = num_buckets(k, o->delta);
    int64_t tr = ((int64_t)k * o->alpha_num + o->alpha_den - 1) / o->alpha_den;
    const int32_t trunc = (int32_t)std::max<int64_t>(1, std::min<int64_t>(k, tr));

    im_status s = build_partition(p, P, o->partition_seed, st);
    if (s != IM_OK) return s;
    // the largest part sizes the producers' shared memory
    std::vector<int32_t> hoff(P + 1);
    IM_CUDA(cudaMemcpyAsync(hoff.data(), p->part_off, (P + 1) * 4, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    int32_t max_np = 0;
    for (int q = 0; q < P; ++q) max_np = std::max(max_np, hoff[q + 1] - hoff[q]);
    const size_t prod_smem = (size_t)std::max(max_np, 1) * 4;
    if (prod_smem > 200 * 1024) {
        set_error("RandGreedi: a vertex part is too large for shared memory; use more partitions");
        return IM_ERR_UNSUPPORTED;
    }

    // result buffers kept in the pool for im_randgreedi_details
    const size_t need = align256((size_t)P * k * 4) + align256((size_t)P * k * 8) +
                        align256((size_t)P * 4) + align256((size_t)P * 8) +
                        align256((size_t)B * 8) * 2 + align256((size_t)B * 4) +
                        align256((size_t)B * k * 4) + align256((size_t)B * k * 8);
    if (p->rg_cap_bytes < need) {
        if (p->rg_block) cudaFree(p->rg_block);
        p->rg_block = nullptr;
        p->rg_cap_bytes = 0;
        IM_CUDA(cudaMalloc(&p->rg_block, need));
        p->rg_cap_bytes = need;
    }
    {
        char *R = (char *)p->rg_block;
        size_t at = 0;
        auto grab = [&](size_t bytes) {
            char *q = R + at;
            at += align256(bytes);
            return q;
        };
        p->rg_local_seeds = (int32_t *)grab((size_t)P * k * 4);
        p->rg_local_gains = (int64_t *)grab((size_t)P * k * 8);
        p->rg_local_n = (int32_t *)grab((size_t)P * 4);
        p->rg_local_cov = (int64_t *)grab((size_t)P * 8);
        p->rg_thr = (int64_t *)grab((size_t)B * 8);
        p->rg_bucket_cov = (int64_t *)grab((size_t)B * 8);
        p->rg_bucket_n = (int32_t *)grab((size_t)B * 4);
        p->rg_bucket_seeds = (int32_t *)grab((size_t)B * k * 4);
        p->rg_bucket_gains = (int64_t *)grab((size_t)B * k * 8);
    }
    p->rg_P = P;
    p->rg_B = B;
    p->rg_k = k;

    // scratch: producer + bucket bitmaps, stream slots, flags, l
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align256(bytes);
        return at;
    };
    const size_t o_cov = take((size_t)P * words * 4);
    const size_t o_bcov = take((size_t)B * words * 4);
    const size_t o_flags = take((size_t)trunc * P * 4);
    const size_t o_elems = take((size_t)trunc * P * 4);
    const size_t o_l = take(8);
    void *base = nullptr;
    s = pool_scratch(p, off, &base);
    if (s != IM_OK) return s;
    char *Bs = (char *)base;
    IM_CUDA(cudaMemsetAsync(Bs + o_flags, 0, (size_t)trunc * P * 4, st));
    // l = max_v |S(v)|: a lower bound on the optimum of the stream, u = k l
    int64_t l = 0;
    {
        s = max_segment_length(p->vtx_off, n, (int64_t *)(Bs + o_l), st);
        if (s != IM_OK) return s;
        IM_CUDA(cudaMemcpyAsync(&l, Bs + o_l, 8, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> thr(B);
    {
        double guess = (double)l;
        for (int32_t b = 0; b < B; ++b) {
            thr[b] = (int64_t)std::ceil(guess / (2.0 * (double)k));
            guess *= 1.0 + o->delta;
        }
    }
    IM_CUDA(cudaMemcpyAsync(p->rg_thr, thr.data(), (size_t)B * 8, cudaMemcpyHostToDevice, st));

    RGArgs a;
    a.n = n;
    a.theta = theta;
    a.words = words;
    a.k = k;
    a.P = P;
    a.trunc = trunc;
    a.B = B;
    a.set_off = p->set_off;
    a.pkeys = p->pkeys;
    a.vtx_off = p->vtx_off;
    a.set_ids = p->set_ids;
    a.part_off = p->part_off;
    a.part_vtx = p->part_vtx;
    a.covered = (uint32_t *)(Bs + o_cov);
    a.bcovered = (uint32_t *)(Bs + o_bcov);
    a.local_seeds = p->rg_local_seeds;
    a.local_gains = p->rg_local_gains;
    a.local_n = p->rg_local_n;
    a.local_cov = p->rg_local_cov;
    a.thr = p->rg_thr;
    a.bucket_cov = p->rg_bucket_cov;
    a.bucket_n = p->rg_bucket_n;
    a.bucket_seeds = p->rg_bucket_seeds;
    a.bucket_gains = p->rg_bucket_gains;
    a.flags = (uint32_t *)(Bs + o_flags);
    a.elems = (int32_t *)(Bs + o_elems);
    a.status = d_status;

    IM_CUDA(cudaFuncSetAttribute(k_randgreedi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)prod_smem));
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_randgreedi, kRGThreads,
                                                          prod_smem));
    if (per_sm < 1) return IM_ERR_UNSUPPORTED;
    const int resident = per_sm * num_sms();
    bool fused = o->fused != 0 && resident >= 2;
    if (fused) {
        a.ncons = std::min<int32_t>(B, resident / 2);
        a.nprod = std::min<int32_t>(P, resident - a.ncons);
        a.first_role = 0;
        void *args[] = {&a};
        KernelTimer kt(st, "randgreedi_fused");
        IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_randgreedi,
                                            dim3(a.nprod + a.ncons), dim3(kRGThreads), args,
                                            prod_smem, st));
    } else {
        // producers alone, then consumers alone (the stream is complete by then)
        a.nprod = std::min<int32_t>(P, resident);
        a.ncons = 0;
        a.first_role = 0;
        {
            KernelTimer kt(st, "randgreedi_local");
            k_randgreedi<<<a.nprod, kRGThreads, prod_smem, st>>>(a);
        }
        IM_CUDA(cudaGetLastError());
        a.ncons = std::min<int32_t>(B, resident);
        a.first_role = 1;
        {
            KernelTimer kt(st, "randgreedi_stream");
            k_randgreedi<<<a.ncons, kRGThreads, prod_smem, st>>>(a);
        }
        IM_CUDA(cudaGetLastError());
    }
    int32_t *d_chosen = (int32_t *)(Bs + o_l);   // l is no longer needed
    {
        KernelTimer kt(st, "randgreedi_final");
        k_rg_final<<<1, 32, 0, st>>>(a, d_seeds, d_gains, d_nseeds, d_cov, d_chosen);
    }
    IM_CUDA(cudaGetLastError());
    int32_t chosen = 0;
    IM_CUDA(cudaMemcpyAsync(&chosen, d_chosen, 4, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    p->rg_chosen = chosen;
    return IM_OK;
}

}  // namespace im

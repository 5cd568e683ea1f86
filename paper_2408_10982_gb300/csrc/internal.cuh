// internal.cuh -- shared device helpers and handle layouts of libim (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/im.h"

namespace im {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with the round constants,
// xor-mixed with the other words and the key, key bumped by the Weyl pair.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a_lo = 0xD2511F53u * x.x, a_hi = __umulhi(0xD2511F53u, x.x);
        const uint32_t b_lo = 0xCD9E8D57u * x.z, b_hi = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(b_hi ^ x.y ^ k0, b_lo, a_hi ^ x.w ^ k1, a_lo);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

// Counter-word-3 domain tags: one independent stream per kind of draw.
constexpr uint32_t kStreamRoot = 1;   // root of sample s: (s, 0, 0)
constexpr uint32_t kStreamCoin = 2;   // IC coins of edges 4g..4g+3: (s, g lo, g hi)
constexpr uint32_t kStreamPick = 3;   // LT in-edge pick of vertex v: (s, v, 0)
constexpr uint32_t kStreamPart = 4;   // partition label of vertex v: (v, 0, 0)

__device__ __forceinline__ uint32_t seed_lo(uint64_t seed) { return (uint32_t)seed; }
__device__ __forceinline__ uint32_t seed_hi(uint64_t seed) { return (uint32_t)(seed >> 32); }

// Uniform pick in [0, N) from a 32-bit draw: floor(r * N / 2^32).
__device__ __forceinline__ uint32_t scale_u32(uint32_t r, uint32_t N) { return __umulhi(r, N); }

__device__ __forceinline__ uint32_t rrr_root(uint64_t seed, uint32_t s, uint32_t n) {
    return scale_u32(philox4x32_10(make_uint4(s, 0u, 0u, kStreamRoot), seed_lo(seed),
                                   seed_hi(seed)).x, n);
}

__device__ __forceinline__ int32_t vertex_part(uint64_t pseed, uint32_t v, uint32_t P) {
    return (int32_t)scale_u32(
        philox4x32_10(make_uint4(v, 0u, 0u, kStreamPart), seed_lo(pseed), seed_hi(pseed)).x, P);
}

// ---------------------------------------------------------------------------
// memory-model helpers and bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Fire-and-forget add to global memory (no value returned).
__device__ __forceinline__ void red_add_s32(int32_t *p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device status codes written to a status word (mapped to im_status on the host).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;
constexpr int kDevQueueOverflow = 2;
constexpr int kDevStageOverflow = 3;
constexpr int kDevBadInput = 4;

__device__ __forceinline__ void raise_status(int *status, int code) { atomicCAS(status, 0, code); }

// Every device spin-wait gives up after this many nanoseconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Software grid barrier for cooperative launches (all blocks co-resident).
// The barrier word is one 64-bit arrival counter, zeroed before the launch and
// never reset: arrival a (counting from 0) belongs to barrier floor(a / nblocks),
// which every block passes once the counter reaches nblocks times its number
// plus one.  A block's arrival is one atomic add after a fence (its writes are
// then visible to every block that passes), its wait a poll of the counter
// with acquire loads.  Returns false (and raises kDevTimeout) if the other
// blocks did not arrive within kWaitLimitNs; callers then leave the kernel,
// and the blocks still waiting give up at their next barrier.
struct GridBarrier {
    unsigned long long count;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, uint32_t nblocks, int *status) {
    __shared__ int ok_flag;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned long long old = atomicAdd(&bar->count, 1ull);
        const unsigned long long target = (old / nblocks + 1ull) * nblocks;
        uint64_t t0 = 0;
        for (uint32_t spin = 0; ld_acquire_u64(&bar->count) < target; ++spin) {
            if ((spin & 31u) == 31u) {       // the clock is read once per 32 polls
                const uint64_t t = global_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > kWaitLimitNs) {
                    raise_status(status, kDevTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        ok_flag = ok;
    }
    __syncthreads();
    return ok_flag != 0;
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sets bit `id` of a bitmap for every lane with id >= 0 (all 32 lanes call
// it) and returns whether the lane's bit was clear before.  Lanes whose bits
// share a word combine them first, so a run of nearby ids -- S(v) lists are
// close to ascending -- costs one atomic per word instead of one per id.
__device__ __forceinline__ bool warp_bitmap_set(uint32_t *bits, int64_t id, int lane) {
    const uint32_t w = id >= 0 ? (uint32_t)(id >> 5) : 0xffffffffu;
    const uint32_t bit = id >= 0 ? 1u << (id & 31) : 0u;
    const unsigned grp = __match_any_sync(kFull, w);
    const uint32_t all = __reduce_or_sync(grp, bit);
    const int leader = __ffs(grp) - 1;
    uint32_t old = 0;
    if (lane == leader && id >= 0) old = atomicOr(bits + w, all);
    old = __shfl_sync(grp, old, leader);
    return id >= 0 && !(old & bit);
}

// The same without the answer (a reduction instead of a returning atomic).
__device__ __forceinline__ void warp_bitmap_or(uint32_t *bits, int64_t id, int lane) {
    const uint32_t w = id >= 0 ? (uint32_t)(id >> 5) : 0xffffffffu;
    const uint32_t bit = id >= 0 ? 1u << (id & 31) : 0u;
    const unsigned grp = __match_any_sync(kFull, w);
    const uint32_t all = __reduce_or_sync(grp, bit);
    if (lane == __ffs(grp) - 1 && id >= 0) atomicOr(bits + w, all);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    return v;
}

}  // namespace im

// What a sampling kernel needs of one query: its graph and random stream.
// A launch reads a table of these; a single-query launch has one entry.
struct QueryView {
    const int64_t *in_off;
    const int32_t *in_src;
    const uint32_t *w;
    const uint4 *lt_vrec;
    const unsigned long long *lt_leaf;
    const unsigned long long *lt_tree;
    const uint4 *lt_guide;
    uint64_t seed;
    uint32_t n;
    uint32_t first;      // sample id of the query's first sample
};

// ---------------------------------------------------------------------------
// handle layouts (host side)
// ---------------------------------------------------------------------------
struct im_graph {
    int device;
    int64_t n, m;
    int64_t *in_off;     // [n+1]
    int32_t *in_src;     // [m]
    uint32_t *w;         // [m], 16-byte aligned
    // LT search index, built on first LT use: per-vertex records, per-edge
    // leaves (running weight sum << 31 | source) and upper tree levels
    uint4 *lt_vrec;                  // [n] {edge offset, in-degree, tree offset | levels << 28, equal in-weight or 0}
    unsigned long long *lt_leaf;     // [m]
    unsigned long long *lt_tree;     // [sum over vertices of the upper-level sizes]
    uint4 *lt_guide;                 // [m] inverse-CDF cut points (see k_lt_guide)
    // out-edge index, built on first im_spread: per source, the in-CSR ids
    // of its out-edges and their heads
    int64_t *out_off;                // [n+1]
    uint4 *out_rec;                  // [m] {head, in-CSR id, weight, LT interval start}
    int32_t lt_valid;
    int64_t max_indeg;
};

struct im_pool {
    const im_graph *g;
    int device;
    int64_t max_sets, max_entries;
    int64_t theta, total, examined;   // host copies, valid after every call
    int64_t sample_bytes;             // algorithmic bytes of all sampling so far
    int64_t *set_off;                 // [max_sets+1]
    int32_t *members;                 // [max_entries]
    // covering subsets
    bool index_valid;
    int64_t *vtx_off;                 // [n+1]
    int32_t *set_ids;                 // [max_entries]; also the sampling stage
    int32_t *vtx_cursor;              // [n] scratch
    // RandGreedi vertex partition (labels, per-part ascending vertex lists)
    int32_t part_P;                   // partition count / seed the lists were built for
    uint64_t part_seed;
    bool part_valid;
    int32_t *part;                    // [n]
    int32_t *part_off;                // [P+1]
    int32_t *part_vtx;                // [n]
    int32_t *part_loc;                // [n]
    int32_t part_cap;                 // allocated P capacity of part_off
    // last RandGreedi results (device)
    int32_t rg_P, rg_B, rg_k, rg_chosen;
    int32_t *rg_local_seeds;          // [P*k]
    int64_t *rg_local_gains;          // [P*k]
    int32_t *rg_local_n;              // [P]
    int64_t *rg_local_cov;            // [P]
    int64_t *rg_thr;                  // [B]
    int64_t *rg_bucket_cov;           // [B]
    int32_t *rg_bucket_n;             // [B]
    int32_t *rg_bucket_seeds;         // [B*k]
    int64_t *rg_bucket_gains;         // [B*k]
    long long *rg_stats;              // [(P+B)*6] diagnostics
    size_t rg_cap_bytes;
    void *rg_block;
    // last lazy greedy: rounds, candidate evaluations, entries scanned, list builds
    long long lz_stats[4];
    // scratch arena (grown on demand) and per-call results
    void *scratch;
    size_t scratch_bytes;
    void *res;
    size_t res_bytes;
};

namespace im {

// error plumbing (api.cu)
void set_error(const std::string &msg);
im_status cuda_fail(cudaError_t e, const char *what);
#define IM_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::im::cuda_fail(_e, #call);  \
    } while (0)
im_status map_dev_status(int code, const char *where);

#define IM_TRY(expr)                   \
    do {                               \
        im_status _s = (expr);         \
        if (_s != IM_OK) return _s;    \
    } while (0)

// Device (or managed) memory, as opposed to host memory.
inline bool is_device_ptr(const void *ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Makes a handle's device current for the scope of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Brackets the kernels launched in its scope with timing events when the
// profiler is on (im_profile_enable); a no-op otherwise.
class KernelTimer {
  public:
    KernelTimer(cudaStream_t st, const char *name);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    cudaStream_t st_;
    const char *name_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    bool on_ = false;
};

// process-wide tuning knobs (im_tune_set); results never depend on them
int64_t tune_value(int32_t knob);
constexpr int32_t kMaxIndexReplicas = 8;   // largest IM_TUNE_INDEX_REPLICAS value

// Device buffers owned by pools (api.cu).  They come from one stream-ordered
// memory pool per device that keeps up to an eighth of the device's memory
// cached after a free, so a pool created after another was destroyed reuses
// its pages instead of mapping new ones (im_trim_memory hands the cache back).
// dev_alloc returns memory usable on any stream (allocations of 0 bytes give
// 16); dev_free waits for the device to go idle before it returns p to the
// cache, and ignores nullptr.  Every field of im_pool that holds device memory
// uses this pair.  Graph buffers (edges, LT index, forward index) stay plain
// cudaMalloc: the LT walk's random gathers from them measured 7% faster there
// than from pool memory, while the index build's random counter atomics ran
// faster on pool memory.
im_status dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
template <typename T>
inline im_status dev_alloc(T **p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

// scratch arena of a pool: returns a pointer to at least `bytes` (256-aligned)
im_status pool_scratch(im_pool *p, size_t bytes, void **out);

int num_sms();

// imm.cu
im_status pool_grow(im_pool *p, int64_t max_sets, int64_t max_entries, cudaStream_t st);

// scan.cu
im_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t count,
                                    const int64_t *base, void *tmp, size_t tmp_bytes,
                                    cudaStream_t st);
size_t scan_tmp_bytes(int64_t count);

// sample.cu
// One sampling launch of one model over a table of queries: query q draws
// counts[q] samples (ids first_q ..) into stage[]; sizes / stage_off are
// indexed by the flattened sample index.  Scratch comes from `alloc`.
struct SamplingJob {
    im_model model;
    std::vector<QueryView> views;
    std::vector<int64_t> counts;
    int64_t n_max;
    int32_t *stage;
    int64_t stage_cap;
};
struct SamplingResult {
    int64_t *stage_off;      // [total]
    int32_t *sizes;          // [total]
    void *scan_tmp;          // scan_tmp_bytes(total) bytes
    void *sort_tmp;          // (2 + 2 total) * 8 bytes
    int64_t total;           // samples
    int64_t added;           // members written to the stage
    int64_t examined;
    int64_t alg_bytes;
};
im_status run_sampling(const SamplingJob &job, const std::function<im_status(size_t, void **)> &alloc,
                       cudaStream_t st, SamplingResult *res);
im_status segmented_sort_sets(int32_t *dst, const int64_t *seg_off, int64_t nseg, const int32_t *stage,
                              const int64_t *stage_off, void *tmp, int64_t n_max, cudaStream_t st);
QueryView query_view(const im_graph *g, uint64_t seed, uint64_t first);
im_status sample_append(const im_graph *g, im_model model, uint64_t seed, uint64_t first,
                        uint64_t count, im_pool *pool, cudaStream_t st);
im_status build_lt_index(im_graph *g, cudaStream_t st);

// index.cu
im_status build_index(im_pool *p, cudaStream_t st);
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it (api.cu).  Launches of one kernel from
// several host threads with different sizes (serving workers) then all stay
// within the limit; setting the attribute to each launch's own size would let
// one thread lower it under another's launch.
im_status raise_dyn_smem(const void *func, size_t bytes);

// covering subsets by a stable radix sort (index.cu): scratch bytes, and the build
size_t radix_index_bytes(int64_t T, int64_t n);
im_status build_index_radix(const int64_t *set_off, const int32_t *members, int64_t theta,
                            int64_t T, int64_t n, int64_t *vtx_off, int32_t *set_ids,
                            int32_t *cnt, void *scratch, cudaStream_t st);
im_status build_index_raw(const int64_t *set_off, const int32_t *members, int64_t theta, int64_t T,
                          int64_t n, int64_t *vtx_off, int32_t *set_ids, int32_t *cursor,
                          int32_t replicas, void *tmp, cudaStream_t st);
im_status build_partition(im_pool *p, int32_t P, uint64_t pseed, cudaStream_t st);
im_status launch_partition_labels(int64_t n, int32_t P, uint64_t pseed, int32_t *part,
                                  cudaStream_t st);
im_status max_segment_length(const int64_t *off, int64_t n, int64_t *d_out, cudaStream_t st);

// cover.cu
int32_t num_buckets(int32_t k, double delta);
im_status greedy_plain(im_pool *p, int32_t k, int32_t *d_seeds, int64_t *d_gains,
                       int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st, int *d_status);
im_status greedy_launch(int64_t n, int64_t theta, const int64_t *set_off, const int32_t *members,
                        const int64_t *vtx_off, const int32_t *set_ids, int32_t k, int32_t *counts,
                        uint32_t *covered, unsigned long long *block_best, int max_grid,
                        void *barrier, int32_t *seeds, int64_t *gains, int32_t *nseeds,
                        int64_t *coverage, int *status, cudaStream_t st);
im_status greedy_launch_view(int64_t n, int64_t theta, const int64_t *set_off,
                             const int32_t *members, const int64_t *vtx_off,
                             const int32_t *set_ids, int64_t sshift, int64_t vshift, int32_t k,
                             int32_t *counts, uint32_t *covered, unsigned long long *block_best,
                             int max_grid, void *barrier, int32_t *seeds, int64_t *gains,
                             int32_t *nseeds, int64_t *coverage, int *status, cudaStream_t st);
// The standard greedy's result on a pool: the lazy kernel (lazy = true, or
// IM_TUNE_GREEDY_EVALS > 0) or the counts-decrement kernel (cover.cu).
im_status greedy_select(im_pool *p, int32_t k, bool lazy, int32_t *d_seeds, int64_t *d_gains,
                        int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st, int *d_status);
// imm.cu: append ids [first, first + count) to a pool, growing it; and one
// SelectSeeds (index build + the cover opts asks for) with its coverage
// read back to the host.
im_status sample_growing(const im_graph *g, im_model model, uint64_t seed, uint64_t first,
                         uint64_t count, im_pool *p, cudaStream_t st);
im_status select_seeds(im_pool *p, int32_t k, const im_cover_opts *o, int32_t *d_seeds,
                       int64_t *d_gains, int32_t *d_ns, int64_t *d_cov, int *d_status,
                       int64_t *coverage, cudaStream_t st);
// lazy greedy (lazy.cu): scratch bytes, and the launch on caller scratch
size_t lazy_greedy_scratch(int64_t n, int64_t theta);
// With cand_seeds, the candidates are the first cand_take seeds of each of
// cand_parts local solutions (RandGreedi's gathered seeds, Alg. 4).
im_status greedy_lazy_launch(int64_t n, int64_t theta, const int64_t *vtx_off,
                             const int32_t *set_ids, int32_t k, int32_t W, void *scratch,
                             int32_t *seeds, int64_t *gains, int32_t *nseeds, int64_t *coverage,
                             long long *stats_out, int *status, cudaStream_t st,
                             const int32_t *cand_seeds = nullptr, const int32_t *cand_n = nullptr,
                             int32_t cand_parts = 0, int32_t cand_take = 0,
                             int32_t cand_stride = 0);
im_status randgreedi(im_pool *p, int32_t k, const im_cover_opts *o, int32_t *d_seeds,
                     int64_t *d_gains, int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st,
                     int *d_status);

}  // namespace im

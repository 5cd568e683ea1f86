// spread.cu -- forward simulation of the diffusion from a seed set (im_spread).
//
// The influence spread sigma(S) (Sec. 2) is the expected number of vertices
// the seeds activate; the paper judges the selected seeds by it (Sec. 4.1).
// Run r simulates the live-edge world of RRR sample r -- the same IC coins
// and LT picks the sampler uses -- forward from S by a BFS
// over out-edges (one block per run, level by level, each warp expanding 32
// queued vertices at a time).
//   IC: in-edge e is live iff lane (e & 3) of Philox(r, e >> 2, e >> 34, coin
//       tag) is below w[e];
//   LT: in-edge e into v is live iff v's pick draw x = Philox(r, v, 0, pick
//       tag).x falls in [sum(e) - w[e], sum(e)), sum(e) being the running
//       in-weight sum of v up to and including e (the LT index's leaves), i.e.
//       iff e is the first in-edge whose running sum exceeds x.
// Because run r and RRR sample r share their world, the run's root is
// activated exactly when S meets RRR set r (the RIS identity).
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace im {

namespace {

constexpr int kSpreadThreads = 512;

// Out-edge index: for every source u, one 16-byte record per out-edge
// {head v, in-CSR id e, w[e], lo(e)} where lo(e) is v's running in-weight sum
// before e (mod 2^32).  An LT draw x of v picks e iff (x - lo(e)) mod 2^32 <
// w[e]: with valid LT weights lo(e) + w[e] <= 2^32, so the difference wraps to
// at least 2^32 - lo(e) >= w[e] whenever x < lo(e).
__global__ void k_out_hist(const int32_t *in_src, int64_t m, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[in_src[e]], 1);
}

__global__ void k_out_fill(const int64_t *in_off, const int32_t *in_src, const uint32_t *w,
                           int64_t n, const int64_t *out_off, int32_t *cursor, uint4 *out_rec) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += nw) {
        const int64_t b = in_off[v], e1 = in_off[v + 1];
        unsigned long long carry = 0;
        for (int64_t base = b; base < e1; base += 32) {
            const int64_t e = base + lane;
            const uint32_t we = e < e1 ? w[e] : 0u;
            const unsigned long long incl = warp_incl_scan<unsigned long long>(we, lane);
            if (e < e1) {
                const int32_t u = in_src[e];
                const int64_t pos = out_off[u] + atomicAdd(&cursor[u], 1);
                out_rec[pos] = make_uint4((uint32_t)v, (uint32_t)e, we,
                                          (uint32_t)(carry + incl - we));
            }
            carry += __shfl_sync(kFull, incl, 31);
        }
    }
}

struct SpreadArgs {
    int64_t n;
    int32_t model;
    uint64_t seed;
    uint64_t first;
    int64_t runs;
    const int32_t *seeds;
    int32_t k;
    const int64_t *out_off;
    const uint4 *out_rec;
    uint32_t *vis;                    // [blocks][words]
    int64_t words;
    int32_t *queues;                  // [blocks][n]
    unsigned long long *work;
    unsigned long long *total;
    int64_t *activated;               // [runs] or null
    uint8_t *root_hit;                // [runs] or null
    int *status;
};

// One run per block: a level-synchronous BFS whose warps take 32 vertices
// of the current level at a time and append the vertices they activate to
// the block's queue (one atomic per warp and step).
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs a) {
    __shared__ unsigned long long s_run;
    __shared__ unsigned long long s_tail, s_cursor;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *vis = a.vis + (int64_t)blockIdx.x * a.words;
    int32_t *q = a.queues + (int64_t)blockIdx.x * a.n;
    const uint32_t k0 = seed_lo(a.seed), k1 = seed_hi(a.seed);
    unsigned long long my_total = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_run = atomicAdd(a.work, 1ull);
            s_tail = 0;
        }
        __syncthreads();
        const unsigned long long i = s_run;
        if (i >= (unsigned long long)a.runs) break;
        const uint32_t s = (uint32_t)(a.first + i);
        // the seeds, each once
        if (warp == 0) {
            for (int32_t b = 0; b < a.k; b += 32) {
                bool fresh = false;
                int32_t u = -1;
                if (b + lane < a.k) {
                    u = a.seeds[b + lane];
                    if (u < 0 || u >= a.n) {
                        raise_status(a.status, kDevBadInput);
                        u = -1;
                    } else {
                        const uint32_t bit = 1u << (u & 31);
                        fresh = !(atomicOr(&vis[u >> 5], bit) & bit);
                    }
                }
                const unsigned fm = __ballot_sync(kFull, fresh);
                if (fresh) q[s_tail + __popc(fm & ((1u << lane) - 1u))] = u;
                __syncwarp();
                if (lane == 0) s_tail += __popc(fm);
                __syncwarp();
            }
        }
        __syncthreads();
        long long head = 0;
        for (;;) {
            const long long lvl_end = (long long)s_tail;
            if (head >= lvl_end) break;
            if (threadIdx.x == 0) s_cursor = (unsigned long long)head;
            __syncthreads();
            for (;;) {
                long long base = 0;
                if (lane == 0) base = (long long)atomicAdd(&s_cursor, 32ull);
                base = __shfl_sync(kFull, base, 0);
                if (base >= lvl_end) break;
                const int nb = (int)(lvl_end - base < 32 ? lvl_end - base : 32);
                int64_t ob = 0, oe = 0;
                if (lane < nb) {
                    const int32_t u = q[base + lane];
                    ob = a.out_off[u];
                    oe = a.out_off[u + 1];
                }
                const int64_t len = oe - ob;
                const int64_t incl = warp_incl_scan<int64_t>(len, lane);
                const int64_t total = __shfl_sync(kFull, incl, 31);
                for (int64_t eb = 0; eb < total; eb += 32) {
                    const int64_t t = eb + lane;
                    int owner = 0;   // first lane whose inclusive count exceeds t
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int64_t c = __shfl_sync(kFull, incl, owner + step - 1);
                        if (c <= t) owner += step;
                    }
                    const int64_t o_incl = __shfl_sync(kFull, incl, owner);
                    const int64_t o_len = __shfl_sync(kFull, len, owner);
                    const int64_t o_ob = __shfl_sync(kFull, ob, owner);
                    bool fresh = false;
                    uint32_t v = 0;
                    if (t < total) {
                        const uint4 r = __ldg(a.out_rec + o_ob + (t - (o_incl - o_len)));
                        v = r.x;
                        if (!((__ldcg(vis + (v >> 5)) >> (v & 31)) & 1u)) {
                            bool live;
                            if (a.model == IM_IC) {
                                const uint32_t e = r.y;   // in-CSR id (< 2^31)
                                const uint4 c = philox4x32_10(
                                    make_uint4(s, e >> 2, 0u, kStreamCoin), k0, k1);
                                const int ln = (int)(e & 3);
                                const uint32_t coin =
                                    ln == 0 ? c.x : ln == 1 ? c.y : ln == 2 ? c.z : c.w;
                                live = coin < r.z;
                            } else {
                                const uint32_t x =
                                    philox4x32_10(make_uint4(s, v, 0u, kStreamPick), k0, k1).x;
                                live = x - r.w < r.z;
                            }
                            if (live) {
                                const uint32_t bit = 1u << (v & 31);
                                fresh = !(atomicOr(&vis[v >> 5], bit) & bit);
                            }
                        }
                    }
                    const unsigned fm = __ballot_sync(kFull, fresh);
                    if (fm) {
                        long long at = 0;
                        if (lane == 0) at = (long long)atomicAdd(&s_tail, (unsigned long long)__popc(fm));
                        at = __shfl_sync(kFull, at, 0);
                        if (fresh) q[at + __popc(fm & ((1u << lane) - 1u))] = (int32_t)v;
                    }
                }
            }
            __syncthreads();
            head = lvl_end;
        }
        const long long tail = (long long)s_tail;
        if (threadIdx.x == 0) {
            const uint32_t root = rrr_root(a.seed, s, (uint32_t)a.n);
            const bool hit = (vis[root >> 5] >> (root & 31)) & 1u;
            if (a.activated) a.activated[i] = tail;
            if (a.root_hit) a.root_hit[i] = hit ? 1 : 0;
            my_total += (unsigned long long)tail;
        }
        __syncthreads();
        // clear this run's visited bits
        if (tail > a.words) {
            for (int64_t x = threadIdx.x; x < a.words; x += blockDim.x) vis[x] = 0u;
        } else {
            for (int64_t x = threadIdx.x; x < tail; x += blockDim.x) vis[q[x] >> 5] = 0u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && my_total) atomicAdd(a.total, my_total);
}

std::mutex g_out_index_mu;   // graphs are shared between threads

im_status build_out_index(im_graph *g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_out_index_mu);
    if (g->out_off) return IM_OK;   // set only once the whole index is built
    const int64_t n = g->n, m = g->m;
    // stream-ordered temporaries, freed on every exit; the index itself is
    // handed to g once complete and freed on any failure
    struct Parts {
        cudaStream_t st;
        int32_t *cnt = nullptr;
        void *scan_tmp = nullptr;
        int64_t *off = nullptr;
        uint4 *rec = nullptr;
        ~Parts() {
            if (off || rec) {
                cudaDeviceSynchronize();
                cudaFree(off);
                cudaFree(rec);
            }
            if (cnt) cudaFreeAsync(cnt, st);
            if (scan_tmp) cudaFreeAsync(scan_tmp, st);
        }
    } t{st};
    IM_CUDA(cudaMallocAsync((void **)&t.cnt, (size_t)n * 4, st));
    IM_CUDA(cudaMallocAsync(&t.scan_tmp, scan_tmp_bytes(n), st));
    IM_CUDA(cudaMalloc(&t.off, (size_t)(n + 1) * 8));
    IM_CUDA(cudaMalloc(&t.rec, (size_t)std::max<int64_t>(m, 1) * sizeof(uint4)));
    IM_CUDA(cudaMemsetAsync(t.cnt, 0, (size_t)n * 4, st));
    {
        KernelTimer kt(st, "out_index");
        if (m > 0) k_out_hist<<<num_sms() * 4, 256, 0, st>>>(g->in_src, m, t.cnt);
    }
    IM_CUDA(cudaGetLastError());
    IM_TRY(exclusive_scan_i32_to_i64(t.cnt, t.off, n, nullptr, t.scan_tmp, scan_tmp_bytes(n), st));
    IM_CUDA(cudaMemsetAsync(t.cnt, 0, (size_t)n * 4, st));
    {
        KernelTimer kt(st, "out_index");
        if (m > 0)
            k_out_fill<<<num_sms() * 8, 256, 0, st>>>(g->in_off, g->in_src, g->w, n, t.off,
                                                      t.cnt, t.rec);
    }
    IM_CUDA(cudaGetLastError());
    IM_CUDA(cudaStreamSynchronize(st));
    g->out_rec = t.rec;
    g->out_off = t.off;
    t.off = nullptr;
    t.rec = nullptr;
    return IM_OK;
}

}  // namespace

}  // namespace im

using namespace im;

extern "C" im_status im_spread(const im_graph *gc, im_model model, const int32_t *seeds, int32_t k,
                               uint64_t seed, uint64_t first_run, uint64_t runs, int64_t *activated,
                               uint8_t *root_hit, int64_t *total, void *stream) {
    if (!gc || k < 0 || (k > 0 && !seeds) || (model != IM_IC && model != IM_LT) ||
        first_run + runs > (1ull << 32) || runs > (1ull << 32)) {
        set_error("im_spread: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    im_graph *g = const_cast<im_graph *>(gc);
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    if (model == IM_LT) {
        IM_TRY(build_lt_index(g, st));
        if (!g->lt_valid) {
            set_error("im_spread: LT needs every vertex's in-weights to sum to at most 2^32");
            return IM_ERR_INVALID_ARG;
        }
    }
    IM_TRY(build_out_index(g, st));
    if (total) *total = 0;
    if (runs == 0) return IM_OK;
    const int64_t n = g->n, words = (n + 31) / 32;
    // blocks (one run each at a time): occupancy-sized, and the per-block
    // queue (n entries) and bitmap within about 2 GB
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread, kSpreadThreads, 0));
    const int64_t per_block = (int64_t)n * 4 + words * 4;
    int64_t blocks = std::max(1, per_sm) * (int64_t)num_sms();
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(1, (2ll << 30) / per_block));
    blocks = std::min<int64_t>(blocks, (int64_t)runs);
    const int64_t warps = blocks;   // one visited bitmap and queue per block
    const bool host_act = activated && !is_device_ptr(activated);
    const bool host_hit = root_hit && !is_device_ptr(root_hit);
    const bool host_seeds = k > 0 && !is_device_ptr(seeds);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t o_ctr = take(4 * 8), o_seeds = take((size_t)std::max(k, 1) * 4),
                 o_vis = take((size_t)warps * words * 4), o_q = take((size_t)warps * n * 4),
                 o_act = take(host_act ? (size_t)runs * 8 : 0),
                 o_hit = take(host_hit ? (size_t)runs : 0);
    char *B = nullptr;
    IM_CUDA(cudaMallocAsync((void **)&B, off, st));
    IM_CUDA(cudaMemsetAsync(B + o_ctr, 0, 4 * 8, st));
    IM_CUDA(cudaMemsetAsync(B + o_vis, 0, (size_t)warps * words * 4, st));
    if (k > 0) IM_CUDA(cudaMemcpyAsync(B + o_seeds, seeds, (size_t)k * 4, cudaMemcpyDefault, st));
    SpreadArgs a;
    a.n = n;
    a.model = model;
    a.seed = seed;
    a.first = first_run;
    a.runs = (int64_t)runs;
    a.seeds = (const int32_t *)(B + o_seeds);
    a.k = k;
    a.out_off = g->out_off;
    a.out_rec = g->out_rec;
    a.vis = (uint32_t *)(B + o_vis);
    a.words = words;
    a.queues = (int32_t *)(B + o_q);
    unsigned long long *ctr = (unsigned long long *)(B + o_ctr);
    a.work = ctr;
    a.total = ctr + 1;
    a.status = (int *)(ctr + 2);
    a.activated = host_act ? (int64_t *)(B + o_act) : activated;
    a.root_hit = host_hit ? (uint8_t *)(B + o_hit) : root_hit;
    {
        KernelTimer kt(st, model == IM_LT ? "spread_lt" : "spread_ic");
        k_spread<<<(unsigned)blocks, kSpreadThreads, 0, st>>>(a);
    }
    IM_CUDA(cudaGetLastError());
    unsigned long long hc[3] = {0, 0, 0};
    IM_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    if (host_act) IM_CUDA(cudaMemcpyAsync(activated, B + o_act, (size_t)runs * 8, cudaMemcpyDeviceToHost, st));
    if (host_hit) IM_CUDA(cudaMemcpyAsync(root_hit, B + o_hit, (size_t)runs, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaFreeAsync(B, st));
    IM_CUDA(cudaStreamSynchronize(st));
    (void)host_seeds;
    const int dev_status = (int)(hc[2] & 0xffffffffu);
    if (dev_status != kDevOk) {
        if (dev_status == kDevBadInput) {
            set_error("im_spread: a seed id is outside [0, n)");
            return IM_ERR_INVALID_ARG;
        }
        return map_dev_status(dev_status, "im_spread");
    }
    if (total) *total = (int64_t)hc[1];
    return IM_OK;
}

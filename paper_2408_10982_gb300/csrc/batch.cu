// batch.cu -- many independent IM queries solved together (im_solve_batch).
//
// Queries may differ in graph, model, k and theta.  The batch runs in a fixed
// number of launches whatever the number of queries:
//   1. one sampling launch per model over the flattened samples of all its
//      queries (each sample finds its query and that query's graph, see
//      run_sampling in sample.cu);
//   2. one scan and one segmented sort over all sets;
//   3. members are moved into one vertex space (query q's vertex u becomes
//      vbase[q] + u) so that one histogram / scan / scatter builds the covering
//      subsets of every query at once;
//   4. one greedy launch, one block per query, running the lazy greedy of
//      Alg. 2 with exact tie handling -- the standard greedy's result -- over
//      a tournament: stale gains of the query's vertices in global memory,
//      the maximum of every 1024-vertex chunk in shared memory.
// Each query's result equals what it gets alone (the random stream of a
// sample depends only on the query's seed and the sample id).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "internal.cuh"

struct im_batch {
    int device = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    void *sscratch = nullptr;  // sampling scratch
    size_t sscratch_bytes = 0;
    // members per set to reserve, per graph and model: twice the most seen in
    // earlier batches (64 before any), four times more after a capacity miss
    std::map<std::pair<const im_graph *, int32_t>, int64_t> entry_hint;
    // RandGreedi queries: a pool view per graph (its partition and RandGreedi
    // buffers are owned, the index is the batch's), and the partition count
    // picked for each (graph, model, power-of-two theta)
    std::map<const im_graph *, im_pool *> views;
    std::map<std::tuple<const im_graph *, int32_t, int32_t>, int32_t> rg_parts;
};

namespace im {
namespace {

constexpr int kBGThreads = 1024;
constexpr int kChunkV = 1024;      // vertices per tournament chunk

struct BatchQuery {
    int64_t vbase;     // first vertex of the query in the batch vertex space
    int64_t n;
    int64_t sbase;     // first set of the query in the batch
    int64_t theta;
    int64_t cbase;     // first word of the query's covered bitmap
    int64_t out;       // row of the query in the seeds output (original index)
    int32_t k;
    int32_t pad;       // 1: the query runs the grid-wide greedy, not a block
};

// First member position of every query's sets: out[i] = set_off[qset[i]].
__global__ void k_query_bounds(const int64_t *set_off, const int64_t *qset, int32_t nq,
                               int64_t *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nq; i += gridDim.x * blockDim.x)
        out[i] = set_off[qset[i]];
}

// A RandGreedi query reads its covering subsets with its own set ids: the
// batch ids of its entries [vtx_off[0], vtx_off[n]) lose the query's first set.
__global__ void k_localize(int32_t *set_ids, const int64_t *vtx_off, int64_t n, int64_t sbase) {
    const int64_t b = vtx_off[0], e = vtx_off[n];
    for (int64_t t = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < e;
         t += (int64_t)gridDim.x * blockDim.x)
        set_ids[t] -= (int32_t)sbase;
}

__global__ void k_globalize(const int64_t *set_off, int32_t *members, int64_t nsets,
                            const int64_t *qset, const int64_t *vbase, int32_t nq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsets;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (qset[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int32_t vb = (int32_t)vbase[lo];
        for (int64_t t = set_off[i]; t < set_off[i + 1]; ++t) members[t] += vb;
    }
}

__device__ __forceinline__ unsigned long long bmax(unsigned long long v, unsigned long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(kFull, x, o);
            x = t > x ? t : x;
        }
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    const unsigned long long r = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ long long bsum(long long v, long long *sh) {
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

__device__ __forceinline__ unsigned long long pack(int32_t gain, int64_t l) {
    return gain > 0 ? (((unsigned long long)(uint32_t)gain << 32) | (0xffffffffu - (uint32_t)l)) : 0ull;
}

// Lazy greedy of one query per block.  key[v] is v's marginal gain, exact
// when stamp[v] equals the current round and an upper bound otherwise; cm[c]
// is the packed maximum of chunk c.  A fresh winner is the standard greedy's
// pick (ties to the smallest id); a stale one is re-evaluated.
__global__ void __launch_bounds__(kBGThreads) k_batch_greedy(
    const BatchQuery *bq, int32_t nq, const int64_t *vtx_off, const int32_t *set_ids, int32_t *key,
    int32_t *stamp, uint32_t *covered, int32_t *seeds, int64_t *gains, int32_t kmax,
    int32_t *nseeds, int64_t *coverage) {
    extern __shared__ unsigned long long cm[];
    __shared__ unsigned long long shm[33];
    __shared__ long long shs[33];
    for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const BatchQuery Q = bq[qi];
        if (Q.pad) continue;                 // run by the grid-wide greedy instead
        const int64_t nch = (Q.n + kChunkV - 1) / kChunkV;
        int32_t *kq = key + Q.vbase;
        int32_t *sq = stamp + Q.vbase;
        uint32_t *cov = covered + Q.cbase;
        const int64_t words = (Q.theta + 31) / 32;
        for (int64_t x = threadIdx.x; x < words; x += blockDim.x) cov[x] = 0u;
        for (int64_t v = threadIdx.x; v < Q.n; v += blockDim.x) {
            const int64_t gv = Q.vbase + v;
            kq[v] = (int32_t)(vtx_off[gv + 1] - vtx_off[gv]);   // exact: nothing covered yet
            sq[v] = 0;
        }
        __syncthreads();
        // chunk maxima: one warp per chunk
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int64_t c = warp; c < nch; c += blockDim.x >> 5) {
                unsigned long long m = 0;
                for (int64_t l = c * kChunkV + lane; l < min(Q.n, (c + 1) * kChunkV); l += 32) {
                    const unsigned long long p = pack(kq[l], l);
                    m = p > m ? p : m;
                }
                m = warp_max_u64(m);
                if (lane == 0) cm[c] = m;
            }
        }
        __syncthreads();
        int32_t j = 0;
        int64_t total = 0;
        while (j < Q.k) {
            unsigned long long best = 0;
            for (int64_t c = threadIdx.x; c < nch; c += blockDim.x) best = cm[c] > best ? cm[c] : best;
            best = bmax(best, shm);
            if (best == 0) break;                                   // every gain is zero
            const int64_t l = (int64_t)(0xffffffffu - (uint32_t)(best & 0xffffffffu));
            const int64_t gv = Q.vbase + l;
            const int64_t sb = vtx_off[gv], se = vtx_off[gv + 1];
            if (sq[l] != j) {
                long long miss = 0;
                for (int64_t t = sb + threadIdx.x; t < se; t += blockDim.x) {
                    const int64_t i = (int64_t)set_ids[t] - Q.sbase;
                    miss += !((cov[i >> 5] >> (i & 31)) & 1u);
                }
                const long long g = bsum(miss, shs);
                if (threadIdx.x == 0) {
                    kq[l] = (int32_t)g;
                    sq[l] = j;
                }
            } else {
                const int64_t gain = (int64_t)(best >> 32);
                if (threadIdx.x == 0) {
                    seeds[Q.out * kmax + j] = (int32_t)l;
                    gains[Q.out * kmax + j] = gain;
                    kq[l] = 0;
                }
                for (int64_t t = sb + threadIdx.x; t < se; t += blockDim.x) {
                    const int64_t i = (int64_t)set_ids[t] - Q.sbase;
                    atomicOr(&cov[i >> 5], 1u << (i & 31));
                }
                total += gain;
                ++j;
            }
            __syncthreads();
            // refresh the maximum of l's chunk
            const int64_t c = l / kChunkV;
            const int64_t v = c * kChunkV + threadIdx.x;
            const unsigned long long p = v < Q.n ? pack(kq[v], v) : 0ull;
            const unsigned long long m = bmax(p, shm);
            if (threadIdx.x == 0) cm[c] = m;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            nseeds[Q.out] = j;
            coverage[Q.out] = total;
        }
        __syncthreads();
    }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

im_status grow(void **p, size_t *have, size_t need) {
    if (need <= *have) return IM_OK;
    if (*p) {
        IM_CUDA(cudaDeviceSynchronize());
        cudaFree(*p);
        *p = nullptr;
        *have = 0;
    }
    const size_t want = need + need / 4 + 4096;
    if (cudaMalloc(p, want) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("im_solve_batch: device memory exhausted");
        return IM_ERR_OOM;
    }
    *have = want;
    return IM_OK;
}

// A pool that borrows a batch's covering subsets for one query at a time:
// theta, vtx_off and set_ids are set per query; the partition, RandGreedi and
// scratch buffers are its own, kept between queries on the same graph.
im_pool *make_pool_view(const im_graph *g, int device) {
    im_pool *v = new (std::nothrow) im_pool();
    if (!v) return nullptr;
    std::memset(v, 0, sizeof(*v));
    v->g = g;
    v->device = device;
    return v;
}

void release_pool_view(im_pool *v) {
    if (!v) return;
    for (void *b : {(void *)v->vtx_cursor, (void *)v->part, (void *)v->part_off,
                    (void *)v->part_vtx, (void *)v->part_loc, (void *)v->rg_block, v->scratch,
                    v->res})
        dev_free(b);
    delete v;
}

// The partition counts a RandGreedi query may use: powers of two from 16 and
// the SM count, each part small enough for one producer block.
std::vector<int32_t> partition_candidates(int64_t n) {
    std::vector<int32_t> c;
    for (int32_t P = 16; P < num_sms(); P *= 2) c.push_back(P);
    c.push_back(num_sms());
    std::vector<int32_t> ok;
    for (int32_t P : c)
        if (P <= n && (n + P - 1) / P <= 16384) ok.push_back(P);
    if (ok.empty()) ok.push_back((int32_t)std::min<int64_t>(n, std::max<int64_t>(1, (n + 16383) / 16384)));
    return ok;
}

}  // namespace
}  // namespace im

using namespace im;

extern "C" {

im_status im_batch_create(im_batch **out) {
    if (!out) return IM_ERR_INVALID_ARG;
    im_batch *b = new (std::nothrow) im_batch();
    if (!b) return IM_ERR_OOM;
    cudaGetDevice(&b->device);
    *out = b;
    return IM_OK;
}

im_status im_batch_destroy(im_batch *b) {
    if (!b) return IM_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    for (auto &kv : b->views) release_pool_view(kv.second);
    cudaFree(b->arena);
    cudaFree(b->sscratch);
    delete b;
    return IM_OK;
}

im_status im_solve_batch(im_batch *b, const im_query *qs, int32_t nq, int32_t kmax, int32_t *seeds,
                         int64_t *gains, im_result *res, void *stream) {
    if (!b || !qs || nq < 1 || kmax < 1 || !seeds || !res) {
        set_error("im_solve_batch: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // validate; LT queries need their graph's LT index
    int64_t n_total = 0, sets_total = 0, n_max = 1;
    for (int32_t q = 0; q < nq; ++q) {
        const im_query &Q = qs[q];
        if (!Q.graph || (Q.model != IM_IC && Q.model != IM_LT) || Q.k < 1 || Q.k > kmax ||
            Q.k > Q.graph->n || Q.theta < 0 || Q.theta >= ((int64_t)1 << 31) ||
            Q.graph->device != b->device) {
            set_error("im_solve_batch: query out of range");
            return IM_ERR_INVALID_ARG;
        }
        const im_cover_opts &o = Q.cover;
        if (o.algo == IM_RANDGREEDI) {
            if (o.partitions < 0 || o.partitions > 4096 || o.partitions > Q.graph->n ||
                o.alpha_num < 1 || o.alpha_den < 1 || o.alpha_num > o.alpha_den ||
                !(o.delta > 0.0 && o.delta < 0.5) ||
                (o.aggregator != IM_AGG_STREAM && o.aggregator != IM_AGG_GREEDY)) {
                set_error("im_solve_batch: RandGreedi options out of range");
                return IM_ERR_INVALID_ARG;
            }
        } else if (o.algo != IM_GREEDY_PLAIN && o.algo != IM_GREEDY_LAZY) {
            set_error("im_solve_batch: unknown algorithm");
            return IM_ERR_INVALID_ARG;
        }
        if (Q.model == IM_LT) {
            im_status s = build_lt_index(const_cast<im_graph *>(Q.graph), st);
            if (s != IM_OK) return s;
            if (!Q.graph->lt_valid) {
                set_error("im_solve_batch: LT query on a graph whose in-weights exceed 1");
                return IM_ERR_INVALID_ARG;
            }
        }
        n_total += Q.graph->n;
        sets_total += Q.theta;
        n_max = std::max<int64_t>(n_max, Q.graph->n);
    }
    if (n_total >= ((int64_t)1 << 31)) {
        set_error("im_solve_batch: the batch's vertices exceed 2^31");
        return IM_ERR_CAPACITY;
    }
    // batch order: IC queries, then LT queries (one sampling launch each)
    std::vector<int32_t> order(nq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_partition(order.begin(), order.end(), [&](int32_t q) { return qs[q].model == IM_IC; });
    std::vector<BatchQuery> bq(nq);
    std::vector<int64_t> qset(nq + 1, 0), vbase(nq, 0);
    int64_t vb = 0, sb = 0, cb = 0;
    for (int32_t i = 0; i < nq; ++i) {
        const im_query &Q = qs[order[i]];
        bq[i].vbase = vb;
        bq[i].n = Q.graph->n;
        bq[i].sbase = sb;
        bq[i].theta = Q.theta;
        bq[i].cbase = cb;
        bq[i].out = order[i];
        bq[i].k = Q.k;
        bq[i].pad = 0;
        vbase[i] = vb;
        qset[i] = sb;
        vb += Q.graph->n;
        sb += Q.theta;
        cb += (Q.theta + 31) / 32;
    }
    qset[nq] = sb;
    const int64_t cov_words = std::max<int64_t>(cb, 1);

    for (int attempt = 0; attempt < 8; ++attempt) {
        int64_t cap = 1024;
        for (int32_t q = 0; q < nq; ++q) {
            auto it = b->entry_hint.find({qs[q].graph, qs[q].model});
            cap += qs[q].theta * (it == b->entry_hint.end() ? 64 : it->second);
        }
        // arena layout
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t at = off;
            off += up256(bytes);
            return at;
        };
        const size_t o_stage = take((size_t)cap * 4), o_mem = take((size_t)cap * 4),
                     o_sids = take((size_t)cap * 4), o_soff = take((size_t)(sets_total + 1) * 8),
                     o_sizes = take((size_t)std::max<int64_t>(sets_total, 1) * 4),
                     o_stoff = take((size_t)std::max<int64_t>(sets_total, 1) * 8),
                     o_voff = take((size_t)(n_total + 1) * 8), o_cur = take((size_t)n_total * 4),
                     o_key = take((size_t)n_total * 4), o_stamp = take((size_t)n_total * 4),
                     o_cov = take((size_t)cov_words * 4), o_bq = take((size_t)nq * sizeof(BatchQuery)),
                     o_qset = take((size_t)(nq + 1) * 8), o_vbase = take((size_t)nq * 8),
                     o_tmp = take(std::max(scan_tmp_bytes(std::max(sets_total, n_total)),
                                           (size_t)(2 + 2 * std::max<int64_t>(sets_total, 1)) * 8)),
                     o_out = take(up256((size_t)nq * kmax * 4) + up256((size_t)nq * kmax * 8) +
                                  up256((size_t)nq * 4) + up256((size_t)nq * 8)),
                     o_bounds = take((size_t)(nq + 1) * 8),
                     o_best = take((size_t)num_sms() * 8 * 8), o_gbar = take(256);
        im_status s = grow(&b->arena, &b->arena_bytes, off);
        if (s != IM_OK) return s;
        char *A = (char *)b->arena;
        int32_t *stage = (int32_t *)(A + o_stage);
        int64_t *set_off = (int64_t *)(A + o_soff);
        int32_t *sizes = (int32_t *)(A + o_sizes);
        int64_t *stage_off = (int64_t *)(A + o_stoff);

        // 1. sampling: one launch per model
        int64_t added = 0, examined = 0;
        bool capacity = false;
        int64_t done_sets = 0;
        for (int mi = 0; mi < 2 && !capacity; ++mi) {
            const im_model model = mi == 0 ? IM_IC : IM_LT;
            SamplingJob job;
            job.model = model;
            job.n_max = 1;
            for (int32_t i = 0; i < nq; ++i) {
                const im_query &Q = qs[order[i]];
                if (Q.model != model) continue;
                job.views.push_back(query_view(Q.graph, Q.seed, 0));
                job.counts.push_back(Q.theta);
                job.n_max = std::max<int64_t>(job.n_max, Q.graph->n);
            }
            if (job.views.empty()) continue;
            int64_t nsets = 0;
            for (int64_t c : job.counts) nsets += c;
            job.stage = stage + added;
            job.stage_cap = cap - added;
            SamplingResult r;
            s = run_sampling(job,
                             [&](size_t bytes, void **p) {
                                 im_status g2 = grow(&b->sscratch, &b->sscratch_bytes, bytes);
                                 *p = b->sscratch;
                                 return g2;
                             },
                             st, &r);
            if (s == IM_ERR_CAPACITY) {
                capacity = true;
                break;
            }
            if (s != IM_OK) return s;
            // gather sizes and stage offsets (relative to `stage`) in batch order
            IM_CUDA(cudaMemcpyAsync(sizes + done_sets, r.sizes, (size_t)nsets * 4,
                                    cudaMemcpyDeviceToDevice, st));
            if (added == 0) {
                IM_CUDA(cudaMemcpyAsync(stage_off + done_sets, r.stage_off, (size_t)nsets * 8,
                                        cudaMemcpyDeviceToDevice, st));
            } else {
                // offsets of the second launch are relative to stage + added: shift them
                std::vector<int64_t> h(nsets);
                IM_CUDA(cudaMemcpyAsync(h.data(), r.stage_off, (size_t)nsets * 8,
                                        cudaMemcpyDeviceToHost, st));
                IM_CUDA(cudaStreamSynchronize(st));
                for (auto &x : h) x += added;
                IM_CUDA(cudaMemcpyAsync(stage_off + done_sets, h.data(), (size_t)nsets * 8,
                                        cudaMemcpyHostToDevice, st));
                IM_CUDA(cudaStreamSynchronize(st));
            }
            done_sets += nsets;
            added += r.added;
            examined += r.examined;
        }
        if (capacity) {
            std::map<std::pair<const im_graph *, int32_t>, bool> seen;
            for (int32_t q = 0; q < nq; ++q) {
                const auto key = std::make_pair(qs[q].graph, (int32_t)qs[q].model);
                if (seen[key]) continue;                 // once per graph and model
                seen[key] = true;
                auto &h = b->entry_hint[key];
                h = std::max<int64_t>(h, 64) * 4;
            }
            continue;
        }
        IM_CUDA(cudaStreamSynchronize(st));


        // 2. set offsets and sorted members
        void *tmp = A + o_tmp;
        s = exclusive_scan_i32_to_i64(sizes, set_off, sets_total, nullptr, tmp,
                                      scan_tmp_bytes(sets_total), st);
        if (s != IM_OK) return s;
        int32_t *members = (int32_t *)(A + o_mem);
        s = segmented_sort_sets(members, set_off, sets_total, stage, stage_off, tmp, n_max, st);
        if (s != IM_OK) return s;
        // 3. one vertex space, one index
        IM_CUDA(cudaMemcpyAsync(A + o_bq, bq.data(), (size_t)nq * sizeof(BatchQuery),
                                cudaMemcpyHostToDevice, st));
        IM_CUDA(cudaMemcpyAsync(A + o_qset, qset.data(), (size_t)(nq + 1) * 8, cudaMemcpyHostToDevice, st));
        IM_CUDA(cudaMemcpyAsync(A + o_vbase, vbase.data(), (size_t)nq * 8, cudaMemcpyHostToDevice, st));
        if (sets_total > 0) {
            KernelTimer kt(st, "batch_globalize");
            k_globalize<<<num_sms() * 4, 256, 0, st>>>(set_off, members, sets_total,
                                                       (const int64_t *)(A + o_qset),
                                                       (const int64_t *)(A + o_vbase), nq);
        }
        IM_CUDA(cudaGetLastError());
        int64_t *vtx_off = (int64_t *)(A + o_voff);
        int32_t *set_ids = (int32_t *)(A + o_sids);
        s = build_index_raw(set_off, members, sets_total, added, n_total, vtx_off, set_ids,
                            (int32_t *)(A + o_cur), 1, tmp, st);
        if (s != IM_OK) return s;
        // 4. seed selection.  A block-per-query lazy greedy suits many small
        // queries; a query holding a large share of the batch's members would
        // keep one SM busy long after the rest finish, so those run the
        // grid-wide greedy, one cooperative launch each.  Cost model (rates
        // measured on GB300 at the batched mix): a block scans ~0.36 G
        // entries/s, the grid greedy ~17 G entries/s over a ~0.8 ms floor of
        // k barrier-bound steps; the largest queries are moved to the grid
        // while that lowers max(block phase) + sum(grid launches).
        int32_t *d_seeds = (int32_t *)(A + o_out);
        int64_t *d_gains = (int64_t *)(A + o_out + up256((size_t)nq * kmax * 4));
        int32_t *d_ns = (int32_t *)((char *)d_gains + up256((size_t)nq * kmax * 8));
        int64_t *d_cov = (int64_t *)((char *)d_ns + up256((size_t)nq * 4));
        int64_t *d_bounds = (int64_t *)(A + o_bounds);
        {
            KernelTimer kt(st, "batch_bounds");
            k_query_bounds<<<std::max(1, std::min(num_sms(), (nq + 256) / 256)), 256, 0, st>>>(
                set_off, (const int64_t *)(A + o_qset), nq, d_bounds);
        }
        IM_CUDA(cudaGetLastError());
        std::vector<int64_t> hb(nq + 1);
        IM_CUDA(cudaMemcpyAsync(hb.data(), d_bounds, (size_t)(nq + 1) * 8, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        // RandGreedi queries (pad 2) run after the greedy launches, one by one
        std::vector<int32_t> by_size;
        for (int32_t i = 0; i < nq; ++i)
            if (qs[order[i]].cover.algo != IM_RANDGREEDI) by_size.push_back(i);
        const int32_t ng = (int32_t)by_size.size();
        std::sort(by_size.begin(), by_size.end(), [&](int32_t x, int32_t y) {
            return hb[x + 1] - hb[x] > hb[y + 1] - hb[y];
        });
        const double rb = 0.36e9, rg = 17e9, t0 = 0.8e-3;
        const double slots = 2.0 * num_sms();
        double rest = 0.0, grid_t = 0.0;
        for (int32_t x : by_size) rest += (double)(hb[x + 1] - hb[x]);
        double best_t = std::max((ng ? (double)(hb[by_size[0] + 1] - hb[by_size[0]]) : 0.0) / rb,
                                 rest / (rb * slots));
        int32_t n_grid = 0;
        for (int32_t r = 0; r < ng; ++r) {
            const double w = (double)(hb[by_size[r] + 1] - hb[by_size[r]]);
            grid_t += t0 + w / rg;
            rest -= w;
            const double next = r + 1 < ng ? (double)(hb[by_size[r + 1] + 1] - hb[by_size[r + 1]]) : 0.0;
            const double t = grid_t + std::max(next / rb, rest / (rb * slots));
            if (t < best_t) {
                best_t = t;
                n_grid = r + 1;
            }
        }
        for (int32_t i = 0; i < nq; ++i) bq[i].pad = 2;
        for (int32_t r = 0; r < ng; ++r) bq[by_size[r]].pad = r < n_grid ? 1 : 0;
        IM_CUDA(cudaMemcpyAsync(A + o_bq, bq.data(), (size_t)nq * sizeof(BatchQuery),
                                cudaMemcpyHostToDevice, st));
        int64_t max_nch = 1;
        for (auto &x : bq) max_nch = std::max<int64_t>(max_nch, (x.n + kChunkV - 1) / kChunkV);
        const size_t smem = (size_t)max_nch * 8;
        if (smem > 200 * 1024) {
            set_error("im_solve_batch: a query graph is too large for the batched greedy");
            return IM_ERR_UNSUPPORTED;
        }
        IM_TRY(raise_dyn_smem((const void *)k_batch_greedy, smem));
        if (n_grid < ng) {
            KernelTimer kt(st, "batch_greedy");
            k_batch_greedy<<<(unsigned)std::min<int64_t>(nq, (int64_t)num_sms() * 2), kBGThreads, smem,
                             st>>>((const BatchQuery *)(A + o_bq), nq, vtx_off, set_ids,
                                   (int32_t *)(A + o_key), (int32_t *)(A + o_stamp),
                                   (uint32_t *)(A + o_cov), d_seeds, d_gains, kmax, d_ns, d_cov);
        }
        IM_CUDA(cudaGetLastError());
        int *d_gstatus = (int *)(A + o_gbar + sizeof(GridBarrier) + 64);
        IM_CUDA(cudaMemsetAsync(d_gstatus, 0, sizeof(int), st));
        for (int32_t r = 0; r < n_grid; ++r) {
            const BatchQuery &Q = bq[by_size[r]];
            IM_CUDA(cudaMemsetAsync(A + o_gbar, 0, sizeof(GridBarrier), st));
            s = greedy_launch_view(Q.n, Q.theta, set_off, members, vtx_off + Q.vbase, set_ids,
                                   Q.sbase, Q.vbase, Q.k, (int32_t *)(A + o_key) + Q.vbase,
                                   (uint32_t *)(A + o_cov) + Q.cbase,
                                   (unsigned long long *)(A + o_best), num_sms() * 8,
                                   A + o_gbar, d_seeds + Q.out * kmax, d_gains + Q.out * kmax,
                                   d_ns + Q.out, d_cov + Q.out, d_gstatus, st);
            if (s != IM_OK) return s;
        }
        // RandGreedi queries: each on a view of the batch's index, with its own
        // set ids; the partition count picked by timing when the query leaves it open
        std::vector<int32_t> parts_used(nq, 0);
        for (int32_t i = 0; i < nq; ++i) {
            const BatchQuery &Q = bq[i];
            if (Q.pad != 2) continue;
            const im_query &q = qs[order[i]];
            {
                KernelTimer kt(st, "batch_localize");
                k_localize<<<num_sms() * 4, 256, 0, st>>>(set_ids, vtx_off + Q.vbase, Q.n, Q.sbase);
            }
            IM_CUDA(cudaGetLastError());
            im_pool *&view = b->views[q.graph];
            if (!view) view = make_pool_view(q.graph, b->device);
            if (!view) return IM_ERR_OOM;
            view->theta = Q.theta;
            view->total = hb[i + 1] - hb[i];
            view->vtx_off = vtx_off + Q.vbase;
            view->set_ids = set_ids;
            view->index_valid = true;
            im_cover_opts o = q.cover;
            o.fused = 0;
            if (o.partitions == 0) {
                int32_t lg = 0;
                while (((int64_t)1 << (lg + 1)) <= Q.theta) ++lg;
                const auto key = std::make_tuple(q.graph, (int32_t)q.model, lg);
                auto it = b->rg_parts.find(key);
                if (it == b->rg_parts.end()) {
                    // time every candidate count (second of two runs) and keep the fastest
                    cudaEvent_t e0, e1;
                    IM_CUDA(cudaEventCreate(&e0));
                    IM_CUDA(cudaEventCreate(&e1));
                    float best = 0.f;
                    int32_t bestP = 0;
                    for (int32_t P : partition_candidates(Q.n)) {
                        o.partitions = P;
                        float ms = 0.f;
                        for (int rep = 0; rep < 2 && s == IM_OK; ++rep) {
                            cudaEventRecord(e0, st);
                            s = randgreedi(view, Q.k, &o, d_seeds + Q.out * kmax,
                                           d_gains + Q.out * kmax, d_ns + Q.out, d_cov + Q.out, st,
                                           d_gstatus);
                            cudaEventRecord(e1, st);
                            cudaEventSynchronize(e1);
                            cudaEventElapsedTime(&ms, e0, e1);
                        }
                        if (s != IM_OK) break;
                        if (bestP == 0 || ms < best) {
                            best = ms;
                            bestP = P;
                        }
                    }
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    if (s != IM_OK) return s;
                    it = b->rg_parts.emplace(key, bestP).first;
                }
                o.partitions = it->second;
            }
            s = randgreedi(view, Q.k, &o, d_seeds + Q.out * kmax, d_gains + Q.out * kmax,
                           d_ns + Q.out, d_cov + Q.out, st, d_gstatus);
            if (s != IM_OK) return s;
            parts_used[i] = o.partitions;
        }
        // 5. results
        std::vector<int32_t> hns(nq);
        std::vector<int64_t> hcov(nq);
        IM_CUDA(cudaMemcpyAsync(seeds, d_seeds, (size_t)nq * kmax * 4, cudaMemcpyDefault, st));
        if (gains) IM_CUDA(cudaMemcpyAsync(gains, d_gains, (size_t)nq * kmax * 8, cudaMemcpyDefault, st));
        IM_CUDA(cudaMemcpyAsync(hns.data(), d_ns, (size_t)nq * 4, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaMemcpyAsync(hcov.data(), d_cov, (size_t)nq * 8, cudaMemcpyDeviceToHost, st));
        int gstatus = 0;
        IM_CUDA(cudaMemcpyAsync(&gstatus, d_gstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        if (gstatus != 0) return map_dev_status(gstatus, "im_solve_batch greedy");
        for (int32_t i = 0; i < nq; ++i) {
            const int32_t q = order[i];
            res[q].num_seeds = hns[q];
            res[q].status = IM_OK;
            res[q].coverage = hcov[q];
            res[q].entries = hb[i + 1] - hb[i];
            res[q].partitions = parts_used[i];
            res[q].reserved = 0;
            // the hint for the next batches with this graph and model
            const int64_t per = qs[q].theta ? (2 * (hb[i + 1] - hb[i]) + qs[q].theta - 1) / qs[q].theta : 1;
            auto &h = b->entry_hint[{qs[q].graph, qs[q].model}];
            h = std::max<int64_t>({h, per, 1});
        }
        (void)examined;
        return IM_OK;
    }
    set_error("im_solve_batch: RRR sets did not fit after growing the arena");
    return IM_ERR_CAPACITY;
}

}  // extern "C"

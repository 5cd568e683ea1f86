// tune.cu -- im_autotune: pick the launch-shape knobs of a workload by timing.
//
// Every knob tried here leaves the results unchanged (lanes per LT walk,
// counter replicas of the covering-subset build, candidates re-evaluated per
// round by RandGreedi's local greedy, the layout of its bucket stage), so the
// tuner only measures: it samples a probe pool of the caller's workload,
// times the step each knob governs for every allowed value (CUDA events on the
// caller's stream, the best of two runs), and leaves the fastest values set.
// The RandGreedi partition count is the paper's m and changes the result; it
// stays the caller's choice.
#include <cfloat>
#include <vector>

#include "internal.cuh"

using namespace im;

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~EventPair() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Best of two runs of f, in milliseconds (negative on failure).
template <typename F>
double time_best(cudaStream_t st, F &&f, im_status *err) {
    EventPair ev;
    double best = DBL_MAX;
    for (int r = 0; r < 2; ++r) {
        if (cudaEventRecord(ev.a, st) != cudaSuccess) return -1.0;
        const im_status s = f();
        if (s != IM_OK) {
            *err = s;
            return -1.0;
        }
        if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess)
            return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.a, ev.b);
        best = ms < best ? ms : best;
    }
    return best;
}

}  // namespace

extern "C" im_status im_autotune(const im_graph *g, im_model model, uint64_t seed, int64_t theta,
                                 int32_t k, const im_cover_opts *rg_opts, im_tune_result *out,
                                 void *stream) {
    if (!g || !out || theta < 1 || k < 1 || (model != IM_IC && model != IM_LT)) {
        set_error("im_autotune: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 8; ++j) out->ms[i][j] = -1.0;
    out->lt_group = out->rg_evals = out->rg_cluster = -1;
    out->index_replicas = out->lt_cache = out->greedy_hot = -1;
    // the probe pool: grow the member capacity until the sample fits
    int64_t cap = theta * 64;
    im_pool *p = nullptr;
    im_status s = IM_OK;
    for (int attempt = 0; attempt < 6; ++attempt) {
        s = im_pool_create(g, theta, cap, &p);
        if (s != IM_OK) return s;
        s = im_sample_rrr(g, model, seed, 0, (uint64_t)theta, p, stream);
        if (s == IM_OK) break;
        im_pool_destroy(p);
        p = nullptr;
        if (s != IM_ERR_CAPACITY) return s;
        cap *= 4;
    }
    if (!p) return s;
    im_status err = IM_OK;
    auto resample = [&]() {
        im_status r = im_pool_reset(p);
        return r != IM_OK ? r : im_sample_rrr(g, model, seed, 0, (uint64_t)theta, p, stream);
    };
    auto pick = [&](int32_t knob, const int64_t *vals, int nv, int row, auto &&body) -> int32_t {
        double best = DBL_MAX;
        int64_t bv = vals[0];
        for (int i = 0; i < nv; ++i) {
            im_tune_set(knob, vals[i]);
            const double ms = body();
            out->ms[row][i] = ms;
            if (ms >= 0.0 && ms < best) {
                best = ms;
                bv = vals[i];
            }
        }
        im_tune_set(knob, bv);
        return (int32_t)bv;
    };
    // lanes per LT walk
    if (model == IM_LT) {
        const int64_t v[4] = {1, 8, 16, 32};
        out->lt_group = pick(IM_TUNE_LT_GROUP, v, 4, 0, [&]() {
            return time_best(st, [&]() { return resample(); }, &err);
        });
    }
    // L2 policy of the one-walk-per-thread LT sampler
    if (model == IM_LT && out->lt_group == 1) {
        const int64_t v[3] = {0, 1, 2};
        out->lt_cache = pick(IM_TUNE_LT_CACHE, v, 3, 4, [&]() {
            return time_best(st, [&]() { return resample(); }, &err);
        });
    }
    // covering-subset build: radix sort, or counting with 1-8 counter replicas
    {
        const int64_t v[5] = {0, 1, 2, 4, 8};
        out->index_replicas = pick(IM_TUNE_INDEX_REPLICAS, v, 5, 1, [&]() {
            return time_best(st, [&]() {
                im_status r = resample();
                return r != IM_OK ? r : im_pool_index(p, stream);
            }, &err);
        });
    }
    // the standard greedy's tau
    if (err == IM_OK) {
        s = im_pool_index(p, stream);
        int32_t *d = nullptr;
        if (s == IM_OK && cudaMalloc(&d, (size_t)k * 16 + 64) != cudaSuccess) s = IM_ERR_OOM;
        if (s == IM_OK) {
            int32_t *seeds = d;
            int64_t *gains = (int64_t *)((char *)d + (((size_t)k * 4 + 15) & ~(size_t)15));
            int32_t *ns = (int32_t *)(gains + k);
            int64_t *cov = (int64_t *)((char *)ns + 16);
            const int64_t v[4] = {0, 7, 8, 10};
            out->greedy_hot = pick(IM_TUNE_GREEDY_HOT, v, 4, 5, [&]() {
                return time_best(st, [&]() {
                    return im_max_k_cover(p, k, nullptr, seeds, gains, ns, cov, stream);
                }, &err);
            });
            cudaFree(d);
        }
    }
    // RandGreedi: local-greedy evaluation width, bucket-stage layout
    if (rg_opts && rg_opts->algo == IM_RANDGREEDI && err == IM_OK) {
        s = im_pool_index(p, stream);
        int32_t *d = nullptr;
        if (s == IM_OK && cudaMalloc(&d, (size_t)k * 16 + 64) != cudaSuccess) s = IM_ERR_OOM;
        if (s == IM_OK) {
            int32_t *seeds = d;
            int64_t *gains = (int64_t *)((char *)d + (((size_t)k * 4 + 15) & ~(size_t)15));
            int32_t *ns = (int32_t *)(gains + k);
            int64_t *cov = (int64_t *)((char *)ns + 16);
            auto cover = [&]() {
                return time_best(st, [&]() {
                    return im_max_k_cover(p, k, rg_opts, seeds, gains, ns, cov, stream);
                }, &err);
            };
            const int64_t ve[4] = {1, 2, 4, 8};
            out->rg_evals = pick(IM_TUNE_RG_EVALS, ve, 4, 2, cover);
            if (!rg_opts->fused) {
                const int64_t vc[6] = {0, 1, 2, 4, 8, -1};
                out->rg_cluster = pick(IM_TUNE_RG_CLUSTER, vc, 6, 3, cover);
            }
            cudaFree(d);
        }
    }
    im_pool_destroy(p);
    if (s != IM_OK) return s;
    return err;
}

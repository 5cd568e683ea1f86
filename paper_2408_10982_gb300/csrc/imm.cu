// imm.cu -- im_solve: the IMM driver of Alg. 1 on the device path, and pool growth.
//
// Alg. 1: Estimate, then martingale rounds i = 1, 2, ... that extend one pool
// (Sample appends sets whose ids keep counting, Sec. 3.2), SelectSeeds and
// CheckGoodness; once a round passes, theta = f(LB) fresh samples and a final
// SelectSeeds.  The paper defers Estimate / CheckGoodness / f to Tang et al.
// (SIGMOD 2015) and Chen (2018); their closed forms, natural logs:
//   l' = l (1 + ln 2 / ln n), e' = sqrt(2) e
//   lambda' = (2 + 2e'/3) (ln C(n,k) + l' ln n + ln log2 n) n / e'^2
//   alpha = sqrt(l' ln n + ln 2), beta = sqrt((1 - 1/e)(ln C(n,k) + l' ln n + ln 2))
//   lambda* = 2 n ((1 - 1/e) alpha + beta)^2 / e^2
//   round i = 1 .. floor(log2 n) - 1: x_i = n / 2^i, theta_i = ceil(lambda' / x_i);
//   pass iff n (cov / theta_i) >= (1 + e') x_i, then LB = n (cov / theta_i) / (1 + e')
//   theta = ceil(lambda* / LB) (LB = 1 if no round passes)
// All of it is host double arithmetic; the sampling and covers are the
// library's kernels.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace im {

im_status pool_grow(im_pool *p, int64_t max_sets, int64_t max_entries, cudaStream_t st) {
    max_sets = std::max(max_sets, p->max_sets);
    max_entries = std::max(max_entries, p->max_entries);
    if (max_sets == p->max_sets && max_entries == p->max_entries) return IM_OK;
    int64_t *so = nullptr;
    int32_t *mem = nullptr, *sid = nullptr;
    if (dev_alloc(&so, (size_t)(max_sets + 1) * 8) != IM_OK ||
        dev_alloc(&mem, (size_t)std::max<int64_t>(max_entries, 1) * 4) != IM_OK ||
        dev_alloc(&sid, (size_t)std::max<int64_t>(max_entries, 1) * 4) != IM_OK) {
        dev_free(so);
        dev_free(mem);
        dev_free(sid);
        set_error("pool growth: device memory exhausted");
        return IM_ERR_OOM;
    }
    IM_CUDA(cudaMemcpyAsync(so, p->set_off, (size_t)(p->theta + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (p->total > 0)
        IM_CUDA(cudaMemcpyAsync(mem, p->members, (size_t)p->total * 4, cudaMemcpyDeviceToDevice, st));
    IM_CUDA(cudaStreamSynchronize(st));
    dev_free(p->set_off);
    dev_free(p->members);
    dev_free(p->set_ids);
    p->set_off = so;
    p->members = mem;
    p->set_ids = sid;
    p->max_sets = max_sets;
    p->max_entries = max_entries;
    p->index_valid = false;
    return IM_OK;
}

// Appends ids [first, first + count) to the pool, growing it when needed.
im_status sample_growing(const im_graph *g, im_model model, uint64_t seed, uint64_t first,
                         uint64_t count, im_pool *p, cudaStream_t st) {
    const uint64_t kChunk = 1u << 22;
    for (uint64_t done = 0; done < count;) {
        const uint64_t c = std::min<uint64_t>(kChunk, count - done);
        if (p->theta + (int64_t)c > p->max_sets) {
            im_status s = pool_grow(p, std::max<int64_t>(p->theta + (int64_t)c, p->max_sets * 2),
                                    p->max_entries, st);
            if (s != IM_OK) return s;
        }
        im_status s = sample_append(g, model, seed, first + done, c, p, st);
        if (s == IM_ERR_CAPACITY) {
            // grow by what the sets so far suggest (at least double) and retry
            const double per = p->theta > 0 ? (double)p->total / (double)p->theta : 64.0;
            const int64_t want = std::max<int64_t>(p->max_entries * 2,
                                                   (int64_t)(per * (double)(p->theta + (int64_t)c) * 1.5) + 1024);
            s = pool_grow(p, p->max_sets, want, st);
            if (s != IM_OK) return s;
            continue;
        }
        if (s != IM_OK) return s;
        done += c;
    }
    return IM_OK;
}

im_status select_seeds(im_pool *p, int32_t k, const im_cover_opts *o, int32_t *d_seeds,
                       int64_t *d_gains, int32_t *d_ns, int64_t *d_cov, int *d_status,
                       int64_t *coverage, cudaStream_t st) {
    im_status s = build_index(p, st);
    if (s != IM_OK) return s;
    IM_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    s = (o && o->algo == IM_RANDGREEDI)
            ? randgreedi(p, k, o, d_seeds, d_gains, d_ns, d_cov, st, d_status)
            : greedy_select(p, k, o && o->algo == IM_GREEDY_LAZY, d_seeds, d_gains, d_ns, d_cov,
                            st, d_status);
    if (s != IM_OK) return s;
    int64_t hc[3] = {0, 0, 0};
    IM_CUDA(cudaMemcpyAsync(&hc[0], d_cov, 8, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaMemcpyAsync(&hc[1], d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if ((int)hc[1] != kDevOk) return map_dev_status((int)hc[1], "im_solve");
    *coverage = hc[0];
    return IM_OK;
}

}  // namespace im

using namespace im;

extern "C" {

im_status im_pool_reserve(im_pool *p, int64_t max_sets, int64_t max_entries) {
    if (!p || max_sets < 0 || max_entries < 0 || max_sets >= ((int64_t)1 << 31)) {
        set_error("im_pool_reserve: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    im_status s = pool_grow(p, max_sets, max_entries, 0);
    if (prev != p->device) cudaSetDevice(prev);
    return s;
}

im_status im_solve(const im_graph *g, im_model model, int32_t k, double eps, double ell,
                   uint64_t seed, const im_cover_opts *opts, int32_t *seeds, int32_t *num_seeds,
                   int64_t *coverage_out, int64_t *theta_out, im_solve_info *info, void *stream) {
    if (!g || (model != IM_IC && model != IM_LT) || k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) ||
        !(ell > 0.0) || !seeds || !num_seeds || !coverage_out) {
        set_error("im_solve: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = g->n;
    const double dn = (double)n;
    const double ln_n = std::log(dn);
    const double lncnk = std::lgamma(dn + 1.0) - std::lgamma((double)k + 1.0) -
                         std::lgamma(dn - (double)k + 1.0);
    const double l2 = ell * (1.0 + std::log(2.0) / ln_n);
    const double e2 = std::sqrt(2.0) * eps;
    const double lam1 = (2.0 + 2.0 * e2 / 3.0) * (lncnk + l2 * ln_n + std::log(std::log2(dn))) * dn /
                        (e2 * e2);
    const double one_e = 1.0 - std::exp(-1.0);
    const double alpha = std::sqrt(l2 * ln_n + std::log(2.0));
    const double beta = std::sqrt(one_e * (lncnk + l2 * ln_n + std::log(2.0)));
    const double lamstar = 2.0 * dn * (one_e * alpha + beta) * (one_e * alpha + beta) / (eps * eps);
    int32_t rounds = 0;
    while (((int64_t)1 << (rounds + 2)) <= n) ++rounds;

    im_status s = IM_OK;
    im_pool *p = nullptr, *kept = nullptr;
    void *res = nullptr;
    im_solve_info loc;
    std::memset(&loc, 0, sizeof(loc));
    const bool keep = info && info->keep_pools;
    loc.keep_pools = keep ? 1 : 0;
    double lb = 1.0;
    int64_t have = 0;
    auto fail = [&](im_status code) {
        if (p) im_pool_destroy(p);
        if (kept) im_pool_destroy(kept);
        cudaFree(res);
        if (prev != g->device) cudaSetDevice(prev);
        return code;
    };
    if (cudaMalloc(&res, (size_t)k * 12 + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(IM_ERR_OOM);
    }
    int32_t *d_seeds = (int32_t *)res;
    int64_t *d_gains = (int64_t *)((char *)res + (((size_t)k * 4 + 15) & ~(size_t)15));
    int64_t *d_cov = (int64_t *)((char *)res + (size_t)k * 12 + 128);
    int32_t *d_ns = (int32_t *)((char *)d_cov + 8);
    int *d_status = (int *)((char *)d_cov + 16);

    s = im_pool_create(g, 1 << 16, (int64_t)1 << 22, &p);
    if (s != IM_OK) return fail(s);
    for (int32_t i = 1; i <= rounds; ++i) {
        const double x = dn / std::ldexp(1.0, i);
        const int64_t th = (int64_t)std::ceil(lam1 / x);
        if (loc.rounds < 64) loc.theta_rounds[loc.rounds] = th;
        loc.rounds++;
        if (th > have) {                              // Sample(G, theta_i - |R|, R)
            s = sample_growing(g, model, seed, (uint64_t)have, (uint64_t)(th - have), p, st);
            if (s != IM_OK) return fail(s);
            have = th;
        }
        int64_t cov = 0;
        s = select_seeds(p, k, opts, d_seeds, d_gains, d_ns, d_cov, d_status, &cov, st);
        if (s != IM_OK) return fail(s);
        if (loc.rounds <= 64) loc.cov_rounds[loc.rounds - 1] = cov;
        const double spread = dn * ((double)cov / (double)th);   // CheckGoodness
        if (spread >= (1.0 + e2) * x) {
            lb = spread / (1.0 + e2);
            break;
        }
    }
    const int64_t theta = (int64_t)std::ceil(lamstar / lb);
    loc.lb = lb;
    loc.theta = theta;
    loc.round_entries = p->total;
    // final phase: theta fresh samples, ids after the rounds' ids
    const double per = p->theta > 0 ? (double)p->total / (double)p->theta : 64.0;
    if (keep) kept = p;
    else im_pool_destroy(p);
    p = nullptr;
    if ((uint64_t)have + (uint64_t)theta > ((uint64_t)1 << 32) || theta >= ((int64_t)1 << 31)) {
        set_error("im_solve: theta exceeds the 2^31 sets one pool holds");
        return fail(IM_ERR_CAPACITY);
    }
    s = im_pool_create(g, theta, std::max<int64_t>(1024, (int64_t)(per * (double)theta * 1.25)), &p);
    if (s != IM_OK) return fail(s);
    s = sample_growing(g, model, seed, (uint64_t)have, (uint64_t)theta, p, st);
    if (s != IM_OK) return fail(s);
    int64_t cov = 0;
    s = select_seeds(p, k, opts, d_seeds, d_gains, d_ns, d_cov, d_status, &cov, st);
    if (s != IM_OK) return fail(s);
    int32_t ns = 0;
    if (cudaMemcpyAsync(&ns, d_ns, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(seeds, d_seeds, (size_t)k * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "im_solve: result copy"));
    *num_seeds = ns;
    *coverage_out = cov;
    if (theta_out) *theta_out = theta;
    loc.final_entries = p->total;
    loc.examined = p->examined;
    if (keep) {
        loc.round_pool = kept;
        loc.final_pool = p;
        kept = p = nullptr;
    }
    if (info) *info = loc;
    return fail(IM_OK);
}

}  // extern "C"

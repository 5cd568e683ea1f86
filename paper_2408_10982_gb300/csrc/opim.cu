// opim.cu -- im_opim: GreediRIS inside OPIM's rounds (Sec. 3.3.2, Sec. 4.4).
//
// OPIM (Tang et al. 2018) splits each round's samples into a selection half R1
// and a validation half R2 drawn with disjoint sample ids (R1 from 0, R2 from
// 2^31).  Seeds are selected on R1 -- standard greedy, or RandGreedi with
// truncation -- and scored twice: their coverage of R2 (sets that hold a
// seed: the RIS estimate of their spread) gives a lower confidence bound on
// their spread, and an upper bound on the optimal k-set's coverage of R1 (the
// seeds' coverage plus the k largest marginal gains left on R1, valid for any
// seed set by submodularity) gives an upper confidence bound on OPT.  Their
// ratio is the round's instance-wise guarantee; the rounds double both halves
// (appending ids) until it reaches 1 - 1/e - eps or the last round.  The
// paper prints none of these formulas; natural logs:
//   theta_max = 2n ((1-1/e) sqrt(ln(6/delta)) + sqrt((1-1/e)(ln C(n,k) + ln(6/delta))))^2 / (eps^2 k)
//   theta_0 = ceil(theta_max eps^2 k / n), theta_i = theta_0 2^(i-1)
//   i_max = max(1, ceil(log2(theta_max / theta_0))), or the last round within the cap
//   a = ln(3 i_max / delta)
//   sigma_l = ((sqrt(cov2 + 2a/9) - sqrt(a/2))^2 - a/18) n / theta
//   sigma_u = (sqrt(cov1u + a/2) + sqrt(a/2))^2 n / theta
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace im {
namespace {

constexpr int kOpimThreads = 256;

__global__ void k_seed_bits(const int32_t *seeds, int32_t ns, uint32_t *bits) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)seeds[i];
        atomicOr(bits + (v >> 5), 1u << (v & 31));
    }
}

// One warp per RRR set: does it hold a seed?  count_hits: count the sets that
// do; otherwise add one to the marginal-gain counter of every member of each
// set that does not (the gains |S(v) \ C(seeds)| of all vertices).
__global__ void __launch_bounds__(kOpimThreads) k_set_scan(const int64_t *set_off,
                                                           const int32_t *members, int64_t theta,
                                                           const uint32_t *bits, int count_hits,
                                                           unsigned long long *hits,
                                                           int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_hits = 0;
    for (int64_t i = warp; i < theta; i += nwarps) {
        const int64_t b = __ldg(set_off + i), e = __ldg(set_off + i + 1);
        bool found = false;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t t = base + lane;
            bool f = false;
            if (t < e) {
                const uint32_t u = (uint32_t)__ldg(members + t);
                f = (__ldg(bits + (u >> 5)) >> (u & 31)) & 1u;
            }
            if (__any_sync(kFull, f)) {
                found = true;
                break;
            }
        }
        if (count_hits) {
            my_hits += found ? 1 : 0;
        } else if (!found) {
            for (int64_t t = b + lane; t < e; t += 32) atomicAdd(cnt + __ldg(members + t), 1);
        }
    }
    if (count_hits && lane == 0 && my_hits) atomicAdd(hits, my_hits);
}

// Histogram of one 8-bit digit (at shift) of the counters whose higher digits
// equal want under mask: per digit, how many counters and their sum.
__global__ void __launch_bounds__(kOpimThreads) k_digit_hist(const int32_t *cnt, int64_t n,
                                                             uint32_t mask, uint32_t want,
                                                             int shift, unsigned long long *hc,
                                                             unsigned long long *hs) {
    __shared__ unsigned long long sc[256], ss[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sc[i] = ss[i] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const uint32_t x = v < n ? (uint32_t)cnt[v] : 0u;
        const bool in = v < n && (x & mask) == want;
        const int d = in ? (int)((x >> shift) & 255u) : -1;
        const unsigned grp = __match_any_sync(kFull, d);
        // the group's lanes share the digit; the leader adds the count, every
        // lane its own value
        if (in) {
            if (lane == __ffs(grp) - 1) atomicAdd(&sc[d], (unsigned long long)__popc(grp));
            atomicAdd(&ss[d], (unsigned long long)x);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        if (sc[i]) atomicAdd(hc + i, sc[i]);
        if (ss[i]) atomicAdd(hs + i, ss[i]);
    }
}

// Sum of the k largest counters (radix selection, 8 bits a pass).
im_status topk_sum(const int32_t *cnt, int64_t n, int64_t k, unsigned long long *hist,
                   cudaStream_t st, int64_t *out) {
    uint32_t mask = 0, want = 0;
    int64_t remaining = k, sum = 0;
    const int grid = num_sms() * 4;
    for (int shift = 24; shift >= 0 && remaining > 0; shift -= 8) {
        IM_CUDA(cudaMemsetAsync(hist, 0, 512 * 8, st));
        {
            KernelTimer kt(st, "opim_topk");
            k_digit_hist<<<grid, kOpimThreads, 0, st>>>(cnt, n, mask, want, shift, hist,
                                                         hist + 256);
        }
        IM_CUDA(cudaGetLastError());
        unsigned long long h[512];
        IM_CUDA(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        int d = 255;
        for (; d >= 0; --d) {
            if ((int64_t)h[d] < remaining) {
                remaining -= (int64_t)h[d];
                sum += (int64_t)h[256 + d];
            } else {
                break;
            }
        }
        if (d < 0) break;                     // fewer than k counters left: all counted
        want |= (uint32_t)d << shift;
        mask |= 255u << shift;
        if (shift == 0) {
            sum += remaining * (int64_t)want;   // ties at the k-th largest value
            remaining = 0;
        }
    }
    *out = sum;
    return IM_OK;
}

}  // namespace
}  // namespace im

using namespace im;

extern "C" im_status im_opim(const im_graph *g, im_model model, int32_t k, double eps,
                             double delta, uint64_t seed, int64_t theta_cap,
                             const im_cover_opts *opts, int32_t *seeds, int32_t *num_seeds,
                             im_opim_info *info, void *stream) {
    if (!g || (model != IM_IC && model != IM_LT) || k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) ||
        !(delta > 0.0 && delta < 1.0) || theta_cap < 0 || !seeds || !num_seeds) {
        set_error("im_opim: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    const int64_t n = g->n;
    const double dn = (double)n;
    const double lncnk = std::lgamma(dn + 1.0) - std::lgamma((double)k + 1.0) -
                         std::lgamma(dn - (double)k + 1.0);
    const double one_e = 1.0 - std::exp(-1.0);
    const double l6 = std::log(6.0 / delta);
    const double sroot = one_e * std::sqrt(l6) + std::sqrt(one_e * (lncnk + l6));
    const double tmax = 2.0 * dn * sroot * sroot / (eps * eps * (double)k);
    const double t0d = std::ceil(tmax * eps * eps * (double)k / dn);
    int32_t imax = (int32_t)std::ceil(std::log2(tmax / t0d));
    if (imax < 1) imax = 1;
    if (theta_cap > 0) {
        int32_t fit = 1;
        while (fit < imax && std::ldexp(t0d, fit) <= (double)theta_cap) ++fit;
        imax = fit;
    }
    if (imax > 64) imax = 64;
    const double a = std::log(3.0 * (double)imax / delta);
    const int64_t theta0 = (int64_t)t0d;
    if (theta0 < 1 || (double)theta0 * std::ldexp(1.0, imax - 1) >= 2147483648.0) {
        set_error("im_opim: the rounds would need 2^31 or more sets per half; pass a theta cap");
        return IM_ERR_CAPACITY;
    }
    const bool keep = info && info->keep_pools;
    im_opim_info loc;
    std::memset(&loc, 0, sizeof(loc));
    loc.keep_pools = keep ? 1 : 0;
    loc.theta_max = tmax;
    loc.theta0 = theta0;
    loc.max_rounds = imax;
    loc.a = a;

    im_pool *r1 = nullptr, *r2 = nullptr;
    void *res = nullptr;
    auto finish = [&](im_status code) {
        if (r1) im_pool_destroy(r1);
        if (r2) im_pool_destroy(r2);
        cudaFree(res);
        return code;
    };
    // results + scratch: seeds[k] gains[k] cov ns status | bits[n/32] | cnt[n] | hist[512] hits
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_gains = up((size_t)k * 4), o_tail = o_gains + up((size_t)k * 8);
    const size_t o_bits = o_tail + 256, o_cnt = o_bits + up((size_t)((n + 31) / 32) * 4);
    const size_t o_hist = o_cnt + up((size_t)n * 4), total = o_hist + up(513 * 8);
    if (cudaMalloc(&res, total) != cudaSuccess) {
        cudaGetLastError();
        set_error("im_opim: device memory exhausted");
        return IM_ERR_OOM;
    }
    char *R = (char *)res;
    int32_t *d_seeds = (int32_t *)R;
    int64_t *d_gains = (int64_t *)(R + o_gains);
    int64_t *d_cov = (int64_t *)(R + o_tail);
    int32_t *d_ns = (int32_t *)(R + o_tail + 8);
    int *d_status = (int *)(R + o_tail + 16);
    uint32_t *d_bits = (uint32_t *)(R + o_bits);
    int32_t *d_cnt = (int32_t *)(R + o_cnt);
    unsigned long long *d_hist = (unsigned long long *)(R + o_hist);
    unsigned long long *d_hits = d_hist + 512;

    im_status s = im_pool_create(g, theta0, theta0 * 64, &r1);
    if (s != IM_OK) return finish(s);
    s = im_pool_create(g, theta0, theta0 * 64, &r2);
    if (s != IM_OK) return finish(s);
    const double target = 1.0 - std::exp(-1.0) - eps;
    int64_t have = 0;
    int32_t ns = 0;
    double sl = 0.0, su = 0.0;
    const int grid = num_sms() * 8;
    for (int32_t i = 1; i <= imax; ++i) {
        const int64_t th = theta0 << (i - 1);
        s = sample_growing(g, model, seed, (uint64_t)have, (uint64_t)(th - have), r1, st);
        if (s != IM_OK) return finish(s);
        s = sample_growing(g, model, seed, (1ull << 31) + (uint64_t)have, (uint64_t)(th - have), r2,
                           st);
        if (s != IM_OK) return finish(s);
        have = th;
        int64_t cov1 = 0;
        s = select_seeds(r1, k, opts, d_seeds, d_gains, d_ns, d_cov, d_status, &cov1, st);
        if (s != IM_OK) return finish(s);
        IM_CUDA(cudaMemcpyAsync(&ns, d_ns, 4, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaMemsetAsync(d_bits, 0, (size_t)((n + 31) / 32) * 4, st));
        IM_CUDA(cudaMemsetAsync(d_hits, 0, 8, st));
        IM_CUDA(cudaMemsetAsync(d_cnt, 0, (size_t)n * 4, st));
        IM_CUDA(cudaStreamSynchronize(st));
        {
            KernelTimer kt(st, "opim_scan");
            k_seed_bits<<<std::max(1, (ns + 255) / 256), 256, 0, st>>>(d_seeds, ns, d_bits);
            k_set_scan<<<grid, kOpimThreads, 0, st>>>(r2->set_off, r2->members, r2->theta, d_bits,
                                                      1, d_hits, nullptr);
            k_set_scan<<<grid, kOpimThreads, 0, st>>>(r1->set_off, r1->members, r1->theta, d_bits,
                                                      0, nullptr, d_cnt);
        }
        IM_CUDA(cudaGetLastError());
        unsigned long long cov2 = 0;
        IM_CUDA(cudaMemcpyAsync(&cov2, d_hits, 8, cudaMemcpyDeviceToHost, st));
        int64_t top = 0;
        s = topk_sum(d_cnt, n, k, d_hist, st, &top);
        if (s != IM_OK) return finish(s);
        const int64_t cov1u = cov1 + top;
        double r = std::sqrt((double)cov2 + 2.0 * a / 9.0) - std::sqrt(a / 2.0);
        sl = (r * r - a / 18.0) * dn / (double)th;
        r = std::sqrt((double)cov1u + a / 2.0) + std::sqrt(a / 2.0);
        su = r * r * dn / (double)th;
        const int32_t q = loc.rounds++;
        loc.theta[q] = th;
        loc.cov1[q] = cov1;
        loc.cov2[q] = (int64_t)cov2;
        loc.cov1_upper[q] = cov1u;
        loc.alpha[q] = sl / su;
        if (sl / su >= target) break;
    }
    if (cudaMemcpyAsync(seeds, d_seeds, (size_t)ns * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return finish(cuda_fail(cudaGetLastError(), "im_opim: result copy"));
    *num_seeds = ns;
    loc.sigma_lower = sl;
    loc.sigma_upper = su;
    loc.guarantee = sl / su;
    if (keep) {
        loc.r1_pool = r1;
        loc.r2_pool = r2;
        r1 = r2 = nullptr;
    }
    if (info) *info = loc;
    return finish(IM_OK);
}

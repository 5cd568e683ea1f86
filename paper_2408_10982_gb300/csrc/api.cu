// api.cu -- the extern "C" entry points of libim (declared in include/im.h).
//
// Each entry point validates its arguments, runs the kernels of sample.cu,
// index.cu and cover.cu on the caller's stream, and maps device status words
// and CUDA errors to im_status.  No C++ exception crosses the boundary.  The
// device memory of RRR pools comes from dev_alloc / dev_free below (a cached
// stream-ordered memory pool per device); graphs use plain cudaMalloc.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace im {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

im_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? IM_ERR_OOM : IM_ERR_CUDA;
}

im_status map_dev_status(int code, const char *where) {
    switch (code) {
        case kDevOk: return IM_OK;
        case kDevTimeout:
            set_error(std::string(where) + ": a bounded device wait expired");
            return IM_ERR_TIMEOUT;
        case kDevQueueOverflow:
        case kDevStageOverflow:
            set_error(std::string(where) + ": capacity exceeded");
            return IM_ERR_CAPACITY;
        case kDevBadInput:
            set_error(std::string(where) + ": invalid input");
            return IM_ERR_INVALID_ARG;
        default:
            set_error(std::string(where) + ": unknown device status");
            return IM_ERR_CUDA;
    }
}

// ---- profiler -------------------------------------------------------------
namespace {
struct PendingTiming {
    std::string name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<PendingTiming> g_prof_pending;
std::map<std::string, std::pair<int64_t, double>> g_prof_acc;

void prof_drain_locked() {
    for (auto &t : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) ==
                                                            cudaSuccess) {
            auto &acc = g_prof_acc[t.name];
            acc.first += 1;
            acc.second += ms;
        } else {
            cudaGetLastError();
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_prof_pending.clear();
}
}  // namespace

KernelTimer::KernelTimer(cudaStream_t st, const char *name) : st_(st), name_(name) {
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        on_ = g_prof_on;
    }
    if (on_) {
        if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
            cudaGetLastError();
            on_ = false;
            return;
        }
        cudaEventRecord(a_, st_);
    }
}

KernelTimer::~KernelTimer() {
    if (!on_) return;
    cudaEventRecord(b_, st_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back({name_, a_, b_});
    if (g_prof_pending.size() > 4096) prof_drain_locked();
}

namespace {
std::mutex g_tune_mu;
// IM_TUNE_LT_GROUP, IM_TUNE_RG_CLUSTER, IM_TUNE_INDEX_REPLICAS, IM_TUNE_RG_EVALS,
// IM_TUNE_GREEDY_EVALS, IM_TUNE_LT_CACHE, IM_TUNE_GREEDY_HOT
constexpr int kKnobs = 7;
int64_t g_tune[kKnobs] = {1, 0, 0, 2, 0, 0, 8};
}  // namespace

int64_t tune_value(int32_t knob) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (knob >= 0 && knob < kKnobs) ? g_tune[knob] : 0;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

namespace {

constexpr int kMaxDevices = 64;

struct DevHeap {
    cudaMemPool_t pool = nullptr;
    cudaStream_t st = nullptr;   // allocations and frees are ordered on this stream
};

std::mutex g_heap_mu;
DevHeap g_heap[kMaxDevices];

// The heap of the current device, created on first use.
cudaError_t dev_heap(DevHeap **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_heap_mu);
    DevHeap &h = g_heap[dev];
    if (!h.pool) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        uint64_t keep = (uint64_t)total_b / 8;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaStream_t st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        h.pool = pool;
        h.st = st;
    }
    *out = &h;
    return cudaSuccess;
}

}  // namespace

im_status dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    DevHeap *h = nullptr;
    IM_CUDA(dev_heap(&h));
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, h->pool, h->st);
    if (e == cudaErrorMemoryAllocation) {
        // pages cached for sizes that do not fit: hand them back and retry once
        cudaGetLastError();
        IM_CUDA(cudaDeviceSynchronize());
        cudaMemPoolTrimTo(h->pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes, h->pool, h->st);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "device allocation");
    }
    // ordered before any later use on another stream
    if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return cuda_fail(e, "device allocation");
    return IM_OK;
}

im_status raise_dyn_smem(const void *func, size_t bytes) {
    constexpr size_t kDefault = 48 * 1024;   // the limit without opting in
    if (bytes <= kDefault) return IM_OK;
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    IM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[{dev, func}];
    if (bytes <= cur) return IM_OK;
    IM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return IM_OK;
}

void dev_free(void *p) {
    if (!p) return;
    DevHeap *h = nullptr;
    if (dev_heap(&h) != cudaSuccess) return;
    cudaDeviceSynchronize();   // no kernel on any stream may still use p
    cudaFreeAsync(p, h->st);
}

im_status pool_scratch(im_pool *p, size_t bytes, void **out) {
    if (bytes > p->scratch_bytes) {
        if (p->scratch) {
            dev_free(p->scratch);
            p->scratch = nullptr;
            p->scratch_bytes = 0;
        }
        size_t want = bytes + bytes / 4 + 4096;
        IM_TRY(dev_alloc(&p->scratch, want));
        p->scratch_bytes = want;
    }
    *out = p->scratch;
    return IM_OK;
}

namespace {


__global__ void k_validate_graph(const int64_t *in_off, const int32_t *in_src, int64_t n,
                                 int64_t m, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (in_off[v + 1] < in_off[v]) atomicExch(bad, 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t u = in_src[e];
        if (u < 0 || (int64_t)u >= n) atomicExch(bad, 2);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (in_off[0] != 0 || in_off[n] != m))
        atomicExch(bad, 3);
}


// copy to a caller buffer (host or device); returns whether it was host memory
im_status copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st, bool *host) {
    if (!dst || bytes == 0) return IM_OK;
    if (!is_device_ptr(dst)) *host = true;
    IM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return IM_OK;
}

im_status pool_results(im_pool *p, size_t bytes, void **out) {
    if (bytes > p->res_bytes) {
        if (p->res) {
            dev_free(p->res);
            p->res = nullptr;
            p->res_bytes = 0;
        }
        IM_TRY(dev_alloc(&p->res, bytes));
        p->res_bytes = bytes;
    }
    *out = p->res;
    return IM_OK;
}


}  // namespace
}  // namespace im

using namespace im;

extern "C" {

const char *im_status_str(im_status s) {
    switch (s) {
        case IM_OK: return "ok";
        case IM_ERR_INVALID_ARG: return "invalid argument";
        case IM_ERR_OOM: return "out of device memory";
        case IM_ERR_CUDA: return "CUDA error";
        case IM_ERR_TIMEOUT: return "bounded device wait expired";
        case IM_ERR_CAPACITY: return "capacity exceeded";
        case IM_ERR_BUSY: return "busy";
        case IM_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *im_last_error(void) { return g_last_error.c_str(); }

im_status im_device_info(int32_t *sms, int32_t *device) {
    int dev = 0, count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return IM_ERR_UNSUPPORTED;
    }
    IM_CUDA(cudaGetDevice(&dev));
    if (sms) *sms = num_sms();
    if (device) *device = dev;
    return IM_OK;
}

im_status im_trim_memory(void) {
    int dev = 0, count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return IM_ERR_UNSUPPORTED;
    }
    IM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return IM_OK;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_heap_mu);
        pool = g_heap[dev].pool;
    }
    if (!pool) return IM_OK;
    IM_CUDA(cudaDeviceSynchronize());
    IM_CUDA(cudaMemPoolTrimTo(pool, 0));
    return IM_OK;
}

im_status im_graph_create(const int64_t *in_off, const int32_t *in_src, const uint32_t *w,
                          int64_t n, int64_t m, void *stream, im_graph **out) {
    if (!out || !in_off || n < 1 || n > INT32_MAX || m < 0 || m >= ((int64_t)1 << 31) ||
        (m > 0 && (!in_src || !w))) {
        set_error("im_graph_create: bad sizes or null pointers");
        return IM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cudaStream_t st = as_stream(stream);
    im_graph *g = new (std::nothrow) im_graph();
    if (!g) return IM_ERR_OOM;
    std::memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    g->n = n;
    g->m = m;
    const int64_t mpad = (m + 3) & ~(int64_t)3;   // 16-byte groups of four edges
    auto fail = [&](im_status s) {
        cudaFree(g->in_off);
        cudaFree(g->in_src);
        cudaFree(g->w);
        delete g;
        return s;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&g->in_off, (size_t)(n + 1) * 8)) != cudaSuccess ||
        (e = cudaMalloc(&g->in_src, (size_t)std::max<int64_t>(mpad, 4) * 4)) != cudaSuccess ||
        (e = cudaMalloc(&g->w, (size_t)std::max<int64_t>(mpad, 4) * 4)) != cudaSuccess)
        return fail(cuda_fail(e, "im_graph_create: cudaMalloc"));
    if ((e = cudaMemcpyAsync(g->in_off, in_off, (size_t)(n + 1) * 8, cudaMemcpyDefault, st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(g->in_src, 0, (size_t)std::max<int64_t>(mpad, 4) * 4, st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(g->w, 0, (size_t)std::max<int64_t>(mpad, 4) * 4, st)) != cudaSuccess)
        return fail(cuda_fail(e, "im_graph_create: copy"));
    if (m > 0 &&
        ((e = cudaMemcpyAsync(g->in_src, in_src, (size_t)m * 4, cudaMemcpyDefault, st)) !=
             cudaSuccess ||
         (e = cudaMemcpyAsync(g->w, w, (size_t)m * 4, cudaMemcpyDefault, st)) != cudaSuccess))
        return fail(cuda_fail(e, "im_graph_create: copy"));
    int *d_bad = nullptr;
    if ((e = cudaMallocAsync((void **)&d_bad, sizeof(int), st)) != cudaSuccess)
        return fail(cuda_fail(e, "im_graph_create: cudaMallocAsync"));
    cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    {
        KernelTimer kt(st, "validate_graph");
        k_validate_graph<<<num_sms() * 4, 256, 0, st>>>(g->in_off, g->in_src, n, m, d_bad);
    }
    int bad = 0;
    cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_bad, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(cuda_fail(e, "im_graph_create: validation"));
    if (bad) {
        set_error(bad == 2 ? "im_graph_create: source id out of range"
                           : "im_graph_create: offsets not a valid CSR of m edges");
        return fail(IM_ERR_INVALID_ARG);
    }
    g->lt_valid = -1;   // unknown until the LT weights are summed
    *out = g;
    return IM_OK;
}

im_status im_graph_destroy(im_graph *g) {
    if (!g) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    for (void *b : {(void *)g->in_off, (void *)g->in_src, (void *)g->w, (void *)g->lt_vrec,
                    (void *)g->lt_leaf, (void *)g->lt_tree, (void *)g->lt_guide,
                    (void *)g->out_off, (void *)g->out_rec})
        cudaFree(b);
    delete g;
    return IM_OK;
}

im_status im_graph_info(const im_graph *g, int64_t *n, int64_t *m, int32_t *lt_valid) {
    if (!g) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (lt_valid) {
        IM_TRY(build_lt_index(const_cast<im_graph *>(g), 0));   // returns at once when built
        *lt_valid = g->lt_valid;
    }
    return IM_OK;
}

im_status im_pool_create(const im_graph *g, int64_t max_sets, int64_t max_entries,
                         im_pool **out) {
    if (!g || !out || max_sets < 0 || max_entries < 0 || max_sets >= ((int64_t)1 << 31)) {
        set_error("im_pool_create: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(g->device);
    *out = nullptr;
    im_pool *p = new (std::nothrow) im_pool();
    if (!p) return IM_ERR_OOM;
    std::memset(p, 0, sizeof(*p));
    p->g = g;
    p->device = g->device;
    p->max_sets = max_sets;
    p->max_entries = max_entries;
    const int64_t n = g->n;
    cudaError_t e;
    im_status as;
    if ((as = dev_alloc(&p->set_off, (size_t)(max_sets + 1) * 8)) != IM_OK ||
        (as = dev_alloc(&p->members, (size_t)std::max<int64_t>(max_entries, 1) * 4)) != IM_OK ||
        (as = dev_alloc(&p->vtx_off, (size_t)(n + 1) * 8)) != IM_OK ||
        (as = dev_alloc(&p->set_ids, (size_t)std::max<int64_t>(max_entries, 1) * 4)) != IM_OK ||
        (as = dev_alloc(&p->vtx_cursor, (size_t)(kMaxIndexReplicas + 1) * n * 4)) != IM_OK) {
        im_pool_destroy(p);
        return as;
    }
    cudaMemset(p->set_off, 0, 8);
    cudaMemset(p->vtx_off, 0, (size_t)(n + 1) * 8);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        im_status s = cuda_fail(e, "im_pool_create");
        im_pool_destroy(p);
        return s;
    }
    *out = p;
    return IM_OK;
}

im_status im_pool_destroy(im_pool *p) {
    if (!p) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    for (void *b : {(void *)p->set_off, (void *)p->members, (void *)p->vtx_off,
                    (void *)p->set_ids, (void *)p->vtx_cursor, (void *)p->part,
                    (void *)p->part_off, (void *)p->part_vtx, (void *)p->part_loc,
                    (void *)p->rg_block, p->scratch, p->res})
        dev_free(b);
    delete p;
    return IM_OK;
}

im_status im_pool_reset(im_pool *p) {
    if (!p) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    p->theta = p->total = p->examined = p->sample_bytes = 0;
    p->index_valid = false;
    IM_CUDA(cudaMemset(p->set_off, 0, 8));
    return IM_OK;
}

im_status im_pool_info(const im_pool *p, int64_t *theta, int64_t *total, int64_t *examined) {
    if (!p) return IM_ERR_INVALID_ARG;
    if (theta) *theta = p->theta;
    if (total) *total = p->total;
    if (examined) *examined = p->examined;
    return IM_OK;
}

im_status im_sample_rrr(const im_graph *g, im_model model, uint64_t seed,
                        uint64_t first_sample_id, uint64_t num_samples, im_pool *pool,
                        void *stream) {
    if (!g || !pool || pool->g != g || (model != IM_IC && model != IM_LT) ||
        first_sample_id + num_samples > ((uint64_t)1 << 32) || num_samples >= ((uint64_t)1 << 31)) {
        set_error("im_sample_rrr: bad arguments (graph/pool mismatch, model or sample ids)");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(g->device);
    return sample_append(g, model, seed, first_sample_id, num_samples, pool, as_stream(stream));
}

im_status im_pool_export(const im_pool *p, int64_t *set_off, int32_t *members, void *stream) {
    if (!p) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    cudaStream_t st = as_stream(stream);
    bool host = false;
    IM_TRY(copy_out(set_off, p->set_off, (size_t)(p->theta + 1) * 8, st, &host));
    IM_TRY(copy_out(members, p->members, (size_t)p->total * 4, st, &host));
    if (host) IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

im_status im_pool_index(im_pool *p, void *stream) {
    if (!p) return IM_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    return build_index(p, as_stream(stream));
}

im_status im_index_export(const im_pool *pc, int64_t *vtx_off, int32_t *set_ids, void *stream) {
    if (!pc) return IM_ERR_INVALID_ARG;
    im_pool *p = const_cast<im_pool *>(pc);
    DeviceGuard dg(p->device);
    cudaStream_t st = as_stream(stream);
    IM_TRY(build_index(p, st));
    bool host = false;
    IM_TRY(copy_out(vtx_off, p->vtx_off, (size_t)(p->g->n + 1) * 8, st, &host));
    IM_TRY(copy_out(set_ids, p->set_ids, (size_t)p->total * 4, st, &host));
    if (host) IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

im_status im_max_k_cover(im_pool *p, int32_t k, const im_cover_opts *opts, int32_t *seeds,
                         int64_t *gains, int32_t *num_seeds, int64_t *coverage, void *stream) {
    if (!p || k < 1 || k > (1 << 24)) {
        set_error("im_max_k_cover: bad arguments");
        return IM_ERR_INVALID_ARG;
    }
    im_cover_opts o;
    std::memset(&o, 0, sizeof(o));
    o.algo = IM_GREEDY_PLAIN;
    if (opts) o = *opts;
    if (o.algo == IM_RANDGREEDI) {
        if (o.partitions < 1 || o.partitions > 4096 || o.alpha_num < 1 || o.alpha_den < 1 ||
            o.alpha_num > o.alpha_den || !(o.delta > 0.0 && o.delta < 0.5) ||
            (o.aggregator != IM_AGG_STREAM && o.aggregator != IM_AGG_GREEDY)) {
            set_error("im_max_k_cover: RandGreedi options out of range");
            return IM_ERR_INVALID_ARG;
        }
    } else if (o.algo != IM_GREEDY_PLAIN && o.algo != IM_GREEDY_LAZY) {
        set_error("im_max_k_cover: unknown algorithm");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t st = as_stream(stream);
    IM_TRY(build_index(p, st));
    // results: seeds[k] gains[k] nseeds cov status
    const size_t o_seeds = 0, o_gains = ((size_t)k * 4 + 255) & ~(size_t)255;
    const size_t o_tail = o_gains + (((size_t)k * 8 + 255) & ~(size_t)255);
    void *res = nullptr;
    IM_TRY(pool_results(p, o_tail + 64, &res));
    char *R = (char *)res;
    int32_t *d_seeds = (int32_t *)(R + o_seeds);
    int64_t *d_gains = (int64_t *)(R + o_gains);
    int64_t *d_cov = (int64_t *)(R + o_tail);
    int32_t *d_nseeds = (int32_t *)(R + o_tail + 8);
    int *d_status = (int *)(R + o_tail + 16);
    IM_CUDA(cudaMemsetAsync(R + o_tail, 0, 64, st));
    im_status s = o.algo == IM_RANDGREEDI
                      ? randgreedi(p, k, &o, d_seeds, d_gains, d_nseeds, d_cov, st, d_status)
                      : greedy_select(p, k, o.algo == IM_GREEDY_LAZY, d_seeds, d_gains, d_nseeds,
                                      d_cov, st, d_status);
    if (s != IM_OK) return s;
    int32_t hdr[6];
    IM_CUDA(cudaMemcpyAsync(hdr, R + o_tail, sizeof(hdr), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (hdr[4] != kDevOk) return map_dev_status(hdr[4], "im_max_k_cover");
    const int32_t ns = hdr[2];
    bool host = false;
    IM_TRY(copy_out(seeds, d_seeds, (size_t)ns * 4, st, &host));
    IM_TRY(copy_out(gains, d_gains, (size_t)ns * 8, st, &host));
    IM_TRY(copy_out(num_seeds, d_nseeds, 4, st, &host));
    IM_TRY(copy_out(coverage, d_cov, 8, st, &host));
    if (host) IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

im_status im_randgreedi_details(const im_pool *p, int32_t *P_out, int32_t *B_out,
                                int32_t *local_seeds, int64_t *local_gains, int32_t *local_n,
                                int64_t *local_cov, int64_t *thr, int64_t *bucket_cov,
                                int32_t *bucket_n, int32_t *bucket_seeds, int64_t *bucket_gains,
                                int32_t *chosen, void *stream) {
    if (!p || p->rg_P == 0) {
        set_error("im_randgreedi_details: no RandGreedi run on this pool");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t st = as_stream(stream);
    const size_t P = p->rg_P, B = p->rg_B, k = p->rg_k;
    if (P_out) *P_out = (int32_t)P;
    if (B_out) *B_out = (int32_t)B;
    if (chosen) *chosen = p->rg_chosen;
    bool host = false;
    IM_TRY(copy_out(local_seeds, p->rg_local_seeds, P * k * 4, st, &host));
    IM_TRY(copy_out(local_gains, p->rg_local_gains, P * k * 8, st, &host));
    IM_TRY(copy_out(local_n, p->rg_local_n, P * 4, st, &host));
    IM_TRY(copy_out(local_cov, p->rg_local_cov, P * 8, st, &host));
    IM_TRY(copy_out(thr, p->rg_thr, B * 8, st, &host));
    IM_TRY(copy_out(bucket_cov, p->rg_bucket_cov, B * 8, st, &host));
    IM_TRY(copy_out(bucket_n, p->rg_bucket_n, B * 4, st, &host));
    IM_TRY(copy_out(bucket_seeds, p->rg_bucket_seeds, B * k * 4, st, &host));
    IM_TRY(copy_out(bucket_gains, p->rg_bucket_gains, B * k * 8, st, &host));
    if (host) IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

im_status im_randgreedi_stats(const im_pool *p, int64_t *stats, void *stream) {
    if (!p || p->rg_P == 0 || !stats) {
        set_error("im_randgreedi_stats: no RandGreedi run on this pool");
        return IM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t st = as_stream(stream);
    bool host = false;
    IM_TRY(copy_out(stats, p->rg_stats, (size_t)(p->rg_P + p->rg_B) * 6 * 8, st, &host));
    if (host) IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

im_status im_pool_sample_bytes(const im_pool *p, int64_t *bytes) {
    if (!p || !bytes) return IM_ERR_INVALID_ARG;
    *bytes = p->sample_bytes;
    return IM_OK;
}

im_status im_tune_set(int32_t knob, int64_t value) {
    const bool ok = (knob == IM_TUNE_LT_GROUP && (value == 1 || value == 8 || value == 16 || value == 32)) ||
                    (knob == IM_TUNE_RG_CLUSTER &&
                     (value == -1 || value == 0 || value == 1 || value == 2 || value == 4 ||
                      value == 8)) ||
                    (knob == IM_TUNE_INDEX_REPLICAS && (value == 0 || value == 1 || value == 2 || value == 4 ||
                                                        value == 8)) ||
                    (knob == IM_TUNE_RG_EVALS && (value == 1 || value == 2 || value == 4 ||
                                                  value == 8)) ||
                    (knob == IM_TUNE_GREEDY_EVALS && (value == 0 || value == 1 || value == 2 ||
                                                      value == 4 || value == 8 || value == 16 ||
                                                      value == 32)) ||
                    (knob == IM_TUNE_LT_CACHE && value >= 0 && value <= 2) ||
                    (knob == IM_TUNE_GREEDY_HOT && (value == 0 || (value >= 4 && value <= 16)));
    if (ok) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[knob] = value;
        return IM_OK;
    }
    set_error("im_tune_set: unknown knob or value out of range");
    return IM_ERR_INVALID_ARG;
}

im_status im_tune_get(int32_t knob, int64_t *value) {
    if (!value || knob < IM_TUNE_LT_GROUP || knob > IM_TUNE_GREEDY_HOT)
        return IM_ERR_INVALID_ARG;
    *value = tune_value(knob);
    return IM_OK;
}

im_status im_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return IM_OK;
}

im_status im_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    g_prof_acc.clear();
    return IM_OK;
}

im_status im_profile_read(int32_t max_entries, char *names, int64_t *launches, double *total_ms,
                          int32_t *count) {
    if (max_entries < 0 || !count) return IM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    int32_t i = 0;
    for (auto &kv : g_prof_acc) {
        if (i >= max_entries) break;
        if (names) {
            std::strncpy(names + 48 * i, kv.first.c_str(), 47);
            names[48 * i + 47] = 0;
        }
        if (launches) launches[i] = kv.second.first;
        if (total_ms) total_ms[i] = kv.second.second;
        ++i;
    }
    *count = i;
    return IM_OK;
}

im_status im_partition(int64_t n, int32_t P, uint64_t partition_seed, int32_t *part,
                       void *stream) {
    if (n < 1 || n > INT32_MAX || P < 1 || !part) return IM_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const bool dev = is_device_ptr(part);
    int32_t *d = part;
    if (!dev) IM_CUDA(cudaMallocAsync((void **)&d, (size_t)n * 4, st));
    IM_TRY(launch_partition_labels(n, P, partition_seed, d, st));
    if (!dev) {
        IM_CUDA(cudaMemcpyAsync(part, d, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaFreeAsync(d, st));
        IM_CUDA(cudaStreamSynchronize(st));
    }
    return IM_OK;
}

}  // extern "C"

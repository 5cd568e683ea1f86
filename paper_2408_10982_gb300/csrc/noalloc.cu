// noalloc.cu -- standard greedy max-k-cover that allocates no device memory.
//
// Some callers must not have a library allocate GPU memory behind their back:
// a framework whose caching allocator already holds (almost) all device memory
// and would see a cudaMalloc fail or fragment its pool, a serving loop that
// cannot afford cudaMalloc's latency or implicit synchronisation in the middle
// of a request, or a process whose device-memory budget is fixed up front.
// im_max_k_cover_noalloc gives them the standard greedy over arrays they own:
// its scratch space is this file's static device array, which every GPU that
// loads the library holds until the process exits.
#include "internal.cuh"

namespace im {
namespace {

// Scratch of every im_max_k_cover_noalloc call on a device, 256-byte aligned:
//   [0, 256)                 grid barrier and device status word
//   [256, 256 + 8 * 4096)    per-block maxima (at most 4096 blocks)
//   then counts int32[n], then the covered bitmap uint32[ceil(theta / 32)].
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB
constexpr int kNoAllocMaxGrid = 4096;
constexpr size_t kCtrlBytes = 256;
constexpr size_t kBestBytes = (size_t)kNoAllocMaxGrid * 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the static array on the current device.  The host-side
// symbol is only a stand-in, not an address; the runtime maps it per device
// (and again in a new context after cudaDeviceReset), so it is looked up with
// the device current on every call -- a lookup, not an allocation.  The first
// call on a device also loads this module there.
im_status scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "im_max_k_cover_noalloc: cudaGetSymbolAddress");
    *out = p;
    return IM_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Every array handed to this entry point must be memory the current device
// can reach: its own device memory, or managed memory.  Another GPU's memory
// is refused (without peer access the kernel would fault on it).
bool on_device(const void *p, int dev) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// The caller's arrays are checked before the greedy writes anything indexed by
// them: both offset arrays start at 0 and never decrease, both end at the same
// total T, every member id is below n and every set id below theta.  A
// violation raises kDevBadInput (the call then returns IM_ERR_INVALID_ARG and
// the greedy does not run).
__global__ void k_noalloc_validate(const int64_t *set_off, const int32_t *members,
                                   const int64_t *vtx_off, const int32_t *set_ids, int64_t n,
                                   int64_t theta, int *status) {
    const int64_t T = set_off[theta];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (set_off[0] != 0 || vtx_off[0] != 0 || vtx_off[n] != T || T < 0))
        raise_status(status, kDevBadInput);
    if (T < 0 || vtx_off[n] != T) return;
    bool bad = false;
    for (int64_t i = tid; i < theta; i += stride) bad |= set_off[i + 1] < set_off[i];
    for (int64_t v = tid; v < n; v += stride) bad |= vtx_off[v + 1] < vtx_off[v];
    for (int64_t t = tid; t < T; t += stride)
        bad |= (uint32_t)members[t] >= (uint64_t)n || (uint32_t)set_ids[t] >= (uint64_t)theta;
    if (bad) raise_status(status, kDevBadInput);
}

}  // namespace
}  // namespace im

using namespace im;

extern "C" im_status im_max_k_cover_noalloc(const int64_t *set_off, const int32_t *members,
                                            const int64_t *vtx_off, const int32_t *set_ids,
                                            int64_t n, int64_t theta, int32_t k, int32_t *seeds,
                                            int64_t *gains, int32_t *num_seeds,
                                            int64_t *coverage, void *stream) {
    if (!set_off || !vtx_off || n < 1 || n > INT32_MAX || theta < 0 || theta >= ((int64_t)1 << 31) ||
        k < 1 || !seeds || !gains || !num_seeds || !coverage ||
        (theta > 0 && (!members || !set_ids))) {
        set_error("im_max_k_cover_noalloc: bad sizes or null pointers");
        return IM_ERR_INVALID_ARG;
    }
    const size_t need = kCtrlBytes + kBestBytes + up256((size_t)n * 4) +
                        up256((size_t)((theta + 31) / 32) * 4);
    if (need > kNoAllocScratchBytes) {
        set_error("im_max_k_cover_noalloc: 4 n + theta / 8 bytes of scratch exceed the fixed "
                  "64 MiB array (use im_max_k_cover for larger instances)");
        return IM_ERR_CAPACITY;
    }
    int dev = 0;
    IM_CUDA(cudaGetDevice(&dev));
    if (!on_device(set_off, dev) || !on_device(members, dev) || !on_device(vtx_off, dev) ||
        !on_device(set_ids, dev) || !on_device(seeds, dev) || !on_device(gains, dev) ||
        !on_device(num_seeds, dev) || !on_device(coverage, dev)) {
        set_error("im_max_k_cover_noalloc: every array must be memory of the current device "
                  "(or managed memory)");
        return IM_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    im_status s = scratch_address(&base);
    if (s != IM_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *B = (char *)base;
    int *d_status = (int *)(B + 64);
    // the barrier and the status word must start at zero; the kernel fills the rest
    IM_CUDA(cudaMemsetAsync(B, 0, kCtrlBytes, st));
    IM_CUDA(cudaMemsetAsync(num_seeds, 0, sizeof(int32_t), st));
    IM_CUDA(cudaMemsetAsync(coverage, 0, sizeof(int64_t), st));
    int hstatus = 0;
    k_noalloc_validate<<<num_sms() * 4, 256, 0, st>>>(set_off, members, vtx_off, set_ids, n, theta,
                                                      d_status);
    IM_CUDA(cudaGetLastError());
    IM_CUDA(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (hstatus != kDevOk) {
        set_error("im_max_k_cover_noalloc: offsets must start at 0, never decrease and end at "
                  "the same total; member ids must be < n and set ids < theta");
        return IM_ERR_INVALID_ARG;
    }
    s = greedy_launch(n, theta, set_off, members, vtx_off, set_ids, k,
                      (int32_t *)(B + kCtrlBytes + kBestBytes),
                      (uint32_t *)(B + kCtrlBytes + kBestBytes + up256((size_t)n * 4)),
                      (unsigned long long *)(B + kCtrlBytes), kNoAllocMaxGrid, B, seeds, gains,
                      num_seeds, coverage, d_status, st);
    if (s != IM_OK) return s;
    IM_CUDA(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (hstatus != kDevOk) return map_dev_status(hstatus, "im_max_k_cover_noalloc");
    return IM_OK;
}

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
#include <mutex>

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

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Resolve the device address of the static array once per device, with that
// device current (the host-side symbol is only a stand-in, not an address).
im_status scratch_address(void **out) {
    int dev = 0;
    IM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("im_max_k_cover_noalloc: device ordinal out of range");
        return IM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "im_max_k_cover_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return IM_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Every array handed to this entry point must be device memory: the kernel
// reads and writes it directly.
bool on_device(const void *p) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
    if (!on_device(set_off) || !on_device(members) || !on_device(vtx_off) || !on_device(set_ids) ||
        !on_device(seeds) || !on_device(gains) || !on_device(num_seeds) || !on_device(coverage)) {
        set_error("im_max_k_cover_noalloc: every array must be device memory");
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
    s = greedy_launch(n, theta, set_off, members, vtx_off, set_ids, k,
                      (int32_t *)(B + kCtrlBytes + kBestBytes),
                      (uint32_t *)(B + kCtrlBytes + kBestBytes + up256((size_t)n * 4)),
                      (unsigned long long *)(B + kCtrlBytes), kNoAllocMaxGrid, B, seeds, gains,
                      num_seeds, coverage, d_status, st);
    if (s != IM_OK) return s;
    int hstatus = 0;
    IM_CUDA(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (hstatus != kDevOk) return map_dev_status(hstatus, "im_max_k_cover_noalloc");
    return IM_OK;
}

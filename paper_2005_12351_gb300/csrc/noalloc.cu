// noalloc.cu -- fmm_morton_order_noalloc: the Morton order of a point set
// without any device allocation.
//
// Some callers cannot allocate device memory while they call this library:
// code running inside a custom allocator or a memory-pool callback (an
// allocation there would re-enter the allocator), runtimes that hand the
// library a fixed arena and forbid cudaMalloc/cudaFree because those calls
// synchronise the whole device, and latency-critical loops where an
// allocation would stall other streams.  For them this entry point runs the
// same kernels as fmm_morton_order (bounding box, keys, stable radix sort)
// with its scratch in a file-scope device array sized for at most
// FMM_NOALLOC_MAX_POINTS points.  The array exists on every GPU that loads
// the library and stays allocated until the process exits.
#include <mutex>

#include "fmm_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = FMM_NOALLOC_MAX_POINTS;
constexpr int64_t kHistWords = fmm::radix_hist_words(kMaxPoints);
constexpr size_t kOffKeys2 = 0;                                          // uint64 [max]
constexpr size_t kOffIdx2 = kOffKeys2 + 8 * (size_t)kMaxPoints;          // uint32 [max]
constexpr size_t kOffHist = kOffIdx2 + 4 * (size_t)kMaxPoints;           // sort scratch
constexpr size_t kOffBox = kOffHist + 4 * (size_t)kHistWords;            // 6 x uint64 + 4 x f64
constexpr size_t kOffErr = kOffBox + 256;                                // int error word
constexpr size_t kScratchBytes = kOffErr + 256;

// Shared by every call on a device: each call leaves its contents behind.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
fmm_status scratch_address(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return FMM_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return FMM_OK;
}

}  // namespace

extern "C" fmm_status fmm_morton_order_noalloc(void *cuda_stream, const double *positions,
                                               int64_t n, uint64_t *keys_out, int32_t *perm_out)
{
    if (n < 0) return FMM_EINVAL;
    if (n > kMaxPoints) return FMM_EBUDGET;       // larger than the fixed scratch array
    unsigned char *base = nullptr;
    if (n == 0) {
        // the per-device set-up alone: load the kernels and this file's module
        // (which holds the scratch array), look up its address, raise the
        // sort's shared-memory limit -- everything a later call would
        // otherwise do on its first use
        fmm::morton_order_prepare();
        return scratch_address(&base);
    }
    if (!positions || !keys_out || !perm_out) return FMM_EINVAL;
    fmm_status st = scratch_address(&base);
    if (st != FMM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int *err = (int *)(base + kOffErr);
    // only the error word must start at zero; the sort clears its own
    // counters, and every other region is fully written before it is read
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    int64_t launches = 0;
    fmm::morton_order_raw(s, positions, n, keys_out, (uint32_t *)perm_out,
                          (uint64_t *)(base + kOffKeys2), (uint32_t *)(base + kOffIdx2),
                          (uint32_t *)(base + kOffHist), (unsigned long long *)(base + kOffBox), (double *)(base + kOffBox) + 8,
                          err, &launches);
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    if (herr & fmm::kErrNonFinite) return FMM_EINVAL;
    return (herr & fmm::kErrSortWait) ? FMM_ETIMEOUT : FMM_OK;
}

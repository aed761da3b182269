// noalloc.cu — an entry point for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running inside a
// pre-sized memory pool that already owns all of the device's memory, or a
// plug-in that must not change the process's device footprint after
// start-up.  For them,
// nl_k_gemv_residual_noalloc computes the same single-precision residual and
// norm as nl_k_gemv_residual, but keeps its scratch (one partial sum per
// block of eight rows, and the finishing counter) in a fixed array that is
// part of the library image, instead of asking the allocator for it.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace nl {

// Largest N accepted by the entry point, and the scratch it needs:
// ceil(N / 8) doubles of per-block partial sums plus one counter word.
constexpr int kNoAllocMaxN = 32768;
constexpr size_t kNoAllocPartials = (kNoAllocMaxN + 7) / 8;
constexpr size_t kNoAllocBytes = kNoAllocPartials * sizeof(double) + 256;

// Every GPU that loads the library holds these 33 KB until the process ends.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array (a host-side name of a __device__ array is
// not a device address).  It is looked up again on every call made outside a
// stream capture, so an address cached before a device reset (which tears the
// context down and loads the module again) is never used; during a capture
// the address cached by the last call on that device is used, so the first
// call on a device must come before any capture.
static constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static nl_status scratch_for_current_device(cudaStream_t st, void** out)
{
    int dev = 0;
    NL_CUDA_OK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gemv_residual_noalloc: device index %d out of range", dev);
        return NL_EINVAL;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NL_CUDA_OK(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("gemv_residual_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return NL_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NL_OK;
}

}  // namespace nl

using namespace nl;

extern "C" nl_status nl_k_gemv_residual_noalloc(int64_t N, const float* A, int64_t ld, const float* b, const float* u,
                                                float* r, double* rnorm_dev, void* stream)
{
    if (N < 1 || N > kNoAllocMaxN || !A || !u || !r || ld < N) {
        set_error("nl_k_gemv_residual_noalloc: need 1 <= N <= %d (got %lld), non-NULL A, u, r and ld >= N",
                  kNoAllocMaxN, (long long)N);
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    nl_status s = scratch_for_current_device(st, &scratch);
    if (s != NL_OK) return s;
    double* partial = (double*)scratch;
    unsigned* counter = (unsigned*)((char*)scratch + kNoAllocPartials * sizeof(double));
    // the finishing counter must start at zero whatever the last call left
    NL_CUDA_OK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    return launch_gemv_residual((int)N, A, ld, b, u, r, partial, counter, rnorm_dev, st);
}

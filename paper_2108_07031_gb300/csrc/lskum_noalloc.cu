// lskum_residue_noalloc: the residue reduction for callers that cannot
// allocate device memory.
//
// Some host programs may not call cudaMalloc at all: code running inside a
// CUDA-graph capture it does not own, a plug-in whose host framework owns
// every device allocation (a fixed memory pool with its own accounting), or
// an embedded runtime that forbids allocation after start-up. They still
// need the residue of a residual they already hold. This entry point computes
// it with no allocation: the per-block partial sums live in a file-scope
// __device__ array that exists once per device for the life of the process.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "lskum_internal.h"

namespace lskum {
namespace {

constexpr int kNoAllocBlock = 256;
constexpr int kNoAllocPerBlock = 8192;      // points reduced by one block
constexpr int kNoAllocMaxPartials = 8192;   // 64 KiB of partial sums per device
constexpr int kMaxDevices = 64;

// Partial sums of the residue. In host code this name is only a stand-in for
// the device array: it is never dereferenced or passed to a kernel from the
// host; kernels receive the device address from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

std::mutex g_setup_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kNoAllocBlock)
k_noalloc_partials(const double* __restrict__ R, int64_t n, double* __restrict__ scratch) {
    const int64_t base = int64_t(blockIdx.x) * kNoAllocPerBlock;
    double s = 0.0;
    for (int k = threadIdx.x; k < kNoAllocPerBlock; k += kNoAllocBlock) {
        const int64_t i = base + k;
        if (i < n) {
            const double r = R[4 * i];  // mass component of point i
            s += r * r;
        }
    }
    __shared__ double part[kNoAllocBlock / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kNoAllocBlock / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) scratch[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(512)
k_noalloc_final(const double* __restrict__ scratch, int nblocks, int64_t n, double* out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 512) s += scratch[b];
    __shared__ double part[16];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < 16 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) *out = sqrt(t) / double(n);
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress allocates nothing) and kept for the life of
// the process. A device reset reloads the module at another address, which
// makes the kept address stale; the header states that the entry point is not
// to be called on a device after it was reset.
int scratch_for_current_device(double** ptr, std::string& err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return LSKUM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device ordinal out of range";
        return LSKUM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || p == nullptr) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LSKUM_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *ptr = g_scratch[dev];
    return LSKUM_OK;
}

}  // namespace
}  // namespace lskum

extern "C" int lskum_residue_noalloc(const double* R, int64_t n, double* out, void* stream) {
    using namespace lskum;
    if (!R || !out) {
        set_last_error("lskum_residue_noalloc: null device pointer");
        return LSKUM_ERR_INVALID_ARG;
    }
    const int64_t max_n = int64_t(kNoAllocMaxPartials) * kNoAllocPerBlock;
    if (n < 1 || n > max_n) {
        set_last_error("lskum_residue_noalloc: n = " + std::to_string(n) + " outside [1, " +
                       std::to_string(max_n) + "] (the fixed scratch holds " +
                       std::to_string(kNoAllocMaxPartials) + " partial sums of " +
                       std::to_string(kNoAllocPerBlock) + " points each)");
        return LSKUM_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    std::string err;
    int rc = scratch_for_current_device(&scratch, err);
    if (rc != LSKUM_OK) {
        set_last_error("lskum_residue_noalloc: " + err);
        return rc;
    }
    const int nblocks = int((n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_partials<<<nblocks, kNoAllocBlock, 0, s>>>(R, n, scratch);
    k_noalloc_final<<<1, 512, 0, s>>>(scratch, nblocks, n, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("lskum_residue_noalloc launch: ") + cudaGetErrorString(e));
        return LSKUM_ERR_CUDA;
    }
    return LSKUM_OK;
}

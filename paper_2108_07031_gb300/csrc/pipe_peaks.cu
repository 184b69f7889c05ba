// Arithmetic-pipe throughput probe for the roofline denominators of the
// solver kernels: FP64 FMA, FP32 FMA, MUFU ex2 (FP32) and the FP64 libdevice
// calls the flux kernel leans on (erfc, exp, log, sqrt, reciprocal).
//
// The flux residual is a stencil gather whose per-neighbour cost is dominated
// by FP64 arithmetic (kinetic split fluxes with erfc/exp, q -> primitive
// conversions with exp/log), so its roofline is the FP64 pipe, not HBM. The
// measured numbers printed here are the peaks the benchmark divides by.
//
// Output: one JSON object on stdout. Every kernel writes one value per thread
// into a buffer sized grid*block, so all stores are in bounds.

#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
    exit(1); } } while (0)

constexpr int kIters = 4096;
constexpr int kChains = 8;

__global__ void fp64_fma_kernel(double* out, double a, double b) {
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fp32_fma_kernel(float* out, float a, float b) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void mufu_ex2_kernel(float* out, float a) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = -1.0f - threadIdx.x * 1e-6f - c * 1e-3f;
    for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = ex2_approx(acc[c]) * a - 1.0f;
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 library-call throughput: op 0 erfc, 1 exp, 2 log, 3 sqrt, 4 1/x.
template <int OP>
__global__ void fp64_call_kernel(double* out, double a) {
    double acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = 0.5 + threadIdx.x * 1e-6 + c * 1e-3;
    for (int it = 0; it < kIters / 64; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = acc[c];
            double r;
            if (OP == 0) r = erfc(v);
            else if (OP == 1) r = exp(-v);
            else if (OP == 2) r = log(v + 1.0);
            else if (OP == 3) r = sqrt(v + 1.0);
            else r = 1.0 / (v + 1.0);
            acc[c] = fma(r, a, 0.25);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc[0] + acc[1] + acc[2] + acc[3];
}

template <typename F>
static double time_ms(F launch, int reps) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    launch();  // warm-up
    CK(cudaDeviceSynchronize());
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(e0));
        launch();
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    std::sort(t.begin(), t.end());
    return t[0];
}

int main() {
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, 0));
    int sms = prop.multiProcessorCount;
    const int block = 256;
    const int grid = sms * 8;
    const size_t nthreads = size_t(grid) * block;
    double* d64 = nullptr;
    float* d32 = nullptr;
    CK(cudaMalloc(&d64, nthreads * sizeof(double)));
    CK(cudaMalloc(&d32, nthreads * sizeof(float)));

    const int reps = 5;
    double t64 = time_ms([&] { fp64_fma_kernel<<<grid, block>>>(d64, 0.999999, 1e-7); }, reps);
    double t32 = time_ms([&] { fp32_fma_kernel<<<grid, block>>>(d32, 0.9999f, 1e-5f); }, reps);
    double tmu = time_ms([&] { mufu_ex2_kernel<<<grid, block>>>(d32, 0.5f); }, reps);
    CK(cudaGetLastError());
    double fma64 = double(nthreads) * kIters * kChains;
    double fma32 = double(nthreads) * kIters * kChains;
    double ex2 = double(nthreads) * (kIters / 4) * kChains;
    double ncall = double(nthreads) * (kIters / 64) * 4;
    double tc[5];
    tc[0] = time_ms([&] { fp64_call_kernel<0><<<grid, block>>>(d64, 0.5); }, reps);
    tc[1] = time_ms([&] { fp64_call_kernel<1><<<grid, block>>>(d64, 0.5); }, reps);
    tc[2] = time_ms([&] { fp64_call_kernel<2><<<grid, block>>>(d64, 0.5); }, reps);
    tc[3] = time_ms([&] { fp64_call_kernel<3><<<grid, block>>>(d64, 0.5); }, reps);
    tc[4] = time_ms([&] { fp64_call_kernel<4><<<grid, block>>>(d64, 0.5); }, reps);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());

    printf("{\"device\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\", "
           "\"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, \"mufu_ex2_gops\": %.1f, "
           "\"fp64_fma_per_sm_per_clk_at_max\": %.3f, "
           "\"fp64_calls_gcalls_per_s\": {\"erfc\": %.2f, \"exp\": %.2f, \"log\": %.2f, "
           "\"sqrt\": %.2f, \"rcp\": %.2f}, \"l2_bytes\": %d, \"clock_khz\": %d}\n",
           prop.name, sms, prop.major, prop.minor,
           2.0 * fma64 / (t64 * 1e-3) / 1e12, 2.0 * fma32 / (t32 * 1e-3) / 1e12,
           ex2 / (tmu * 1e-3) / 1e9,
           fma64 / (t64 * 1e-3) / (double(sms) * 2.07e9),
           ncall / (tc[0] * 1e-3) / 1e9, ncall / (tc[1] * 1e-3) / 1e9,
           ncall / (tc[2] * 1e-3) / 1e9, ncall / (tc[3] * 1e-3) / 1e9,
           ncall / (tc[4] * 1e-3) / 1e9, prop.l2CacheSize, 0);
    CK(cudaFree(d64));
    CK(cudaFree(d32));
    return 0;
}

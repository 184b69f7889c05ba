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

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int kIters = 4096;
constexpr int kChains = 8;

// CHAINS independent FMA chains per thread; thread 0 of every block also
// records the SM cycles the block ran for (cycles[blockIdx.x]), so the host
// can tell the SM clock during the run from the elapsed time.
template <int CHAINS>
__global__ void fp64_fma_kernel(double* out, double a, double b, long long* cycles) {
    const long long c0 = clock64();
    const unsigned long long t0 = global_ns();
    double acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < kIters * kChains / CHAINS; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[2 * blockIdx.x] = clock64() - c0;
        cycles[2 * blockIdx.x + 1] = (long long)(global_ns() - t0);
    }
}

// Sustained FP64 FMA rate: every thread keeps 8 independent FMA chains going
// until `window_ns` after its own start (global timer), so all warps of an SM
// stay busy to the end (a fixed amount of work per thread leaves a ragged
// tail in which few warps feed the pipe). The loop is also capped at
// max_chunks chunks. Each thread adds its FMA count to *fmas.
__global__ void fp64_window_kernel(double* out, double a, double b, unsigned long long window_ns,
                                   long long max_chunks, unsigned long long* fmas) {
    const unsigned long long t_end = global_ns() + window_ns;
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    long long chunks = 0;
    while (chunks < max_chunks) {
        for (int it = 0; it < 64; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
        }
        ++chunks;
        if (global_ns() >= t_end) break;
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    atomicAdd(fmas, (unsigned long long)(chunks * 64 * kChains));
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

    long long* dcyc = nullptr;
    CK(cudaMalloc(&dcyc, 2 * size_t(grid) * sizeof(long long)));
    const int reps = 5;
    // FP64: exactly one wave of resident blocks (a partial second wave would
    // run at lower occupancy and understate the pipe's rate)
    int occ8 = 0, occ16 = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ8, fp64_fma_kernel<8>, block, 0));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ16, fp64_fma_kernel<16>, block, 0));
    const int g8 = sms * std::min(occ8, 8), g16 = sms * std::min(occ16, 8);
    double t64 = time_ms([&] { fp64_fma_kernel<8><<<g8, block>>>(d64, 0.999999, 1e-7, dcyc); }, reps);
    std::vector<long long> cyc(2 * size_t(g8));
    CK(cudaMemcpy(cyc.data(), dcyc, 2 * size_t(g8) * sizeof(long long), cudaMemcpyDeviceToHost));
    double cyc_sum = 0, ns_sum = 0;
    for (int i = 0; i < g8; ++i) {
        cyc_sum += double(cyc[2 * i]);
        ns_sum += double(cyc[2 * i + 1]);
    }
    double t64b = time_ms([&] { fp64_fma_kernel<16><<<g16, block>>>(d64, 0.999999, 1e-7, dcyc); }, reps);
    const double fma64_8 = double(g8) * block * kIters * kChains;
    unsigned long long* dfmas = nullptr;
    CK(cudaMalloc(&dfmas, sizeof(unsigned long long)));
    double win_tflops = 0;
    for (int r = 0; r < 3; ++r) {  // 20 ms windows, best of 3
        CK(cudaMemset(dfmas, 0, sizeof(unsigned long long)));
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        CK(cudaEventCreate(&a1));
        CK(cudaEventRecord(a0));
        fp64_window_kernel<<<g8, block>>>(d64, 0.999999, 1e-7, 20000000ull, 4096ll, dfmas);
        CK(cudaEventRecord(a1));
        CK(cudaEventSynchronize(a1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a0, a1));
        unsigned long long n = 0;
        CK(cudaMemcpy(&n, dfmas, sizeof(n), cudaMemcpyDeviceToHost));
        win_tflops = std::max(win_tflops, 2.0 * double(n) / (ms * 1e-3) / 1e12);
        CK(cudaEventDestroy(a0));
        CK(cudaEventDestroy(a1));
    }
    CK(cudaFree(dfmas));
    const double fma64_16 = double(g16) * block * kIters * kChains;
    double t32 = time_ms([&] { fp32_fma_kernel<<<grid, block>>>(d32, 0.9999f, 1e-5f); }, reps);
    double tmu = time_ms([&] { mufu_ex2_kernel<<<grid, block>>>(d32, 0.5f); }, reps);
    CK(cudaGetLastError());
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

    // SM clock during the run: the blocks' SM cycles over their global-timer
    // nanoseconds
    const double clk_ghz = ns_sum > 0 ? cyc_sum / ns_sum : 0.0;
    const double block_ms = ns_sum / g8 * 1e-6;
    long long ns_min = cyc[1], ns_max = cyc[1];
    for (int i = 0; i < g8; ++i) {
        ns_min = std::min(ns_min, cyc[2 * i + 1]);
        ns_max = std::max(ns_max, cyc[2 * i + 1]);
    }
    fprintf(stderr, "fp64 probe: %d blocks/SM resident (occupancy), block time min %.3f max %.3f ms\n",
            std::min(occ8, 8), ns_min * 1e-6, ns_max * 1e-6);
    printf("{\"device\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\", "
           "\"fp64_fma_tflops_sustained_window\": %.4f, "
           "\"fp64_fma_tflops\": %.4f, \"fp64_fma_tflops_16_chains\": %.4f, "
           "\"sm_clock_ghz_during_fp64\": %.3f, \"fp64_block_ms\": %.3f, \"fp64_kernel_ms\": %.3f, "
           "\"fp64_fma_per_sm_per_clk\": %.3f, "
           "\"fp32_fma_tflops\": %.3f, \"mufu_ex2_gops\": %.1f, "
           "\"fp64_fma_per_sm_per_clk_at_max\": %.3f, "
           "\"fp64_calls_gcalls_per_s\": {\"erfc\": %.2f, \"exp\": %.2f, \"log\": %.2f, "
           "\"sqrt\": %.2f, \"rcp\": %.2f}, \"l2_bytes\": %d, \"clock_khz\": %d}\n",
           prop.name, sms, prop.major, prop.minor, win_tflops,
           2.0 * fma64_8 / (t64 * 1e-3) / 1e12, 2.0 * fma64_16 / (t64b * 1e-3) / 1e12, clk_ghz,
           block_ms, t64,
           fma64_8 / (t64 * 1e-3) / (double(sms) * clk_ghz * 1e9), 2.0 * fma32 / (t32 * 1e-3) / 1e12,
           ex2 / (tmu * 1e-3) / 1e9,
           fma64_8 / (t64 * 1e-3) / (double(sms) * 2.07e9),
           ncall / (tc[0] * 1e-3) / 1e9, ncall / (tc[1] * 1e-3) / 1e9,
           ncall / (tc[2] * 1e-3) / 1e9, ncall / (tc[3] * 1e-3) / 1e9,
           ncall / (tc[4] * 1e-3) / 1e9, prop.l2CacheSize, 0);
    CK(cudaFree(d64));
    CK(cudaFree(d32));
    CK(cudaFree(dcyc));
    return 0;
}

// Warm-start surrogate: a coordinate/condition MLP trained and evaluated on
// the GPU with hand-written BF16 tensor-core kernels (FP32 accumulation).
//
// Network (include/lskum_mlp.h): 21 input features (zero-padded to 32) ->
// 5 hidden layers of 256 (tanh) -> 4 outputs (linear): six linear layers.
// Z_l = X_l W_l^T + b_l, X_{l+1} = tanh(Z_l). Weights are kept in FP32
// (Adam master copy) and in BF16 (W) for the GEMMs;
// activations are stored FP32 (for tanh') and BF16 (GEMM input).
//
// GEMM: C[M x N] = A[M x K] B[K x N], A and B BF16 in global memory with
// arbitrary element strides (so the forward X W^T, the backward dZ W and
// the weight gradient dZ^T X all use one kernel), staged through shared
// memory as A[m][k] and B[n][k] (k contiguous), 64 x 64 tiles per block of
// four warps, mma.sync m16n8k16 (bf16 x bf16 -> f32).

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lskum_mlp.h"
#include "lskum_internal.h"

namespace mlpk {

constexpr int kTile = 64;
constexpr int kKt = 32;             // k per shared-memory stage
constexpr int kSmemPad = 8;         // bf16 padding per row (bank spread)
constexpr int kLayers = LSKUM_MLP_LAYERS;
constexpr int kWidth = LSKUM_MLP_WIDTH;
constexpr int kIn = LSKUM_MLP_IN_PADDED;
constexpr int kOut = LSKUM_MLP_OUT;

__host__ __device__ inline int layer_in(int l) { return l == 0 ? kIn : kWidth; }
__host__ __device__ inline int layer_out(int l) { return l == kLayers - 1 ? kOut : kWidth; }

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

enum Epilogue { kStoreF32 = 0, kBiasTanh = 1, kBiasLinear = 2 };

// C = A B with A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].
// Epilogue kBiasTanh: Zf = C + bias[n], Af = tanh(Zf), Ab = bf16(Af);
// kBiasLinear: Cf = C + bias[n]; kStoreF32: Cf = C. Row-major outputs with
// leading dimension ldc.
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int64_t sam,
                                                   int64_t sak, const __nv_bfloat16* __restrict__ B,
                                                   int64_t sbk, int64_t sbn, int M, int N, int K,
                                                   const float* __restrict__ bias,
                                                   float* __restrict__ Cf,
                                                   __nv_bfloat16* __restrict__ Cb, int64_t ldc,
                                                   int kchunk) {
    __shared__ __align__(16) __nv_bfloat16 As[kTile][kKt + kSmemPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[kTile][kKt + kSmemPad];
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    const bool a_kfast = sak == 1, b_kfast = sbk == 1;
    // split-K: block z reduces k in [z kchunk, (z+1) kchunk) into its own
    // slice of Cf (summed afterwards in slice order)
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    if (EPI == kStoreF32) Cf += int64_t(blockIdx.z) * M * ldc;
    for (int k0 = kbeg; k0 < kend; k0 += kKt) {
        // stage: 64 x 32 elements of each operand, 16 per thread; consecutive
        // threads walk the operand's contiguous dimension (coalesced loads)
        for (int e = tid; e < kTile * kKt; e += 128) {
            const int r = a_kfast ? e / kKt : e % kTile;
            const int kk = a_kfast ? e % kKt : e / kTile;
            const int gm = m0 + r, gk = k0 + kk;
            As[r][kk] = (gm < M && gk < kend) ? A[gm * sam + gk * sak] : zero;
        }
        for (int e = tid; e < kTile * kKt; e += 128) {
            const int r = b_kfast ? e / kKt : e % kTile;
            const int kk = b_kfast ? e % kKt : e / kTile;
            const int gn = n0 + r, gk = k0 + kk;
            Bs[r][kk] = (gn < N && gk < kend) ? B[gk * sbk + gn * sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kKt; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + i * 16 + grp;
                const int col = ks + tig * 2;
                af[i][0] = ld_pair(&As[row][col]);
                af[i][1] = ld_pair(&As[row + 8][col]);
                af[i][2] = ld_pair(&As[row][col + 8]);
                af[i][3] = ld_pair(&As[row + 8][col + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + grp;
                const int k = ks + tig * 2;
                bfr[j][0] = ld_pair(&Bs[n][k]);
                bfr[j][1] = ld_pair(&Bs[n][k + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + i * 16 + grp + ((r & 2) ? 8 : 0);
                const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                if (EPI != kStoreF32) v += bias[n];
                if (EPI == kBiasTanh) {
                    const float a = tanhf(v);
                    Cf[int64_t(m) * ldc + n] = a;
                    Cb[int64_t(m) * ldc + n] = __float2bfloat16(a);
                } else {
                    Cf[int64_t(m) * ldc + n] = v;
                }
            }
}

// Narrow output layer, C(m, n) = sum_k X(m, k) W(n, k) + bias(n) for N <=
// kNarrowMax outputs (the network's 4-wide last layer): one warp per row of
// X, each lane a 16-byte chunk of eight k per step (a row of 256 is one
// coalesced 512-byte read), W staged once per block in shared memory, FP32
// accumulation of the exact BF16 products, a butterfly sum over the lanes.
// The tiled GEMMs would leave 60 of their 64 (or 124 of 128) columns idle.
// Requirements (checked by the caller): K a multiple of 8, X rows and W
// 16-byte aligned, N <= kNarrowMax, N x K <= kNarrowW.
constexpr int kNarrowMax = 8;
constexpr int kNarrowW = 4096;  // bf16 elements of W in shared memory (8 KB)
constexpr int kNarrowRows = 8;  // rows (warps) per block

__global__ void __launch_bounds__(32 * kNarrowRows) k_gemm_narrow(
    const __nv_bfloat16* __restrict__ X, int64_t sxm, const __nv_bfloat16* __restrict__ W, int M,
    int N, int K, const float* __restrict__ bias, float* __restrict__ C, int64_t ldc) {
    __shared__ __align__(16) __nv_bfloat16 Ws[kNarrowW];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int e = tid * 8; e < N * K; e += 32 * kNarrowRows * 8)
        *reinterpret_cast<uint4*>(&Ws[e]) = *reinterpret_cast<const uint4*>(W + e);
    __syncthreads();
    const int m = blockIdx.x * kNarrowRows + (tid >> 5);
    if (m >= M) return;
    float acc[kNarrowMax];
#pragma unroll
    for (int n = 0; n < kNarrowMax; ++n) acc[n] = 0.f;
    const __nv_bfloat16* x = X + int64_t(m) * sxm;
    for (int k0 = lane * 8; k0 < K; k0 += 256) {
        const uint4 xv = *reinterpret_cast<const uint4*>(x + k0);
        const __nv_bfloat162* xp = reinterpret_cast<const __nv_bfloat162*>(&xv);
#pragma unroll
        for (int n = 0; n < kNarrowMax; ++n) {
            if (n < N) {
                const uint4 wv = *reinterpret_cast<const uint4*>(&Ws[n * K + k0]);
                const __nv_bfloat162* wp = reinterpret_cast<const __nv_bfloat162*>(&wv);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 xf = __bfloat1622float2(xp[q]);
                    const float2 wf = __bfloat1622float2(wp[q]);
                    acc[n] = fmaf(xf.x, wf.x, acc[n]);
                    acc[n] = fmaf(xf.y, wf.y, acc[n]);
                }
            }
        }
    }
#pragma unroll
    for (int n = 0; n < kNarrowMax; ++n)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[n] += __shfl_xor_sync(0xffffffffu, acc[n], o);
    if (lane < N) {
        float v = acc[0];
#pragma unroll
        for (int n = 1; n < kNarrowMax; ++n)
            if (lane == n) v = acc[n];
        C[int64_t(m) * ldc + lane] = v + bias[lane];
    }
}

// Pipelined GEMM for the aligned, large shapes: 128 x 128 tiles per block of
// eight warps (each 64 x 32), k in stages of 32 moved global -> shared by
// cp.async (16-byte chunks, three stages in flight), operand fragments by
// ldmatrix -- plain for an operand whose contraction index is contiguous in
// memory (X and W in the forward pass), transposed for one whose row index
// is (dZ^T and X in the weight gradient, W in dZ W) -- and the same
// mma.sync m16n8k16 and epilogues as k_gemm_bf16. Requirements (checked by
// the caller): the contiguous dimension of each operand a multiple of 8
// elements with 16-byte aligned rows, kchunk a multiple of 32.
constexpr int kTB = 128;
constexpr int kTK = 32;
static_assert(kTK == kKt, "split-K slices hold whole k stages of both GEMM kernels");
constexpr int kStages = 3;

template <bool KFAST>
struct TileGeo {  // shared-memory tile: [rows][ld] bf16, 16 bytes of row padding
    static constexpr int ld = KFAST ? kTK + 8 : kTB + 8;
    static constexpr int elems = KFAST ? kTB * ld : kTK * ld;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return uint32_t(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled, nothing is read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t r[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t r[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

constexpr size_t tc_smem_bytes(bool ak, bool bk) {
    return sizeof(__nv_bfloat16) * kStages *
           size_t((ak ? TileGeo<true>::elems : TileGeo<false>::elems) +
                  (bk ? TileGeo<true>::elems : TileGeo<false>::elems));
}

template <int EPI, bool AK, bool BK>
__global__ void __launch_bounds__(256) k_gemm_bf16_tc(const __nv_bfloat16* __restrict__ A, int64_t sam,
                                                      int64_t sak, const __nv_bfloat16* __restrict__ B,
                                                      int64_t sbk, int64_t sbn, int M, int N, int K,
                                                      const float* __restrict__ bias,
                                                      float* __restrict__ Cf,
                                                      __nv_bfloat16* __restrict__ Cb, int64_t ldc,
                                                      int kchunk) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* sB = sA + kStages * TileGeo<AK>::elems;
    const int m0 = blockIdx.y * kTB, n0 = blockIdx.x * kTB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int ktiles = kend > kbeg ? (kend - kbeg + kTK - 1) / kTK : 0;
    if (EPI == kStoreF32) Cf += int64_t(blockIdx.z) * M * ldc;

    // one stage: 512 16-byte chunks of each operand tile, two per thread
    auto load_stage = [&](int stage, int kt) {
        const int k0 = kbeg + kt * kTK;
        __nv_bfloat16* a = sA + stage * TileGeo<AK>::elems;
        __nv_bfloat16* b = sB + stage * TileGeo<BK>::elems;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * 256;
            if (AK) {
                const int r = c >> 2, kc = (c & 3) * 8, gm = m0 + r, gk = k0 + kc;
                const bool ok = gm < M && gk < kend;
                cp_async16(smem_u32(a + r * TileGeo<AK>::ld + kc), ok ? A + int64_t(gm) * sam + gk : A, ok);
            } else {
                const int r = c >> 4, mc = (c & 15) * 8, gk = k0 + r, gm = m0 + mc;
                const bool ok = gk < kend && gm < M;
                cp_async16(smem_u32(a + r * TileGeo<AK>::ld + mc), ok ? A + int64_t(gk) * sak + gm : A, ok);
            }
            if (BK) {
                const int r = c >> 2, kc = (c & 3) * 8, gn = n0 + r, gk = k0 + kc;
                const bool ok = gn < N && gk < kend;
                cp_async16(smem_u32(b + r * TileGeo<BK>::ld + kc), ok ? B + int64_t(gn) * sbn + gk : B, ok);
            } else {
                const int r = c >> 4, nc = (c & 15) * 8, gk = k0 + r, gn = n0 + nc;
                const bool ok = gk < kend && gn < N;
                cp_async16(smem_u32(b + r * TileGeo<BK>::ld + nc), ok ? B + int64_t(gk) * sbk + gn : B, ok);
            }
        }
    };

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

#pragma unroll
    for (int st = 0; st < kStages - 1; ++st) {
        if (st < ktiles) load_stage(st, st);
        cp_async_commit();
    }
    for (int kt = 0; kt < ktiles; ++kt) {
        cp_async_wait<kStages - 2>();  // stage kt has landed (this thread's copies)
        __syncthreads();                // ... everyone's; stage kt-1 is no longer read
        const int nxt = kt + kStages - 1;
        if (nxt < ktiles) load_stage(nxt % kStages, nxt);
        cp_async_commit();
        const __nv_bfloat16* a = sA + (kt % kStages) * TileGeo<AK>::elems;
        const __nv_bfloat16* b = sB + (kt % kStages) * TileGeo<BK>::elems;
#pragma unroll
        for (int ks = 0; ks < kTK; ks += 16) {
            uint32_t af[4][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (AK) {  // [m][k]: matrices (m 0-7 | 8-15) x (k 0-7 | 8-15)
                    const int row = wm + i * 16 + (lane & 15), col = ks + (lane >> 4) * 8;
                    ldsm_x4(smem_u32(a + row * TileGeo<AK>::ld + col), af[i]);
                } else {   // [k][m], transposed on load
                    const int row = ks + (lane & 7) + (lane >> 4) * 8;
                    const int col = wm + i * 16 + ((lane >> 3) & 1) * 8;
                    ldsm_x4_t(smem_u32(a + row * TileGeo<AK>::ld + col), af[i]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j += 2) {  // two n8 fragments per ldmatrix
                uint32_t r[4];
                if (BK) {  // [n][k]
                    const int row = wn + j * 8 + (lane & 7) + (lane >> 4) * 8;
                    const int col = ks + ((lane >> 3) & 1) * 8;
                    ldsm_x4(smem_u32(b + row * TileGeo<BK>::ld + col), r);
                } else {   // [k][n], transposed on load
                    const int row = ks + (lane & 7) + ((lane >> 3) & 1) * 8;
                    const int col = wn + j * 8 + (lane >> 4) * 8;
                    ldsm_x4_t(smem_u32(b + row * TileGeo<BK>::ld + col), r);
                }
                bfr[j][0] = r[0];
                bfr[j][1] = r[1];
                bfr[j + 1][0] = r[2];
                bfr[j + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
    }
    cp_async_wait<0>();

    const int grp = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + i * 16 + grp + ((r & 2) ? 8 : 0);
                const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                if (EPI != kStoreF32) v += bias[n];
                if (EPI == kBiasTanh) {
                    const float t = tanhf(v);
                    Cf[int64_t(m) * ldc + n] = t;
                    Cb[int64_t(m) * ldc + n] = __float2bfloat16(t);
                } else {
                    Cf[int64_t(m) * ldc + n] = v;
                }
            }
}

// ------------------------------------------------- tcgen05 forward GEMM
// Z = X W^T + b (tanh or linear epilogue) of a hidden layer (256 outputs) on
// the fifth-generation tensor cores. One CTA of eight warps per 128-row tile
// of X and 128-column half of the outputs: it stages X[m0:m0+128, 0:K] and
// W[n0:n0+128, 0:K] (K <= 256: at most 2 x 64 KB) in shared memory with
// cp.async in K stages of 64 (one copy group each), and as each stage lands
// one thread issues its four tcgen05.mma (M 128, N 128, K 16, BF16 x BF16 ->
// FP32) into a 128-column accumulator in tensor memory, so the MMAs of a
// stage overlap the copies of the next; the last commit arrives on an
// mbarrier, and each warp reads a 32-lane x 64-column quarter of the
// accumulator back with tcgen05.ld for the epilogue (warp w: lanes 32 (w mod
// 4) .., columns 64 (w div 4) ..).
//
// Shared-memory operand layout: the no-swizzle K-major canonical form of the
// matrix descriptors: core matrices of 8 rows x 16 bytes (8 BF16 along K)
// stored as 128 contiguous bytes; core matrix (r/8, k/8) of an operand at
// byte (r/8) SBO + (k/8) LBO with LBO = 128 (next core matrix along K) and
// SBO = 16 K (next 8-row group). One MMA reads two core matrices along K, so
// consecutive MMAs advance both descriptors' start by 256 bytes.
constexpr int kUmmaM = 128, kUmmaN = 128, kUmmaK = 16, kUmmaStageK = 64, kUmmaThreads = 256;
constexpr int kUmmaOut = 256;  // outputs of a hidden layer (two CTAs' halves)

__host__ __device__ constexpr size_t umma_smem_bytes(int K) {
    return size_t(kUmmaM + kUmmaN) * size_t(K) * 2 + 16;  // A, B, mbarrier, TMEM address
}

// SM100 shared-memory matrix descriptor: bits [0,14) start address >> 4,
// [16,30) leading-dimension byte offset >> 4, [32,46) stride-dimension byte
// offset >> 4, [46,48) descriptor version 1, [61,64) layout 0 (no swizzle).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits [4,6) = 1), A and B BF16
// (bits [7,10) and [10,13) = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Waits for phase `parity` of the mbarrier at shared address `bar`, polling
// at most `limit` times (with a short sleep between polls); false when the
// limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(128);
    }
    return false;
}

// tcgen05.ld of 32 consecutive FP32 accumulator columns of this thread's
// tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// X: M x K BF16 row-major (K a multiple of 16, K <= 256, rows 16-byte
// aligned), W: 256 x K BF16 row-major, bias[256]; outputs row-major with 256
// columns: EPI kBiasTanh writes Cf = tanh(Z) and Cb = bf16(Cf), kBiasLinear
// Cf = Z. Grid (M / 128 rounded up, 2). `err` receives 1 if the accumulator
// wait ran out (the tile's outputs are then not written).
__device__ __forceinline__ void cp_async_wait_dyn(int n) {  // n in 0..3 groups may stay in flight
    if (n <= 0) cp_async_wait<0>();
    else if (n == 1) cp_async_wait<1>();
    else if (n == 2) cp_async_wait<2>();
    else cp_async_wait<3>();
}

template <int EPI>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_gemm_fwd_umma(const __nv_bfloat16* __restrict__ X,
                                                                   int M, int K,
                                                                   const __nv_bfloat16* __restrict__ W,
                                                                   const float* __restrict__ bias,
                                                                   float* __restrict__ Cf,
                                                                   __nv_bfloat16* __restrict__ Cb,
                                                                   int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kUmmaM, n0 = blockIdx.y * kUmmaN;
    const uint32_t sA = smem_u32(smem);
    const uint32_t sB = sA + uint32_t(kUmmaM * K * 2);
    const uint32_t bar = sB + uint32_t(kUmmaN * K * 2);
    const uint32_t tslot = bar + 8;
    const uint32_t sbo = uint32_t(K) * 16;  // bytes between 8-row groups
    const int kc = K / 8;                   // 16-byte chunks per row
    const int nst = (K + kUmmaStageK - 1) / kUmmaStageK;  // 1..4 stages

    // every stage's copies up front, one group per stage: chunk c of row r
    // lands in core matrix (r/8, c)
    for (int st = 0; st < nst; ++st) {
        const int c0 = st * (kUmmaStageK / 8), c1 = min(kc, c0 + kUmmaStageK / 8), w = c1 - c0;
        for (int i = tid; i < kUmmaM * w; i += kUmmaThreads) {
            const int r = i / w, c = c0 + (i - r * w), gm = m0 + r;
            const bool ok = gm < M;
            cp_async16(sA + uint32_t(r >> 3) * sbo + uint32_t(c) * 128 + uint32_t(r & 7) * 16,
                       ok ? X + int64_t(gm) * K + c * 8 : X, ok);
        }
        for (int i = tid; i < kUmmaN * w; i += kUmmaThreads) {
            const int r = i / w, c = c0 + (i - r * w);
            cp_async16(sB + uint32_t(r >> 3) * sbo + uint32_t(c) * 128 + uint32_t(r & 7) * 16,
                       W + int64_t(n0 + r) * K + c * 8, true);
        }
        cp_async_commit();
    }
    if (warp == 0) {  // 128 columns x 128 lanes of 32-bit accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tslot),
                     "r"(kUmmaN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    uint32_t tmem = 0;
    constexpr uint32_t idesc = umma_idesc_bf16_f32(kUmmaM, kUmmaN);
    for (int st = 0; st < nst; ++st) {
        cp_async_wait_dyn(nst - 1 - st);  // this thread's copies of stages 0..st have landed
        // the staged operands become visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();  // ... everyone's
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (st == 0) asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem) : "r"(tslot));
        if (tid == 0) {
            const int k1 = min(K, (st + 1) * kUmmaStageK) / kUmmaK;
            for (int ks = st * (kUmmaStageK / kUmmaK); ks < k1; ++ks) {
                const uint64_t da = umma_desc(sA + uint32_t(ks) * 256, 128, sbo);
                const uint64_t db = umma_desc(sB + uint32_t(ks) * 256, 128, sbo);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(ks));
            }
            if (st == nst - 1)
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                    : "memory");
        }
    }
    // the accumulators are complete when the mbarrier's phase 0 completes
    // (microseconds; the limit, ~0.5 s, only ends a wait that would not)
    const bool done = __all_sync(0xffffffffu, mbar_wait(bar, 0, 1 << 22));
    if (!done && lane == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (done) {
        const int q = warp & 3, h = warp >> 2;
        const int m = m0 + q * 32 + lane;  // this thread's row = its tensor-memory lane
        for (int cc = 0; cc < kUmmaN / 2; cc += 32) {
            const int c0 = h * (kUmmaN / 2) + cc;  // column within this CTA's half
            float v[32];
            tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), v);
            if (m < M) {
                const int n = n0 + c0;
                float4* of = reinterpret_cast<float4*>(Cf + int64_t(m) * kUmmaOut + n);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float4 o;
                    o.x = v[4 * j] + __ldg(bias + n + 4 * j);
                    o.y = v[4 * j + 1] + __ldg(bias + n + 4 * j + 1);
                    o.z = v[4 * j + 2] + __ldg(bias + n + 4 * j + 2);
                    o.w = v[4 * j + 3] + __ldg(bias + n + 4 * j + 3);
                    if (EPI == kBiasTanh) {
                        o.x = tanhf(o.x); o.y = tanhf(o.y); o.z = tanhf(o.z); o.w = tanhf(o.w);
                        __nv_bfloat162* ob =
                            reinterpret_cast<__nv_bfloat162*>(Cb + int64_t(m) * kUmmaOut + n + 4 * j);
                        ob[0] = __floats2bfloat162_rn(o.x, o.y);
                        ob[1] = __floats2bfloat162_rn(o.z, o.w);
                    }
                    of[j] = o;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kUmmaN));
}

// Features: per sample raw (x, y, wall distance, M, alpha_deg) ->
// [x/10, y/10, log(d + 1e-3)/5, (M - 0.55)/0.25, (alpha - 1)/5,
//  sin(P (x, y)), cos(P (x, y)) (8 projections each), 0 x 11 padding],
// stored FP32 (the caller-visible encoding) and BF16 (GEMM input).
__global__ void k_features(const float* __restrict__ raw, int64_t n, const float* __restrict__ proj,
                           float* __restrict__ feat) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* r = raw + 5 * i;
    float* f = feat + int64_t(kIn) * i;
    const float x = r[0], y = r[1];
    f[0] = x * 0.1f;
    f[1] = y * 0.1f;
    f[2] = logf(r[2] + 1e-3f) * 0.2f;
    f[3] = (r[3] - 0.55f) * 4.0f;
    f[4] = (r[4] - 1.0f) * 0.2f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float t = proj[2 * k] * x + proj[2 * k + 1] * y;
        f[5 + k] = sinf(t);
        f[13 + k] = cosf(t);
    }
#pragma unroll
    for (int k = 21; k < kIn; ++k) f[k] = 0.f;
}

// Sum of the split-K slices in slice order (deterministic).
__global__ void k_sum_slices(const float* __restrict__ part, int slices, int64_t n,
                             float* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < slices; ++z) s += part[int64_t(z) * n + i];
    out[i] = s;
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ dst) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// MSE loss pieces: dY = 2 (Y - T) / (n * 4), per-block partial sums of (Y-T)^2.
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Y, const float* __restrict__ T,
                                             int64_t n, float* __restrict__ dY,
                                             double* __restrict__ partial) {
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    double s = 0.0;
    if (i < n * kOut) {
        const float d = Y[i] - T[i];
        dY[i] = 2.0f * d / float(n * kOut);
        s = double(d) * d;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nb, int64_t count,
                               double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    *out = s / double(count);
}

// dZ = dA * (1 - A^2) (tanh'), FP32 and BF16 copies.
__global__ void k_tanh_back(const float* __restrict__ dA, const float* __restrict__ A, int64_t n,
                            float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZb) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = A[i];
    const float v = dA[i] * (1.0f - a * a);
    dZ[i] = v;
    dZb[i] = __float2bfloat16(v);
}

// db[c] = sum over rows of dZ[r][c], rows summed in a fixed order.
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ dZ, int rows, int cols,
                                                float* __restrict__ db) {
    __shared__ float sh[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.f;
    if (c < cols)
        for (int r = threadIdx.y; r < rows; r += 8) s += dZ[int64_t(r) * cols + c];
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += sh[k][threadIdx.x];
        db[c] = t;
    }
}

// Adam on the flat FP32 parameter vector; the BF16 copy W is refreshed after it.
struct LayerPtrs {
    int64_t w_off[kLayers];  // offsets of W_l and b_l in the flat vector
    int64_t b_off[kLayers];
    __nv_bfloat16* W[kLayers];
};

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_weights_bf16(const float* __restrict__ p, LayerPtrs L) {
    const int l = blockIdx.y;
    const int K = layer_in(l), N = layer_out(l);
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(K) * N) return;
    const int nrow = int(e / K), k = int(e % K);
    float w = p[L.w_off[l] + e];
    if (l == 0 && k >= 21) w = 0.f;  // padded inputs carry no weight
    L.W[l][e] = __float2bfloat16(w);
    (void)nrow;
}

}  // namespace mlpk

// ------------------------------------------------------------------ C ABI

using namespace mlpk;

struct lskum_mlp {
    cudaStream_t stream = nullptr;      // stream the handle's work runs on
    cudaStream_t own_stream = nullptr;  // the handle's own (created, destroyed by it)
    int64_t cap = 0;  // samples per call
    int64_t nparam = 0;
    LayerPtrs L{};
    float* p = nullptr;   // FP32 master parameters
    float* g = nullptr;   // gradients
    float* m = nullptr;   // Adam moments
    float* v = nullptr;
    float* proj = nullptr;  // 8 x 2 Fourier projection
    int64_t step = 0;
    // activations: Af[l] (FP32) and Ab[l] (BF16) for l = 0..kLayers (l = 0: features)
    float* Af[kLayers + 1] = {nullptr};
    __nv_bfloat16* Ab[kLayers + 1] = {nullptr};
    float* dA = nullptr;   // cap x 256 scratch
    float* slices = nullptr;  // split-K partial products of the weight gradients
    float* dZ = nullptr;   // cap x 256
    __nv_bfloat16* dZb = nullptr;
    double* partial = nullptr;
    double* loss_dev = nullptr;
    int gemm_path = LSKUM_MLP_GEMM_MMA_SYNC;
    int* err_dev = nullptr;  // set by a tcgen05 GEMM whose accumulator wait ran out
    std::vector<void*> allocs;
};

namespace {

int fail(int code, const std::string& m) {
    lskum::set_last_error(m);
    return code;
}

#define MLP_CUDA(x)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) return fail(LSKUM_ERR_CUDA, std::string(#x) + ": " +     \
                                                           cudaGetErrorString(e_));    \
    } while (0)

template <typename T>
cudaError_t alloc(lskum_mlp* h, T** p, int64_t count) {
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, sizeof(T) * size_t(count > 0 ? count : 1));
    if (e == cudaSuccess) h->allocs.push_back(raw);
    *p = static_cast<T*>(raw);
    return e;
}

inline unsigned blocks(int64_t n, int b) { return unsigned((n + b - 1) / b); }

constexpr int kMaxSlices = 32;

// The pipelined kernel's layout requirements (see k_gemm_bf16_tc); small
// outputs (the 4-wide output layer, the 32-wide input layer's weight
// gradient) stay on the 64 x 64 kernel.
bool tc_ok(const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbk, int64_t sbn, int M,
           int N, int K) {
    if (M < 64 || N < 64) return false;
    const bool ak = sak == 1, bk = sbk == 1;
    if ((!ak && sam != 1) || (!bk && sbn != 1)) return false;
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return false;
    if (ak ? (sam % 8 || K % 8) : (sak % 8 || M % 8)) return false;
    if (bk ? (sbn % 8 || K % 8) : (sbk % 8 || N % 8)) return false;
    return true;
}

template <int EPI, bool AK, bool BK>
cudaError_t launch_tc(lskum_mlp* h, dim3 grid, const __nv_bfloat16* A, int64_t sam, int64_t sak,
                      const __nv_bfloat16* B, int64_t sbk, int64_t sbn, int M, int N, int K,
                      const float* bias, float* Cf, __nv_bfloat16* Cb, int64_t ldc, int kchunk) {
    constexpr size_t smem = tc_smem_bytes(AK, BK);
    // the opt-in above 48 KB of dynamic shared memory (per device, so set on
    // every launch: a cheap host call next to a GEMM)
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_tc<EPI, AK, BK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_gemm_bf16_tc<EPI, AK, BK><<<grid, 256, smem, h->stream>>>(A, sam, sak, B, sbk, sbn, M, N, K, bias,
                                                                Cf, Cb, ldc, kchunk);
    return cudaGetLastError();
}

// The tcgen05 forward GEMM's requirements: 256 outputs, K a multiple of 16 up
// to 256 (16-byte rows), 16-byte aligned operands.
bool umma_ok(const void* X, const void* W, int N, int K) {
    return N == kUmmaOut && K % kUmmaK == 0 && K >= kUmmaK && K <= 256 &&
           !(reinterpret_cast<uintptr_t>(X) & 15) && !(reinterpret_cast<uintptr_t>(W) & 15);
}

template <int EPI>
cudaError_t launch_umma(lskum_mlp* h, const __nv_bfloat16* X, int M, int K, const __nv_bfloat16* W,
                        const float* bias, float* Cf, __nv_bfloat16* Cb) {
    // at least 60 KB, so at most three CTAs share an SM: their 128-column
    // accumulators fit its 512 tensor-memory columns and no allocation waits
    const size_t smem = std::max<size_t>(umma_smem_bytes(K), 60 * 1024);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_fwd_umma<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(umma_smem_bytes(256)));
    if (e != cudaSuccess) return e;
    const dim3 grid(blocks(M, kUmmaM), kUmmaOut / kUmmaN);
    k_gemm_fwd_umma<EPI><<<grid, kUmmaThreads, smem, h->stream>>>(X, M, K, W, bias, Cf, Cb, h->err_dev);
    return cudaGetLastError();
}

// After a synchronising call: LSKUM_ERR_TIMEOUT (and the flag cleared) if a
// tcgen05 GEMM gave up waiting for its accumulators.
int check_gemm_status(lskum_mlp* h) {
    if (h->gemm_path != LSKUM_MLP_GEMM_TCGEN05) return LSKUM_OK;
    int flag = 0;
    MLP_CUDA(cudaMemcpy(&flag, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return LSKUM_OK;
    MLP_CUDA(cudaMemset(h->err_dev, 0, sizeof(int)));
    return fail(LSKUM_ERR_TIMEOUT, "tcgen05 GEMM: accumulator wait ran out");
}

template <int EPI>
cudaError_t gemm(lskum_mlp* h, const __nv_bfloat16* A, int64_t sam, int64_t sak,
                 const __nv_bfloat16* B, int64_t sbk, int64_t sbn, int M, int N, int K,
                 const float* bias, float* Cf, __nv_bfloat16* Cb, int64_t ldc) {
    // forward X W^T into few outputs (the last layer): a warp per row
    if (EPI == kBiasLinear && sak == 1 && sbk == 1 && sbn == K && N <= kNarrowMax &&
        int64_t(N) * K <= kNarrowW && K % 8 == 0 && sam % 8 == 0 &&
        !(reinterpret_cast<uintptr_t>(A) & 15) && !(reinterpret_cast<uintptr_t>(B) & 15)) {
        k_gemm_narrow<<<blocks(M, kNarrowRows), 32 * kNarrowRows, 0, h->stream>>>(A, sam, B, M, N, K,
                                                                                  bias, Cf, ldc);
        return cudaGetLastError();
    }
    if (tc_ok(A, sam, sak, B, sbk, sbn, M, N, K)) {
        const dim3 grid(blocks(N, kTB), blocks(M, kTB), 1);
        const int kchunk = int(blocks(K, kTK)) * kTK;
        if (sak == 1 && sbk == 1)  // forward X W^T
            return launch_tc<EPI, true, true>(h, grid, A, sam, sak, B, sbk, sbn, M, N, K, bias, Cf, Cb,
                                              ldc, kchunk);
        if (EPI == kStoreF32 && sak == 1)  // backward dZ W
            return launch_tc<kStoreF32, true, false>(h, grid, A, sam, sak, B, sbk, sbn, M, N, K,
                                                     nullptr, Cf, nullptr, ldc, kchunk);
    }
    dim3 grid(blocks(N, kTile), blocks(M, kTile), 1);
    k_gemm_bf16<EPI><<<grid, 128, 0, h->stream>>>(A, sam, sak, B, sbk, sbn, M, N, K, bias, Cf, Cb, ldc,
                                                   K);
    return cudaGetLastError();
}

// C[M x N] (ldc = N) = A B with the contraction split over enough slices to
// give ~4 blocks per SM: for the weight gradients, whose M x N is one 256 x
// 256 tile grid while K is the batch.
cudaError_t gemm_splitk(lskum_mlp* h, const __nv_bfloat16* A, int64_t sam, int64_t sak,
                        const __nv_bfloat16* B, int64_t sbk, int64_t sbn, int M, int N, int K,
                        float* C) {
    const bool tc = tc_ok(A, sam, sak, B, sbk, sbn, M, N, K) && sam == 1 && sbn == 1;
    const int tile = tc ? kTB : kTile;
    const int tiles = int(blocks(N, tile) * blocks(M, tile));
    int slices = std::min(kMaxSlices, std::max(1, (tc ? 300 : 600) / tiles));
    int kchunk = int(blocks(K, slices));
    kchunk = (kchunk + kKt - 1) / kKt * kKt;  // kKt == kTK: whole k stages per slice
    slices = int(blocks(K, kchunk));
    dim3 grid(blocks(N, tile), blocks(M, tile), slices);
    cudaError_t e;
    if (tc) {
        // weight gradient dZ^T X: both operands transposed on load
        e = launch_tc<kStoreF32, false, false>(h, grid, A, sam, sak, B, sbk, sbn, M, N, K, nullptr,
                                               h->slices, nullptr, N, kchunk);
    } else {
        k_gemm_bf16<kStoreF32><<<grid, 128, 0, h->stream>>>(A, sam, sak, B, sbk, sbn, M, N, K, nullptr,
                                                            h->slices, nullptr, N, kchunk);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int64_t n = int64_t(M) * N;
    k_sum_slices<<<blocks(n, 256), 256, 0, h->stream>>>(h->slices, slices, n, C);
    return cudaGetLastError();
}

// forward from features (FP32 n x 32 in h->Af[0]); output Af[kLayers] (n x 4)
int forward(lskum_mlp* h, int64_t n) {
    MLP_CUDA((k_to_bf16<<<blocks(n * kIn, 256), 256, 0, h->stream>>>(h->Af[0], n * kIn, h->Ab[0]),
              cudaGetLastError()));
    for (int l = 0; l < kLayers; ++l) {
        const int K = layer_in(l), N = layer_out(l);
        const float* b = h->p + h->L.b_off[l];
        cudaError_t e;
        if (l < kLayers - 1 && h->gemm_path == LSKUM_MLP_GEMM_TCGEN05 && umma_ok(h->Ab[l], h->L.W[l], N, K))
            e = launch_umma<kBiasTanh>(h, h->Ab[l], int(n), K, h->L.W[l], b, h->Af[l + 1], h->Ab[l + 1]);
        else if (l < kLayers - 1)
            e = gemm<kBiasTanh>(h, h->Ab[l], K, 1, h->L.W[l], 1, K, int(n), N, K, b, h->Af[l + 1],
                                h->Ab[l + 1], N);
        else
            e = gemm<kBiasLinear>(h, h->Ab[l], K, 1, h->L.W[l], 1, K, int(n), N, K, b, h->Af[l + 1],
                                  nullptr, N);
        if (e != cudaSuccess) return fail(LSKUM_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    }
    return LSKUM_OK;
}

// backward from targets T (device n x 4): gradients into h->g, loss into loss_dev
int backward(lskum_mlp* h, const float* T, int64_t n) {
    const int nb = int(blocks(n * kOut, 256));
    MLP_CUDA((k_mse<<<nb, 256, 0, h->stream>>>(h->Af[kLayers], T, n, h->dZ, h->partial), cudaGetLastError()));
    MLP_CUDA((k_sum_partials<<<1, 32, 0, h->stream>>>(h->partial, nb, n * kOut, h->loss_dev), cudaGetLastError()));
    // output layer: dZ (n x 4) FP32 in h->dZ
    MLP_CUDA((k_to_bf16<<<blocks(n * kOut, 256), 256, 0, h->stream>>>(h->dZ, n * kOut, h->dZb), cudaGetLastError()));
    for (int l = kLayers - 1; l >= 0; --l) {
        const int K = layer_in(l), N = layer_out(l);
        // dW_l [N x K] = dZ^T X_l : A(m = out unit, k = sample) = dZ[s][m], B(k = sample, n = in) = X[s][n]
        cudaError_t e = gemm_splitk(h, h->dZb, 1, N, h->Ab[l], K, 1, N, K, int(n),
                                    h->g + h->L.w_off[l]);
        if (e != cudaSuccess) return fail(LSKUM_ERR_CUDA, std::string("dW: ") + cudaGetErrorString(e));
        MLP_CUDA((k_colsum<<<blocks(N, 32), dim3(32, 8), 0, h->stream>>>(h->dZ, int(n), N, h->g + h->L.b_off[l]),
                  cudaGetLastError()));
        if (l == 0) break;
        // dA_{l} [n x K] = dZ W_l : A(m = sample, k = out) = dZ, B(k = out, n = in) = W[out][in]
        e = gemm<kStoreF32>(h, h->dZb, N, 1, h->L.W[l], K, 1, int(n), K, N, nullptr, h->dA, nullptr, K);
        if (e != cudaSuccess) return fail(LSKUM_ERR_CUDA, std::string("dA: ") + cudaGetErrorString(e));
        MLP_CUDA((k_tanh_back<<<blocks(n * K, 256), 256, 0, h->stream>>>(h->dA, h->Af[l], n * K, h->dZ, h->dZb),
                  cudaGetLastError()));
    }
    return LSKUM_OK;
}

int check_n(lskum_mlp* h, int64_t n) {
    if (n < 1 || n > h->cap)
        return fail(LSKUM_ERR_INVALID_ARG, "n = " + std::to_string(n) + " outside [1, " +
                                               std::to_string(h->cap) + "]");
    return LSKUM_OK;
}

}  // namespace

extern "C" {

int64_t lskum_mlp_num_params(void) {
    int64_t s = 0;
    for (int l = 0; l < kLayers; ++l) s += int64_t(layer_in(l)) * layer_out(l) + layer_out(l);
    return s;
}

int lskum_mlp_create(int64_t capacity, const float* proj, lskum_mlp** out) {
    if (!out || !proj || capacity < 1 || capacity > (int64_t(1) << 24))
        return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_create: invalid argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(LSKUM_ERR_CUDA, "lskum_mlp_create: no usable CUDA device");
    lskum_mlp* h = new lskum_mlp();
    h->cap = capacity;
    h->nparam = lskum_mlp_num_params();
    auto bail = [&](cudaError_t e) {
        for (void* p : h->allocs) cudaFree(p);
        if (h->own_stream) cudaStreamDestroy(h->own_stream);
        delete h;
        return fail(LSKUM_ERR_CUDA, std::string("lskum_mlp_create: ") + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    h->stream = h->own_stream;
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        h->L.w_off[l] = off;
        off += int64_t(layer_in(l)) * layer_out(l);
        h->L.b_off[l] = off;
        off += layer_out(l);
        if ((e = alloc(h, &h->L.W[l], int64_t(layer_in(l)) * layer_out(l))) != cudaSuccess) return bail(e);
    }
    if ((e = alloc(h, &h->p, h->nparam)) != cudaSuccess || (e = alloc(h, &h->g, h->nparam)) != cudaSuccess ||
        (e = alloc(h, &h->m, h->nparam)) != cudaSuccess || (e = alloc(h, &h->v, h->nparam)) != cudaSuccess ||
        (e = alloc(h, &h->proj, 16)) != cudaSuccess || (e = alloc(h, &h->dA, capacity * kWidth)) != cudaSuccess ||
        (e = alloc(h, &h->dZ, capacity * kWidth)) != cudaSuccess ||
        (e = alloc(h, &h->dZb, capacity * kWidth)) != cudaSuccess ||
        (e = alloc(h, &h->slices, int64_t(kMaxSlices) * kWidth * kWidth)) != cudaSuccess ||
        (e = alloc(h, &h->partial, int64_t(blocks(capacity * kOut, 256)))) != cudaSuccess ||
        (e = alloc(h, &h->loss_dev, 1)) != cudaSuccess ||
        (e = alloc(h, &h->err_dev, 1)) != cudaSuccess ||
        (e = cudaMemset(h->err_dev, 0, sizeof(int))) != cudaSuccess)
        return bail(e);
    for (int l = 0; l <= kLayers; ++l) {
        const int w = l == 0 ? kIn : (l == kLayers ? kOut : kWidth);
        if ((e = alloc(h, &h->Af[l], capacity * w)) != cudaSuccess ||
            (e = alloc(h, &h->Ab[l], capacity * w)) != cudaSuccess)
            return bail(e);
    }
    if ((e = cudaMemcpy(h->proj, proj, 16 * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->p, 0, sizeof(float) * h->nparam)) != cudaSuccess ||
        (e = cudaMemset(h->m, 0, sizeof(float) * h->nparam)) != cudaSuccess ||
        (e = cudaMemset(h->v, 0, sizeof(float) * h->nparam)) != cudaSuccess)
        return bail(e);
    *out = h;
    return LSKUM_OK;
}

void lskum_mlp_destroy(lskum_mlp* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    cudaStreamDestroy(h->own_stream);
    delete h;
}

int lskum_mlp_set_params(lskum_mlp* h, const float* params, int64_t n) {
    if (!h || !params || n != h->nparam) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_set_params: size");
    MLP_CUDA(cudaMemcpyAsync(h->p, params, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->m, 0, sizeof(float) * n, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->v, 0, sizeof(float) * n, h->stream));
    h->step = 0;
    MLP_CUDA((k_weights_bf16<<<dim3(blocks(int64_t(kWidth) * kWidth, 256), kLayers), 256, 0, h->stream>>>(h->p, h->L),
              cudaGetLastError()));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LSKUM_OK;
}

int lskum_mlp_get_params(lskum_mlp* h, float* params, int64_t n) {
    if (!h || !params || n != h->nparam) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_get_params: size");
    MLP_CUDA(cudaMemcpyAsync(params, h->p, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LSKUM_OK;
}

int lskum_mlp_features(lskum_mlp* h, const float* raw, int64_t n, float* feat) {
    if (!h || !raw || !feat) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_features: null");
    if (n < 1) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_features: n < 1");
    MLP_CUDA((k_features<<<blocks(n, 256), 256, 0, h->stream>>>(raw, n, h->proj, feat), cudaGetLastError()));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LSKUM_OK;
}

int lskum_mlp_predict(lskum_mlp* h, const float* feat, int64_t n, float* out) {
    if (!h || !feat || !out) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_predict: null");
    int rc = check_n(h, n);
    if (rc) return rc;
    MLP_CUDA(cudaMemcpyAsync(h->Af[0], feat, sizeof(float) * n * kIn, cudaMemcpyDeviceToDevice, h->stream));
    rc = forward(h, n);
    if (rc) return rc;
    MLP_CUDA(cudaMemcpyAsync(out, h->Af[kLayers], sizeof(float) * n * kOut, cudaMemcpyDeviceToDevice, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return check_gemm_status(h);
}

int lskum_mlp_gradients(lskum_mlp* h, const float* feat, const float* target, int64_t n, float* grads,
                        double* loss) {
    if (!h || !feat || !target) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_gradients: null");
    int rc = check_n(h, n);
    if (rc) return rc;
    MLP_CUDA(cudaMemcpyAsync(h->Af[0], feat, sizeof(float) * n * kIn, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = forward(h, n)) || (rc = backward(h, target, n))) return rc;
    if (grads) MLP_CUDA(cudaMemcpyAsync(grads, h->g, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost, h->stream));
    if (loss) MLP_CUDA(cudaMemcpyAsync(loss, h->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return check_gemm_status(h);
}

int lskum_mlp_train_step(lskum_mlp* h, const float* feat, const float* target, int64_t n, float lr,
                         double* loss) {
    if (!h || !feat || !target || !(lr > 0.f)) return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_train_step: argument");
    int rc = check_n(h, n);
    if (rc) return rc;
    MLP_CUDA(cudaMemcpyAsync(h->Af[0], feat, sizeof(float) * n * kIn, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = forward(h, n)) || (rc = backward(h, target, n))) return rc;
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, float(h->step)));
    const float c2 = 1.f / (1.f - powf(b2, float(h->step)));
    MLP_CUDA((k_adam<<<blocks(h->nparam, 256), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->nparam, lr, b1, b2,
                                                                     1e-8f, c1, c2),
              cudaGetLastError()));
    MLP_CUDA((k_weights_bf16<<<dim3(blocks(int64_t(kWidth) * kWidth, 256), kLayers), 256, 0, h->stream>>>(h->p, h->L),
              cudaGetLastError()));
    if (loss) {
        MLP_CUDA(cudaMemcpyAsync(loss, h->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        MLP_CUDA(cudaStreamSynchronize(h->stream));
        return check_gemm_status(h);
    }
    return LSKUM_OK;
}

int lskum_mlp_sync(lskum_mlp* h) {
    if (!h) return fail(LSKUM_ERR_INVALID_ARG, "null");
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return check_gemm_status(h);
}

int lskum_mlp_set_gemm(lskum_mlp* h, int path) {
    if (!h || (path != LSKUM_MLP_GEMM_MMA_SYNC && path != LSKUM_MLP_GEMM_TCGEN05))
        return fail(LSKUM_ERR_INVALID_ARG, "lskum_mlp_set_gemm: unknown path");
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    h->gemm_path = path;
    return LSKUM_OK;
}

int lskum_mlp_set_stream(lskum_mlp* h, void* stream) {
    if (!h) return fail(LSKUM_ERR_INVALID_ARG, "null");
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    return LSKUM_OK;
}

}  // extern "C"

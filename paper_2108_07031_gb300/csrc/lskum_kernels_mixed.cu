// Mixed-precision kernels of the q-LSKUM hot path (sm_103a).
//
// FP32 for the stencil, least-squares and split-flux arithmetic; FP64 for
// the state accumulation U += dt R, the q-variables derived from U, the 2x2
// least-squares determinants (folded into weights on the host in FP64 and
// stored as FP32), the residue and the force integral.
//
// Differences are what the method consumes -- q_j - q_i in the
// least-squares sums and G(q~_j) - G(q~_0) in the split-flux derivatives --
// and at fine resolution they are 1e-4 of the values, so FP32 values would
// lose four of their seven digits in each subtraction. The FP32 path
// therefore never subtracts two nearby values:
//   * q is stored as a pair of floats (hi + lo = the FP64 q to ~2^-48), so
//     q_j - q_i = (hi_j - hi_i) + (lo_j - lo_i) is accurate to FP32
//     precision relative to the difference itself;
//   * the primitive state of q~_j is formed as base + difference from
//     q~_0 and dq~ = q~_j - q~_0 with quotient identities and log1p/expm1;
//   * each split flux is differenced in closed form: products by the
//     product rule, exp(-S^2) by expm1, and erfc by the midpoint expansion
//     erfc(m-h) - erfc(m+h) = (2/sqrt(pi)) e^{-m^2} sum_k H_2k(m) ...
//     (Hermite polynomials) for small steps, directly for large ones.
// The result is the same residual as the FP64 path to about FP32 relative
// precision of the residual itself, not of the fluxes.

#include <cmath>

#include "device_math.cuh"
#include "lskum_internal.h"
#include "lskum_kernels.cuh"
#include "math_tables.h"

namespace lskum {

namespace {

constexpr float kInvSqrtPiF = 0.5641895835477563f;  // 1 / sqrt(pi)

// q_j - q_i from the hi/lo float pairs.
__device__ __forceinline__ float4 qdiff(const QHL& a, const QHL& b) {
    return make_float4((a.hi.x - b.hi.x) + (a.lo.x - b.lo.x), (a.hi.y - b.hi.y) + (a.lo.y - b.lo.y),
                       (a.hi.z - b.hi.z) + (a.lo.z - b.lo.z), (a.hi.w - b.hi.w) + (a.lo.w - b.lo.w));
}

// ----------------------------------------------------------- q-derivatives

// Both sweeps stream, per neighbour entry, the packed neighbour word and the
// FP32 weight pair {wx, wy}, then gather the neighbour's record with the
// index that word holds. Entries are taken in groups of kLsAhead, and the
// next group's stream loads are issued before the current group's gathers,
// so a thread has a group of DRAM loads in flight while it waits on the
// cache-resident gathers (12-13 % less time per sweep at 10M points than a
// plain unrolled loop; staging the stream or the tile's own records in
// shared memory was slower). Slots at or past the point's count c are not
// read.
constexpr int kLsAhead = 4;

__device__ __forceinline__ void load_ls_entries(const DevGeom& g, const DevGeom32& g32,
                                                const int64_t d, const int k0, const int c,
                                                uint32_t e[kLsAhead], float2 w[kLsAhead]) {
#pragma unroll
    for (int u = 0; u < kLsAhead; ++u) {
        if (k0 + u < c) {
            const int64_t at = int64_t(k0 + u) * g.stride + d;
            e[u] = g.nbr[at];
            w[u] = g32.lw2[at];
        }
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_ls_first_mx(const DevGeom g, const DevGeom32 g32,
                                                       const QHL* __restrict__ q,
                                                       D8f* __restrict__ dq) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    if (d >= g.n) return;
    const int c = g.cnt[d];
    const QHL qi = q[t];
    float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax;
    uint32_t en[kLsAhead] = {};
    float2 wn[kLsAhead] = {};
    load_ls_entries(g, g32, d, 0, c, en, wn);
    for (int k0 = 0; k0 < c; k0 += kLsAhead) {
        uint32_t ec[kLsAhead];
        float2 wc[kLsAhead];
#pragma unroll
        for (int u = 0; u < kLsAhead; ++u) {
            ec[u] = en[u];
            wc[u] = wn[u];
        }
        load_ls_entries(g, g32, d, k0 + kLsAhead, c, en, wn);
#pragma unroll
        for (int u = 0; u < kLsAhead; ++u) {
            if (k0 + u < c) {
                const float wx = wc[u].x, wy = wc[u].y;
                const float4 dqv = qdiff(q[sidx(g, ec[u] & kIndexMask, cc)], qi);
                ax.x += wx * dqv.x; ax.y += wx * dqv.y; ax.z += wx * dqv.z; ax.w += wx * dqv.w;
                ay.x += wy * dqv.x; ay.y += wy * dqv.y; ay.z += wy * dqv.z; ay.w += wy * dqv.w;
            }
        }
    }
    dq[t] = D8f{ax, ay};
}

// One Jacobi sweep of Eq. 29 as the first-order derivative of the stage
// (dq_first, the sum of wx_j (q_j - q_i)) minus the sum of wx_j (hdx_j
// (qx_j - qx_i) + hdy_j (qy_j - qy_i)): the q gathers and their float-pair
// differences are done once per stage, not per sweep; the derivative
// differences stay differences (exact in FP32 for nearby values). The
// per-neighbour stream is the 8-byte weight pair; the half offsets come from
// the gathered coordinate pairs of the neighbour (cache-resident: the
// neighbours of a warp's points are close in the Hilbert order).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_ls_inner_mx(const DevGeom g, const DevGeom32 g32,
                                                       const D8f* __restrict__ dq_first,
                                                       const D8f* __restrict__ din,
                                                       D8f* __restrict__ dout) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    if (d >= g.n) return;
    const int c = g.cnt[d];
    const D8f di = din[t];
    const float4 pi = g32.xyhl[d];
    float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax;
    uint32_t en[kLsAhead] = {};
    float2 wn[kLsAhead] = {};
    load_ls_entries(g, g32, d, 0, c, en, wn);
    for (int k0 = 0; k0 < c; k0 += kLsAhead) {
        uint32_t ec[kLsAhead];
        float2 wc[kLsAhead];
#pragma unroll
        for (int u = 0; u < kLsAhead; ++u) {
            ec[u] = en[u];
            wc[u] = wn[u];
        }
        load_ls_entries(g, g32, d, k0 + kLsAhead, c, en, wn);
#pragma unroll
        for (int u = 0; u < kLsAhead; ++u) {
            if (k0 + u < c) {
                const uint32_t j = ec[u] & kIndexMask;
                const float wx = wc[u].x, wy = wc[u].y;
                const float4 pj = g32.xyhl[j];
                const D8f dj = din[sidx(g, j, cc)];
                const float hx = 0.5f * ((pj.x - pi.x) + (pj.z - pi.z));
                const float hy = 0.5f * ((pj.y - pi.y) + (pj.w - pi.w));
                // (dx (qx_j - qx_i) + dy (qy_j - qy_i)) / 2, the Eq. 28 correction
                const float t0 = hx * (dj.x.x - di.x.x) + hy * (dj.y.x - di.y.x);
                const float t1 = hx * (dj.x.y - di.x.y) + hy * (dj.y.y - di.y.y);
                const float t2 = hx * (dj.x.z - di.x.z) + hy * (dj.y.z - di.y.z);
                const float t3 = hx * (dj.x.w - di.x.w) + hy * (dj.y.w - di.y.w);
                ax.x += wx * t0; ax.y += wx * t1; ax.z += wx * t2; ax.w += wx * t3;
                ay.x += wy * t0; ay.y += wy * t1; ay.z += wy * t2; ay.w += wy * t3;
            }
        }
    }
    const D8f f = dq_first[t];
    dout[t] = D8f{make_float4(f.x.x - ax.x, f.x.y - ax.y, f.x.z - ax.z, f.x.w - ax.w),
                  make_float4(f.y.x - ay.x, f.y.y - ay.y, f.y.z - ay.z, f.y.w - ay.w)};
}

// ------------------------------------------------ primitive base + difference

struct PrimPair {
    float r, u, v, p, sb;       // base state (of q~_0): density, velocity, pressure, sqrt(beta)
    float dr, du, dv, dp, dsb;  // difference state(q~_j) - state(q~_0)
    float isb, isbj;            // 1/sqrt(beta) of the base and of state j
    // frame-invariant factor both split fluxes of the pair share (base and
    // difference): h = p + rho e
    float h, dh;
};

// e^x - 1: its Taylor polynomial to x^5/120 for |x| <= 1/16 (the remainder is
// below 2e-9 of the result), the library function beyond. The arguments
// here are differences of nearby states, almost always far inside 1/16.
__device__ __forceinline__ float expm1_f(const float x) {
    if (fabsf(x) <= 0.0625f)
        return x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f), 0.5f),
                        1.0f);
    return expm1f(x);
}

// ln(1 + x): its Taylor polynomial to x^6/6 for |x| <= 1/16 (remainder below
// 1e-8 of the result), the library function beyond.
__device__ __forceinline__ float log1p_f(const float x) {
    if (fabsf(x) <= 0.0625f)
        return x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f),
                                -0.5f),
                        1.0f);
    return log1pf(x);
}

// The FP32 quotients below are fast (reciprocal approximation times the
// numerator, ~2 ulp): every one scales a difference term, whose own FP32
// rounding error is larger.

// From the base q~_0 and the difference dq~ = q~_j - q~_0 (inverse of Eq. 26).
template <bool G14>
__device__ __forceinline__ PrimPair prim_pair(const float4 b, const float4 dq, const float gm1_inv) {
    PrimPair w;
    const float beta = -0.5f * b.w;
    const float dbeta = -0.5f * dq.w;
    const float qj4 = b.w + dq.w;
    const float inv2b = __fdividef(-1.0f, b.w);  // 1 / (2 beta)
    w.u = b.y * inv2b;
    w.v = b.z * inv2b;
    // u = -q2/q4:  u_j - u_0 = (q2 dq4 - dq2 q4) / (q4 q4_j)
    const float rq = __fdividef(1.0f, b.w * qj4);
    w.du = (b.y * dq.w - dq.y * b.w) * rq;
    w.dv = (b.z * dq.w - dq.z * b.w) * rq;
    const float uj = w.u + w.du, vj = w.v + w.dv;
    const float uu0 = w.u * w.u + w.v * w.v;
    const float uuj = uj * uj + vj * vj;
    const float duu = w.du * (uj + w.u) + w.dv * (vj + w.v);
    w.isb = rsqrtf(beta);
    w.sb = beta * w.isb;
    const float betaj = beta + dbeta;
    w.isbj = rsqrtf(betaj);
    // sqrt(beta_j) - sqrt(beta) = dbeta / (sqrt(beta_j) + sqrt(beta))
    w.dsb = __fdividef(dbeta, betaj * w.isbj + w.sb);
    // ln rho = q1 - ln(beta)/(gamma-1) + beta |u|^2
    if (G14) {
        const float i2 = w.isb * w.isb;
        w.r = __expf(b.x + beta * uu0) * (i2 * i2 * w.isb);
    } else {
        w.r = __expf(b.x - __logf(beta) * gm1_inv + beta * uu0);
    }
    const float dlnr = dq.x - log1p_f(dbeta * (2.0f * inv2b)) * gm1_inv + (dbeta * uuj + beta * duu);
    w.dr = w.r * expm1_f(dlnr);
    // p = rho / (2 beta):  p_j - p_0 = (drho beta - rho dbeta) / (2 beta beta_j)
    w.p = w.r * inv2b;
    w.dp = (w.dr * beta - w.r * dbeta) * (inv2b * (w.isbj * w.isbj));
    // rho e = p/(gamma-1) + rho |u|^2 / 2 (|u|^2 is the same in every frame)
    const float E0 = w.p * gm1_inv + 0.5f * w.r * uu0;
    const float dE = w.dp * gm1_inv + 0.5f * (w.dr * uuj + w.r * duu);
    w.h = w.p + E0;
    w.dh = w.dp + dE;
    return w;
}

// erfc(m - h) - erfc(m + h) = (4/sqrt(pi)) e^{-m^2} (h + H2 h^3/6 + H4 h^5/120
// + H6 h^7/5040 + H8 h^9/362880) with the Hermite polynomials H_k(m): the
// even Taylor terms of e^{-t^2} about m integrated over [m - h, m + h].
// For |h| <= 1/64 the H6 and H8 terms are below 2e-11 of the first (|m| <=
// 6.5, the range where erfc is not negligible) and are left out.
__device__ __forceinline__ float erfc_central_diff(const float m, const float h) {
    const float m2 = m * m;
    const float H2 = 4.0f * m2 - 2.0f;
    const float H4 = (16.0f * m2 - 48.0f) * m2 + 12.0f;
    const float h2 = h * h;
    float tail = H4 * (1.0f / 120.0f);
    if (fabsf(h) > 0.015625f) {
        const float H6 = ((64.0f * m2 - 480.0f) * m2 + 720.0f) * m2 - 120.0f;
        const float H8 = (((256.0f * m2 - 3584.0f) * m2 + 13440.0f) * m2 - 13440.0f) * m2 + 1680.0f;
        tail += h2 * (H6 * (1.0f / 5040.0f) + h2 * (H8 * (1.0f / 362880.0f)));
    }
    const float s = h * (1.0f + h2 * (H2 * (1.0f / 6.0f) + h2 * tail));
    return 4.0f * kInvSqrtPiF * __expf(-m2) * s;
}

// erfc(x)/2 given e = exp(-x^2): e erfcx(|x|)/2 from the FP32 erfcx pieces
// (width 1/4, degree 5, 1.2e-7 relative) for |x| <= 6, then 1 minus it for
// x < 0; the exponential is the one the split flux needs for B anyway.
__device__ __forceinline__ float half_erfc_f(const float x, const float e) {
    const float a = fabsf(x);
    float hc;
    if (a <= 6.0f) {
        const float* c = kErfcxF[min(int(a * kErfcxFInvW), kErfcxFPieces - 1)];
        const float z = a - __ldg(c);
        float pv = __ldg(c + 1 + kErfcxFDeg);
#pragma unroll
        for (int m = kErfcxFDeg - 1; m >= 0; --m) pv = fmaf(pv, z, __ldg(c + 1 + m));
        hc = 0.5f * e * pv;
    } else {
        hc = 0.5f * erfcf(a);
    }
    return x > 0.0f ? hc : 1.0f - hc;
}

// Difference of the kinetic split flux along the frame's first axis ("a",
// velocity ua, transverse ub), sign sg: dG = G(state_j) - G(state_0),
// state_j = base + difference; the frame-invariant factors come from w.
__device__ __forceinline__ void dsplit_flux_a(const PrimPair& w, const float ua0, const float ub0,
                                              const float dua, const float dub, const float sg,
                                              float dG[4]) {
    const float r0 = w.r, dr = w.dr, p0 = w.p, dp = w.dp, sb0 = w.sb, dsb = w.dsb;
    const float isb0 = w.isb, isbj = w.isbj;
    const float sbj = sb0 + dsb;
    const float S0 = ua0 * sb0;
    const float dS = dua * sbj + ua0 * dsb;
    const float Sj = S0 + dS;
    // exponential: e_j - e_0 = e_0 expm1(-(S_j^2 - S_0^2))
    const float e0 = __expf(-S0 * S0);
    const float de = e0 * expm1_f(-dS * (Sj + S0));
    // A = erfc(x)/2 at x = -sg S
    const float x0 = -sg * S0, dx = -sg * dS;
    const float A0 = half_erfc_f(x0, e0);  // e0 = exp(-x0^2)
    float dA;
    if (fabsf(dx) <= 0.25f) {
        // erfc(x0 + dx) - erfc(x0) = -(erfc(m - h) - erfc(m + h)), m = x0 + dx/2, h = dx/2
        dA = -0.5f * erfc_central_diff(x0 + 0.5f * dx, 0.5f * dx);
    } else {
        dA = 0.5f * (erfcf(x0 + dx) - erfcf(x0));
    }
    const float Aj = A0 + dA;
    // B = e / (2 sqrt(pi) sqrt(beta))
    const float c = 0.5f * kInvSqrtPiF;
    const float B0 = c * e0 * isb0;
    const float dB = c * (de * isbj - e0 * dsb * isbj * isb0);
    const float Bj = B0 + dB;
    // t = u_a A + sg B
    const float t0 = ua0 * A0 + sg * B0;
    const float dt = dua * Aj + ua0 * dA + sg * dB;
    const float tj = t0 + dt;
    // mass: G0 = rho t
    const float G00 = r0 * t0;
    dG[0] = dr * tj + r0 * dt;
    const float G0j = G00 + dG[0];
    // a-momentum: (p + rho u_a^2) A + sg rho u_a B = u_a G0 + p A
    dG[1] = dua * G0j + ua0 * dG[0] + (dp * Aj + p0 * dA);
    // b-momentum: rho u_b t = u_b G0
    dG[2] = dub * G0j + ub0 * dG[0];
    // energy: (p + rho e) u_a A + sg (rho e + p/2) B = h t - (p/2) sg B
    dG[3] = w.dh * tj + w.h * dt - 0.5f * sg * (dp * Bj + p0 * dB);
}

__device__ __forceinline__ QHL split_hl(const V4& q) {
    QHL o;
    o.hi = make_float4(__double2float_rn(q.a), __double2float_rn(q.b), __double2float_rn(q.c),
                       __double2float_rn(q.d));
    o.lo = make_float4(__double2float_rn(q.a - double(o.hi.x)), __double2float_rn(q.b - double(o.hi.y)),
                       __double2float_rn(q.c - double(o.hi.z)), __double2float_rn(q.d - double(o.hi.w)));
    return o;
}

__device__ __forceinline__ bool physical(double rho, double u, double v, double p) {
    return rho > 0.0 && p > 0.0 && isfinite(rho) && isfinite(p) && isfinite(u) && isfinite(v);
}

template <int BLOCK>
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double warp_part[BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part[wid] = x;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < BLOCK / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// ------------------------------------------------------- flux residual + RK

// Latency bound (long-scoreboard stalls lead): each neighbour entry's stream
// loads (packed word, FP32 constants) are issued one entry ahead, during the
// previous entry's flux arithmetic, so only the gathers they index are
// waited on. Registers capped at 72 per thread (seven blocks of 128 per SM);
// measured at 10M points: 2.35 ms per launch, against 2.60 without the
// prefetch at 64 registers (eight blocks) and 2.69 with it at 64 (the
// prefetched words then spill).
template <int MODE, int BLOCK, bool G14>
__global__ void __launch_bounds__(BLOCK, 896 / BLOCK) k_flux_mx(const DevGeom g, const DevGeom32 g32,
                                                   const Physics ph, const DevState st,
                                                   const QHL* __restrict__ q_in,
                                                   const D8f* __restrict__ dq,
                                                   QHL* __restrict__ q_out) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    double r2 = 0.0;
    if (d < g.n) {
        const int8_t fl = g.flag[d];
        const bool fixed = ph.outer_fixed && fl == LSKUM_OUTER;
        float R[4] = {0.f, 0.f, 0.f, 0.f};
        if (!fixed) {
            float tx = 1.f, ty = 0.f, nx = 0.f, ny = 1.f;
            const bool local = fl != LSKUM_INTERIOR;
            if (local) {
                const double2 nn = g.nrm[d];
                nx = float(nn.x);
                ny = float(nn.y);
                tx = ny;
                ty = -nx;
            }
            const QHL qi = q_in[t];
            const D8f di = dq[t];
            const float4 qiv = make_float4(qi.hi.x + qi.lo.x, qi.hi.y + qi.lo.y, qi.hi.z + qi.lo.z,
                                           qi.hi.w + qi.lo.w);
            const float gm1_inv = float(ph.gm1_inv);
            const bool second = ph.order == 2;
            const int c = g.cnt[d];
            uint32_t e_next = 0u;
            float4 fw_next = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c > 0) {
                e_next = g.nbr[d];
                fw_next = g32.fxw[d];
            }
            for (int k = 0; k < c; ++k) {
                const uint32_t e = e_next;
                const float4 fw = fw_next;
                if (k + 1 < c) {  // the next entry's stream, in flight during this one
                    const int64_t at = int64_t(k + 1) * g.stride + d;
                    e_next = g.nbr[at];
                    fw_next = g32.fxw[at];
                }
                const uint32_t j = e & kIndexMask;
                const uint32_t sc = (e >> kIndexBits) & 3u;
                const uint32_t nc = (e >> (kIndexBits + 2)) & 3u;
                const int64_t jt = sidx(g, j, cc);
                const float4 dqv = qdiff(q_in[jt], qi);
                float4 base = qiv, dlt = dqv;
                if (second) {
                    const float hx = fw.z, hy = fw.w;
                    const D8f dj = dq[jt];
                    // q~_0 = q_i - (dx q_x,i + dy q_y,i)/2; dq~ = q~_j - q~_0 (Eq. 28)
                    base.x = qiv.x - (hx * di.x.x + hy * di.y.x);
                    base.y = qiv.y - (hx * di.x.y + hy * di.y.y);
                    base.z = qiv.z - (hx * di.x.z + hy * di.y.z);
                    base.w = qiv.w - (hx * di.x.w + hy * di.y.w);
                    dlt.x = dqv.x - (hx * (dj.x.x - di.x.x) + hy * (dj.y.x - di.y.x));
                    dlt.y = dqv.y - (hx * (dj.x.y - di.x.y) + hy * (dj.y.y - di.y.y));
                    dlt.z = dqv.z - (hx * (dj.x.z - di.x.z) + hy * (dj.y.z - di.y.z));
                    dlt.w = dqv.w - (hx * (dj.x.w - di.x.w) + hy * (dj.y.w - di.y.w));
                }
                if (dlt.x == 0.f && dlt.y == 0.f && dlt.z == 0.f && dlt.w == 0.f) continue;
                PrimPair w = prim_pair<G14>(base, dlt, gm1_inv);
                if (local) {
                    const float s0 = w.u * tx + w.v * ty, n0 = w.u * nx + w.v * ny;
                    const float ds = w.du * tx + w.dv * ty, dn = w.du * nx + w.dv * ny;
                    w.u = s0; w.v = n0; w.du = ds; w.dv = dn;
                }
                if (sc) {
                    const float sg = sc == 1u ? 1.f : -1.f;
                    float dG[4];
                    dsplit_flux_a(w, w.u, w.v, w.du, w.dv, sg, dG);
                    const float wt = fw.x;
                    R[0] += wt * dG[0]; R[1] += wt * dG[1]; R[2] += wt * dG[2]; R[3] += wt * dG[3];
                }
                if (nc) {
                    const float sg = nc == 1u ? 1.f : -1.f;
                    float dG[4];
                    dsplit_flux_a(w, w.v, w.u, w.dv, w.du, sg, dG);
                    const float wt = fw.y;
                    R[0] += wt * dG[0]; R[1] += wt * dG[2]; R[2] += wt * dG[1]; R[3] += wt * dG[3];
                }
            }
            if (local) {
                const float rs = R[1], rn = R[2];
                R[1] = rs * tx + rn * nx;
                R[2] = rs * ty + rn * ny;
            }
        }
        // FP64 from here: state accumulation, wall condition, next q, residue
        const double R0 = R[0], R1 = R[1], R2 = R[2], R3 = R[3];
        if (MODE == 0) {
            st.R[t] = V4{R0, R1, R2, R3};
        } else {
            V4 U = st.U[t];
            double dtv;
            if (MODE == 1) {
                // local time step in FP32: it sets the pseudo-time path, not
                // the steady state, and FP32 square roots and quotients cost
                // a fraction of the FP64 pipe's
                const float rho = float(U.a), irho = 1.0f / rho;
                const float u = float(U.b) * irho, v = float(U.c) * irho;
                const float uu = fmaf(u, u, v * v);
                const float p = float(ph.gm1) * (float(U.d) - 0.5f * rho * uu);
                dtv = double(float(ph.cfl * g.dmin[d]) /
                             (sqrtf(uu) + sqrtf(float(ph.gamma) * p * irho)));
                st.dt[t] = dtv;
                st.U0[t] = U;
                r2 = R0 * R0;
            } else {
                dtv = st.dt[t];
            }
            if (!fixed) {
                const double h = 0.5 * dtv;
                if (MODE == 3) {
                    const V4 U0 = st.U0[t];
                    U.a = (2.0 / 3.0) * U0.a + (1.0 / 3.0) * (U.a - h * R0);
                    U.b = (2.0 / 3.0) * U0.b + (1.0 / 3.0) * (U.b - h * R1);
                    U.c = (2.0 / 3.0) * U0.c + (1.0 / 3.0) * (U.c - h * R2);
                    U.d = (2.0 / 3.0) * U0.d + (1.0 / 3.0) * (U.d - h * R3);
                } else {
                    U.a -= h * R0;
                    U.b -= h * R1;
                    U.c -= h * R2;
                    U.d -= h * R3;
                }
                if (fl == LSKUM_WALL) {
                    const double2 nn = g.nrm[d];
                    const double tx = nn.y, ty = -nn.x;
                    const double ms = U.b * tx + U.c * ty;
                    U.b = ms * tx;
                    U.c = ms * ty;
                }
                st.U[t] = U;
            }
            V4 qn;
            double rho, u, v, p;
            cons_to_q64<G14>(U, ph, qn, rho, u, v, p);
            q_out[t] = split_hl(qn);
            if (!physical(rho, u, v, p)) atomicOr(st.status, 1);
        }
    }
    if (MODE == 1) {
        if (g.cshift == 0) {
            const double s = block_sum<BLOCK>(r2);
            if (threadIdx.x == 0) st.partials[blockIdx.x] = s;
        } else if (d < g.n) {
            st.r2[t] = r2;
        }
    }
}

__global__ void k_q_from_U_mx(const DevGeom g, const Physics ph, const V4* __restrict__ U,
                              QHL* __restrict__ q) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if ((t >> g.cshift) >= g.n) return;
    V4 qn;
    double rho, u, v, p;
    if (fabs(ph.gm1_inv - 2.5) < 1e-12)
        cons_to_q64<true>(U[t], ph, qn, rho, u, v, p);
    else
        cons_to_q64<false>(U[t], ph, qn, rho, u, v, p);
    q[t] = split_hl(qn);
}

__global__ void k_dq_to_v8(const DevGeom g, const D8f* __restrict__ src, V8* __restrict__ dst) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t d = t >> g.cshift;
    if (d >= g.n) return;
    const int64_t cc = int64_t(uint32_t(t) & g.cmask);
    const D8f s = src[t];
    V8 o;
    o.x[0] = s.x.x; o.x[1] = s.x.y; o.x[2] = s.x.z; o.x[3] = s.x.w;
    o.y[0] = s.y.x; o.y[1] = s.y.y; o.y[2] = s.y.z; o.y[3] = s.y.w;
    dst[cc * g.n + g.dev_to_user[d]] = o;
}

inline unsigned grid_for(int64_t n, int block) { return unsigned((n + block - 1) / block); }
inline unsigned grid_nc(const DevGeom& g, int block) { return grid_for(g.n << g.cshift, block); }

template <int BLOCK, bool G14>
void flux_mx_dispatch(int mode, const DevGeom& g, const DevGeom32& g32, const Physics& ph,
                      const DevState& st, const QHL* q_in, const D8f* dq, QHL* q_out,
                      cudaStream_t s) {
    const unsigned grid = grid_nc(g, BLOCK);
    switch (mode) {
        case 0: k_flux_mx<0, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, g32, ph, st, q_in, dq, q_out); break;
        case 1: k_flux_mx<1, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, g32, ph, st, q_in, dq, q_out); break;
        case 2: k_flux_mx<2, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, g32, ph, st, q_in, dq, q_out); break;
        case 3: k_flux_mx<3, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, g32, ph, st, q_in, dq, q_out); break;
        default: k_flux_mx<4, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, g32, ph, st, q_in, dq, q_out); break;
    }
}

}  // namespace

cudaError_t launch_ls_first_mx(const DevGeom& g, const DevGeom32& g32, const QHL* q, D8f* dq,
                               int block, cudaStream_t s) {
    if (block == 256)
        k_ls_first_mx<256><<<grid_nc(g, 256), 256, 0, s>>>(g, g32, q, dq);
    else
        k_ls_first_mx<kDefaultBlock><<<grid_nc(g, kDefaultBlock), kDefaultBlock, 0, s>>>(g, g32, q, dq);
    return cudaGetLastError();
}

cudaError_t launch_ls_inner_mx(const DevGeom& g, const DevGeom32& g32, const D8f* dq_first,
                               const D8f* din, D8f* dout, int block, cudaStream_t s) {
    if (block == 256)
        k_ls_inner_mx<256><<<grid_nc(g, 256), 256, 0, s>>>(g, g32, dq_first, din, dout);
    else
        k_ls_inner_mx<kDefaultBlock><<<grid_nc(g, kDefaultBlock), kDefaultBlock, 0, s>>>(g, g32, dq_first,
                                                                                        din, dout);
    return cudaGetLastError();
}

cudaError_t launch_flux_mx(int mode, const DevGeom& g, const DevGeom32& g32, const Physics& ph,
                           const DevState& st, const QHL* q_in, const D8f* dq, QHL* q_out,
                           int block, cudaStream_t s) {
    const bool g14 = fabs(ph.gm1_inv - 2.5) < 1e-12;
    if (block == 256) {
        if (g14) flux_mx_dispatch<256, true>(mode, g, g32, ph, st, q_in, dq, q_out, s);
        else flux_mx_dispatch<256, false>(mode, g, g32, ph, st, q_in, dq, q_out, s);
    } else {
        if (g14) flux_mx_dispatch<kDefaultBlock, true>(mode, g, g32, ph, st, q_in, dq, q_out, s);
        else flux_mx_dispatch<kDefaultBlock, false>(mode, g, g32, ph, st, q_in, dq, q_out, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_q_from_U_mx(const DevGeom& g, const Physics& ph, const V4* U, QHL* q,
                               cudaStream_t s) {
    k_q_from_U_mx<<<grid_nc(g, 256), 256, 0, s>>>(g, ph, U, q);
    return cudaGetLastError();
}

cudaError_t launch_dq_to_user_mx(const DevGeom& g, const D8f* src, V8* dst_user, cudaStream_t s) {
    k_dq_to_v8<<<grid_nc(g, 256), 256, 0, s>>>(g, src, dst_user);
    return cudaGetLastError();
}

}  // namespace lskum

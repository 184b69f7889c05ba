// FP64 device kernels of the q-LSKUM hot path (sm_103a).
//
// Mapping: one thread per point, points in Hilbert-curve order (set-up), so a
// warp's 32 points and their stencils are spatially close. Per-slot data
// (packed neighbour entry, half offsets, least-squares weights) is slot-major
// [slot][point]: consecutive threads read consecutive words (coalesced). The
// gathered per-point records are AoS: q (32 B) and (q_x, q_y) (64 B), so a
// neighbour gather is one or two full sectors.
//
// Per stage (Algorithm 2 re-fused):
//   ls_first  : q_x, q_y from Eq. 11 (full stencil), weights precomputed
//   ls_inner  : Jacobi sweep of Eq. 29 with dq~ of Eq. 28 (x inner_iters)
//   flux<k>   : residual of Eq. 12 -- per neighbour q~_j and q~_0 (Eq. 28),
//               their primitive states, the kinetic split fluxes G+-(q~)
//               along s and n (Eq. 27), accumulated with the precomputed
//               split-stencil weights (Eq. 24 over the Eq. 14 stencils) --
//               fused with the SSP-RK stage update, the wall condition, the
//               next stage's q-variables (Eq. 26), the stage-1 local time
//               step and the stage-1 partial sums of the residue.
//   residue   : fixed-order reduction of the partial sums (deterministic).
//
// The arithmetic is FP64 throughout. On GB300 the FP64 pipe, not HBM,
// bounds the flux kernel.

#include <cmath>

#include "device_math.cuh"
#include "lskum_internal.h"
#include "math_tables.h"
#include "lskum_kernels.cuh"

namespace lskum {

namespace {

constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1 / sqrt(pi)

__device__ __forceinline__ V4 ld4(const V4* p) { return *p; }

// Bit-pattern helpers: comparisons and sign flips of doubles done on the
// integer pipe, which leaves the FP64 pipe (the flux kernel's bound) alone.
constexpr int64_t kSignBit = int64_t(0x8000000000000000ULL);
constexpr int64_t kAbsMask = 0x7FFFFFFFFFFFFFFFLL;
constexpr int64_t kBits700 = 0x4085E00000000000LL;  // 700.0
constexpr int64_t kBits6 = 0x4018000000000000LL;    // 6.0, the end of the erfcx table
static_assert(kErfcxLo == 0.0 && kErfcxInvW == double(1 << kErfcxLog2InvW) && kErfcxHi == 6.0,
              "erfcx_piece assumes pieces of width 2^-kErfcxLog2InvW on [0, 6]");

__device__ __forceinline__ int64_t dbits(const double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(const int64_t b) { return __longlong_as_double(b); }

// Primitive state of one modified state q~ in the flux's frame, with the
// per-state factors the split fluxes share: sqrt(beta), 1/sqrt(pi beta),
// h = p + rho e and mhp = -p/2 (|u|^2 is frame-invariant, so these are too).
struct Prim {
    double r, u, v, p, sb, cb, h, mhp;
};

// exp(x) 2^-HALVE by Tang's table-driven method (math_tables.h): x = k ln2/N
// + r (N = 2^kExpBits = 256), |r| <= ln2/(2N), exp(x) = 2^(k div N)
// 2^((k mod N)/N) e^r with e^r - 1 from its degree-4 Taylor polynomial
// (remainder < 4e-17); max error 1.2 ulp (checked against 200-bit arithmetic
// with exact FMA emulation). About 9 FP64 operations against the library's
// ~18; the power of two, including the optional halving, is an integer add
// to the exponent field (the result stays normal for |x| <= 700). Outside
// that range the library exp.
template <int HALVE>
__device__ __forceinline__ double exp_tab(const double x) {
    if ((dbits(x) & kAbsMask) > kBits700) return HALVE ? 0.5 * exp(x) : exp(x);
    const double shifter = 6755399441055744.0;  // 1.5 * 2^52: rounds k into the low bits
    double kd = fma(x, kInvLn2ByN, shifter);
    const int64_t k = dbits(kd) - 0x4338000000000000LL;
    kd -= shifter;
    const double r = fma(-kd, kLn2ByNLo, fma(-kd, kLn2ByNHi, x));
    const double p = r * fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0);
    const double t = kExp2Tab[k & ((1 << kExpBits) - 1)];
    const double res = fma(t, p, t);
    return bitsd(dbits(res) + (((k >> kExpBits) - HALVE) << 52));
}

// q~ -> primitive (inverse of Eq. 26); velocities in the global frame. With
// gamma = 1.4 (1/(gamma-1) = 5/2) the factor beta^(-1/(gamma-1)) of the
// density is (1/beta)^2 / sqrt(beta), so no logarithm is needed; 1/sqrt(beta)
// is needed by the split fluxes anyway.
template <bool G14>
__device__ __forceinline__ Prim q_to_prim(const double t0, const double t1, const double t2,
                                          const double t3, const double gm1_inv) {
    Prim w;
    const double beta = -0.5 * t3;
    const double isb = rsqrt(beta);
    w.sb = beta * isb;
    w.cb = isb * kInvSqrtPi;
    // 1/beta from (1/sqrt(beta))^2 and one Newton step, i2 (1 + (1 - beta
    // i2)): the residual 1 - beta i2 comes exact from the FMA, so the step
    // leaves ~0.5 ulp, as good as an IEEE division (u, v, p and the density's
    // (1/beta)^2 inherit it) for 4 FP64 instructions instead of ~7.
    const double i20 = isb * isb;
    const double i2 = fma(i20, fma(-beta, i20, 1.0), i20);  // 1 / beta
    const double inv2b = 0.5 * i2;                         // 1 / (2 beta)
    w.u = t1 * inv2b;
    w.v = t2 * inv2b;
    const double uu = fma(w.u, w.u, w.v * w.v);
    if (G14) {
        w.r = exp_tab<0>(fma(beta, uu, t0)) * (i2 * i2 * isb);
    } else {
        w.r = exp_tab<0>(t0 - log(beta) * gm1_inv + beta * uu);
    }
    w.p = w.r * inv2b;
    const double rhoe = fma(0.5 * w.r, uu, w.p * gm1_inv);
    w.h = w.p + rhoe;
    w.mhp = -0.5 * w.p;
    return w;
}

// Index of the erfcx piece holding a (0 <= a <= 6), floor(2^L a) with
// L = kErfcxLog2InvW, from the bit pattern of a = 1.f x 2^e:
// 2^L a = (2^52 + f) / 2^(52 - L - e).
__device__ __forceinline__ int erfcx_piece(const int64_t abits) {
    const int sh = (52 - kErfcxLog2InvW) - (int(abits >> 52) - 1023);
    const int64_t m = (abits & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
    const int k = sh > 52 ? 0 : int(m >> sh);
    return min(k, kErfcxPieces - 1);
}

// Kinetic split flux along the frame's first axis ("a" = ua, "b" = ub) of
// the state w, for molecules with positive (nmask = 0) or negative (nmask =
// sign bit) a-velocity. With S = ua sqrt(beta) and sg = +-1:
//   A = erfc(-sg S)/2, B = exp(-S^2)/(2 sqrt(pi beta)),
//   G = (rho (ua A + sg B), (p + rho ua^2) A + sg rho ua B, rho ub (ua A + sg B),
//        (p + rho e) ua A + sg (rho e + p/2) B).
// erfc(|S|)/2 = exp(-S^2)/2 erfcx(|S|) from the erfcx pieces for every |S| <= 6
// (one path for all lanes), sharing exp(-S^2)/2 with B; the library erfc beyond.
// With t = ua A + sg B the four components are G0 = rho t, G1 = ua G0 + p A,
// G2 = ub G0 and G3 = h t - (p/2) sg B (h - p/2 = rho e + p/2); split_ab
// returns t, A and sg B of one state, split_flux_diff the four differences
// between two states.
struct SplitAB {
    double t, A, Bs;
};

__device__ __forceinline__ SplitAB split_ab(const Prim& w, const double ua, const int64_t nmask) {
    const double S = ua * w.sb;
    const double eh = exp_tab<1>(-(S * S));  // exp(-S^2) / 2
    const int64_t abits = dbits(S) & kAbsMask;
    double hc;  // erfc(|S|) / 2
    if (abits <= kBits6) {
        const double* c = kErfcxC[erfcx_piece(abits)];
        const double z = bitsd(abits) - __ldg(c);
        double pv = __ldg(c + 1 + kErfcxDeg);
#pragma unroll
        for (int m = kErfcxDeg - 1; m >= 0; --m) pv = fma(pv, z, __ldg(c + 1 + m));
        hc = eh * pv;
    } else {
        hc = 0.5 * erfc(bitsd(abits));
    }
    // A = erfc(x)/2 at x = -sg S: erfc(|x|)/2 for x > 0, 1 - erfc(|x|)/2 otherwise
    const int64_t xbits = dbits(S) ^ nmask ^ kSignBit;
    const double A = xbits > 0 ? hc : 1.0 - hc;
    const double Bs = bitsd(dbits(eh * w.cb) ^ nmask);  // sg B
    return SplitAB{fma(ua, A, Bs), A, Bs};
}

// G(state j) - G(state 0) along the frame's first axis (velocities uaj, ubj
// and ua0, ub0): each difference takes state 0's value, rounded once, into
// the FMA chain of state j's, so the four cost 13 FP64 operations where two
// flux evaluations and four subtractions took 16.
__device__ __forceinline__ void split_flux_diff(const Prim& wj, const Prim& w0, const double uaj,
                                                const double ubj, const double ua0, const double ub0,
                                                const SplitAB& aj, const SplitAB& a0, double d[4]) {
    const double g0j = wj.r * aj.t, g00 = w0.r * a0.t;
    d[0] = g0j - g00;
    const double g10 = fma(ua0, g00, w0.p * a0.A);
    d[1] = fma(uaj, g0j, fma(wj.p, aj.A, -g10));
    d[2] = fma(g0j, ubj, -(g00 * ub0));
    const double g30 = fma(w0.h, a0.t, w0.mhp * a0.Bs);
    d[3] = fma(wj.h, aj.t, fma(wj.mhp, aj.Bs, -g30));
}

// Modified states q~_j and q~_0 of Eq. 28 for one neighbour (half offsets
// hx, hy); returns false when they are bitwise equal: then every split-flux
// difference is exactly 0 (free-stream preservation), and the pair is skipped.
__device__ __forceinline__ bool modified_states(const bool second, const double hx, const double hy,
                                                const V8& dj, const V8& di, double tj[4],
                                                double t0[4]) {
    if (second) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            tj[m] = fma(-hx, dj.x[m], fma(-hy, dj.y[m], tj[m]));
            t0[m] = fma(-hx, di.x[m], fma(-hy, di.y[m], t0[m]));
        }
    }
    int64_t diff = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) diff |= dbits(tj[m]) ^ dbits(t0[m]);
    return diff != 0;
}

// Eq. 26 from the primitive state (rho, u, v, p).
__device__ __forceinline__ void prim_to_q(const double rho, const double u, const double v,
                                          const double p, const Physics& ph, V4& q) {
    const double beta = rho / (2.0 * p);
    q.a = log(rho) + log(beta) * ph.gm1_inv - beta * (u * u + v * v);
    q.b = 2.0 * beta * u;
    q.c = 2.0 * beta * v;
    q.d = -2.0 * beta;
}

__device__ __forceinline__ bool physical(double rho, double u, double v, double p) {
    return rho > 0.0 && p > 0.0 && isfinite(rho) && isfinite(p) && isfinite(u) && isfinite(v);
}

// Block-wide sum in a fixed order (warp shuffles, then the warps' partials
// by the first warp), so the result does not depend on timing.
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
    return s;  // valid in thread 0
}

// ----------------------------------------------------------- q-derivatives

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_ls_first(const DevGeom g, const V4* __restrict__ q,
                                                    V8* __restrict__ dq) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    if (d >= g.n) return;
    const V4 qi = ld4(q + t);
    double ax[4] = {0, 0, 0, 0}, ay[4] = {0, 0, 0, 0};
    const int c = g.cnt[d];
    for (int k = 0; k < c; ++k) {
        const int64_t at = int64_t(k) * g.stride + d;
        const uint32_t j = g.nbr[at] & kIndexMask;
        const double wx = g.wx[at], wy = g.wy[at];
        const V4 qj = ld4(q + sidx(g, j, cc));
        const double dq0 = qj.a - qi.a, dq1 = qj.b - qi.b, dq2 = qj.c - qi.c, dq3 = qj.d - qi.d;
        ax[0] += wx * dq0; ax[1] += wx * dq1; ax[2] += wx * dq2; ax[3] += wx * dq3;
        ay[0] += wy * dq0; ay[1] += wy * dq1; ay[2] += wy * dq2; ay[3] += wy * dq3;
    }
    V8 o;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        o.x[m] = ax[m];
        o.y[m] = ay[m];
    }
    dq[t] = o;
}

// One Jacobi sweep of Eq. 29. With dq~_j = (q_j - q_i) - (hdx_j (qx_j - qx_i)
// + hdy_j (qy_j - qy_i)) (Eq. 28, hdx = dx/2) the sweep is
//   q_x = sum_j wx_j (q_j - q_i) - [sum_j (a_j qx_j + b_j qy_j) - (A qx_i + B qy_i)]
// with a_j = wx_j hdx_j, b_j = wx_j hdy_j, A = sum_j a_j, B = sum_j b_j (and
// c, d, C, D from wy for q_y). The first sum is the first-order derivative of
// the same stage (dq_first), so a sweep gathers only the neighbours'
// derivatives: 4 FMAs per component and neighbour instead of 7 FP64
// operations. The bracket is ~1e-4 of q_x at 10M points and is formed to
// ~1e-12 of itself, so q_x keeps FP64 accuracy.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_ls_inner(const DevGeom g, const V8* __restrict__ dq_first,
                                                    const V8* __restrict__ din,
                                                    V8* __restrict__ dout) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    if (d >= g.n) return;
    double ax[4] = {0, 0, 0, 0}, ay[4] = {0, 0, 0, 0};
    const int c = g.cnt[d];
    for (int k = 0; k < c; ++k) {
        const int64_t at = int64_t(k) * g.stride + d;
        const uint32_t j = g.nbr[at] & kIndexMask;
        const V4 p = g.lcoef[at];
        const V8 dj = din[sidx(g, j, cc)];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            ax[m] = fma(p.a, dj.x[m], fma(p.b, dj.y[m], ax[m]));
            ay[m] = fma(p.c, dj.x[m], fma(p.d, dj.y[m], ay[m]));
        }
    }
    const V4 S = g.lsum[d];
    const V8 di = din[t];
    const V8 f = dq_first[t];
    V8 o;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        o.x[m] = f.x[m] - (ax[m] - fma(S.a, di.x[m], S.b * di.y[m]));
        o.y[m] = f.y[m] - (ay[m] - fma(S.c, di.x[m], S.d * di.y[m]));
    }
    dout[t] = o;
}

// ------------------------------------------------------- flux residual + RK

// SSP-RK stage epilogue of one (point, condition), shared by the fused flux
// kernel and the split-flux ablation: mode 0 stores R; modes 1..4 apply the
// stage update, the wall condition and the next q; stage 1 also stores dt
// and U0 and returns R_rho^2 for the residue.
template <int MODE, bool G14>
__device__ __forceinline__ double stage_epilogue(const DevGeom& g, const Physics& ph,
                                                 const DevState& st, const int64_t t,
                                                 const int64_t d, const int8_t fl, const bool fixed,
                                                 const double R[4], V4* __restrict__ q_out) {
    double r2 = 0.0;
    if (MODE == 0) {
        st.R[t] = V4{R[0], R[1], R[2], R[3]};
    } else {
        V4 U = ld4(st.U + t);
        double dtv;
        if (MODE == 1) {
            const double rho = U.a, u = U.b / rho, v = U.c / rho;
            const double p = ph.gm1 * (U.d - 0.5 * rho * (u * u + v * v));
            dtv = ph.cfl * g.dmin[d] / (sqrt(u * u + v * v) + sqrt(ph.gamma * p / rho));
            st.dt[t] = dtv;
            st.U0[t] = U;
            r2 = R[0] * R[0];
        } else {
            dtv = st.dt[t];
        }
        if (!fixed) {
            const double h = 0.5 * dtv;
            if (MODE == 3) {
                const V4 U0 = ld4(st.U0 + t);
                U.a = (2.0 / 3.0) * U0.a + (1.0 / 3.0) * (U.a - h * R[0]);
                U.b = (2.0 / 3.0) * U0.b + (1.0 / 3.0) * (U.b - h * R[1]);
                U.c = (2.0 / 3.0) * U0.c + (1.0 / 3.0) * (U.c - h * R[2]);
                U.d = (2.0 / 3.0) * U0.d + (1.0 / 3.0) * (U.d - h * R[3]);
            } else {
                U.a -= h * R[0];
                U.b -= h * R[1];
                U.c -= h * R[2];
                U.d -= h * R[3];
            }
            if (fl == LSKUM_WALL) {  // remove the wall-normal momentum
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
        q_out[t] = qn;
        if (!physical(rho, u, v, p)) atomicOr(st.status, 1);
    }

    return r2;
}

template <int MODE, int BLOCK, bool G14>
__global__ void __launch_bounds__(BLOCK) k_flux(const DevGeom g, const Physics ph,
                                                const DevState st, const V4* __restrict__ q_in,
                                                const V8* __restrict__ dq, V4* __restrict__ q_out) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;  // (point, condition)
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    double r2 = 0.0;
    if (d < g.n) {
        const int8_t fl = g.flag[d];
        const bool fixed = ph.outer_fixed && fl == LSKUM_OUTER;
        double R[4] = {0.0, 0.0, 0.0, 0.0};
        if (!fixed) {
            double tx = 1.0, ty = 0.0, nx = 0.0, ny = 1.0;
            const bool local = fl != LSKUM_INTERIOR;
            if (local) {
                const double2 nn = g.nrm[d];
                nx = nn.x;
                ny = nn.y;
                tx = ny;
                ty = -nx;
            }
            const V4 qi = ld4(q_in + t);
            const V8 di = dq[t];
            const double qiv[4] = {qi.a, qi.b, qi.c, qi.d};
            const bool second = ph.order == 2;
            const int c = g.cnt[d];
            for (int k = 0; k < c; ++k) {
                const int64_t at = int64_t(k) * g.stride + d;
                const uint32_t e = g.nbr[at];
                const uint32_t j = e & kIndexMask;
                const uint32_t sc = (e >> kIndexBits) & 3u;
                const uint32_t nc = (e >> (kIndexBits + 2)) & 3u;
                const int64_t jt = sidx(g, j, cc);
                const V4 qj = ld4(q_in + jt);
                double tj[4] = {qj.a, qj.b, qj.c, qj.d};
                double t0[4] = {qiv[0], qiv[1], qiv[2], qiv[3]};
                // equal modified states give dG = 0 exactly (free-stream preservation);
                // the two inlined flux evaluations below need not round identically
                if (!modified_states(second, second ? g.hdx[at] : 0.0, second ? g.hdy[at] : 0.0,
                                     second ? dq[jt] : di, di, tj, t0))
                    continue;
                Prim wj = q_to_prim<G14>(tj[0], tj[1], tj[2], tj[3], ph.gm1_inv);
                Prim w0 = q_to_prim<G14>(t0[0], t0[1], t0[2], t0[3], ph.gm1_inv);
                if (local) {  // velocities into (s, n)
                    const double sj = wj.u * tx + wj.v * ty, nj = wj.u * nx + wj.v * ny;
                    const double s0 = w0.u * tx + w0.v * ty, n0 = w0.u * nx + w0.v * ny;
                    wj.u = sj; wj.v = nj;
                    w0.u = s0; w0.v = n0;
                }
                if (sc) {
                    const int64_t nmask = sc == 1u ? 0 : kSignBit;
                    double dg[4];
                    split_flux_diff(wj, w0, wj.u, wj.v, w0.u, w0.v, split_ab(wj, wj.u, nmask),
                                    split_ab(w0, w0.u, nmask), dg);
                    const double w = g.ws[at];
                    R[0] = fma(w, dg[0], R[0]);
                    R[1] = fma(w, dg[1], R[1]);
                    R[2] = fma(w, dg[2], R[2]);
                    R[3] = fma(w, dg[3], R[3]);
                }
                if (nc) {
                    const int64_t nmask = nc == 1u ? 0 : kSignBit;
                    double dg[4];
                    // along n: "a" = n-velocity, "b" = s-velocity
                    split_flux_diff(wj, w0, wj.v, wj.u, w0.v, w0.u, split_ab(wj, wj.v, nmask),
                                    split_ab(w0, w0.v, nmask), dg);
                    const double w = g.wn[at];
                    R[0] = fma(w, dg[0], R[0]);
                    R[1] = fma(w, dg[2], R[1]);  // s-momentum
                    R[2] = fma(w, dg[1], R[2]);  // n-momentum
                    R[3] = fma(w, dg[3], R[3]);
                }
            }
            if (local) {  // momentum back to the global frame
                const double rs = R[1], rn = R[2];
                R[1] = rs * tx + rn * nx;
                R[2] = rs * ty + rn * ny;
            }
        }
        r2 = stage_epilogue<MODE, G14>(g, ph, st, t, d, fl, fixed, R, q_out);
    }
    if (MODE == 1) {
        if (g.cshift == 0) {  // one condition: fused block partial sums
            const double s = block_sum<BLOCK>(r2);
            if (threadIdx.x == 0) st.partials[blockIdx.x] = s;
        } else if (d < g.n) {  // several: per (point, condition), reduced per condition
            st.r2[t] = r2;
        }
    }
}

// ------------------------------------------------ split-flux kernels (ablation)
// The paper's kernel splitting (Section 5, the four split-flux kernels Gx+,
// Gx-, Gy+, Gy-): one kernel per split-flux derivative dGs+/ds, dGs-/ds,
// dGn+/dn, dGn-/dn, each adding its stencil's contribution to the residual
// (local frame) in Racc, then one kernel for the stage update. An ablation of
// the fused kernel: a neighbour's two q~ -> primitive maps are computed once
// per stencil it belongs to (twice), and Racc makes four extra round trips.
template <int PART, int BLOCK, bool G14>
__global__ void __launch_bounds__(BLOCK) k_flux_part(const DevGeom g, const Physics ph,
                                                     const V4* __restrict__ q_in,
                                                     const V8* __restrict__ dq,
                                                     V4* __restrict__ Racc) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;
    const int64_t d = t >> g.cshift;
    const uint32_t cc = uint32_t(t) & g.cmask;
    if (d >= g.n) return;
    const int8_t fl = g.flag[d];
    double R[4] = {0.0, 0.0, 0.0, 0.0};
    if (!(ph.outer_fixed && fl == LSKUM_OUTER)) {
        double tx = 1.0, ty = 0.0, nx = 0.0, ny = 1.0;
        const bool local = fl != LSKUM_INTERIOR;
        if (local) {
            const double2 nn = g.nrm[d];
            nx = nn.x;
            ny = nn.y;
            tx = ny;
            ty = -nx;
        }
        const V4 qi = ld4(q_in + t);
        const V8 di = dq[t];
        const double qiv[4] = {qi.a, qi.b, qi.c, qi.d};
        const bool second = ph.order == 2;
        const uint32_t want = (PART % 2 == 0) ? 1u : 2u;
        const int64_t nmask = (PART % 2 == 0) ? 0 : kSignBit;
        const int c = g.cnt[d];
        for (int k = 0; k < c; ++k) {
            const int64_t at = int64_t(k) * g.stride + d;
            const uint32_t e = g.nbr[at];
            const uint32_t code = PART < 2 ? ((e >> kIndexBits) & 3u) : ((e >> (kIndexBits + 2)) & 3u);
            if (code != want) continue;
            const uint32_t j = e & kIndexMask;
            const int64_t jt = sidx(g, j, cc);
            const V4 qj = ld4(q_in + jt);
            double tj[4] = {qj.a, qj.b, qj.c, qj.d};
            double t0[4] = {qiv[0], qiv[1], qiv[2], qiv[3]};
            if (!modified_states(second, second ? g.hdx[at] : 0.0, second ? g.hdy[at] : 0.0,
                                 second ? dq[jt] : di, di, tj, t0))
                continue;
            Prim wj = q_to_prim<G14>(tj[0], tj[1], tj[2], tj[3], ph.gm1_inv);
            Prim w0 = q_to_prim<G14>(t0[0], t0[1], t0[2], t0[3], ph.gm1_inv);
            if (local) {
                const double sj = wj.u * tx + wj.v * ty, nj = wj.u * nx + wj.v * ny;
                const double s0 = w0.u * tx + w0.v * ty, n0 = w0.u * nx + w0.v * ny;
                wj.u = sj; wj.v = nj;
                w0.u = s0; w0.v = n0;
            }
            double dg[4];
            if (PART < 2) {
                split_flux_diff(wj, w0, wj.u, wj.v, w0.u, w0.v, split_ab(wj, wj.u, nmask),
                                split_ab(w0, w0.u, nmask), dg);
                const double w = g.ws[at];
                R[0] = fma(w, dg[0], R[0]);
                R[1] = fma(w, dg[1], R[1]);
                R[2] = fma(w, dg[2], R[2]);
                R[3] = fma(w, dg[3], R[3]);
            } else {
                split_flux_diff(wj, w0, wj.v, wj.u, w0.v, w0.u, split_ab(wj, wj.v, nmask),
                                split_ab(w0, w0.v, nmask), dg);
                const double w = g.wn[at];
                R[0] = fma(w, dg[0], R[0]);
                R[1] = fma(w, dg[2], R[1]);
                R[2] = fma(w, dg[1], R[2]);
                R[3] = fma(w, dg[3], R[3]);
            }
        }
    }
    if (PART == 0) {
        Racc[t] = V4{R[0], R[1], R[2], R[3]};
    } else {
        V4 a = Racc[t];
        a.a += R[0];
        a.b += R[1];
        a.c += R[2];
        a.d += R[3];
        Racc[t] = a;
    }
}

template <int MODE, int BLOCK, bool G14>
__global__ void __launch_bounds__(BLOCK) k_stage_split(const DevGeom g, const Physics ph,
                                                       const DevState st, const V4* __restrict__ Racc,
                                                       V4* __restrict__ q_out) {
    const int64_t t = int64_t(blockIdx.x) * BLOCK + threadIdx.x;
    const int64_t d = t >> g.cshift;
    double r2 = 0.0;
    if (d < g.n) {
        const int8_t fl = g.flag[d];
        const bool fixed = ph.outer_fixed && fl == LSKUM_OUTER;
        double R[4] = {0.0, 0.0, 0.0, 0.0};
        if (!fixed) {
            const V4 a = Racc[t];
            R[0] = a.a;
            R[1] = a.b;
            R[2] = a.c;
            R[3] = a.d;
            if (fl != LSKUM_INTERIOR) {
                const double2 nn = g.nrm[d];
                const double tx = nn.y, ty = -nn.x;
                const double rs = R[1], rn = R[2];
                R[1] = rs * tx + rn * nn.x;
                R[2] = rs * ty + rn * nn.y;
            }
        }
        r2 = stage_epilogue<MODE, G14>(g, ph, st, t, d, fl, fixed, R, q_out);
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

// Residue = sqrt(sum of the per-block partials) / N, summed in block order by
// one block (deterministic), appended to the history ring buffer.
__global__ void __launch_bounds__(kReduceBlock) k_residue(const DevState st, int nblocks,
                                                          int64_t n) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kReduceBlock) s += st.partials[b];
    s = block_sum<kReduceBlock>(s);
    if (threadIdx.x == 0) {
        const unsigned long long it = *st.iter_counter;
        const double r = sqrt(s) / double(n);
        st.res_hist[it % (unsigned long long)st.res_cap] = r;
        *st.iter_counter = it + 1;
        if (!isfinite(r)) atomicOr(st.status, 1);
    }
}

// ------------------------------------------------------------ state I/O

__global__ void k_set_uniform(const DevGeom g, const Physics ph, const V4* __restrict__ Wc,
                              V4* U, V4* q) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t d = t >> g.cshift;
    if (d >= g.n) return;
    const V4 W = Wc[uint32_t(t) & g.cmask];
    V4 u;
    u.a = W.a;
    u.b = W.a * W.b;
    u.c = W.a * W.c;
    u.d = W.d * ph.gm1_inv + 0.5 * W.a * (W.b * W.b + W.c * W.c);
    U[t] = u;
    // q straight from the given primitive state (no round trip through U)
    V4 qq;
    prim_to_q(W.a, W.b, W.c, W.d, ph, qq);
    q[t] = qq;
}

// W_user is condition-major in the caller's point order: [condition][point].
__global__ void k_set_prim(const DevGeom g, const Physics ph, const V4* __restrict__ W_user,
                           V4* U, V4* q, int* status) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t d = t >> g.cshift;
    if (d >= g.n) return;
    const int64_t cc = int64_t(uint32_t(t) & g.cmask);
    const V4 W = W_user[cc * g.n + g.dev_to_user[d]];
    if (!physical(W.a, W.b, W.c, W.d)) atomicOr(status, 2);
    V4 u;
    u.a = W.a;
    u.b = W.a * W.b;
    u.c = W.a * W.c;
    u.d = W.d * ph.gm1_inv + 0.5 * W.a * (W.b * W.b + W.c * W.c);
    U[t] = u;
    // q straight from the given primitive state (no round trip through U)
    V4 qq;
    prim_to_q(W.a, W.b, W.c, W.d, ph, qq);
    q[t] = qq;
}

__global__ void k_get_prim(const DevGeom g, const Physics ph, const V4* __restrict__ U,
                           V4* __restrict__ W_user) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t d = t >> g.cshift;
    if (d >= g.n) return;
    const int64_t cc = int64_t(uint32_t(t) & g.cmask);
    const V4 u = U[t];
    const double rho = u.a, uu = u.b / rho, vv = u.c / rho;
    const double p = ph.gm1 * (u.d - 0.5 * rho * (uu * uu + vv * vv));
    W_user[cc * g.n + g.dev_to_user[d]] = V4{rho, uu, vv, p};
}

__global__ void k_q_from_U(const DevGeom g, const Physics ph, const V4* __restrict__ U,
                           V4* __restrict__ q) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if ((t >> g.cshift) >= g.n) return;
    V4 qq;
    double rho, uu, vv, p;
    if (fabs(ph.gm1_inv - 2.5) < 1e-12)
        cons_to_q64<true>(U[t], ph, qq, rho, uu, vv, p);
    else
        cons_to_q64<false>(U[t], ph, qq, rho, uu, vv, p);
    q[t] = qq;
}

template <typename T>
__global__ void k_gather(const DevGeom g, const T* __restrict__ src, T* __restrict__ dst) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t d = t >> g.cshift;
    if (d >= g.n) return;
    const int64_t cc = int64_t(uint32_t(t) & g.cmask);
    dst[cc * g.n + g.dev_to_user[d]] = src[t];
}

// Residue per condition (C > 1), phase 1: block b reduces a contiguous range
// of points for every condition into cpartials[b][c] (rows in a fixed order).
__global__ void __launch_bounds__(512) k_residue_cond_p1(const DevGeom g, const DevState st) {
    __shared__ double part[16][33];
    const int64_t C = int64_t(1) << g.cshift;
    const int64_t rows_per_block = (g.n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
    const int64_t r1 = min(g.n, r0 + rows_per_block);
    for (int64_t c0 = 0; c0 < C; c0 += 32) {
        const int64_t c = c0 + threadIdx.x;
        double s = 0.0;
        if (c < C)
            for (int64_t r = r0 + threadIdx.y; r < r1; r += 16) s += st.r2[(r << g.cshift) | c];
        part[threadIdx.y][threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.y == 0 && c < C) {
            double tot = 0.0;
            for (int k = 0; k < 16; ++k) tot += part[k][threadIdx.x];
            st.cpartials[int64_t(blockIdx.x) * C + c] = tot;
        }
        __syncthreads();
    }
}

// Phase 2 (one block): sum the block partials of each condition in block
// order, append sqrt(sum)/N per condition to the history.
__global__ void __launch_bounds__(256) k_residue_cond_p2(const DevGeom g, const DevState st,
                                                         int nblocks) {
    const int64_t C = int64_t(1) << g.cshift;
    const unsigned long long it = *st.iter_counter;
    const int64_t slot = int64_t(it % (unsigned long long)(st.res_cap / C));
    for (int64_t c = threadIdx.x; c < C; c += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += st.cpartials[int64_t(b) * C + c];
        const double r = sqrt(s) / double(g.n);
        st.res_hist[slot * C + c] = r;
        if (!isfinite(r)) atomicOr(st.status, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *st.iter_counter = it + 1;
}

// Pressure force on the wall loops: F = -sum (p_i - p_inf) n_i ds_i; one
// block per condition.
__global__ void __launch_bounds__(kReduceBlock) k_forces(const DevGeom g, const Physics ph,
                                                         const DevState st) {
    const uint32_t cc = blockIdx.x;
    double fx = 0.0, fy = 0.0;
    for (int64_t k = threadIdx.x; k < g.n_wall; k += kReduceBlock) {
        const int32_t d = g.wall_id[k];
        const V4 u = st.U[sidx(g, d, cc)];
        const double rho = u.a, uu = u.b / rho, vv = u.c / rho;
        const double p = ph.gm1 * (u.d - 0.5 * rho * (uu * uu + vv * vv));
        const double2 nds = g.wall_nds[k];
        fx -= (p - ph.p_inf) * nds.x;
        fy -= (p - ph.p_inf) * nds.y;
    }
    fx = block_sum<kReduceBlock>(fx);
    __syncthreads();
    fy = block_sum<kReduceBlock>(fy);
    if (threadIdx.x == 0) {
        st.force_out[2 * cc] = fx;
        st.force_out[2 * cc + 1] = fy;
    }
}

inline unsigned grid_for(int64_t n, int block) { return unsigned((n + block - 1) / block); }
// threads over all (point, condition) pairs
inline unsigned grid_nc(const DevGeom& g, int block) { return grid_for(g.n << g.cshift, block); }

}  // namespace

cudaError_t launch_ls_first(const DevGeom& g, const V4* q, V8* dq, int block, cudaStream_t s) {
    if (block == 256)
        k_ls_first<256><<<grid_nc(g, 256), 256, 0, s>>>(g, q, dq);
    else
        k_ls_first<kDefaultBlock><<<grid_nc(g, kDefaultBlock), kDefaultBlock, 0, s>>>(g, q, dq);
    return cudaGetLastError();
}

cudaError_t launch_ls_inner(const DevGeom& g, const V8* dq_first, const V8* din, V8* dout, int block,
                            cudaStream_t s) {
    if (block == 256)
        k_ls_inner<256><<<grid_nc(g, 256), 256, 0, s>>>(g, dq_first, din, dout);
    else
        k_ls_inner<kDefaultBlock><<<grid_nc(g, kDefaultBlock), kDefaultBlock, 0, s>>>(g, dq_first, din,
                                                                                     dout);
    return cudaGetLastError();
}

template <int BLOCK, bool G14>
static void flux_dispatch(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                          const V4* q_in, const V8* dq, V4* q_out, cudaStream_t s) {
    const unsigned grid = grid_nc(g, BLOCK);
    switch (mode) {
        case 0: k_flux<0, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, q_in, dq, q_out); break;
        case 1: k_flux<1, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, q_in, dq, q_out); break;
        case 2: k_flux<2, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, q_in, dq, q_out); break;
        case 3: k_flux<3, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, q_in, dq, q_out); break;
        default: k_flux<4, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, q_in, dq, q_out); break;
    }
}

cudaError_t launch_flux(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                        const V4* q_in, const V8* dq, V4* q_out, int block, cudaStream_t s) {
    // gamma = 1.4: log-free density (see q_to_prim)
    const bool g14 = fabs(ph.gm1_inv - 2.5) < 1e-12;
    if (block == 256) {
        if (g14) flux_dispatch<256, true>(mode, g, ph, st, q_in, dq, q_out, s);
        else flux_dispatch<256, false>(mode, g, ph, st, q_in, dq, q_out, s);
    } else {
        if (g14) flux_dispatch<kDefaultBlock, true>(mode, g, ph, st, q_in, dq, q_out, s);
        else flux_dispatch<kDefaultBlock, false>(mode, g, ph, st, q_in, dq, q_out, s);
    }
    return cudaGetLastError();
}

template <int BLOCK, bool G14>
static void flux_split_dispatch(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                                const V4* q_in, const V8* dq, V4* q_out, cudaStream_t s) {
    const unsigned grid = grid_nc(g, BLOCK);
    V4* Racc = st.R;  // accumulator (R is an output only of the evaluation mode)
    k_flux_part<0, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, q_in, dq, Racc);
    k_flux_part<1, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, q_in, dq, Racc);
    k_flux_part<2, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, q_in, dq, Racc);
    k_flux_part<3, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, q_in, dq, Racc);
    switch (mode) {
        case 0: k_stage_split<0, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, Racc, q_out); break;
        case 1: k_stage_split<1, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, Racc, q_out); break;
        case 2: k_stage_split<2, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, Racc, q_out); break;
        case 3: k_stage_split<3, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, Racc, q_out); break;
        default: k_stage_split<4, BLOCK, G14><<<grid, BLOCK, 0, s>>>(g, ph, st, Racc, q_out); break;
    }
}

cudaError_t launch_flux_split(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                              const V4* q_in, const V8* dq, V4* q_out, int block, cudaStream_t s) {
    const bool g14 = fabs(ph.gm1_inv - 2.5) < 1e-12;
    if (block == 256) {
        if (g14) flux_split_dispatch<256, true>(mode, g, ph, st, q_in, dq, q_out, s);
        else flux_split_dispatch<256, false>(mode, g, ph, st, q_in, dq, q_out, s);
    } else {
        if (g14) flux_split_dispatch<kDefaultBlock, true>(mode, g, ph, st, q_in, dq, q_out, s);
        else flux_split_dispatch<kDefaultBlock, false>(mode, g, ph, st, q_in, dq, q_out, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_residue(const DevState& st, int nblocks, int64_t n, cudaStream_t s) {
    k_residue<<<1, kReduceBlock, 0, s>>>(st, nblocks, n);
    return cudaGetLastError();
}

cudaError_t launch_residue_cond(const DevGeom& g, const DevState& st, cudaStream_t s) {
    k_residue_cond_p1<<<kCondReduceBlocks, dim3(32, 16), 0, s>>>(g, st);
    k_residue_cond_p2<<<1, 256, 0, s>>>(g, st, kCondReduceBlocks);
    return cudaGetLastError();
}

cudaError_t launch_set_uniform(const DevGeom& g, const Physics& ph, const V4* W_cond, V4* U, V4* q,
                               cudaStream_t s) {
    k_set_uniform<<<grid_nc(g, 256), 256, 0, s>>>(g, ph, W_cond, U, q);
    return cudaGetLastError();
}

cudaError_t launch_set_prim(const DevGeom& g, const Physics& ph, const V4* W_user, V4* U, V4* q,
                            int* status, cudaStream_t s) {
    k_set_prim<<<grid_nc(g, 256), 256, 0, s>>>(g, ph, W_user, U, q, status);
    return cudaGetLastError();
}

cudaError_t launch_get_prim(const DevGeom& g, const Physics& ph, const V4* U, V4* W_user,
                            cudaStream_t s) {
    k_get_prim<<<grid_nc(g, 256), 256, 0, s>>>(g, ph, U, W_user);
    return cudaGetLastError();
}

cudaError_t launch_q_from_U(const DevGeom& g, const Physics& ph, const V4* U, V4* q, cudaStream_t s) {
    k_q_from_U<<<grid_nc(g, 256), 256, 0, s>>>(g, ph, U, q);
    return cudaGetLastError();
}

cudaError_t launch_gather_v4(const DevGeom& g, const V4* src, V4* dst, cudaStream_t s) {
    k_gather<V4><<<grid_nc(g, 256), 256, 0, s>>>(g, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_gather_v8(const DevGeom& g, const V8* src, V8* dst, cudaStream_t s) {
    k_gather<V8><<<grid_nc(g, 256), 256, 0, s>>>(g, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_forces(const DevGeom& g, const Physics& ph, const DevState& st, cudaStream_t s) {
    k_forces<<<unsigned(1u << g.cshift), kReduceBlock, 0, s>>>(g, ph, st);
    return cudaGetLastError();
}

}  // namespace lskum

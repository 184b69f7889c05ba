// Device math shared by the FP64 and the mixed-precision kernels: the
// table-driven logarithm and the q-variables (Eq. 26) from the conserved
// state, both in FP64.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lskum_kernels.cuh"
#include "math_tables.h"

namespace lskum {

// Natural logarithm by the table of math_tables.h (Tang-style reduction):
// x = 2^e m, m in [1, 2), c_j the midpoint of m's 1/128 interval, F_j = 1/c_j
// rounded, r = m F_j - 1 from one fused multiply-add (|r| <= 2^-8), log x =
// e ln2 - log F_j + log1p(r) with the degree-6 Taylor polynomial of log1p
// (remainder below 2e-18) and ln2, -log F_j as pairs of doubles: about 12
// FP64 operations against the library's ~33 (the stage epilogues run it on
// the FP64 pipe, at 1/64 of the FP32 rate on this GPU). Positive normal
// arguments only: the rest (zero, subnormal, negative, non-finite: a
// diverged state) goes to the library function.
__device__ __forceinline__ double log_tab(const double x) {
    const int64_t b = __double_as_longlong(x);
    if (uint64_t(b - 0x0010000000000000LL) >= uint64_t(0x7FE0000000000000LL)) return log(x);
    const double e = double(int(b >> 52) - 1023);
    const double* t = kLogTab[int(b >> (52 - kLogBits)) & ((1 << kLogBits) - 1)];
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double r = fma(m, __ldg(t), -1.0);
    double p = fma(r, -1.0 / 6.0, 0.2);
    p = fma(r, p, -0.25);
    p = fma(r, p, 1.0 / 3.0);
    p = fma(r, p, -0.5);
    p = fma(r, p, 1.0);
    p *= r;
    return fma(e, kLn2Hi, __ldg(t + 1) + (p + fma(e, kLn2Lo, __ldg(t + 2))));
}

// q-variables (Eq. 26) from the conserved state in FP64, to a few ulp (the
// FP64 path's next stage and the mixed path's float-pair split take them).
// With beta = rho/(2p): q2 = 2 beta u1 = m1/p, q3 = m2/p, q4 = -rho/p,
// beta |u|^2 = |m|^2 / (2 rho p), and for gamma = 1.4 ln rho +
// ln(beta)/(gamma-1) = ln(rho^2 beta^5) / 2. rho p = (gamma - 1)(rho E -
// |m|^2/2) needs no division, so 1/rho and 1/p both come from one
// reciprocal of rho^2 p, and the logarithm needs no square root: one
// division and one table logarithm per point instead of three divisions and
// two library logarithms.
template <bool G14>
__device__ __forceinline__ void cons_to_q64(const V4& U, const Physics& ph, V4& q, double& rho,
                                            double& u, double& v, double& p) {
    rho = U.a;
    const double m2 = fma(U.b, U.b, U.c * U.c);           // |m|^2
    const double rp = ph.gm1 * fma(U.d, rho, -0.5 * m2);  // rho p
    const double rr = 1.0 / (rho * rp);                   // 1 / (rho^2 p)
    const double irho = rp * rr;
    const double ip = (rho * rho) * rr;
    u = U.b * irho;
    v = U.c * irho;
    p = rp * irho;
    const double bu2 = 0.5 * m2 * (rho * rr);  // beta |u|^2
    if (G14) {
        const double beta = 0.5 * rho * ip;
        const double b2 = beta * beta;
        q.a = 0.5 * log_tab((rho * rho) * (b2 * b2 * beta)) - bu2;
    } else {
        q.a = log_tab(rho) + log_tab(0.5 * rho * ip) * ph.gm1_inv - bu2;
    }
    q.b = U.b * ip;
    q.c = U.c * ip;
    q.d = -rho * ip;
}

}  // namespace lskum

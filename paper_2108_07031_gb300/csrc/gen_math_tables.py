"""Writes ``math_tables.h``: the FP64 flux kernel's function tables.

1. Polynomial pieces for the split-flux erfc.

The kinetic split fluxes need A = erfc(x) / 2 and B ~ exp(-x^2) at the same
argument. The device code evaluates erfc(a) = exp(-a^2) erfcx(a) for
0 <= a = |x| <= 6, reusing exp(-a^2) from B, with erfcx (the scaled
complementary error function, smooth and positive on the whole range) as a
polynomial of degree 6 in (a - c_k) on 384 intervals of width 1/64 centred
at c_k; the interval index is floor(64 a), which the device takes from the
bits of a. (Narrow pieces keep the degree, and so the FP64 instructions per
evaluation, low: width 1/8 needed degree 9 for the same accuracy.)
One formula for every argument keeps the lanes of a warp on one path.
Each polynomial is the Chebyshev interpolant of erfcx (computed with mpmath
at 50 digits from erfcx(a) = e^(a^2) erfc(a)) converted to the monomial
basis of the local variable; the script checks the relative error of every
piece at 400 points in double-precision Horner evaluation and refuses to
write the header unless it is below 4e-16.

   The mixed-precision path evaluates the same function in FP32 from its own
   table: 24 pieces of width 1/4 and degree 5 (checked below 3e-7 relative
   in float32 Horner evaluation).

2. The exponential by Tang's table-driven method: x = k ln2/256 + r with
|r| <= ln2/512, exp(x) = 2^(k div 256) * 2^((k mod 256)/256) * e^r, with
e^r - 1 from its degree-4 Taylor polynomial (remainder below 4e-17 of e^r on
that interval); the table holds 2^(j/256), j < 256, correctly rounded
(mpmath), and ln2/256 is split into a double and its remainder for an exact
reduction.

3. The natural logarithm by a table-driven reduction (the mixed-precision
path's FP64 epilogue, where the FP64 pipe binds): x = 2^e m, m in [1, 2);
the top 7 bits of m pick c_j = 1 + (j + 1/2)/128, the table holds F_j =
1/c_j rounded to double and -log(F_j) exactly as a pair of doubles (hi, lo),
so log x = e ln2 - log F_j + log1p(r) with r = m F_j - 1 (one fused
multiply-add, |r| <= 2^-8) and log1p(r) from its degree-6 Taylor
polynomial (remainder below 2e-18).

Run: python gen_math_tables.py  (writes math_tables.h next to this file)
"""

import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50

CX_LO, CX_HI, CX_LOG2_INV_W = 0.0, 6.0, 6
CX_W = 2.0 ** -CX_LOG2_INV_W
CX_DEG = 6            # degree in z = a - c on [-1/128, 1/128]
EXP_BITS = 8          # 2^(j / 2^EXP_BITS) table
LOG_BITS = 7          # 2^LOG_BITS mantissa intervals for the log table
CXF_W, CXF_DEG = 0.25, 5  # FP32 table (mixed precision)


def cheb_to_monomial(f, lo, hi, deg, shift):
    """Monomial coefficients (in u - shift) of the Chebyshev interpolant of f on [lo, hi]."""
    n = deg + 1
    nodes = [mp.mpf(lo + hi) / 2 + mp.mpf(hi - lo) / 2 * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n)
             for k in range(n)]
    vals = [f(u) for u in nodes]
    # solve the Vandermonde system in the shifted monomial basis (high precision)
    A = mp.matrix(n, n)
    for i, u in enumerate(nodes):
        for j in range(n):
            A[i, j] = (u - shift) ** j
    coef = mp.lu_solve(A, mp.matrix(vals))
    return [coef[j] for j in range(n)]


def horner(c, z):
    r = np.zeros_like(z) + float(c[-1])
    for k in range(len(c) - 2, -1, -1):
        r = r * z + float(c[k])
    return r


def horner_f32(c, z):
    c = [np.float32(float(v)) for v in c]
    r = np.zeros_like(z, dtype=np.float32) + c[-1]
    for k in range(len(c) - 2, -1, -1):
        r = (r * z + c[k]).astype(np.float32)
    return r


def erfcx_pieces_f32():
    """FP32 pieces of erfcx on [CX_LO, CX_HI]: (centres, coefficients, worst error)."""
    centres, pieces, worst = [], [], 0.0
    a = CX_LO
    while a < CX_HI - 1e-12:
        lo, hi = a, a + CXF_W
        c = (lo + hi) / 2
        C = cheb_to_monomial(lambda u: mp.erfc(u) * mp.exp(u * u), mp.mpf(lo), mp.mpf(hi), CXF_DEG,
                             mp.mpf(c))
        zs = np.linspace(lo, hi, 500)
        ref = np.array([float(mp.erfc(mp.mpf(float(u))) * mp.exp(mp.mpf(float(u)) ** 2))
                        for u in zs])
        got = horner_f32(C, (zs.astype(np.float32) - np.float32(c)).astype(np.float32))
        e = np.max(np.abs(got - ref) / np.abs(ref))
        assert e < 3e-7, ("erfcx f32", lo, e)
        worst = max(worst, e)
        centres.append(c)
        pieces.append([float(np.float32(float(x))) for x in C])
        a = hi
    return centres, pieces, worst


def main(path=None):
    """Writes the header to `path` (default: math_tables.h next to this file)."""
    centres = []
    pieces = []
    worst = 0.0
    a = CX_LO
    while a < CX_HI - 1e-12:
        lo, hi = a, a + CX_W
        c = (lo + hi) / 2
        C = cheb_to_monomial(lambda u: mp.erfc(u) * mp.exp(u * u), mp.mpf(lo), mp.mpf(hi), CX_DEG,
                             mp.mpf(c))
        zs = np.linspace(lo, hi, 400)
        ref = np.array([float(mp.erfc(mp.mpf(float(u))) * mp.exp(mp.mpf(float(u)) ** 2))
                        for u in zs])
        got = horner(C, zs - c)
        e = np.max(np.abs(got - ref) / np.abs(ref))
        assert e < 4e-16, ("erfcx", lo, e)
        worst = max(worst, e)
        centres.append(c)
        pieces.append([float(x) for x in C])
        a = hi

    # 2^(j/256) and the split of ln2/256
    n_exp = 1 << EXP_BITS
    tab = [float(mp.mpf(2) ** (mp.mpf(j) / n_exp)) for j in range(n_exp)]
    ln2_n = mp.log(2) / n_exp
    hi = float(ln2_n)
    lo = float(ln2_n - mp.mpf(hi))
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "math_tables.h")
    with open(path, "w") as f:
        f.write("// Generated by gen_math_tables.py -- do not edit.\n")
        f.write("// Chebyshev interpolants (mpmath, 50 digits) of erfcx(a) = exp(a^2) erfc(a)\n")
        f.write(f"// in (a - c_k) on intervals of width {CX_W} covering [{CX_LO}, {CX_HI}].\n")
        f.write(f"// Max relative error in double Horner: {worst:.2e}.\n")
        f.write("#pragma once\n\nnamespace lskum {\n\n")
        f.write(f"constexpr double kErfcxLo = {CX_LO!r};\nconstexpr double kErfcxHi = {CX_HI!r};\n")
        f.write(f"constexpr double kErfcxInvW = {1.0 / CX_W!r};\n")
        f.write(f"constexpr int kErfcxLog2InvW = {CX_LOG2_INV_W};\n")
        f.write(f"constexpr int kErfcxPieces = {len(pieces)};\nconstexpr int kErfcxDeg = {CX_DEG};\n")
        f.write("__device__ const double kErfcxC[kErfcxPieces][kErfcxDeg + 2] = {\n")
        for c, p in zip(centres, pieces):
            f.write("    {" + f"{c!r}, " + ", ".join(repr(x) for x in p) + "},\n")
        f.write("};\n\n")
        fc, fp, fworst = erfcx_pieces_f32()
        f.write(f"// FP32 erfcx pieces (mixed precision): width {CXF_W}, degree {CXF_DEG}, "
                f"max relative error {fworst:.2e} in float32 Horner.\n")
        f.write(f"constexpr float kErfcxFInvW = {1.0 / CXF_W!r}f;\n")
        f.write(f"constexpr int kErfcxFPieces = {len(fp)};\nconstexpr int kErfcxFDeg = {CXF_DEG};\n")
        f.write("__device__ const float kErfcxF[kErfcxFPieces][kErfcxFDeg + 2] = {\n")
        for c, p in zip(fc, fp):
            f.write("    {" + f"{c!r}f, " + ", ".join(f"{x!r}f" for x in p) + "},\n")
        f.write("};\n\n")
        f.write(f"// exp(x) by Tang's table-driven reduction: 2^(j/{n_exp}), j < {n_exp}, correctly "
                "rounded,\n")
        f.write(f"// and ln2/{n_exp} = kLn2ByNHi + kLn2ByNLo.\n")
        f.write(f"constexpr int kExpBits = {EXP_BITS};\n")
        f.write(f"constexpr double kLn2ByNHi = {hi!r};\nconstexpr double kLn2ByNLo = {lo!r};\n")
        f.write(f"constexpr double kInvLn2ByN = {float(1 / ln2_n)!r};\n")
        f.write(f"__device__ const double kExp2Tab[{n_exp}] = {{\n")
        for j in range(0, n_exp, 4):
            f.write("    " + ", ".join(repr(v) for v in tab[j:j + 4]) + ",\n")
        f.write("};\n\n")
        n_log = 1 << LOG_BITS
        ln2 = mp.log(2)
        ln2_hi = float(mp.mpf(int(float(ln2) * 2 ** 42)) / 2 ** 42)  # 42 significant bits
        ln2_lo = float(ln2 - mp.mpf(ln2_hi))
        f.write(f"// log(x) by table: c_j = 1 + (j + 1/2)/{n_log}; per row {{F_j = 1/c_j rounded, "
                "-log F_j (hi), (lo), 0}; ln2 = kLn2Hi + kLn2Lo with kLn2Hi of 42 significant bits\n")
        f.write("// (e kLn2Hi is exact for |e| < 2048).\n")
        f.write(f"constexpr int kLogBits = {LOG_BITS};\n")
        f.write(f"constexpr double kLn2Hi = {ln2_hi!r};\nconstexpr double kLn2Lo = {ln2_lo!r};\n")
        f.write(f"__device__ const double kLogTab[{n_log}][4] = {{\n")
        for j in range(n_log):
            F = float(1 / (1 + (mp.mpf(j) + mp.mpf(1) / 2) / n_log))
            L = -mp.log(mp.mpf(F))
            hi = float(L)
            lo = float(L - mp.mpf(hi))
            f.write(f"    {{{F!r}, {hi!r}, {lo!r}, 0.0}},\n")
        f.write("};\n\n}  // namespace lskum\n")
    print(f"wrote {path}: erfcx worst {worst:.2e}, {len(pieces)} pieces")


if __name__ == "__main__":
    main()

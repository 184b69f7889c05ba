"""Writes ``math_tables.h``: the FP64 flux kernel's function tables.

1. Polynomial pieces for the split-flux erfc.

The kinetic split fluxes need A = erfc(x) / 2 and B ~ exp(-x^2) at the same
argument. The device code evaluates erfc(a) = exp(-a^2) erfcx(a) for
0 <= a = |x| <= 6, reusing exp(-a^2) from B, with erfcx (the scaled
complementary error function, smooth and positive on the whole range) as a
polynomial in (a - c_k) on 48 intervals of width 1/8 centred at c_k; the
interval index is floor(8 a), which the device takes from the bits of a.
One formula for every argument keeps the lanes of a warp on one path.
Each polynomial is the Chebyshev interpolant of erfcx (computed with mpmath
at 50 digits from erfcx(a) = e^(a^2) erfc(a)) converted to the monomial
basis of the local variable; the script checks the relative error of every
piece at 2000 points in double-precision Horner evaluation and refuses to
write the header unless it is below 4e-16.

   The mixed-precision path evaluates the same function in FP32 from its own
   table: 24 pieces of width 1/4 and degree 5 (checked below 3e-7 relative
   in float32 Horner evaluation).

2. The exponential by Tang's table-driven method: x = k ln2/64 + r with
|r| <= ln2/128, exp(x) = 2^(k div 64) * 2^((k mod 64)/64) * e^r; the table
holds 2^(j/64), j < 64, correctly rounded (mpmath), and ln2/64 is split into
a double and its remainder for an exact reduction.

Run: python gen_math_tables.py  (writes math_tables.h next to this file)
"""

import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50

CX_LO, CX_HI, CX_W = 0.0, 6.0, 0.125
CX_DEG = 9            # degree in z = a - c on [-1/16, 1/16]
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
        zs = np.linspace(lo, hi, 2000)
        ref = np.array([float(mp.erfc(mp.mpf(float(u))) * mp.exp(mp.mpf(float(u)) ** 2))
                        for u in zs])
        got = horner(C, zs - c)
        e = np.max(np.abs(got - ref) / np.abs(ref))
        assert e < 4e-16, ("erfcx", lo, e)
        worst = max(worst, e)
        centres.append(c)
        pieces.append([float(x) for x in C])
        a = hi

    # 2^(j/64) and the split of ln2/64
    tab = [float(mp.mpf(2) ** (mp.mpf(j) / 64)) for j in range(64)]
    ln2_64 = mp.log(2) / 64
    hi = float(ln2_64)
    lo = float(ln2_64 - mp.mpf(hi))
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
        f.write("// exp(x) by Tang's table-driven reduction: 2^(j/64), j < 64, correctly rounded,\n")
        f.write("// and ln2/64 = kLn2By64Hi + kLn2By64Lo.\n")
        f.write(f"constexpr double kLn2By64Hi = {hi!r};\nconstexpr double kLn2By64Lo = {lo!r};\n")
        f.write(f"constexpr double kInvLn2By64 = {float(1 / ln2_64)!r};\n")
        f.write("__device__ const double kExp2Tab[64] = {\n")
        for j in range(0, 64, 4):
            f.write("    " + ", ".join(repr(v) for v in tab[j:j + 4]) + ",\n")
        f.write("};\n\n}  // namespace lskum\n")
    print(f"wrote {path}: erfcx worst {worst:.2e}, {len(pieces)} pieces")


if __name__ == "__main__":
    main()

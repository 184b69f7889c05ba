"""Accuracy of the FP64 kernels' transcendental designs, checked on the CPU:
the table-driven exponential (Tang's reduction with the 2^(j/256) table and
a degree-4 polynomial), erfc(a)/2 = exp(-a^2)/2 erfcx(a) from the erfcx
pieces, 1/beta from (1/sqrt(beta))^2 with one Newton step, and the
table-driven logarithm of the stage epilogues, all evaluated as the kernel
does -- every fused multiply-add rounded once, emulated in 200-bit
arithmetic -- against mpmath at 50 digits, with the table values read from
math_tables.h; and the rewritten forms in which the kernels assemble the
split fluxes, their differences and the q-variables from U, against the
oracle's direct evaluation. CPU only."""

import math
import os
import re
import struct

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2108_07031_gb300", "csrc", "math_tables.h")


@pytest.fixture(scope="module")
def tables():
    src = open(HDR).read()
    num = lambda name: float(re.search(name + r" = ([^;]+);", src).group(1))  # noqa: E731
    exp_tab = [float(v) for v in re.search(r"kExp2Tab\[\d+\] = \{(.*?)\};", src, re.S).group(1)
               .replace("\n", "").split(",") if v.strip()]
    body = re.search(r"kErfcxC\[kErfcxPieces\]\[kErfcxDeg \+ 2\] = \{(.*?)\n\};", src, re.S).group(1)
    pieces = [[float(x) for x in row.split(",") if x.strip()]
              for row in re.findall(r"\{([^{}]*)\}", body)]
    bits = int(num("kExpBits"))
    assert len(exp_tab) == 1 << bits
    log_body = re.search(r"kLogTab\[\d+\]\[4\] = \{(.*?)\n\};", src, re.S).group(1)
    log_rows = [[float(x) for x in row.split(",") if x.strip()]
                for row in re.findall(r"\{([^{}]*)\}", log_body)]
    return {"hi": num("kLn2ByNHi"), "lo": num("kLn2ByNLo"), "inv": num("kInvLn2ByN"),
            "exp2": exp_tab, "bits": bits, "pieces": pieces, "log2_inv_w": int(num("kErfcxLog2InvW")),
            "log": log_rows, "log_bits": int(num("kLogBits")), "ln2_hi": num("kLn2Hi"),
            "ln2_lo": num("kLn2Lo")}


def _fma(a, b, c):
    """a * b + c rounded once to double."""
    with mp.workprec(200):
        return float(mp.mpf(a) * mp.mpf(b) + mp.mpf(c))


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _exp_tab(t, x, halve=0):
    shifter = 6755399441055744.0
    kd = _fma(x, t["inv"], shifter)
    k = _bits(kd) - 0x4338000000000000
    kd = kd - shifter
    r = _fma(-kd, t["lo"], _fma(-kd, t["hi"], x))
    p = 1.0 / 24.0
    for c in (1.0 / 6.0, 0.5, 1.0):
        p = _fma(r, p, c)
    p = r * p
    tj = t["exp2"][k & ((1 << t["bits"]) - 1)]
    res = _fma(tj, p, tj)
    return _from_bits(_bits(res) + (((k >> t["bits"]) - halve) << 52))


def _ulp(x):
    return math.ulp(x)


def test_table_exp_within_1_2_ulp(tables):
    rng = np.random.Generator(np.random.PCG64(3))
    xs = np.concatenate([rng.uniform(-40.0, 0.0, 1500), rng.uniform(-700.0, 700.0, 300),
                         rng.uniform(-1.0, 1.0, 300), [0.0, -1e-300, math.log(2) / 128]])
    worst = 0.0
    for x in xs:
        for halve in (0, 1):
            ref = mp.exp(mp.mpf(float(x))) / (2 if halve else 1)
            got = _exp_tab(tables, float(x), halve)
            worst = max(worst, float(abs(mp.mpf(got) - ref)) / _ulp(float(ref)))
    assert worst <= 1.25, worst


def test_erfc_from_erfcx_pieces(tables):
    """erfc(a)/2 for 0 <= a <= 6: piece floor(2^L a), Horner in (a - c_k), times
    exp(-a^2)/2 from the table exponential. The argument -a^2 is rounded
    (like the exp(-S^2) of the B term in the oracle), so the relative error
    may grow as (1 + a^2) ulp: it stays within 4 (1 + a^2) ulp."""
    rng = np.random.Generator(np.random.PCG64(4))
    pieces = tables["pieces"]
    worst = 0.0
    scale = float(1 << tables["log2_inv_w"])
    for a in np.concatenate([rng.uniform(0.0, 6.0, 1500), [0.0, 0.125, 0.5, 1 / 64, 5.999999, 6.0]]):
        a = float(a)
        c = pieces[min(int(math.floor(scale * a)), len(pieces) - 1)]
        z = a - c[0]
        pv = c[-1]
        for coef in reversed(c[1:-1]):
            pv = _fma(pv, z, coef)
        eh = _exp_tab(tables, -(a * a), 1)
        got = eh * pv
        ref = mp.erfc(mp.mpf(a)) / 2
        rel = float(abs(mp.mpf(got) - ref) / ref)
        worst = max(worst, rel / ((1.0 + a * a) * np.finfo(float).eps))
    assert worst < 4.0, worst


def test_reciprocal_from_rsqrt_with_one_newton_step():
    """1/beta = i (1 + (1 - beta i)) with i = (1/sqrt(beta))^2, the square root
    reciprocal off by up to 2 ulp (the device's rsqrt is within 1): within
    1 ulp of 1/beta, as an IEEE division is within 0.5."""
    rng = np.random.Generator(np.random.PCG64(5))
    worst = 0.0
    for beta in np.concatenate([rng.uniform(0.05, 20.0, 2000), [0.5, 1.0, 0.7]]):
        beta = float(beta)
        for off in (-2, 0, 2):
            isb = float(1 / mp.sqrt(mp.mpf(beta)))
            for _ in range(abs(off)):
                isb = math.nextafter(isb, math.inf if off > 0 else -math.inf)
            i0 = isb * isb
            i2 = _fma(i0, _fma(-beta, i0, 1.0), i0)
            ref = 1 / mp.mpf(beta)
            worst = max(worst, float(abs(mp.mpf(i2) - ref)) / _ulp(float(ref)))
    assert worst <= 1.0, worst


def _log_tab(t, x):
    b = _bits(x)
    e = float((b >> 52) - 1023)
    row = t["log"][(b >> (52 - t["log_bits"])) & ((1 << t["log_bits"]) - 1)]
    m = _from_bits((b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000)
    r = _fma(m, row[0], -1.0)
    p = _fma(r, -1.0 / 6.0, 0.2)
    for c in (-0.25, 1.0 / 3.0, -0.5, 1.0):
        p = _fma(r, p, c)
    p = p * r
    return _fma(e, t["ln2_hi"], row[1] + (p + _fma(e, t["ln2_lo"], row[2])))


def test_table_log(tables):
    """log x within 0.5 ulp of max(|log x|, 1) -- an absolute bound at the
    rounding of the O(1) q-variable it feeds; near x = 1 the reduction's
    e ln2 and -log F_j cancel, so the bound is absolute -- and within 2 ulp
    relative where |log x| > 0.1. Also the reduction constants the generator
    states: ln2 split with a 42-bit high part."""
    assert len(tables["log"]) == 1 << tables["log_bits"]
    assert (mp.mpf(tables["ln2_hi"]) * 2 ** 42) % 1 == 0
    rng = np.random.Generator(np.random.PCG64(6))
    xs = np.concatenate([np.exp(rng.uniform(-30.0, 30.0, 2500)), 1.0 + rng.uniform(-1e-3, 1e-3, 500),
                         [1.0, 0.5, 2.0, 0.168, 1.0 - 2 ** -53, 1.0 + 2 ** -52, 1e-300, 1e300]])
    worst_abs = worst_rel = 0.0
    for x in xs:
        x = float(x)
        ref = mp.log(mp.mpf(x))
        err = float(abs(mp.mpf(_log_tab(tables, x)) - ref))
        worst_abs = max(worst_abs, err / _ulp(max(abs(float(ref)), 1.0)))
        if abs(float(ref)) > 0.1:
            worst_rel = max(worst_rel, err / _ulp(abs(float(ref))))
    assert worst_abs <= 0.5 and worst_rel <= 2.0, (worst_abs, worst_rel)


# ---------------------------------------------------------------- algebra
# The kernels assemble the kinetic split fluxes and the q-variables in
# rewritten forms. These tests evaluate those forms in float64 with the
# library's erfc/exp/log and compare them with the oracle's direct
# evaluation of the same quantities, so a wrong identity (a dropped term, a
# wrong sign) fails here, on the CPU.

def _states(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(0.3, 3.0, n)
    u = rng.uniform(-2.0, 2.0, n)
    v = rng.uniform(-2.0, 2.0, n)
    p = rng.uniform(0.2, 3.0, n)
    return np.stack([rho, u, v, p], axis=1)


def _split_ab(W, ua, sg, gamma=1.4):
    """t = ua A + sg B, A = erfc(-sg S)/2, sg B with B = exp(-S^2)/(2 sqrt(pi beta))."""
    rho, p = W[:, 0], W[:, 3]
    beta = rho / (2.0 * p)
    S = ua * np.sqrt(beta)
    A = np.array([0.5 * math.erfc(-sg * s) for s in S])
    B = np.exp(-S * S) / (2.0 * np.sqrt(math.pi * beta))
    return ua * A + sg * B, A, sg * B


def _device_split_flux(W, direction, sg, gamma=1.4):
    """G0 = rho t, G_a = ua G0 + p A, G_b = ub G0, G3 = h t - (p/2) sg B,
    the forms of the FP64 flux kernel; returned in the global component order."""
    rho, u, v, p = W.T
    ua, ub = (u, v) if direction == 0 else (v, u)
    t, A, Bs = _split_ab(W, ua, sg, gamma)
    h = p + p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    G0 = rho * t
    Ga = ua * G0 + p * A
    Gb = ub * G0
    G3 = h * t - 0.5 * p * Bs
    mom = (Ga, Gb) if direction == 0 else (Gb, Ga)
    return np.stack([G0, mom[0], mom[1], G3], axis=1)


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("sg", [1, -1])
def test_split_flux_assembly_matches_the_oracle(direction, sg):
    from oracle import oracle as O
    W = _states(400, 11 + direction + (sg > 0))
    ref = O.split_flux(W, direction, sg)
    got = _device_split_flux(W, direction, sg)
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(got - ref).max(axis=0) <= 1e-13 * scale)


@pytest.mark.parametrize("direction", [0, 1])
def test_split_flux_differences_in_one_chain(direction):
    """The kernel's differences G(j) - G(0) (state 0's component rounded once
    into state j's FMA chain) against the oracle's two fluxes subtracted, for
    nearby pairs, within the rounding of the fluxes themselves."""
    from oracle import oracle as O
    W0 = _states(300, 29 + direction)
    rng = np.random.Generator(np.random.PCG64(31 + direction))
    Wj = W0 * (1.0 + 1e-3 * rng.standard_normal(W0.shape))
    for sg in (1, -1):
        rho0, u0, v0, p0 = W0.T
        rhoj, uj, vj, pj = Wj.T
        ua0, ub0 = (u0, v0) if direction == 0 else (v0, u0)
        uaj, ubj = (uj, vj) if direction == 0 else (vj, uj)
        t0, A0, B0 = _split_ab(W0, ua0, sg)
        tj, Aj, Bj = _split_ab(Wj, uaj, sg)
        h0 = p0 / 0.4 + p0 + 0.5 * rho0 * (u0 * u0 + v0 * v0)
        hj = pj / 0.4 + pj + 0.5 * rhoj * (uj * uj + vj * vj)
        g0j, g00 = rhoj * tj, rho0 * t0
        d0 = g0j - g00
        d1 = uaj * g0j + (pj * Aj - (ua0 * g00 + p0 * A0))
        d2 = g0j * ubj - g00 * ub0
        d3 = hj * tj + (-0.5 * pj * Bj - (h0 * t0 - 0.5 * p0 * B0))
        da, db = (d1, d2) if direction == 0 else (d2, d1)
        got = np.stack([d0, da, db, d3], axis=1)
        ref = O.split_flux(Wj, direction, sg) - O.split_flux(W0, direction, sg)
        scale = np.abs(O.split_flux(W0, direction, sg)).max(axis=0)
        assert np.all(np.abs(got - ref).max(axis=0) <= 1e-13 * scale)


def test_q_variables_from_conserved_state():
    """q from U as the stage epilogues form it: rho p without a division, one
    reciprocal of rho^2 p for 1/rho and 1/p, and for gamma = 1.4
    q1 = ln(rho^2 beta^5)/2 - beta |u|^2 -- against Eq. 26 of the oracle
    applied to the primitive state."""
    from oracle import oracle as O
    W = _states(500, 5)
    U = O.prim_to_cons(W)
    gm1 = 0.4
    rho = U[:, 0]
    m2 = U[:, 1] ** 2 + U[:, 2] ** 2
    rp = gm1 * (U[:, 3] * rho - 0.5 * m2)
    rr = 1.0 / (rho * rp)
    ip = rho * rho * rr
    beta = 0.5 * rho * ip
    q = np.stack([0.5 * np.log(rho * rho * beta ** 5) - 0.5 * m2 * (rho * rr),
                  U[:, 1] * ip, U[:, 2] * ip, -rho * ip], axis=1)
    ref = O.prim_to_q(O.cons_to_prim(U))
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(q - ref).max(axis=0) <= 1e-13 * scale)


def _mixed_dsplit(b, dq, direction, sg, gm1_inv=2.5):
    """The mixed path's difference-form split flux, G(q~_0 + dq~) - G(q~_0),
    as its kernel assembles it (base state and difference from the
    q-variables, expm1/log1p of the small arguments, the erfc midpoint
    series), evaluated here in float64 rows."""
    bx, by, bz, bw = b.T
    dx_, dy_, dz_, dw_ = dq.T
    beta, dbeta, qj4 = -0.5 * bw, -0.5 * dw_, bw + dw_
    inv2b = -1.0 / bw
    u, v = by * inv2b, bz * inv2b
    rq = 1.0 / (bw * qj4)
    du = (by * dw_ - dy_ * bw) * rq
    dv = (bz * dw_ - dz_ * bw) * rq
    uj, vj = u + du, v + dv
    uu0, uuj = u * u + v * v, uj * uj + vj * vj
    duu = du * (uj + u) + dv * (vj + v)
    isb = 1.0 / np.sqrt(beta)
    sb = beta * isb
    betaj = beta + dbeta
    isbj = 1.0 / np.sqrt(betaj)
    dsb = dbeta / (betaj * isbj + sb)
    i2 = isb * isb
    r = np.exp(bx + beta * uu0) * (i2 * i2 * isb)
    dlnr = dx_ - np.log1p(dbeta * (2.0 * inv2b)) * gm1_inv + (dbeta * uuj + beta * duu)
    dr = r * np.expm1(dlnr)
    p = r * inv2b
    dp = (dr * beta - r * dbeta) * (inv2b * (isbj * isbj))
    E0 = p * gm1_inv + 0.5 * r * uu0
    dE = dp * gm1_inv + 0.5 * (dr * uuj + r * duu)
    h, dh = p + E0, dp + dE
    ua0, ub0, dua, dub = (u, v, du, dv) if direction == 0 else (v, u, dv, du)
    sbj = sb + dsb
    S0 = ua0 * sb
    dS = dua * sbj + ua0 * dsb
    Sj = S0 + dS
    e0 = np.exp(-S0 * S0)
    de = e0 * np.expm1(-dS * (Sj + S0))
    x0, dx = -sg * S0, -sg * dS
    A0 = np.array([0.5 * math.erfc(x) for x in x0])

    def central(m, hh):  # erfc(m - h) - erfc(m + h), Hermite midpoint series
        m2, h2 = m * m, hh * hh
        H2 = 4 * m2 - 2
        H4 = (16 * m2 - 48) * m2 + 12
        H6 = ((64 * m2 - 480) * m2 + 720) * m2 - 120
        H8 = (((256 * m2 - 3584) * m2 + 13440) * m2 - 13440) * m2 + 1680
        tail = H4 / 120 + np.where(np.abs(hh) > 1 / 64, h2 * (H6 / 5040 + h2 * H8 / 362880), 0.0)
        return 4 / math.sqrt(math.pi) * np.exp(-m2) * hh * (1 + h2 * (H2 / 6 + h2 * tail))

    small = np.abs(dx) <= 0.25
    dA = np.where(small, -0.5 * central(x0 + 0.5 * dx, 0.5 * dx),
                  np.array([0.5 * (math.erfc(a + d) - math.erfc(a)) for a, d in zip(x0, dx)]))
    Aj = A0 + dA
    c = 0.5 / math.sqrt(math.pi)
    B0 = c * e0 * isb
    dB = c * (de * isbj - e0 * dsb * isbj * isb)
    Bj = B0 + dB
    t0 = ua0 * A0 + sg * B0
    dt = dua * Aj + ua0 * dA + sg * dB
    tj = t0 + dt
    G00 = r * t0
    dG0 = dr * tj + r * dt
    G0j = G00 + dG0
    dGa = dua * G0j + ua0 * dG0 + (dp * Aj + p * dA)
    dGb = dub * G0j + ub0 * dG0
    dG3 = dh * tj + h * dt - 0.5 * sg * (dp * Bj + p * dB)
    mom = (dGa, dGb) if direction == 0 else (dGb, dGa)
    return np.stack([dG0, mom[0], mom[1], dG3], axis=1)


@pytest.mark.parametrize("direction", [0, 1])
def test_mixed_difference_form_matches_the_oracle(direction):
    """The mixed kernel's difference-form split flux (base + difference of
    the modified states, product rule, expm1/log1p, erfc midpoint series) in
    float64 against the oracle's two fluxes subtracted: the forms are exact
    up to rounding and the series' truncation, far below the FP32 the kernel
    evaluates them in."""
    from oracle import oracle as O
    W0 = _states(400, 41 + direction)
    b = O.prim_to_q(W0)
    rng = np.random.Generator(np.random.PCG64(43 + direction))
    dq = 1e-3 * np.abs(b) * rng.standard_normal(b.shape)
    Wj = O.q_to_prim(b + dq)
    for sg in (1, -1):
        got = _mixed_dsplit(b, dq, direction, sg)
        ref = O.split_flux(Wj, direction, sg) - O.split_flux(W0, direction, sg)
        scale = np.abs(O.split_flux(W0, direction, sg)).max(axis=0)
        assert np.all(np.abs(got - ref).max(axis=0) <= 1e-12 * scale), \
            (np.abs(got - ref).max(axis=0) / scale)

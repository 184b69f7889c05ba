"""Accuracy of the FP64 flux kernel's transcendental designs, checked on the
CPU: the table-driven exponential (Tang's reduction with the 2^(j/64) table
and a degree-5 polynomial) and erfc(a)/2 = exp(-a^2)/2 erfcx(a) from the
erfcx pieces, both evaluated as the kernel does -- every fused multiply-add
rounded once, emulated in 200-bit arithmetic -- against mpmath at 50
digits, with the table values read from math_tables.h. CPU only."""

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
    exp_tab = [float(v) for v in re.search(r"kExp2Tab\[64\] = \{(.*?)\};", src, re.S).group(1)
               .replace("\n", "").split(",") if v.strip()]
    body = re.search(r"kErfcxC\[kErfcxPieces\]\[kErfcxDeg \+ 2\] = \{(.*?)\n\};", src, re.S).group(1)
    pieces = [[float(x) for x in row.split(",") if x.strip()]
              for row in re.findall(r"\{([^{}]*)\}", body)]
    return {"hi": num("kLn2By64Hi"), "lo": num("kLn2By64Lo"), "inv": num("kInvLn2By64"),
            "exp2": exp_tab, "pieces": pieces}


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
    p = 1.0 / 120.0
    for c in (1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0):
        p = _fma(r, p, c)
    p = r * p
    tj = t["exp2"][k & 63]
    res = _fma(tj, p, tj)
    return _from_bits(_bits(res) + (((k >> 6) - halve) << 52))


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
    """erfc(a)/2 for 0 <= a <= 6: piece floor(8a), Horner in (a - c_k), times
    exp(-a^2)/2 from the table exponential. The argument -a^2 is rounded
    (like the exp(-S^2) of the B term in the oracle), so the relative error
    may grow as (1 + a^2) ulp: it stays within 4 (1 + a^2) ulp."""
    rng = np.random.Generator(np.random.PCG64(4))
    pieces = tables["pieces"]
    worst = 0.0
    for a in np.concatenate([rng.uniform(0.0, 6.0, 1500), [0.0, 0.125, 0.5, 5.999999]]):
        a = float(a)
        c = pieces[min(int(math.floor(8.0 * a)), len(pieces) - 1)]
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

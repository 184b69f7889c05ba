"""The device function tables (paper_2108_07031_gb300/csrc/math_tables.h) are
exactly what their generator writes: the generator computes them with mpmath
and asserts their accuracy (erfcx pieces below 4e-16 relative in FP64 and
3e-7 in FP32 Horner evaluation), so a hand edit or a stale header fails here.
CPU only (a few seconds)."""

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_07031_gb300", "csrc")


def test_header_matches_its_generator(tmp_path):
    pytest.importorskip("mpmath")
    spec = importlib.util.spec_from_file_location("gen_math_tables",
                                                  os.path.join(CSRC, "gen_math_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    out = tmp_path / "math_tables.h"
    gen.main(str(out))
    with open(os.path.join(CSRC, "math_tables.h")) as f:
        committed = f.read()
    assert out.read_text() == committed

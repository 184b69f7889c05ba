"""The library from plain C: tests/c_abi/solve_from_files.c is compiled with
the system C compiler against include/lskum.h and the built liblskum.so.
Without a GPU it must report the missing CUDA device through the ABI's
error code and message; on a GPU its 20 iterations must equal the Python
binding's bit for bit (the same library on the same inputs)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2108_07031_gb300 import build as B
from paper_2108_07031_gb300 import cloud as Cl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "solve_from_files.c")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = B.build()
    out = str(tmp_path_factory.mktemp("cabi") / "solve_from_files")
    subprocess.run([cc, "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    SRC, "-o", out, "-L", os.path.dirname(lib), "-llskum",
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return out


def _write_cloud(c, d):
    np.array([c.n], dtype=np.int64).tofile(os.path.join(d, "n.bin"))
    np.ascontiguousarray(c.xy, dtype=np.float64).tofile(os.path.join(d, "xy.bin"))
    np.ascontiguousarray(c.normals, dtype=np.float64).tofile(os.path.join(d, "normals.bin"))
    np.ascontiguousarray(c.flags, dtype=np.int8).tofile(os.path.join(d, "flags.bin"))
    np.ascontiguousarray(c.nbr_offsets, dtype=np.int32).tofile(os.path.join(d, "off.bin"))
    np.ascontiguousarray(c.nbr_idx, dtype=np.int32).tofile(os.path.join(d, "idx.bin"))


def _cuda_present():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def test_c_consumer_reports_missing_device(exe, tmp_path):
    if _cuda_present():
        pytest.skip("a GPU is present: covered by the gpu test")
    _write_cloud(Cl.naca0012_cloud(24, 8), str(tmp_path))
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 3
    assert r.stdout.startswith("create -4") and "CUDA device" in r.stdout


@pytest.mark.gpu
def test_c_consumer_matches_python_binding(exe, tmp_path):
    if not _cuda_present():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_07031_gb300 import lskum as L
    c = Cl.naca0012_cloud(24, 8)
    _write_cloud(c, str(tmp_path))
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    vals = [float(v) for v in r.stdout.split()[1:]]
    with L.Solver.from_cloud(c) as s:
        s.set_freestream(0.63, 2.0)
        s.step(20)
        res = s.residual_norm()
        cl, cd = s.forces()
        W = s.get_state()
    assert vals[0] == res and vals[1] == cl and vals[2] == cd
    assert vals[3:7] == list(W[0])

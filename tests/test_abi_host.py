"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point that include/lskum.h declares, and rejects bad clouds in its
host-side validation with the documented error codes."""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2108_07031_gb300 import build as B
from paper_2108_07031_gb300 import cloud as Cl
from paper_2108_07031_gb300 import lskum as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("lskum.h", "lskum_mlp.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lskum_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (lskum_[a-z_0-9]+)$", out, flags=re.M))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    from paper_2108_07031_gb300 import surrogate as S
    assert set(declared) == set(L.EXPORTED) | set(S.EXPORTED)
    lib = L.load()
    for s in declared:
        assert hasattr(lib, s)


def test_build_targets_sm_103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_options():
    o = L.default_options()
    assert o.gamma == 1.4 and o.cfl == 0.2 and o.inner_iters == 2 and o.order == 2
    assert o.wall_factor == 2.0 and o.outer_mode == L.OUTER_FREESTREAM and o.reorder == 1
    assert o.weight_power == 0.0 and o.flux_split == 0 and o.n_conditions == 1


def test_error_strings():
    lib = L.load()
    assert lib.lskum_error_string(0) == b"ok"
    assert lib.lskum_error_string(-3) == b"degenerate stencil"
    assert lib.lskum_error_string(-99) == b"unknown error"


def _small_cloud():
    return Cl.naca0012_cloud(24, 8)


def _create_code(c, **kw):
    xy = kw.get("xy", c.xy)
    nrm = kw.get("normals", c.normals)
    fl = kw.get("flags", c.flags)
    off = kw.get("off", c.nbr_offsets)
    idx = kw.get("idx", c.nbr_idx)
    lib = L.load()
    o = L.default_options(**kw.get("options", {}))
    h = C.c_void_p()
    xy = np.ascontiguousarray(xy, np.float64)
    nrm = np.ascontiguousarray(nrm, np.float64)
    fl = np.ascontiguousarray(fl, np.int8)
    off = np.ascontiguousarray(off, np.int32)
    idx = np.ascontiguousarray(idx, np.int32)
    code = lib.lskum_create(kw.get("n", fl.shape[0]), L._ptr(xy), L._ptr(nrm), L._ptr(fl),
                            L._ptr(off), L._ptr(idx), C.byref(o), C.byref(h))
    if code == 0:
        lib.lskum_destroy(h)
    else:
        assert not h.value
    return code, lib.lskum_last_error().decode()


@pytest.mark.parametrize("bad", [dict(weight_power=-1.0), dict(weight_power=9.0),
                                 dict(weight_power=float("nan")), dict(n_conditions=3),
                                 dict(flux_split=1, precision=1), dict(order=3)])
def test_create_rejects_invalid_options(bad):
    code, msg = _create_code(_small_cloud(), options=bad)
    assert code == -1 and "option" in msg


def test_create_rejects_out_of_range_neighbour():
    c = _small_cloud()
    idx = c.nbr_idx.copy()
    idx[5] = c.n + 3
    code, msg = _create_code(c, idx=idx)
    assert code == -2 and "neighbour" in msg


def test_create_rejects_self_and_repeated_neighbours():
    c = _small_cloud()
    idx = c.nbr_idx.copy()
    i = 7
    idx[c.nbr_offsets[i]] = i
    assert _create_code(c, idx=idx)[0] == -2
    idx = c.nbr_idx.copy()
    idx[c.nbr_offsets[i] + 1] = idx[c.nbr_offsets[i]]
    code, msg = _create_code(c, idx=idx)
    assert code == -2 and "twice" in msg


def test_create_rejects_bad_offsets_and_sizes():
    c = _small_cloud()
    off = c.nbr_offsets.copy()
    off[0] = 1
    assert _create_code(c, off=off)[0] == -2
    off = c.nbr_offsets.copy()
    off[4] = off[3] + 21  # 21 neighbours
    assert _create_code(c, off=off)[0] == -2
    assert _create_code(c, n=0)[0] == -1


def test_create_rejects_bad_flags_and_normals():
    c = _small_cloud()
    fl = c.flags.copy()
    fl[10] = 5
    assert _create_code(c, flags=fl)[0] == -1
    nrm = c.normals.copy()
    nrm[0] = (0.5, 0.5)  # wall point 0: not unit length
    assert _create_code(c, normals=nrm)[0] == -1
    xy = c.xy.copy()
    xy[3, 0] = np.nan
    assert _create_code(c, xy=xy)[0] == -1


def test_create_rejects_degenerate_split_stencil():
    """A point whose neighbours all lie on one side leaves a split stencil empty."""
    c = _small_cloud()
    off = c.nbr_offsets.copy()
    idx = c.nbr_idx.copy()
    i = 3 * c.n_c + 5  # an interior point
    nb = c.neighbours(i)
    right = [j for j in nb if c.xy[j, 0] > c.xy[i, 0]]
    keep = right[:3]
    new_idx = np.concatenate([idx[:off[i]], keep, idx[off[i + 1]:]]).astype(np.int32)
    delta = len(keep) - len(nb)
    new_off = off.copy()
    new_off[i + 1:] += delta
    code, msg = _create_code(c, off=new_off, idx=new_idx)
    assert code == -3 and "degenerate" in msg


def test_valid_cloud_passes_validation_and_needs_a_device():
    """A valid cloud passes the host checks; without a CUDA device the library
    fails loudly (there is no CPU fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by the gpu tests")
    c = _small_cloud()
    code, msg = _create_code(c)
    assert code == -4 and "CUDA device" in msg
    with pytest.raises(L.LskumError):
        L.Solver.from_cloud(c)

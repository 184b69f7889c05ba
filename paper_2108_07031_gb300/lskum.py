"""Thin ctypes binding of the C ABI in ``include/lskum.h`` (``_build/liblskum.so``).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels. Importing this module never falls back to anything: if the
native library is missing or no CUDA device is usable, ``load()`` /
``Solver(...)`` raise.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "BAD_CONNECTIVITY", -3: "DEGENERATE_STENCIL", -4: "CUDA",
    -5: "DIVERGED", -6: "TIMEOUT", -7: "STATE",
}
ERR_DIVERGED = -5

INTERIOR, WALL, OUTER = 0, 1, 2
OUTER_KINETIC, OUTER_FREESTREAM = 0, 1
FP64, MIXED = 0, 1
KERNEL_FLUX, KERNEL_LS_FIRST, KERNEL_LS_INNER, KERNEL_REDUCE = 0, 1, 2, 3

# every exported entry point of include/lskum.h
EXPORTED = (
    "lskum_default_options", "lskum_create", "lskum_destroy", "lskum_set_stream",
    "lskum_set_freestream", "lskum_set_conditions", "lskum_set_state", "lskum_get_state", "lskum_step", "lskum_solve",
    "lskum_residual_norm", "lskum_forces", "lskum_eval_residual", "lskum_eval_q_derivatives",
    "lskum_info", "lskum_autotune", "lskum_profile", "lskum_kernel_time", "lskum_last_launch_count",
    "lskum_error_string", "lskum_last_error", "lskum_residue_noalloc",
)

NOALLOC_MAX_POINTS = 8192 * 8192


class LskumError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({detail})")


class Options(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("inner_iters", C.c_int),
                ("order", C.c_int), ("wall_factor", C.c_double), ("outer_mode", C.c_int),
                ("precision", C.c_int), ("reorder", C.c_int), ("block_size", C.c_int),
                ("check_every", C.c_int), ("n_conditions", C.c_int), ("flux_split", C.c_int),
                ("weight_power", C.c_double)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``liblskum.so`` (building it first if absent) and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"native library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
        sig = {
            "lskum_default_options": ([P], I),
            "lskum_create": ([I64, P, P, P, P, P, P, P], I),
            "lskum_destroy": ([P], None),
            "lskum_set_stream": ([P, P], I),
            "lskum_set_freestream": ([P, D, D], I),
            "lskum_set_conditions": ([P, I, P, P], I),
            "lskum_set_state": ([P, P], I),
            "lskum_get_state": ([P, P], I),
            "lskum_step": ([P, I], I),
            "lskum_solve": ([P, I, D, P], I),
            "lskum_residual_norm": ([P, P], I),
            "lskum_forces": ([P, P, P], I),
            "lskum_eval_residual": ([P, P], I),
            "lskum_eval_q_derivatives": ([P, P, P], I),
            "lskum_info": ([P, P, P, P, P], I),
            "lskum_autotune": ([P, I, P], I),
            "lskum_profile": ([P, I], I),
            "lskum_kernel_time": ([P, I, P, P], I),
            "lskum_last_launch_count": ([P], I64),
            "lskum_error_string": ([I], C.c_char_p),
            "lskum_last_error": ([], C.c_char_p),
            "lskum_residue_noalloc": ([P, I64, P, P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def default_options(**overrides) -> Options:
    lib = load()
    o = Options()
    lib.lskum_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _check(code: int, where: str):
    if code != OK:
        detail = load().lskum_last_error().decode(errors="replace")
        raise LskumError(code, where, detail)


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _host_f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


def residue_noalloc(R_device_ptr: int, n: int, out_device_ptr: int, stream_handle: int = 0):
    """``lskum_residue_noalloc``: residue sqrt(sum R_rho^2) / n of a device-resident
    n x 4 residual into one device double, with no allocation (fixed scratch)."""
    lib = load()
    _check(lib.lskum_residue_noalloc(C.c_void_p(R_device_ptr), int(n),
                                     C.c_void_p(out_device_ptr), C.c_void_p(stream_handle)),
           "lskum_residue_noalloc")


class Solver:
    """One point cloud on the GPU (``lskum_create`` ... ``lskum_destroy``)."""

    def __init__(self, xy, normals, flags, nbr_offsets, nbr_idx, options: Options | None = None,
                 **overrides):
        lib = load()
        self._lib = lib
        n = int(np.asarray(flags).shape[0])
        self.n = n
        xy = _host_f64(xy, (n, 2))
        nrm = _host_f64(normals, (n, 2))
        fl = np.ascontiguousarray(flags, dtype=np.int8)
        off = np.ascontiguousarray(nbr_offsets, dtype=np.int32)
        idx = np.ascontiguousarray(nbr_idx, dtype=np.int32)
        if off.shape != (n + 1,):
            raise ValueError("nbr_offsets must have n + 1 entries")
        opt = options if options is not None else default_options(**overrides)
        self.options = opt
        self.n_cond = int(opt.n_conditions)
        h = C.c_void_p()
        _check(lib.lskum_create(n, _ptr(xy), _ptr(nrm), _ptr(fl), _ptr(off), _ptr(idx),
                                C.byref(opt), C.byref(h)), "lskum_create")
        self._h = h

    @classmethod
    def from_cloud(cls, cloud, **overrides):
        return cls(cloud.xy, cloud.normals, cloud.flags, cloud.nbr_offsets, cloud.nbr_idx,
                   **overrides)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lskum_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state
    def set_stream(self, stream_handle: int | None):
        _check(self._lib.lskum_set_stream(self._h, C.c_void_p(stream_handle or 0)),
               "lskum_set_stream")

    def set_freestream(self, mach: float, alpha_deg: float):
        _check(self._lib.lskum_set_freestream(self._h, float(mach), float(alpha_deg)),
               "lskum_set_freestream")

    def set_conditions(self, mach, alpha_deg):
        m = np.ascontiguousarray(mach, dtype=np.float64).reshape(-1)
        a = np.ascontiguousarray(alpha_deg, dtype=np.float64).reshape(-1)
        if m.size != a.size:
            raise ValueError("mach and alpha_deg differ in length")
        _check(self._lib.lskum_set_conditions(self._h, int(m.size), _ptr(m), _ptr(a)),
               "lskum_set_conditions")

    def _shape(self, m=4):
        return (self.n, m) if self.n_cond == 1 else (self.n_cond, self.n, m)

    def set_state(self, prim):
        W = _host_f64(prim, self._shape())
        _check(self._lib.lskum_set_state(self._h, _ptr(W)), "lskum_set_state")

    def set_state_ptr(self, host_ptr: int):
        """set_state from a host address (e.g. a pinned torch tensor's data_ptr)."""
        _check(self._lib.lskum_set_state(self._h, C.c_void_p(host_ptr)), "lskum_set_state")

    def get_state_ptr(self, host_ptr: int):
        """get_state into a host address (e.g. a pinned torch tensor's data_ptr)."""
        _check(self._lib.lskum_get_state(self._h, C.c_void_p(host_ptr)), "lskum_get_state")

    def get_state(self) -> np.ndarray:
        W = np.empty(self._shape(), dtype=np.float64)
        _check(self._lib.lskum_get_state(self._h, _ptr(W)), "lskum_get_state")
        return W

    # -- iteration
    def step(self, n_iters: int = 1):
        _check(self._lib.lskum_step(self._h, int(n_iters)), "lskum_step")

    def solve(self, max_iters: int, tol: float) -> int:
        done = C.c_int()
        _check(self._lib.lskum_solve(self._h, int(max_iters), float(tol), C.byref(done)),
               "lskum_solve")
        return done.value

    def residual_norm(self):
        """Residue of the last iteration (a float, or an array per condition)."""
        r = np.zeros(self.n_cond, dtype=np.float64)
        _check(self._lib.lskum_residual_norm(self._h, _ptr(r)), "lskum_residual_norm")
        return float(r[0]) if self.n_cond == 1 else r

    def forces(self):
        """(Cl, Cd), as floats or as arrays per condition."""
        cl = np.zeros(self.n_cond, dtype=np.float64)
        cd = np.zeros(self.n_cond, dtype=np.float64)
        _check(self._lib.lskum_forces(self._h, _ptr(cl), _ptr(cd)), "lskum_forces")
        if self.n_cond == 1:
            return float(cl[0]), float(cd[0])
        return cl, cd

    # -- evaluation hooks (tests, diagnostics)
    def eval_residual(self) -> np.ndarray:
        R = np.empty(self._shape(), dtype=np.float64)
        _check(self._lib.lskum_eval_residual(self._h, _ptr(R)), "lskum_eval_residual")
        return R

    def eval_q_derivatives(self):
        qx = np.empty(self._shape(), dtype=np.float64)
        qy = np.empty(self._shape(), dtype=np.float64)
        _check(self._lib.lskum_eval_q_derivatives(self._h, _ptr(qx), _ptr(qy)),
               "lskum_eval_q_derivatives")
        return qx, qy

    def info(self):
        n, nw, mx, nc = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        _check(self._lib.lskum_info(self._h, C.byref(n), C.byref(nw), C.byref(mx), C.byref(nc)),
               "lskum_info")
        return {"n_points": n.value, "n_wall": nw.value, "max_neighbours": mx.value,
                "n_conditions": nc.value}

    def autotune(self, trial_iters: int = 2):
        """Pick the fastest (flux block, derivative block); returns the pair."""
        best = C.c_int()
        _check(self._lib.lskum_autotune(self._h, int(trial_iters), C.byref(best)),
               "lskum_autotune")
        return divmod(best.value, 1000)

    def profile(self, enable: bool):
        _check(self._lib.lskum_profile(self._h, 1 if enable else 0), "lskum_profile")

    def kernel_time(self, kernel: int):
        ms, nl = C.c_double(), C.c_int64()
        _check(self._lib.lskum_kernel_time(self._h, int(kernel), C.byref(ms), C.byref(nl)),
               "lskum_kernel_time")
        return ms.value, nl.value

    def last_launch_count(self) -> int:
        return int(self._lib.lskum_last_launch_count(self._h))

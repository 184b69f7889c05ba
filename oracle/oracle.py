"""numpy front end of the plain FP64 CPU oracle (``lskum_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg, never by the solver package. The C file is
compiled here with gcc (``-O2 -ffp-contract=off -fopenmp``) into
``oracle/_build/liblskum_oracle.so``; nothing of the CUDA path is linked.

Each function cites the part of the paper it follows (see the C file's
header for the full list and for the readings of what the paper leaves open).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lskum_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblskum_oracle.so")
_lock = threading.Lock()
_lib = None

GAMMA = 1.4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cloud(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("nx", C.c_void_p),
                ("ny", C.c_void_p), ("flag", C.c_void_p), ("off", C.c_void_p),
                ("nbr", C.c_void_p), ("gamma", C.c_double), ("wall_factor", C.c_double),
                ("order", C.c_int), ("outer_mode", C.c_int), ("weight_power", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_prim_to_q.argtypes = [P, C.c_double, P]
            lib.orc_q_to_prim.argtypes = [P, C.c_double, P]
            lib.orc_q_to_prim.restype = C.c_int
            lib.orc_prim_to_cons.argtypes = [P, C.c_double, P]
            lib.orc_cons_to_prim.argtypes = [P, C.c_double, P]
            lib.orc_split_flux.argtypes = [P, C.c_int, C.c_int, C.c_double, P]
            for nm in ("orc_prim_to_q_n", "orc_q_to_prim_n", "orc_prim_to_cons_n",
                       "orc_cons_to_prim_n"):
                getattr(lib, nm).argtypes = [C.c_int64, P, C.c_double, P]
            lib.orc_split_flux_n.argtypes = [C.c_int64, P, C.c_int, C.c_int, C.c_double, P]
            lib.orc_q_derivatives.argtypes = [P, P, C.c_int, P, P]
            lib.orc_ls_sweep.argtypes = [P, P, P, P, P, P]
            lib.orc_flux_residual.argtypes = [P, P, P, P, P]
            lib.orc_flux_residual.restype = C.c_int
            lib.orc_flux_residual_subset.argtypes = [P, P, P, P, P, C.c_int64, P]
            lib.orc_flux_residual_subset.restype = C.c_int
            lib.orc_timestep.argtypes = [P, P, C.c_double, P]
            lib.orc_rk_stage.argtypes = [C.c_int, P, P, P, C.c_double, P]
            lib.orc_wall_project.argtypes = [P, C.c_double, C.c_double]
            lib.orc_residue.argtypes = [C.c_int64, P]
            lib.orc_residue.restype = C.c_double
            lib.orc_forces.argtypes = [P, P, P, C.c_int64, C.c_double, C.c_double, P, P]
            lib.orc_freestream.argtypes = [C.c_double, C.c_double, C.c_double, P]
            lib.orc_iterate.argtypes = [P, P, C.c_int, C.c_double, C.c_int, P, P]
            lib.orc_iterate.restype = C.c_int
            lib.orc_residual_of_state.argtypes = [P, P, C.c_int, P]
            lib.orc_residual_of_state.restype = C.c_int
            lib.orc_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleCloud:
    """Holds contiguous copies of a cloud's arrays for the C oracle."""

    def __init__(self, xy, normals, flags, nbr_offsets, nbr_idx, gamma: float = GAMMA,
                 wall_factor: float = 2.0, order: int = 2, outer_mode: int = 1,
                 weight_power: float = 0.0):
        xy = np.asarray(xy, dtype=np.float64)
        self.x = np.ascontiguousarray(xy[:, 0])
        self.y = np.ascontiguousarray(xy[:, 1])
        nrm = np.asarray(normals, dtype=np.float64)
        self.nx = np.ascontiguousarray(nrm[:, 0])
        self.ny = np.ascontiguousarray(nrm[:, 1])
        self.flag = np.ascontiguousarray(flags, dtype=np.int8)
        self.off = np.ascontiguousarray(nbr_offsets, dtype=np.int32)
        self.nbr = np.ascontiguousarray(nbr_idx, dtype=np.int32)
        self.n = int(self.x.shape[0])
        self.gamma = float(gamma)
        self._s = _Cloud(self.n, _ptr(self.x).value, _ptr(self.y).value, _ptr(self.nx).value,
                         _ptr(self.ny).value, _ptr(self.flag).value, _ptr(self.off).value,
                         _ptr(self.nbr).value, self.gamma, float(wall_factor), int(order),
                         int(outer_mode), float(weight_power))

    @classmethod
    def from_cloud(cls, cloud, gamma: float = GAMMA, wall_factor: float = 2.0, order: int = 2,
                   outer_mode: int = 1, weight_power: float = 0.0):
        return cls(cloud.xy, cloud.normals, cloud.flags, cloud.nbr_offsets, cloud.nbr_idx, gamma,
                   wall_factor, order, outer_mode, weight_power)

    @property
    def ref(self):
        return C.byref(self._s)


# ------------------------------------------------------------------ point maps

def prim_to_q(W, gamma=GAMMA):
    """Eq. 26 for each row of W = (rho, u1, u2, p)."""
    lib = _load()
    W = _f64(W, (-1, 4))
    q = np.empty_like(W)
    lib.orc_prim_to_q_n(W.shape[0], _ptr(W), float(gamma), _ptr(q))
    return q


def q_to_prim(q, gamma=GAMMA):
    """Inverse of Eq. 26 for each row."""
    lib = _load()
    q = _f64(q, (-1, 4))
    W = np.empty_like(q)
    lib.orc_q_to_prim_n(q.shape[0], _ptr(q), float(gamma), _ptr(W))
    return W


def prim_to_cons(W, gamma=GAMMA):
    lib = _load()
    W = _f64(W, (-1, 4))
    U = np.empty_like(W)
    lib.orc_prim_to_cons_n(W.shape[0], _ptr(W), float(gamma), _ptr(U))
    return U


def cons_to_prim(U, gamma=GAMMA):
    lib = _load()
    U = _f64(U, (-1, 4))
    W = np.empty_like(U)
    lib.orc_cons_to_prim_n(U.shape[0], _ptr(U), float(gamma), _ptr(W))
    return W


def split_flux(W, direction: int, sign: int, gamma=GAMMA):
    """Kinetic split flux G^(sign) along x (direction 0) or y (1), per row of W."""
    lib = _load()
    W = _f64(W, (-1, 4))
    G = np.empty_like(W)
    lib.orc_split_flux_n(W.shape[0], _ptr(W), int(direction), int(sign), float(gamma), _ptr(G))
    return G


# --------------------------------------------------------------- cloud sweeps

def q_derivatives(oc: OracleCloud, q, inner: int):
    """Eq. 11 then `inner` Jacobi sweeps of Eq. 29 (full stencil, global frame)."""
    lib = _load()
    q = _f64(q, (oc.n, 4))
    qx = np.empty_like(q)
    qy = np.empty_like(q)
    lib.orc_q_derivatives(oc.ref, _ptr(q), int(inner), _ptr(qx), _ptr(qy))
    return qx, qy


def ls_sweep(oc: OracleCloud, q, px=None, py=None):
    """One sweep: Eq. 11 on q (px, py None) or Eq. 29 with q~ from (px, py)."""
    lib = _load()
    q = _f64(q, (oc.n, 4))
    if px is not None:
        px = _f64(px, (oc.n, 4))
        py = _f64(py, (oc.n, 4))
    qx = np.empty_like(q)
    qy = np.empty_like(q)
    lib.orc_ls_sweep(oc.ref, _ptr(q), _ptr(px), _ptr(py), _ptr(qx), _ptr(qy))
    return qx, qy


def flux_residual(oc: OracleCloud, q, qx, qy):
    """Eq. 12 residual per point (conserved components, global frame)."""
    lib = _load()
    q, qx, qy = (_f64(a, (oc.n, 4)) for a in (q, qx, qy))
    R = np.empty_like(q)
    bad = lib.orc_flux_residual(oc.ref, _ptr(q), _ptr(qx), _ptr(qy), _ptr(R))
    return R, bad


def flux_residual_subset(oc: OracleCloud, q, qx, qy, idx):
    lib = _load()
    q, qx, qy = (_f64(a, (oc.n, 4)) for a in (q, qx, qy))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    R = np.empty((idx.size, 4), dtype=np.float64)
    bad = lib.orc_flux_residual_subset(oc.ref, _ptr(q), _ptr(qx), _ptr(qy), _ptr(idx),
                                       idx.size, _ptr(R))
    return R, bad


def timestep(oc: OracleCloud, W, cfl: float):
    lib = _load()
    W = _f64(W, (oc.n, 4))
    dt = np.empty(oc.n, dtype=np.float64)
    lib.orc_timestep(oc.ref, _ptr(W), float(cfl), _ptr(dt))
    return dt


def rk_stage(stage: int, U0, U, R, dt: float):
    lib = _load()
    U0, U, R = (_f64(a, (4,)) for a in (U0, U, R))
    out = np.empty(4, dtype=np.float64)
    lib.orc_rk_stage(int(stage), _ptr(U0), _ptr(U), _ptr(R), float(dt), _ptr(out))
    return out


def wall_project(U, nx: float, ny: float):
    lib = _load()
    U = _f64(U, (4,)).copy()
    lib.orc_wall_project(_ptr(U), float(nx), float(ny))
    return U


def residue(R):
    lib = _load()
    R = _f64(R, (-1, 4))
    return lib.orc_residue(R.shape[0], _ptr(R))


def forces(oc: OracleCloud, W, wall_loop, mach: float, alpha_deg: float):
    lib = _load()
    W = _f64(W, (oc.n, 4))
    loop = np.ascontiguousarray(wall_loop, dtype=np.int64)
    cl = C.c_double()
    cd = C.c_double()
    lib.orc_forces(oc.ref, _ptr(W), _ptr(loop), loop.size, float(mach), float(alpha_deg),
                   C.byref(cl), C.byref(cd))
    return cl.value, cd.value


def freestream(mach: float, alpha_deg: float, gamma=GAMMA):
    lib = _load()
    W = np.empty(4, dtype=np.float64)
    lib.orc_freestream(float(gamma), float(mach), float(alpha_deg), _ptr(W))
    return W


def iterate(oc: OracleCloud, W, iters: int, cfl: float = 0.2, inner: int = 2,
            want_r1: bool = False):
    """Algorithm 1 for `iters` iterations from W (returned updated, not in place).

    Returns (W, residue history, status[, stage-1 residual of the last iteration]).
    """
    lib = _load()
    W = _f64(W, (oc.n, 4)).copy()
    res = np.empty(max(iters, 1), dtype=np.float64)
    R1 = np.empty((oc.n, 4), dtype=np.float64) if want_r1 else None
    st = lib.orc_iterate(oc.ref, _ptr(W), int(iters), float(cfl), int(inner), _ptr(res),
                         _ptr(R1))
    res = res[:iters]
    if want_r1:
        return W, res, st, R1
    return W, res, st


def residual_of_state(oc: OracleCloud, W, inner: int = 2):
    lib = _load()
    W = _f64(W, (oc.n, 4))
    R = np.empty_like(W)
    bad = lib.orc_residual_of_state(oc.ref, _ptr(W), int(inner), _ptr(R))
    return R, bad


def num_threads() -> int:
    return int(_load().orc_num_threads())

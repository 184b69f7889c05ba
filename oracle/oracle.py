"""numpy front end of the plain FP64 CPU oracle (``lskum_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg, never by the solver package. The C file is
compiled here with gcc (``-O2 -ffp-contract=off -fopenmp``) into
``oracle/_build/liblskum_oracle.so``; nothing of the CUDA path is linked.
The same C file compiled with ``-DORC_QUAD`` (``liblskum_oracle_q.so``) runs
the same formulas in IEEE binary128: ``residual_at`` uses it as the
extended-precision reference of a residual evaluation (see its docstring).

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
_LIB_Q = os.path.join(_BUILD, "liblskum_oracle_q.so")
_lock = threading.Lock()
_libs = {}

GAMMA = 1.4


def build(force: bool = False, quad: bool = False) -> str:
    """Compile the oracle shared library (idempotent): the FP64 build, or with
    ``quad`` the binary128 build of the same source."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_Q if quad else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=gnu11", "-Wl,-Bsymbolic", "-o", tmp, _SRC, "-lm"]
        if quad:
            cmd.insert(1, "-DORC_QUAD")
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


class _Cloud(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("nx", C.c_void_p),
                ("ny", C.c_void_p), ("flag", C.c_void_p), ("off", C.c_void_p),
                ("nbr", C.c_void_p), ("gamma", C.c_double), ("wall_factor", C.c_double),
                ("order", C.c_int), ("outer_mode", C.c_int), ("weight_power", C.c_double)]


def _load(quad: bool = False):
    """The FP64 library, or (quad) the binary128 one. In the binary128 build
    every array argument is a buffer of binary128 values (see ``_RealBuf``)."""
    with _lock:
        if quad not in _libs:
            lib = C.CDLL(build(quad=quad))
            P = C.c_void_p
            lib.orc_real_bytes.restype = C.c_int
            lib.orc_to_real.argtypes = [C.c_int64, P, P, P]
            lib.orc_from_real.argtypes = [C.c_int64, P, P, P]
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
            assert lib.orc_real_bytes() == (16 if quad else 8)
            _libs[quad] = lib
    return _libs[quad]


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
        self.options = dict(gamma=float(gamma), wall_factor=float(wall_factor), order=int(order),
                            outer_mode=int(outer_mode), weight_power=float(weight_power))
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

    def neighbourhood(self, seeds, hops: int):
        """Hop distance (0 .. hops) from `seeds` along the neighbour lists, -1
        beyond: point j is one hop from i when j is in N(i)."""
        level = np.full(self.n, -1, dtype=np.int8)
        frontier = np.unique(np.asarray(seeds, dtype=np.int64))
        level[frontier] = 0
        for h in range(1, hops + 1):
            starts, ends = self.off[frontier], self.off[frontier + 1]
            lens = (ends - starts).astype(np.int64)
            first = np.repeat(starts.astype(np.int64) - np.cumsum(lens) + lens, lens)
            cand = self.nbr[first + np.arange(lens.sum())]
            cand = np.unique(cand[level[cand] < 0])
            level[cand] = h
            frontier = cand.astype(np.int64)
        return level

    def subcloud(self, seeds, hops: int):
        """The points within `hops` of `seeds` as a cloud of their own, with
        this cloud's options. Points closer than `hops` keep their whole
        neighbour list in its order; the outermost ring keeps only the
        neighbours inside. Returns (sub-cloud, members (global indices, sorted),
        the seeds' indices in the sub-cloud)."""
        level = self.neighbourhood(seeds, hops)
        members = np.flatnonzero(level >= 0)
        local = np.full(self.n, -1, dtype=np.int64)
        local[members] = np.arange(members.size)
        starts, ends = self.off[members], self.off[members + 1]
        lens = (ends - starts).astype(np.int64)
        first = np.repeat(starts.astype(np.int64) - np.cumsum(lens) + lens, lens)
        edges = local[self.nbr[first + np.arange(lens.sum())]]
        owner = np.repeat(np.arange(members.size), lens)
        keep = edges >= 0
        assert np.all(keep[level[members][owner] < hops])  # inner rings are complete
        off = np.zeros(members.size + 1, dtype=np.int32)
        off[1:] = np.cumsum(np.bincount(owner[keep], minlength=members.size))
        sub = OracleCloud(np.stack([self.x[members], self.y[members]], 1),
                          np.stack([self.nx[members], self.ny[members]], 1), self.flag[members],
                          off, edges[keep].astype(np.int32), **self.options)
        return sub, members, local[np.asarray(seeds, dtype=np.int64)]


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


# ------------------------------------------------- extended-precision reference

class _RealBuf:
    """An array of `count` values of the library's `real` type (opaque bytes)."""

    def __init__(self, lib, count: int):
        self.lib, self.count = lib, int(count)
        self.raw = np.zeros(self.count * lib.orc_real_bytes(), dtype=np.uint8)

    @classmethod
    def of(cls, lib, hi, lo=None):
        hi = np.ascontiguousarray(hi, dtype=np.float64).ravel()
        buf = cls(lib, hi.size)
        lo = None if lo is None else np.ascontiguousarray(lo, dtype=np.float64).ravel()
        lib.orc_to_real(hi.size, _ptr(hi), _ptr(lo), _ptr(buf.raw))
        return buf

    def split(self):
        """(hi, lo): the values rounded to double and the remainders."""
        hi = np.empty(self.count, dtype=np.float64)
        lo = np.empty(self.count, dtype=np.float64)
        self.lib.orc_from_real(self.count, _ptr(self.raw), _ptr(hi), _ptr(lo))
        return hi, lo

    @property
    def ptr(self):
        return _ptr(self.raw)


def split_flux_real(W, direction: int, sign: int, quad: bool = True, gamma=GAMMA, W_lo=None):
    """``split_flux`` in the chosen build on W (+ W_lo); returns (hi, lo) rows."""
    lib = _load(quad)
    W = _f64(W, (-1, 4))
    Wr, G = _RealBuf.of(lib, W, W_lo), _RealBuf(lib, W.size)
    lib.orc_split_flux_n(W.shape[0], Wr.ptr, int(direction), int(sign), float(gamma), G.ptr)
    hi, lo = G.split()
    return hi.reshape(-1, 4), lo.reshape(-1, 4)


def q_to_prim_real(q_hi, q_lo=None, quad: bool = True, gamma=GAMMA):
    """Inverse of Eq. 26 in the chosen build on q = hi + lo; returns (hi, lo)."""
    lib = _load(quad)
    q_hi = _f64(q_hi, (-1, 4))
    qr, W = _RealBuf.of(lib, q_hi, q_lo), _RealBuf(lib, q_hi.size)
    lib.orc_q_to_prim_n(q_hi.shape[0], qr.ptr, float(gamma), W.ptr)
    hi, lo = W.split()
    return hi.reshape(-1, 4), lo.reshape(-1, 4)


def prim_to_q_real(W, quad: bool = True, gamma=GAMMA, W_lo=None):
    """Eq. 26 in the chosen build on W (+ W_lo); returns (hi, lo)."""
    lib = _load(quad)
    W = _f64(W, (-1, 4))
    Wr, q = _RealBuf.of(lib, W, W_lo), _RealBuf(lib, W.size)
    lib.orc_prim_to_q_n(W.shape[0], Wr.ptr, float(gamma), q.ptr)
    hi, lo = q.split()
    return hi.reshape(-1, 4), lo.reshape(-1, 4)


def q_derivatives_real(oc: OracleCloud, q_hi, q_lo=None, inner: int = 2, quad: bool = True):
    """``q_derivatives`` in the chosen build on q = hi + lo; returns
    ((qx hi, qx lo), (qy hi, qy lo))."""
    lib = _load(quad)
    q_hi = _f64(q_hi, (oc.n, 4))
    qr = _RealBuf.of(lib, q_hi, q_lo)
    qx, qy = _RealBuf(lib, q_hi.size), _RealBuf(lib, q_hi.size)
    lib.orc_q_derivatives(oc.ref, qr.ptr, int(inner), qx.ptr, qy.ptr)
    return tuple(tuple(a.reshape(-1, 4) for a in b.split()) for b in (qx, qy))


def ls_sweep_real(oc: OracleCloud, q, px=None, py=None, quad: bool = True):
    """``ls_sweep`` in the chosen build; q, px, py are arrays or (hi, lo)
    pairs; returns ((qx hi, lo), (qy hi, lo))."""
    lib = _load(quad)

    def buf(a):
        if a is None:
            return None
        hi, lo = a if isinstance(a, tuple) else (a, None)
        return _RealBuf.of(lib, _f64(hi, (oc.n, 4)), lo)

    qr, pxr, pyr = buf(q), buf(px), buf(py)
    q = qr.count
    qx, qy = _RealBuf(lib, q), _RealBuf(lib, q)
    lib.orc_ls_sweep(oc.ref, qr.ptr, pxr.ptr if pxr else None, pyr.ptr if pyr else None,
                     qx.ptr, qy.ptr)
    return tuple(tuple(a.reshape(-1, 4) for a in b.split()) for b in (qx, qy))


def residual_at(oc: OracleCloud, W, idx, inner: int = 2, quad: bool = True):
    """The stage-1 residual R(W) (Eq. 12, with the q-derivatives of Eqs. 11,
    28-29) and the final q-derivatives at the points `idx`, evaluated on the
    (inner + 2)-hop neighbourhood of those points only -- all that R at them
    depends on: R_i reads the derivatives of N(i), each inner sweep reaches one
    hop further, the first-order sweep one more, and it reads q of its
    neighbours. With ``quad`` the binary128 build computes it from the same
    double inputs: the extended-precision reference of an FP64 evaluation
    (its own rounding error is ~1e-30 of the values, far below FP64's).

    Returns a dict of (hi, lo) pairs: "R", "qx", "qy" (rows follow `idx`), and
    "bad" (split stencils with a non-positive determinant at `idx`).
    """
    lib = _load(quad)
    idx = np.asarray(idx, dtype=np.int64)
    sub, members, loc = oc.subcloud(idx, inner + 2)
    Ws = _f64(W, (oc.n, 4))[members]
    Wr = _RealBuf.of(lib, Ws)
    q = _RealBuf(lib, Ws.size)
    lib.orc_prim_to_q_n(sub.n, Wr.ptr, float(sub.gamma), q.ptr)
    qx, qy = _RealBuf(lib, Ws.size), _RealBuf(lib, Ws.size)
    lib.orc_q_derivatives(sub.ref, q.ptr, int(inner), qx.ptr, qy.ptr)
    R = _RealBuf(lib, 4 * idx.size)
    loc = np.ascontiguousarray(loc, dtype=np.int64)
    bad = lib.orc_flux_residual_subset(sub.ref, q.ptr, qx.ptr, qy.ptr, _ptr(loc), loc.size,
                                       R.ptr)
    out = {"bad": int(bad), "R": tuple(a.reshape(-1, 4) for a in R.split())}
    for name, buf in (("qx", qx), ("qy", qy)):
        hi, lo = buf.split()
        out[name] = (hi.reshape(-1, 4)[loc], lo.reshape(-1, 4)[loc])
    return out

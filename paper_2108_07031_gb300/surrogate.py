"""Learned warm start for the q-LSKUM solver.

A coordinate/condition MLP (include/lskum_mlp.h) maps (x, y, wall distance,
Mach, alpha) at every point to the flow state (rho, u1, u2, p). It is
trained on converged solutions that the batched solver itself produces and
is used only to choose the starting state of a solve: the solver iterates to
convergence from it, so the converged answer (Cl, Cd, the field) is the
solver's, not the network's; a non-physical prediction falls back to the
free-stream start. The paper always starts from the free stream.

Everything numerical runs in the library's CUDA kernels (BF16 tensor-core
GEMMs with FP32 accumulation for the network, the solver for the data and
the solves); this module marshals arguments and keeps the training loop.
Tensors on the GPU are torch tensors (device memory only).
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import cloud as Cl
from . import lskum as L

GAMMA = 1.4
OUT_SCALE = 0.25  # network output o -> W = W_inf + OUT_SCALE * o


def _lib():
    lib = L.load()
    if not getattr(lib, "_mlp_declared", False):
        P, I64, I, D, F = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_float
        sig = {
            "lskum_mlp_num_params": ([], I64),
            "lskum_mlp_create": ([I64, P, P], I),
            "lskum_mlp_destroy": ([P], None),
            "lskum_mlp_set_params": ([P, P, I64], I),
            "lskum_mlp_get_params": ([P, P, I64], I),
            "lskum_mlp_features": ([P, P, I64, P], I),
            "lskum_mlp_predict": ([P, P, I64, P], I),
            "lskum_mlp_gradients": ([P, P, P, I64, P, P], I),
            "lskum_mlp_train_step": ([P, P, P, I64, F, P], I),
            "lskum_mlp_sync": ([P], I),
            "lskum_mlp_set_stream": ([P, P], I),
            "lskum_mlp_set_gemm": ([P, I], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        lib._mlp_declared = True
    return lib


EXPORTED = ("lskum_mlp_num_params", "lskum_mlp_create", "lskum_mlp_destroy",
            "lskum_mlp_set_params", "lskum_mlp_get_params", "lskum_mlp_features",
            "lskum_mlp_predict", "lskum_mlp_gradients", "lskum_mlp_train_step", "lskum_mlp_sync",
            "lskum_mlp_set_stream", "lskum_mlp_set_gemm")

GEMM_MMA_SYNC, GEMM_TCGEN05 = 0, 1


def projection(seed: int = 2108, scales=(1.0,) * 8) -> np.ndarray:
    """Seeded 8 x 2 Gaussian projection of (x, y) for the Fourier features;
    row k has standard deviation scales[k] (its spatial frequency)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = rng.normal(0.0, 1.0, size=(8, 2))
    return (P * np.asarray(scales, dtype=np.float64)[:, None]).astype(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """Xavier-uniform weights, zero biases (W_0's padding columns zero)."""
    lib = _lib()
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l in range(6):
        k = 32 if l == 0 else 256
        n = 4 if l == 5 else 256
        fan_in = 21 if l == 0 else k
        lim = math.sqrt(6.0 / (fan_in + n))
        W = rng.uniform(-lim, lim, size=(n, k))
        if l == 0:
            W[:, 21:] = 0.0
        parts += [W.ravel(), np.zeros(n)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == lib.lskum_mlp_num_params()
    return p


class MLP:
    """The surrogate network on the GPU (``lskum_mlp_*``)."""

    def __init__(self, capacity: int = 65536, proj: np.ndarray | None = None, seed: int = 0):
        lib = _lib()
        self._lib = lib
        self.capacity = int(capacity)
        self.proj = np.ascontiguousarray(projection() if proj is None else proj, dtype=np.float32)
        h = C.c_void_p()
        L._check(lib.lskum_mlp_create(self.capacity, self.proj.ctypes.data_as(C.c_void_p),
                                      C.byref(h)), "lskum_mlp_create")
        self._h = h
        self.n_params = int(lib.lskum_mlp_num_params())
        self.set_params(init_params(seed))
        # run on torch's current stream: the batches torch gathers for
        # train_step are then written only after the previous step read them
        import torch
        if torch.cuda.is_available():
            self.set_stream(torch.cuda.current_stream().cuda_stream)

    def set_stream(self, handle: int):
        """Run on CUDA stream `handle` (torch's `cuda_stream`; 0, the legacy
        default stream, is passed as cudaStreamLegacy)."""
        h = int(handle) if handle else 1  # 1 == cudaStreamLegacy
        L._check(self._lib.lskum_mlp_set_stream(self._h, C.c_void_p(h)), "lskum_mlp_set_stream")

    def set_gemm(self, path: int):
        """GEMM path of the forward pass's 256-wide layers (GEMM_MMA_SYNC or
        GEMM_TCGEN05)."""
        L._check(self._lib.lskum_mlp_set_gemm(self._h, int(path)), "lskum_mlp_set_gemm")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lskum_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        L._check(self._lib.lskum_mlp_set_params(self._h, p.ctypes.data_as(C.c_void_p), p.size),
                 "lskum_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, dtype=np.float32)
        L._check(self._lib.lskum_mlp_get_params(self._h, p.ctypes.data_as(C.c_void_p), p.size),
                 "lskum_mlp_get_params")
        return p

    def features(self, raw_dev):
        """raw (torch, cuda, float32, n x 5) -> features (n x 32)."""
        import torch
        n = raw_dev.shape[0]
        feat = torch.empty((n, 32), dtype=torch.float32, device=raw_dev.device)
        L._check(self._lib.lskum_mlp_features(self._h, C.c_void_p(raw_dev.data_ptr()), n,
                                              C.c_void_p(feat.data_ptr())), "lskum_mlp_features")
        return feat

    def predict(self, feat_dev):
        import torch
        n = feat_dev.shape[0]
        out = torch.empty((n, 4), dtype=torch.float32, device=feat_dev.device)
        for a in range(0, n, self.capacity):
            b = min(n, a + self.capacity)
            L._check(self._lib.lskum_mlp_predict(self._h, C.c_void_p(feat_dev[a:b].data_ptr()),
                                                 b - a, C.c_void_p(out[a:b].data_ptr())),
                     "lskum_mlp_predict")
        return out

    def gradients(self, feat_dev, target_dev):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_double()
        L._check(self._lib.lskum_mlp_gradients(self._h, C.c_void_p(feat_dev.data_ptr()),
                                               C.c_void_p(target_dev.data_ptr()),
                                               feat_dev.shape[0], g.ctypes.data_as(C.c_void_p),
                                               C.byref(loss)), "lskum_mlp_gradients")
        return loss.value, g

    def train_step(self, feat_dev, target_dev, lr: float, want_loss: bool = True):
        loss = C.c_double()
        L._check(self._lib.lskum_mlp_train_step(self._h, C.c_void_p(feat_dev.data_ptr()),
                                                C.c_void_p(target_dev.data_ptr()),
                                                feat_dev.shape[0], float(lr),
                                                C.byref(loss) if want_loss else None),
                 "lskum_mlp_train_step")
        return loss.value if want_loss else None


# ---------------------------------------------------------------- data

def wall_distance(cloud) -> np.ndarray:
    """Distance of every point to the nearest wall point (input geometry)."""
    walls = cloud.xy[cloud.flags == Cl.FLAG_WALL]
    d = np.full(cloud.n, np.inf)
    for a in range(0, cloud.n, 4096):
        diff = cloud.xy[a:a + 4096, None, :] - walls[None, :, :]
        d[a:a + 4096] = np.sqrt((diff ** 2).sum(-1)).min(axis=1)
    return d


def wall_arc(cloud) -> np.ndarray:
    """Position (0..1) along the wall loop of every point's nearest wall point."""
    wall_idx = np.flatnonzero(cloud.flags == Cl.FLAG_WALL)
    walls = cloud.xy[wall_idx]
    s = np.empty(cloud.n)
    for a in range(0, cloud.n, 4096):
        diff = cloud.xy[a:a + 4096, None, :] - walls[None, :, :]
        s[a:a + 4096] = np.argmin((diff ** 2).sum(-1), axis=1) / float(len(wall_idx))
    return s


def wall_features(cloud, wall_d, arc, mach, alpha_deg, proj) -> np.ndarray:
    """Alternative 21 (+ 11 zero) inputs, computed on the host: (x, y, wall
    distance, M, alpha) scaled as in lskum_mlp_features, then sin/cos of
    2 pi k s (k = 1..4) of the wall-loop position s of the nearest wall
    point, then sin/cos of the first 4 Fourier projections of (x, y).
    n x 32 float32."""
    x, y = cloud.xy[:, 0], cloud.xy[:, 1]
    f = np.zeros((cloud.n, 32))
    f[:, 0] = x / 10.0
    f[:, 1] = y / 10.0
    f[:, 2] = np.log(wall_d + 1e-3) / 5.0
    f[:, 3] = (mach - 0.55) * 4.0
    f[:, 4] = (alpha_deg - 1.0) / 5.0
    for k in range(4):
        f[:, 5 + k] = np.sin(2 * np.pi * (k + 1) * arc)
        f[:, 9 + k] = np.cos(2 * np.pi * (k + 1) * arc)
    t = cloud.xy @ np.asarray(proj, dtype=np.float64)[:4].T
    f[:, 13:17] = np.sin(t)
    f[:, 17:21] = np.cos(t)
    return f.astype(np.float32)


def raw_inputs(cloud, wall_d, mach, alpha_deg) -> np.ndarray:
    """n_cond x n x 5 float32: (x, y, wall distance, M, alpha)."""
    mach = np.atleast_1d(np.asarray(mach, dtype=np.float64))
    alpha = np.atleast_1d(np.asarray(alpha_deg, dtype=np.float64))
    out = np.empty((mach.size, cloud.n, 5), dtype=np.float32)
    out[:, :, 0] = cloud.xy[:, 0]
    out[:, :, 1] = cloud.xy[:, 1]
    out[:, :, 2] = wall_d
    out[:, :, 3] = mach[:, None]
    out[:, :, 4] = alpha[:, None]
    return out


def freestream(mach, alpha_deg):
    a = math.radians(alpha_deg)
    return np.array([1.0, mach * math.cos(a), mach * math.sin(a), 1.0 / GAMMA])


def targets(W, mach, alpha_deg) -> np.ndarray:
    """Normalised deviations from the free stream (the network's outputs)."""
    return ((W - freestream(mach, alpha_deg)) / OUT_SCALE).astype(np.float32)


def state_from_output(out, mach, alpha_deg) -> np.ndarray:
    return freestream(mach, alpha_deg) + OUT_SCALE * np.asarray(out, dtype=np.float64)


def converged_solutions(cloud, mach, alpha, tol=1e-6, max_iters=60_000, batch=64, cfl=0.8,
                        precision=L.MIXED):
    """Solve every (M, alpha) with the batched solver to a `tol` residue drop.

    Returns (states n_cond x n x 4, iterations used per batch). The converged
    state does not depend on the pseudo-time step, so the data is generated
    at a larger CFL than the evaluation uses.
    """
    mach = np.asarray(mach, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    states, iters = [], []
    for a in range(0, mach.size, batch):
        m = mach[a:a + batch]
        al = alpha[a:a + batch]
        nc = 1 << int(math.ceil(math.log2(max(1, m.size))))
        mm = np.concatenate([m, np.repeat(m[-1:], nc - m.size)])
        aa = np.concatenate([al, np.repeat(al[-1:], nc - al.size)])
        with L.Solver.from_cloud(cloud, precision=precision, cfl=cfl, n_conditions=nc,
                                 check_every=500) as s:
            s.set_conditions(mm, aa)
            done = s.solve(max_iters, tol)
            W = s.get_state()
        W = W.reshape(nc, cloud.n, 4)[: m.size]
        states.append(W)
        iters.append(done)
    return np.concatenate(states), iters


def train(mlp: MLP, feats_dev, targets_dev, epochs=40, batch=8192, lr=2e-3, lr_final=1e-4,
          seed=0, log=None):
    """Adam over shuffled mini-batches with a cosine learning-rate decay."""
    import torch
    n = feats_dev.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(feats_dev.device)
        for k in range(steps_per_epoch):
            idx = perm[k * batch:(k + 1) * batch]
            lr_k = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / total))
            # the loss is read back (a host synchronisation) once per epoch
            last = k == steps_per_epoch - 1
            loss = mlp.train_step(feats_dev[idx].contiguous(), targets_dev[idx].contiguous(), lr_k,
                                  want_loss=last)
            step += 1
        losses.append(loss)  # loss of the epoch's last mini-batch
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    return losses


def predict_state(mlp: MLP, cloud, wall_d, mach, alpha_deg, arc=None):
    """Network prediction of the primitive state for one condition (n x 4),
    or None when it is not physical (the caller keeps the free stream).
    With `arc` (wall_arc) the inputs are wall_features, else the library's
    Fourier encoding."""
    import torch
    if arc is None:
        raw = torch.from_numpy(raw_inputs(cloud, wall_d, [mach], [alpha_deg])[0]).cuda()
        feat = mlp.features(raw)
    else:
        feat = torch.from_numpy(wall_features(cloud, wall_d, arc, mach, alpha_deg, mlp.proj)).cuda()
    out = mlp.predict(feat).cpu().numpy()
    W = state_from_output(out, mach, alpha_deg)
    if not np.all(np.isfinite(W)) or np.any(W[:, 0] <= 0.05) or np.any(W[:, 3] <= 0.05):
        return None
    # far-field points are boundary data, held at whatever state they are
    # given: they keep the exact free stream (a predicted far field would fix
    # a different circulation around the aerofoil for good)
    W[cloud.flags == Cl.FLAG_OUTER] = freestream(mach, alpha_deg)
    # the wall condition holds no normal momentum: project the prediction
    wall = cloud.flags == Cl.FLAG_WALL
    n = cloud.normals[wall]
    un = (W[wall, 1] * n[:, 0] + W[wall, 2] * n[:, 1])
    W[wall, 1] -= un * n[:, 0]
    W[wall, 2] -= un * n[:, 1]
    return W


def _time_predict(batches, repeats):
    """Host-timed predict of random feature batches with each forward GEMM path."""
    import time

    import torch
    net = MLP(capacity=max(batches), seed=1)
    try:
        for n in batches:
            fd = torch.randn(n, 32, device="cuda")
            fd[:, 21:] = 0
            for path, name in ((GEMM_MMA_SYNC, "mma.sync"), (GEMM_TCGEN05, "tcgen05")):
                net.set_gemm(path)
                net.predict(fd)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(repeats):
                    net.predict(fd)
                torch.cuda.synchronize()
                print(f"batch {n}, {name}: predict {(time.perf_counter() - t0) / repeats * 1e6:.1f} us",
                      flush=True)
    finally:
        net.set_gemm(GEMM_MMA_SYNC)
        net.close()


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="time the surrogate's predict with both GEMM paths")
    ap.add_argument("--batches", default="4096", help="comma-separated batch sizes")
    ap.add_argument("--repeats", type=int, default=50)
    a = ap.parse_args()
    _time_predict([int(v) for v in a.batches.split(",")], a.repeats)

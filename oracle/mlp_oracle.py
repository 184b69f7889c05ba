"""Plain numpy FP64 reference of the warm-start MLP (forward, loss, backward).

TEST INFRASTRUCTURE ONLY (imported by tests/, never by the package). It
follows the network of include/lskum_mlp.h written out layer by layer:
six linear layers, tanh between them, mean squared error. With
``emulate=True`` it rounds to BF16 (round to nearest even) exactly where the
GPU keeps BF16 operands -- the features, the weights, the hidden activations
fed to the next layer and the error signals fed to the gradient GEMMs -- and
does all sums in FP64, so the GPU (FP32 accumulation) can be compared with it
at BF16-appropriate tolerance. With ``emulate=False`` it is the plain FP64
network whose gradient the tests pin by central finite differences.
"""

from __future__ import annotations

import numpy as np

LAYERS = 6
WIDTH = 256
IN = 21
IN_PADDED = 32
OUT = 4


def layer_shapes():
    """(out, in) of W_l for l = 0..5."""
    shapes = []
    for l in range(LAYERS):
        k = IN_PADDED if l == 0 else WIDTH
        n = OUT if l == LAYERS - 1 else WIDTH
        shapes.append((n, k))
    return shapes


def num_params():
    return sum(n * k + n for n, k in layer_shapes())


def unpack(params):
    """Flat vector -> [(W_l, b_l)] (views); W_0's padded columns read as zero."""
    out = []
    off = 0
    for l, (n, k) in enumerate(layer_shapes()):
        W = params[off:off + n * k].reshape(n, k)
        off += n * k
        b = params[off:off + n]
        off += n
        out.append((W, b))
    return out


def bf16(a):
    """Round to BF16 (via FP32, round to nearest even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def features(raw, proj):
    """raw n x 5 (x, y, wall distance, M, alpha_deg) -> n x 32 (FP64)."""
    raw = np.asarray(raw, dtype=np.float64)
    proj = np.asarray(proj, dtype=np.float64).reshape(8, 2)
    x, y, d, m, a = raw.T
    f = np.zeros((raw.shape[0], IN_PADDED))
    f[:, 0] = x / 10.0
    f[:, 1] = y / 10.0
    f[:, 2] = np.log(d + 1e-3) / 5.0
    f[:, 3] = (m - 0.55) * 4.0
    f[:, 4] = (a - 1.0) / 5.0
    t = raw[:, :2] @ proj.T
    f[:, 5:13] = np.sin(t)
    f[:, 13:21] = np.cos(t)
    return f


def forward(params, feat, emulate=True):
    """Returns (Y, cache). feat is n x 32 (the GPU's FP32 features)."""
    layers = unpack(np.asarray(params, dtype=np.float64))
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    X = r(feat)
    xs, acts = [X], []
    for l, (W, b) in enumerate(layers):
        Wl = W.copy()
        if l == 0:
            Wl[:, IN:] = 0.0
        Z = X @ r(Wl).T + b
        if l < LAYERS - 1:
            A = np.tanh(Z)
            acts.append(A)
            X = r(A)
            xs.append(X)
        else:
            return Z, (xs, acts)


def loss_and_grad(params, feat, target, emulate=True):
    """Mean squared error over n x 4 outputs and its gradient (flat)."""
    params = np.asarray(params, dtype=np.float64)
    layers = unpack(params)
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    Y, (xs, acts) = forward(params, feat, emulate)
    T = np.asarray(target, dtype=np.float64)
    n = T.shape[0]
    loss = float(np.mean((Y - T) ** 2))
    dZ = 2.0 * (Y - T) / (n * OUT)
    grads = []
    for l in range(LAYERS - 1, -1, -1):
        W, _ = layers[l]
        dZb = r(dZ)
        dW = dZb.T @ xs[l]
        db = dZ.sum(axis=0)
        if l == 0:
            dW[:, IN:] = 0.0
        grads.append((dW, db))
        if l == 0:
            break
        Wl = W.copy()
        if l == 0:
            Wl[:, IN:] = 0.0
        dA = dZb @ r(Wl)
        dZ = dA * (1.0 - acts[l - 1] ** 2)
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat

"""Helpers shared by the GPU parity tests (no GPU needed to import)."""

import numpy as np

from oracle import oracle as O


def normwise(a, b):
    """max over components of max_i |a - b| / max_i |b|."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return float((np.abs(a - b).max(axis=0) / scale).max())


def linf_rel(a, b):
    """||a - b||_inf / ||b||_inf over all entries: the one-step parity measure."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def residual_conditioning_bound(oc, W, inner=2, factor=8.0, floor=1e-12, seed=11):
    """Tolerance for an FP64 residual comparison from the problem's conditioning.

    The oracle alone evaluates the residual of W and of W perturbed by one ulp
    (random sign per entry); the norm-wise spread is what any two correct FP64
    evaluations may differ by. Returns (reference residual, max(floor, factor
    x spread), spread).
    """
    R, bad = O.residual_of_state(oc, W, inner=inner)
    assert bad == 0
    rng = np.random.Generator(np.random.PCG64(seed))
    Wp = W * (1.0 + np.finfo(np.float64).eps * rng.choice([-1.0, 1.0], size=W.shape))
    Rp, _ = O.residual_of_state(oc, Wp, inner=inner)
    spread = normwise(Rp, R)
    return R, max(floor, factor * spread), spread

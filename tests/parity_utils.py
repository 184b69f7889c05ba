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


def exact_errors(oc, W, got, idx=None, inner=2):
    """Errors of a GPU evaluation and of the FP64 oracle against the binary128
    reference (the same formulas on the same inputs, ``oracle.residual_at``).

    `got` maps "R", "qx", "qy" (any subset) to the GPU's full n x 4 arrays;
    `idx` picks the points compared (all by default). Returns, per name, the
    per-component errors relative to the reference's largest magnitude in
    that component: {"gpu_max", "oracle_max", "gpu_rms", "oracle_rms"}, and
    "gpu_linf", "oracle_linf": the largest error over all entries relative to
    the reference's largest entry (the infinity-norm measure).
    """
    idx = np.arange(oc.n) if idx is None else np.asarray(idx)
    ref = O.residual_at(oc, W, idx, inner, quad=True)
    f64 = O.residual_at(oc, W, idx, inner, quad=False)
    assert ref["bad"] == 0 and f64["bad"] == 0
    out = {}
    for name, arr in got.items():
        hi, lo = ref[name]
        scale = np.abs(hi).max(axis=0)
        scale = np.where(scale > 0, scale, 1.0)
        res = {}
        for who, val in (("gpu", np.asarray(arr)[idx]), ("oracle", f64[name][0])):
            e = np.abs((val - hi) - lo)
            res[who + "_max"] = e.max(axis=0) / scale
            res[who + "_rms"] = np.sqrt((e ** 2).mean(axis=0)) / scale
            res[who + "_linf"] = float(e.max() / scale.max())
        out[name] = res
    return out


def describe(errs):
    """One line per quantity: GPU and oracle errors and their ratios."""
    lines = []
    for name, e in errs.items():
        lines.append(f"{name}: linf gpu {e['gpu_linf']:.2e} oracle {e['oracle_linf']:.2e} | "
                     f"gpu max {np.array2string(e['gpu_max'], precision=2)} oracle max "
                     f"{np.array2string(e['oracle_max'], precision=2)} | rms ratio "
                     f"{np.array2string(e['gpu_rms'] / np.maximum(e['oracle_rms'], 1e-300), precision=2)}")
    return "\n".join(lines)

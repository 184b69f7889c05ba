"""Pins of the warm-start MLP's CPU reference (no GPU needed)."""

import math

import numpy as np

from oracle import mlp_oracle as M


def _random_params(rng, scale=0.3):
    p = np.concatenate([rng.normal(0, scale / math.sqrt(k), n * k).tolist() + rng.normal(0, 0.1, n).tolist()
                        for n, k in M.layer_shapes()])
    return p


def test_gradient_matches_central_differences():
    """The FP64 backward pass equals d(loss)/d(param) by central differences."""
    rng = np.random.Generator(np.random.PCG64(3))
    p = _random_params(rng)
    feat = rng.normal(0, 1, (6, M.IN_PADDED))
    feat[:, M.IN:] = 0.0
    T = rng.normal(0, 1, (6, M.OUT))
    loss, g = M.loss_and_grad(p, feat, T, emulate=False)
    # weights of W_0's live columns, inner layers, biases and the output layer
    idx = [0, 5, 20, 40, 33 + 256 * 7, 8448, 8500, 8448 + 65536 + 17, M.num_params() - 1,
           M.num_params() - 5, M.num_params() - 1030]
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, feat, T, emulate=False)[0] -
              M.loss_and_grad(pm, feat, T, emulate=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, g[i])


def test_padded_input_columns_carry_no_weight():
    rng = np.random.Generator(np.random.PCG64(4))
    p = _random_params(rng)
    feat = rng.normal(0, 1, (3, M.IN_PADDED))
    y1, _ = M.forward(p, feat, emulate=False)
    feat[:, M.IN:] = 123.0
    y2, _ = M.forward(p, feat, emulate=False)
    assert np.array_equal(y1, y2)
    _, g = M.loss_and_grad(p, feat, np.zeros((3, 4)), emulate=False)
    W0g = g[: 256 * 32].reshape(256, 32)
    assert np.all(W0g[:, M.IN:] == 0.0)


def test_bf16_rounding_is_round_to_nearest_even():
    eps = 2.0 ** -7  # bf16 spacing at 1
    vals = np.array([1.0, 1 + eps / 2, 1 + 1.5 * eps, 1 + 0.75 * eps, -(1 + eps / 2), 3.0e38])
    r = M.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                # tie -> even (1.0)
    assert r[2] == 1 + 2 * eps        # tie -> even mantissa
    assert r[3] == 1 + eps
    assert r[4] == -1.0
    assert np.isfinite(r[5])


def test_feature_encoding_closed_form():
    proj = np.arange(16, dtype=np.float64).reshape(8, 2) / 10.0
    raw = np.array([[0.5, -0.25, 0.01, 0.63, 2.0]])
    f = M.features(raw, proj)[0]
    assert f[0] == 0.05 and f[1] == -0.025
    assert abs(f[2] - math.log(0.011) / 5) < 1e-15
    assert abs(f[3] - 0.32) < 1e-15 and abs(f[4] - 0.2) < 1e-15
    t = proj @ np.array([0.5, -0.25])
    assert np.allclose(f[5:13], np.sin(t)) and np.allclose(f[13:21], np.cos(t))
    assert np.all(f[21:] == 0.0)

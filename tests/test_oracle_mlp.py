"""Pins of the float64 surrogate-network oracle (CPU only): closed-form GELU
values, a network that reduces to an affine map, and central finite
differences of the loss for every parameter block."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_forms():
    # gelu(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array(-1.0)) + (1 - 0.8413447460685429)) < 1e-15
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-16
    z = np.linspace(-4, 4, 101)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-9


def test_parameter_count():
    assert mlp.N_PARAMS == 2 * 128 + 128 + 3 * (128 * 128 + 128) + 2 * 128 + 2 == 50178


def test_network_reduces_to_affine_map_without_hidden_weights():
    """With W2..W4 = 0 every sample sees the same hidden state gelu(b4)."""
    rng = np.random.default_rng(0)
    p = mlp.unpack(rng.normal(size=mlp.N_PARAMS) * 0.1)
    for k in (2, 3, 4):
        p[f"W{k}"][:] = 0.0
    x = rng.uniform(-1, 1, size=(7, 2))
    out, _ = mlp.forward(mlp.pack(p), x)
    expect = p["W5"] @ mlp.gelu(p["b4"]) + p["b5"]
    assert np.abs(out - expect).max() < 1e-14


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(size=mlp.N_PARAMS) * 0.2
    x = rng.uniform(-1, 1, size=(9, 2))
    y = np.stack([rng.normal(size=9), (rng.uniform(size=9) > 0.5).astype(float)], axis=1)
    L, g = mlp.grad(p, x, y)
    assert abs(L - mlp.loss(mlp.forward(p, x)[0], y)) < 1e-15
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    h = 1e-6
    for (name, _), lo, hi in zip(mlp.SHAPES, offs[:-1], offs[1:]):
        for j in rng.choice(np.arange(lo, hi), size=min(6, hi - lo), replace=False):
            e = np.zeros_like(p)
            e[j] = h
            fd = (mlp.loss(mlp.forward(p + e, x)[0], y) - mlp.loss(mlp.forward(p - e, x)[0], y)) / (2 * h)
            assert abs(fd - g[j]) < 1e-8 * max(1.0, abs(g[j])), (name, j, fd, g[j])


def test_bce_and_mse_parts():
    out = np.array([[0.3, 2.0], [-1.0, -3.0]])
    y = np.array([[0.0, 1.0], [1.0, 0.0]])
    mse = (0.3 ** 2 + 2.0 ** 2) / 2
    bce = (math.log1p(math.exp(-2.0)) + math.log1p(math.exp(-3.0))) / 2
    assert abs(mlp.loss(out, y) - (mse + bce)) < 1e-15

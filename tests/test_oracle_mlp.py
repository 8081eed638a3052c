"""Pins of the FP64 MLP oracle: closed-form GELU values and finite differences of the loss."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_forms():
    # GELU(z) = z Phi(z); Phi(1) and Phi(-1) are the standard normal CDF values
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    # derivative: Phi(z) + z phi(z); at 0 it is 1/2
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    z = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_bias_only_network_adds_bias_to_the_skip_features():
    flat = np.zeros(mlp.NPARAM)
    p = mlp.unpack(flat)
    p["b4"] = np.array([1.0, -2.0, 0.5, 3.0])
    x = np.random.default_rng(0).standard_normal((5, 10))
    y, _ = mlp.forward(mlp.pack(p), x)
    assert np.array_equal(y, x[:, 6:10] + p["b4"][None])


def test_layout_size():
    assert mlp.NPARAM == 34948


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    flat = mlp.init(1) * 0.5
    x = rng.standard_normal((7, 10))
    t = rng.standard_normal((7, 4))
    g = mlp.backward(flat, x, t)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    # include every layer and every bias block
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    idx = np.concatenate([idx, offs[:-1], offs[1:] - 1])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (mlp.loss(flat + e, x, t) - mlp.loss(flat - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])

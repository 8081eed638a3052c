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


def _gelu_scalar(z):
    # GELU(z) = z Phi(z), Phi the standard normal CDF: an independent scalar closed form
    return 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))


def test_single_path_network_matches_hand_computation():
    """One non-zero weight per layer, each at a non-symmetric [out][in] position, routes one
    input feature through one unit of every layer; the output is a closed form of that feature.
    A transposed weight matrix (reading [in][out]) or two layers in the wrong order route the
    path through other units, whose activations are GELU(0) = 0, and the output changes."""
    p = mlp.unpack(np.zeros(mlp.NPARAM))
    p["W1"][5, 2] = 2.0        # unit 5 of layer 1 reads input feature 2
    p["b1"][5] = 0.25
    p["W2"][7, 5] = -1.5       # unit 7 of layer 2 reads unit 5 of layer 1
    p["W3"][0, 7] = 3.0        # unit 0 of layer 3 reads unit 7 of layer 2
    p["b3"][0] = -0.5
    p["W4"][3, 0] = 0.75       # output 3 reads unit 0 of layer 3
    p["b4"][1] = -0.125
    flat = mlp.pack(p)
    rng = np.random.default_rng(11)
    x = rng.uniform(-1.5, 1.5, size=(6, 10))
    y, _ = mlp.forward(flat, x)
    for r in range(x.shape[0]):
        a1 = _gelu_scalar(2.0 * x[r, 2] + 0.25)
        a2 = _gelu_scalar(-1.5 * a1)
        a3 = _gelu_scalar(3.0 * a2 - 0.5)
        want = [x[r, 6], x[r, 7] - 0.125, x[r, 8], x[r, 9] + 0.75 * a3]
        # every other unit of layers 1-3 has pre-activation 0 (b = 0) and contributes GELU(0) = 0,
        # except layer-3 units j != 0 with zero weights into the output
        assert np.allclose(y[r], want, rtol=0, atol=1e-14), (r, y[r], want)


def test_forward_matches_torch_fp64_layers_on_a_random_network():
    """The oracle's forward pass against PyTorch's FP64 linear and exact-erf GELU applied to
    the same flat parameters read in the documented [out][in] layout (a library computation
    that shares nothing with the oracle's code)."""
    torch = __import__("pytest").importorskip("torch")
    import torch.nn.functional as F
    rng = np.random.default_rng(5)
    flat = rng.standard_normal(mlp.NPARAM) * 0.3
    x = rng.standard_normal((9, 10))
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    t = {name: torch.tensor(flat[offs[i]:offs[i + 1]].reshape(shp), dtype=torch.float64)
         for i, (name, shp) in enumerate(mlp.SHAPES)}
    xt = torch.tensor(x, dtype=torch.float64)
    h = F.gelu(F.linear(xt, t["W1"], t["b1"]), approximate="none")
    h = F.gelu(F.linear(h, t["W2"], t["b2"]), approximate="none")
    h = F.gelu(F.linear(h, t["W3"], t["b3"]), approximate="none")
    want = (F.linear(h, t["W4"], t["b4"]) + xt[:, 6:10]).numpy()
    y, _ = mlp.forward(flat, x)
    assert np.max(np.abs(y - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))

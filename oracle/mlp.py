"""FP64 numpy reference of the warm-start multilayer perceptron (test infrastructure only).

Network: Linear(10 -> 128) GELU, Linear(128 -> 128) GELU, Linear(128 -> 128) GELU,
Linear(128 -> 4) plus the skip term x[6:10] (previous-interval gains passed through),
GELU(z) = z (1 + erf(z / sqrt 2)) / 2, mean-squared-error loss.
Parameters use the flat layout of the library: W1 [128][10], b1, W2 [128][128], b2,
W3 [128][128], b3, W4 [4][128], b4.  Written directly from the chain rule; pinned by
closed-form GELU values and central finite differences of the loss.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 10, 128, 4
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)), ("b3", (HID,)),
          ("W4", (OUT, HID)), ("b4", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf)


def unpack(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(flat, x):
    p = unpack(flat)
    z1 = x @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = gelu(z3)
    y = a3 @ p["W4"].T + p["b4"] + x[:, 6:10]
    return y, (z1, a1, z2, a2, z3, a3)


def loss(flat, x, t):
    y, _ = forward(flat, x)
    return float(np.mean((y - t) ** 2))


def backward(flat, x, t):
    """Gradient of the mean-squared-error loss with respect to the flat parameters."""
    p = unpack(flat)
    y, (z1, a1, z2, a2, z3, a3) = forward(flat, x)
    n = x.shape[0]
    d4 = 2.0 * (y - t) / (n * OUT)
    g = {"W4": d4.T @ a3, "b4": d4.sum(0)}
    d3 = (d4 @ p["W4"]) * gelu_grad(z3)
    g["W3"], g["b3"] = d3.T @ a2, d3.sum(0)
    d2 = (d3 @ p["W3"]) * gelu_grad(z2)
    g["W2"], g["b2"] = d2.T @ a1, d2.sum(0)
    d1 = (d2 @ p["W2"]) * gelu_grad(z1)
    g["W1"], g["b1"] = d1.T @ x, d1.sum(0)
    return pack(g)


def init(seed: int = 0):
    """He-style initialisation used by the library's trainer (for tests)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * math.sqrt(2.0 / shp[1])
        else:
            p[name] = np.zeros(shp)
    return pack(p)

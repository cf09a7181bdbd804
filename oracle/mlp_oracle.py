"""FP64 CPU reference of the selection controller's network - TEST INFRASTRUCTURE ONLY.

The controller (no counterpart in the paper, which fixes the window count k by hand,
Section 5.2) is a fully connected ReLU network 24 -> 64 -> 64 -> 64 -> 1 trained on the
loss 0.5 * mean((y - target)^2).  Parameters are one flat vector, layer by layer,
weights row-major [out][in] then biases.  This module gives the plain definitions
(forward, loss, hand-derived backward); the tests pin the backward pass to central
finite differences of the loss and compare the GPU kernels against it.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 24
N_HIDDEN = 64
SHAPES = [("W1", (N_HIDDEN, N_FEATURES)), ("b1", (N_HIDDEN,)), ("W2", (N_HIDDEN, N_HIDDEN)), ("b2", (N_HIDDEN,)),
          ("W3", (N_HIDDEN, N_HIDDEN)), ("b3", (N_HIDDEN,)), ("W4", (N_HIDDEN,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation from a seeded splitmix stream (no torch / numpy RNG)."""
    from paper_1305_1293_gb300.meshgen import SplitMix64
    rng = SplitMix64(seed)
    d = {}
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            fan_in = shape[-1] if len(shape) == 2 else N_HIDDEN
            d[name] = rng.normal(n).reshape(shape) * np.sqrt(2.0 / fan_in)
        else:
            d[name] = np.zeros(shape)
    d["W4"] = d["W4"] * 0.1
    return pack(d)


def forward(p, X):
    """Returns y (n,) and the hidden activations (post-ReLU)."""
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ q["W1"].T + q["b1"], 0.0)
    h2 = np.maximum(h1 @ q["W2"].T + q["b2"], 0.0)
    h3 = np.maximum(h2 @ q["W3"].T + q["b3"], 0.0)
    y = h3 @ q["W4"] + q["b4"][0]
    return y, (h1, h2, h3)


def loss(p, X, t):
    y, _ = forward(p, X)
    return 0.5 * float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, X, t):
    """Gradient of loss() by the chain rule, layer by layer."""
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    y, (h1, h2, h3) = forward(p, X)
    dy = (y - np.asarray(t, dtype=np.float64)) / n            # dL/dy
    g = {"W4": h3.T @ dy, "b4": np.array([dy.sum()])}
    d3 = np.outer(dy, q["W4"]) * (h3 > 0)                     # dL/dz3
    g["W3"], g["b3"] = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ q["W3"]) * (h2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ q["W2"]) * (h1 > 0)
    g["W1"], g["b1"] = d1.T @ X, d1.sum(0)
    return pack(g)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v

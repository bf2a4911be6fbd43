"""FP64 reference of the cost-model network -- TEST INFRASTRUCTURE ONLY.

Written from the definition (no code shared with the CUDA library):
    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
    loss = mean over the batch of (y - t)^2,
and its gradient by the chain rule, layer by layer. The flat parameter
layout is W1 (64 x 24, row-major), b1, W2 (64 x 64), b2, w3, b3.
"""

import numpy as np

F, H = 24, 64
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = p[off: off + size].reshape(shape)
        off += size
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, x):
    w = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["w3"] + w["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss(p, x, t):
    y, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(p, x, t):
    """Gradient of the mean squared error with respect to the flat parameters."""
    w = unpack(p)
    y, (x, z1, h1, z2, h2) = forward(p, x)
    b = len(y)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / b          # d loss / d y
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, w["w3"]) * (z2 > 0)                        # through relu
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return pack(g)

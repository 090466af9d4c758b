"""FP64 numpy reference of the warm-start network (features, forward, loss,
backward), written from the definition in include/gp.h.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: it checks the GPU kernels' gradients
and is itself checked against central finite differences.  It shares no code
with the CUDA path.

Parameters are one flat float array in the order W0 (16x64, [in][out]), b0,
W1 (64x64), b1, W2 (64x64), b2, w3 (64), b3.
"""
from __future__ import annotations

import math

import numpy as np

IN, H = 16, 64
SIZES = [("W0", IN * H), ("b0", H), ("W1", H * H), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)]
COUNT = sum(n for _, n in SIZES)


def unpack(theta):
    out, off = {}, 0
    for name, n in SIZES:
        v = np.asarray(theta[off:off + n], dtype=np.float64)
        out[name] = v.reshape(IN, H) if name == "W0" else v.reshape(H, H) if name in ("W1", "W2") else v
        off += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(shape, d, omega, g, sites):
    """Feature rows of the given flat node indices of one condensate."""
    nx, ny, nz = shape
    sites = np.asarray(sites, dtype=np.int64)
    k = sites % nz
    j = (sites // nz) % ny
    i = sites // (nz * ny)
    x = [(idx - 0.5 * (n - 1)) * dd for idx, n, dd in zip((i, j, k), shape, d)]
    w = np.asarray(omega, dtype=np.float64)
    mu_tf = 0.5 * (15.0 * abs(g) * w[0] * w[1] * w[2] / (4.0 * math.pi)) ** 0.4
    r = np.sqrt(2.0 * mu_tf) / w
    f = np.zeros((sites.size, IN))
    su = np.zeros(sites.size)
    sq = np.zeros(sites.size)
    for a in range(3):
        u = x[a] * math.sqrt(w[a])
        f[:, a] = 0.125 * np.minimum(u * u, 16.0) - 1.0
        su += u * u
        sq += (x[a] / r[a]) ** 2
    f[:, 3] = 0.5 * np.minimum(sq, 4.0) - 1.0
    f[:, 4] = 0.125 * np.minimum(su, 16.0) - 1.0
    f[:, 5] = (math.log(max(abs(g), 1e-12)) - 3.1) / 3.1
    for a in range(3):
        f[:, 6 + a] = (w[a] - 1.75) / 1.25
    return f


def softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def forward(theta, x):
    p = unpack(theta)
    h1 = np.tanh(x @ p["W0"] + p["b0"])
    h2 = np.tanh(h1 @ p["W1"] + p["b1"])
    h3 = np.tanh(h2 @ p["W2"] + p["b2"])
    z4 = h3 @ p["w3"] + p["b3"][0]
    return softplus(z4), (x, h1, h2, h3, z4)


def loss_and_grad(theta, x, t):
    """Mean squared error (1/P) sum (y - t)^2 and its gradient."""
    p = unpack(theta)
    y, (x, h1, h2, h3, z4) = forward(theta, x)
    P = x.shape[0]
    r = y - t
    loss = float(np.sum(r * r) / P)
    dz4 = 2.0 / P * r / (1.0 + np.exp(-z4))
    g = {"w3": h3.T @ dz4, "b3": np.array([dz4.sum()])}
    d3 = np.outer(dz4, p["w3"]) * (1.0 - h3 * h3)
    g["W2"], g["b2"] = h2.T @ d3, d3.sum(0)
    d2 = (d3 @ p["W2"].T) * (1.0 - h2 * h2)
    g["W1"], g["b1"] = h1.T @ d2, d2.sum(0)
    d1 = (d2 @ p["W1"].T) * (1.0 - h1 * h1)
    g["W0"], g["b0"] = x.T @ d1, d1.sum(0)
    return loss, pack(g)


def init(seed):
    """Random parameters for tests (not the library's initialisation)."""
    rng = np.random.default_rng(seed)
    parts = {"W0": rng.uniform(-0.5, 0.5, (IN, H)), "b0": rng.uniform(-0.1, 0.1, H),
             "W1": rng.uniform(-0.3, 0.3, (H, H)), "b1": rng.uniform(-0.1, 0.1, H),
             "W2": rng.uniform(-0.3, 0.3, (H, H)), "b2": rng.uniform(-0.1, 0.1, H),
             "w3": rng.uniform(-0.3, 0.3, H), "b3": np.array([0.1])}
    parts["W0"][9:, :] = 0.0
    return pack(parts)

"""FP64 CPU oracle of the learned warm start -- TEST INFRASTRUCTURE ONLY.

Only tests/ may import this module.  The warm start is not in the paper; it
follows the benchmark spec: an MLP over each site's 24 nearest-neighbour
offsets, previous weight, velocity and previous weight change (77 inputs,
padded to 80), three hidden layers of width 128 with ReLU, one output, BF16
weights and activations with FP32 accumulation, trained with Adam on the mean
squared error.

The GPU rounds the weights, the inputs and every hidden activation to BF16
(round to nearest even) and accumulates in FP32; `forward` reproduces those
roundings in FP64 so the two can be compared element by element, and
`backward` gives the exact FP64 gradient of that network (the roundings are
treated as the identity, as in the GPU's backward pass, where the gradients
of the hidden layers are rounded to BF16 too when `bf16_grads` is set).

Pins (tests/test_oracle_mlp.py): finite differences of the loss in every
parameter block on the unrounded FP64 network; Adam against its closed-form
first step; kNN features against a brute-force sort.
"""
from __future__ import annotations

import numpy as np

N_IN, N_FEAT, N_HID, N_KNN = 80, 77, 128, 24


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def param_shapes():
    return [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
            ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("w4", (N_HID,)), ("b4", (1,))]


def unflatten(flat):
    out, k = {}, 0
    for name, shp in param_shapes():
        size = int(np.prod(shp))
        out[name] = np.asarray(flat[k:k + size], np.float64).reshape(shp)
        k += size
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in param_shapes()])


def forward(p, X, rounding=True):
    """out (B,), cache.  Weights W_l: (in, out).  With rounding, the matrix
    weights, inputs and hidden activations are BF16 as on the GPU (biases and
    the head weight w4 stay FP32, the head reads the BF16 h3)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    X = r(X)
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    z1 = X @ W1 + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    z3 = h2 @ W3 + p["b3"]
    h3 = r(np.maximum(z3, 0.0))
    out = h3 @ p["w4"] + p["b4"][0]
    return out, dict(X=X, W1=W1, W2=W2, W3=W3, h1=h1, h2=h2, h3=h3)


def loss(out, y):
    return float(np.mean((np.asarray(out) - np.asarray(y)) ** 2))


def backward(p, cache, out, y, bf16_grads=False):
    """Gradients of mean((out - y)^2) for every parameter block."""
    B = out.shape[0]
    g = bf16 if bf16_grads else (lambda a: a)
    dout = 2.0 * (out - y) / B
    h1, h2, h3, X = cache["h1"], cache["h2"], cache["h3"], cache["X"]
    grads = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}
    dz3 = g(np.outer(dout, p["w4"]) * (h3 > 0))
    grads["W3"] = h2.T @ dz3
    grads["b3"] = dz3.sum(0)
    dz2 = g((dz3 @ cache["W3"].T) * (h2 > 0))
    grads["W2"] = h1.T @ dz2
    grads["b2"] = dz2.sum(0)
    dz1 = g((dz2 @ cache["W2"].T) * (h1 > 0))
    grads["W1"] = X.T @ dz1
    grads["b1"] = dz1.sum(0)
    return grads


def adam(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on flat arrays; step counts from 1."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed=0):
    """He-uniform initialisation (the GPU takes the same flat vector)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes():
        if name.startswith("W") or name == "w4":
            fan_in = shp[0]
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shp)
            if name == "W1":
                p[name][N_FEAT:, :] = 0.0  # padding inputs
            if name == "w4":
                p[name] *= 0.1
        else:
            p[name] = np.zeros(shp)
    return flatten(p)


def knn_features(pos, psi_prev, vel, nu, dt, radius=None, psi_old=None):
    """Features of every site, brute force: offsets to the (up to) 24 nearest
    other sites closer than `radius` (default 2 h_i), by increasing
    distance, over h = nu^(1/3), zero-padded; psi_prev / h^2; vel * dt / h;
    (psi_prev - psi_old) / h^2 (0 when psi_old is None); 3 zeros.
    (n, 80) float64."""
    pos = np.asarray(pos, np.float64)
    n = pos.shape[0]
    h = np.cbrt(np.asarray(nu, np.float64))
    F = np.zeros((n, N_IN))
    for i in range(n):
        rad = 2.0 * h[i] if radius is None else radius
        d = pos - pos[i]
        d2 = np.sum(d * d, 1)
        d2[i] = np.inf
        d2[d2 >= rad * rad] = np.inf
        order = np.argsort(d2, kind="stable")[:N_KNN]
        order = order[np.isfinite(d2[order])]
        off = d[order] / h[i]
        F[i, : 3 * len(order)] = off.ravel()
        F[i, 72] = psi_prev[i] / h[i] ** 2
        F[i, 73:76] = np.asarray(vel[i], np.float64) * dt / h[i]
        if psi_old is not None:
            F[i, 76] = (psi_prev[i] - psi_old[i]) / h[i] ** 2
    return F

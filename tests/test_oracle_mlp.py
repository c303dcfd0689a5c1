"""Pins of the FP64 MLP oracle (learned warm start, not in the paper):
finite differences of the loss in every parameter block, Adam's first step in
closed form, BF16 rounding against torch's conversion, kNN features against
scipy's KD-tree."""
import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

from oracle import mlp_oracle as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-8, 8, 5000), [0.0, -0.0, 1.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


@pytest.mark.parametrize("block", ["W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"])
def test_backward_finite_differences(block):
    rng = np.random.default_rng(1)
    flat = M.init_params(seed=3)
    p = M.unflatten(flat)
    for k in ("b1", "b2", "b3"):  # non-zero biases so every path is exercised
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    X = rng.normal(size=(16, M.N_IN))
    X[:, M.N_FEAT:] = 0.0
    y = rng.normal(size=16)
    out, cache = M.forward(p, X, rounding=False)
    g = M.backward(p, cache, out, y)[block]
    arr = p[block]
    idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]
    for ix in idx:
        if block == "W1" and ix[0] >= M.N_FEAT:
            continue
        old = arr[ix]
        eps = 1e-6
        arr[ix] = old + eps
        lp = M.loss(M.forward(p, X, rounding=False)[0], y)
        arr[ix] = old - eps
        lm = M.loss(M.forward(p, X, rounding=False)[0], y)
        arr[ix] = old
        fd = (lp - lm) / (2 * eps)
        assert fd == pytest.approx(g[ix], rel=1e-5, abs=1e-9)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = M.adam(p0, g, np.zeros(100), np.zeros(100), step=1, lr=1e-3)
    # bias-corrected moments equal g and g^2 on the first step
    np.testing.assert_allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_knn_features_against_kdtree():
    rng = np.random.default_rng(4)
    n = 400
    pos = rng.uniform(0, 0.3, size=(n, 3))
    psi = rng.uniform(0.03, 0.05, size=n) ** 2
    vel = rng.normal(size=(n, 3))
    nu = np.full(n, 2e-5)
    F = M.knn_features(pos, psi, vel, nu, dt=1e-3)
    tree = cKDTree(pos)
    h = np.cbrt(nu)
    radius = 2 * h[0]
    for i in range(0, n, 17):
        d, j = tree.query(pos[i], k=25)
        keep = (j != i) & (d < radius)
        j = j[keep][:24]
        off = (pos[j] - pos[i]) / h[i]
        np.testing.assert_allclose(F[i, : 3 * len(j)], off.ravel(), rtol=1e-12)
        assert np.all(F[i, 3 * len(j):72] == 0)
        assert F[i, 72] == pytest.approx(psi[i] / h[i] ** 2)
        np.testing.assert_allclose(F[i, 73:76], vel[i] * 1e-3 / h[i])
        assert np.all(F[i, 76:] == 0)
    # history: an unchanged weight gives the no-history features; a change of
    # c h^2 per site gives c in input 76 and nothing else moves
    np.testing.assert_array_equal(M.knn_features(pos, psi, vel, nu, dt=1e-3, psi_old=psi), F)
    c = rng.uniform(-0.3, 0.3, size=n)
    G = M.knn_features(pos, psi, vel, nu, dt=1e-3, psi_old=psi - c * h ** 2)
    np.testing.assert_allclose(G[:, 76], c, rtol=1e-9, atol=1e-12)
    G[:, 76] = 0.0
    np.testing.assert_array_equal(G, F)

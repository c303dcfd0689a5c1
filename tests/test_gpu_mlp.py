"""GPU kernels of the learned warm start against the FP64 oracle:
tcgen05 forward (BF16 operands, FP32 accumulation) and back-propagation,
Adam, and the kNN features."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M
from paper_2601_05765_b300 import pot, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlp():
    m = pot.Mlp(200000, 0)
    yield m
    m.close()


def rand_params(seed):
    rng = np.random.default_rng(seed)
    flat = M.init_params(seed)
    p = M.unflatten(flat)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    p["b4"] = np.array([0.05])
    return M.flatten(p)


def rand_x(rows, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(rows, M.N_IN))
    x[:, M.N_FEAT:] = 0.0
    return M.bf16(x)


def to_dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


@pytest.mark.parametrize("rows", [1000, 12345])
def test_forward_matches_oracle(mlp, rows):
    flat = rand_params(1)
    mlp.set_params(to_dev(flat, torch.float32))
    x = rand_x(rows, 2)
    out = mlp.forward(to_dev(x, torch.bfloat16)).cpu().numpy().astype(np.float64)
    # the oracle sees the FP32-rounded parameters the GPU holds
    p = M.unflatten(flat.astype(np.float32).astype(np.float64))
    ref, _ = M.forward(p, x, rounding=True)
    scale = np.sqrt(np.mean(ref ** 2))
    err = np.abs(out - ref)
    # BF16 rounding of the hidden layers may tie-break differently after a
    # different FP32 summation order: a few entries per row differ by one ulp
    assert np.percentile(err, 99) <= 1e-2 * scale
    assert err.max() <= 5e-2 * scale
    assert np.corrcoef(out, ref)[0, 1] > 0.9999


def test_gradients_match_oracle(mlp):
    flat = rand_params(3)
    mlp.set_params(to_dev(flat, torch.float32))
    n_all, batch = 5000, 2048
    x = rand_x(n_all, 4)
    y = np.random.default_rng(5).normal(size=n_all)
    idx = np.random.default_rng(6).choice(n_all, size=batch, replace=False).astype(np.int32)
    g, loss = mlp.gradients(to_dev(x, torch.bfloat16), to_dev(y, torch.float32), to_dev(idx, torch.int32))
    g = g.cpu().numpy().astype(np.float64)
    p = M.unflatten(flat.astype(np.float32).astype(np.float64))
    out, cache = M.forward(p, x[idx], rounding=True)
    yb = y[idx].astype(np.float32).astype(np.float64)
    ref = M.flatten(M.backward(p, cache, out, yb, bf16_grads=True))
    assert float(loss.item()) == pytest.approx(M.loss(out, yb), rel=1e-3)
    gd, rd = M.unflatten(g), M.unflatten(ref)
    for name, _ in M.param_shapes():
        a, b = gd[name].ravel(), rd[name].ravel()
        if name == "W1":
            a, b = gd[name][: M.N_FEAT].ravel(), rd[name][: M.N_FEAT].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300)
        assert cos > 0.999 and rel < 3e-2, (name, cos, rel)


def test_adam_step(mlp):
    flat = rand_params(7)
    mlp.set_params(to_dev(flat, torch.float32))
    n_all, batch = 4096, 1024
    x = to_dev(rand_x(n_all, 8), torch.bfloat16)
    y = to_dev(np.random.default_rng(9).normal(size=n_all), torch.float32)
    idx = to_dev(np.arange(batch, dtype=np.int32), torch.int32)
    g, _ = mlp.gradients(x, y, idx)
    loss = torch.empty(1, dtype=torch.float32, device="cuda:0")
    mlp.train_step(x, y, idx, lr=1e-3, loss=loss)
    got = mlp.get_params().cpu().numpy().astype(np.float64)
    p0 = flat.astype(np.float32).astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    exp, _, _ = M.adam(p0, gg, np.zeros_like(p0), np.zeros_like(p0), step=1, lr=1e-3)
    np.testing.assert_allclose(got, exp, rtol=0, atol=2e-6)
    mlp.check()


@pytest.mark.parametrize("history", [False, True])
def test_features_match_oracle(mlp, history):
    sc = scenes.jittered_block(n_side=10, seed=0)
    n = sc.n
    rng = np.random.default_rng(10)
    vel = (rng.normal(size=(n, 3)) * 0.2).astype(np.float32)
    h2 = np.cbrt(sc.nu) ** 2
    old = (sc.psi - rng.uniform(-0.2, 0.2, size=n) * h2).astype(np.float32) if history else None
    ctx = pot.Context(n, 64, 0, fp64=False)
    prm = pot.default_params(dt=1e-3)
    feat = pot.pot_mlp_features(ctx, mlp, to_dev(sc.pos, torch.float32), to_dev(vel, torch.float32),
                                to_dev(sc.psi, torch.float32), to_dev(sc.nu, torch.float64), params=prm,
                                psi_old=to_dev(old, torch.float32) if history else None)
    got = feat.float().cpu().numpy().astype(np.float64)
    x1 = np.clip(sc.pos.astype(np.float32) + np.float32(1e-3) * vel, 1e-6, 1 - 1e-6).astype(np.float64)
    ref = M.bf16(M.knn_features(x1, sc.psi.astype(np.float64), vel.astype(np.float64), sc.nu, 1e-3,
                                psi_old=old.astype(np.float64) if history else None))
    diff = np.abs(got - ref)
    # one BF16 ulp of the offsets (values ~1) or of the scaled psi
    assert np.mean(diff <= 1e-2 * np.abs(ref) + 1e-6) > 0.999
    # the weight change: an FP32 difference, then one BF16 rounding
    np.testing.assert_allclose(got[:, 76], ref[:, 76], rtol=1e-2, atol=1e-5)
    assert np.all(got[:, 77:] == 0)
    ctx.close()

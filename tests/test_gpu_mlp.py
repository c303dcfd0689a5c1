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
    print("realistic forward: err / scale p50 %.2e p99 %.2e max %.2e" % tuple(
        np.percentile(err, [50, 99, 100]) / scale))
    # BF16 rounding of the hidden layers may tie-break differently after a
    # different FP32 summation order (the exact-arithmetic test below pins
    # the kernels bit-exactly): a few entries per row differ by one ulp
    assert np.percentile(err, 99) <= 1e-2 * scale
    assert err.max() <= 5e-2 * scale
    assert np.corrcoef(out, ref)[0, 1] > 0.9999


def exact_network(seed):
    """A network whose every hidden pre-activation is exact in FP32 for the
    inputs of exact_x: inputs in {0, +-1/2, +-1}, W1 entries in {0, +-1/8},
    biases on the grid of their layer, W2 and W3 entries in {0, +-1/32}.  Then
    z1 is a multiple of 1/16 below 2^8/16 (so relu(z1) is already BF16), and
    z2, z3 are multiples of 2^-9 and 2^-14 far inside FP32's 24 bits: the
    GPU's FP32 accumulation, in whatever order, gives the exact sums, and the
    BF16 roundings of the hidden layers are the oracle's."""
    rng = np.random.default_rng(seed)
    p = M.unflatten(np.zeros(sum(int(np.prod(shp)) for _, shp in M.param_shapes())))
    p["W1"] = rng.integers(-1, 2, size=(M.N_IN, M.N_HID)) / 8.0
    p["W1"][M.N_FEAT:] = 0.0
    p["b1"] = rng.integers(-16, 17, size=M.N_HID) / 16.0
    p["W2"] = rng.integers(-1, 2, size=(M.N_HID, M.N_HID)) / 32.0
    p["b2"] = rng.integers(-512, 513, size=M.N_HID) / 512.0
    p["W3"] = rng.integers(-1, 2, size=(M.N_HID, M.N_HID)) / 32.0
    p["b3"] = rng.integers(-2 ** 14, 2 ** 14 + 1, size=M.N_HID) / 2.0 ** 14
    p["w4"] = rng.integers(-4, 5, size=M.N_HID) / 16.0
    p["b4"] = np.array([0.25])
    return M.flatten(p)


def exact_x(rows, seed):
    x = np.random.default_rng(seed).integers(-2, 3, size=(rows, M.N_IN)) / 2.0
    x[:, M.N_FEAT:] = 0.0
    return x


def test_forward_exact_arithmetic(mlp):
    """Bit-level check of the tensor-core forward (layouts, bias, ReLU, BF16
    packing between layers, head): on exact_network every hidden activation
    is determined, so the output may differ from the oracle's only by the
    FP32 rounding of the head's sum, bounded by K u sum |h3 w4| + u |out|."""
    flat = exact_network(11)
    p = M.unflatten(flat)
    x = exact_x(5000, 12)
    ref, cache = M.forward(p, x, rounding=True)
    # the construction: each layer's FP32 sums, in two different orders,
    # equal the FP64 ones
    for h, W, b in ((x, p["W1"], p["b1"]), (cache["h1"], p["W2"], p["b2"]),
                    (cache["h2"], p["W3"], p["b3"])):
        z64 = h @ W + b
        for order in (slice(None), slice(None, None, -1)):
            z32 = h[:, order].astype(np.float32) @ W[order].astype(np.float32) + b.astype(np.float32)
            assert np.array_equal(z32.astype(np.float64), z64)
    assert np.array_equal(cache["h1"], np.maximum(x @ p["W1"] + p["b1"], 0.0))  # no rounding in layer 1
    mlp.set_params(to_dev(flat, torch.float32))
    out = mlp.forward(to_dev(x, torch.bfloat16)).cpu().numpy().astype(np.float64)
    u = 2.0 ** -24
    bound = M.N_HID * u * (np.abs(cache["h3"]) @ np.abs(p["w4"]) + abs(p["b4"][0])) + u * np.abs(ref)
    err = np.abs(out - ref)
    print("exact-arithmetic forward: max err", err.max(), "max bound", bound.max(),
          "rows with nonzero err", int(np.sum(err > 0)), "of", len(err))
    assert np.all(err <= bound)


def test_gradients_exact_arithmetic(mlp):
    """Bit-level check of back-propagation, the split-K weight gradients and
    the bias sums: on exact_network with targets y = out - delta (delta a
    small multiple of 2^-10, so dL/dout = 2 delta / B is exact), every FP32
    sum of the backward pass is exact in any order (checked on the CPU in
    two orders), and the BF16 roundings of the hidden deltas see the same
    values, so the GPU's gradients must equal the oracle's."""
    flat = exact_network(13)
    p = M.unflatten(flat)
    n_all, batch = 4096, 2048
    x = exact_x(n_all, 14)
    idx = np.random.default_rng(15).choice(n_all, size=batch, replace=False).astype(np.int32)
    out_all, _ = M.forward(p, x, rounding=True)
    delta = np.random.default_rng(16).integers(-8, 9, size=n_all) / 1024.0
    y = out_all - delta
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)
    out, cache = M.forward(p, x[idx], rounding=True)
    ref = M.backward(p, cache, out, y[idx], bf16_grads=True)
    # the construction: the backward's sums in FP32, in two orders, equal FP64
    for order in (slice(None), slice(None, None, -1)):
        c32 = {k: v[order].astype(np.float32) for k, v in cache.items() if k in ("X", "h1", "h2", "h3")}
        d = (2.0 * (out[order] - y[idx][order]) / batch).astype(np.float32)
        dz3 = M.bf16(np.outer(d, p["w4"]) * (c32["h3"] > 0)).astype(np.float32)
        dz2 = M.bf16((dz3 @ p["W3"].T.astype(np.float32)) * (c32["h2"] > 0)).astype(np.float32)
        dz1 = M.bf16((dz2 @ p["W2"].T.astype(np.float32)) * (c32["h1"] > 0)).astype(np.float32)
        for name, a in (("W3", c32["h2"].T @ dz3), ("W2", c32["h1"].T @ dz2), ("W1", c32["X"].T @ dz1),
                        ("b3", dz3.sum(0)), ("b2", dz2.sum(0)), ("b1", dz1.sum(0)),
                        ("w4", c32["h3"].T @ d), ("b4", np.array([d.sum()]))):
            assert np.array_equal(a.astype(np.float64), ref[name]), name
    mlp.set_params(to_dev(flat, torch.float32))
    g, loss = mlp.gradients(to_dev(x, torch.bfloat16), to_dev(y, torch.float32), to_dev(idx, torch.int32))
    gd = M.unflatten(g.cpu().numpy().astype(np.float64))
    assert float(loss.item()) == pytest.approx(M.loss(out, y[idx]), rel=1e-6)
    for name, _ in M.param_shapes():
        a, b = gd[name], ref[name]
        if name == "W1":
            a, b = a[: M.N_FEAT], b[: M.N_FEAT]
        print(name, "max |diff|", float(np.max(np.abs(a - b))), "max |ref|", float(np.max(np.abs(b))))
        assert np.array_equal(a, b), name


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


def bf16_ulp(v):
    """Spacing of the BF16 numbers at |v| (8 significant bits)."""
    v = np.abs(np.asarray(v, np.float64))
    e = np.floor(np.log2(np.where(v > 0, v, 1.0)))
    return np.where(v > 0, 2.0 ** (e - 7), 2.0 ** -133)


@pytest.mark.parametrize("history", [False, True])
def test_features_match_oracle(mlp, history):
    """kNN features entry by entry.  The GPU computes each value in FP32 and
    rounds it to BF16, the oracle in FP64 and rounds it to BF16, so every
    entry may differ by one BF16 ulp (the weight change, an FP32 difference
    of two weights, also by the FP32 rounding of those weights).  Where two
    neighbours' distances agree within FP32 rounding (relative 2^-18: the
    positions x + dt v themselves may round differently, by a fused
    multiply-add) their order is not determined: a slot may hold either
    one's offsets; a neighbour at the search radius within the same rounding
    may be in or out.  Every other entry must agree."""
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
    ctx.close()
    x1 = np.clip(sc.pos.astype(np.float32) + np.float32(1e-3) * vel, 1e-6, 1 - 1e-6).astype(np.float64)
    psi64 = sc.psi.astype(np.float64)
    ref = M.bf16(M.knn_features(x1, psi64, vel.astype(np.float64), sc.nu, 1e-3,
                                psi_old=old.astype(np.float64) if history else None))
    # scalar inputs: within one ulp (the weight change also within the FP32
    # rounding of the two weights it subtracts)
    for col in range(72, 76):
        assert np.all(np.abs(got[:, col] - ref[:, col]) <= bf16_ulp(ref[:, col])), col
    slack = 2.0 ** -23 * (np.abs(psi64) + (np.abs(old.astype(np.float64)) if history else 0.0)) / h2
    assert np.all(np.abs(got[:, 76] - ref[:, 76]) <= bf16_ulp(ref[:, 76]) + slack)
    assert np.all(got[:, 77:] == 0)
    # offsets: slot by slot, with the ties above
    h = np.cbrt(sc.nu)
    tie = 2.0 ** -18
    ties = 0
    for i in range(n):
        d = x1 - x1[i]
        dist = np.sqrt(np.sum(d * d, 1))
        dist[i] = np.inf
        order = np.argsort(dist, kind="stable")
        near = order[dist[order] < 2.0 * h[i] * (1.0 + tie)]
        offs = M.bf16(d[near] / h[i])
        g = got[i, :72].reshape(24, 3)
        used = np.zeros(len(near), bool)
        for k in range(24):
            if not np.any(g[k] != 0.0):
                # padding: no neighbour left, or only ones on the radius
                assert k >= len(near) or np.all(dist[near[k:]] >= 2.0 * h[i] * (1.0 - tie)), (i, k)
                continue
            # neighbours whose distance ties with the k-th one
            dk = dist[near[min(k, len(near) - 1)]]
            cand = [m for m in range(len(near)) if not used[m] and abs(dist[near[m]] - dk) <= tie * dk]
            hit = [m for m in cand if np.all(np.abs(g[k] - offs[m]) <= bf16_ulp(offs[m]))]
            assert hit, (i, k, g[k], offs[min(k, len(near) - 1)])
            used[hit[0]] = True
            ties += int(hit[0] != k)
    print("features: slots taken by a tied neighbour", ties)

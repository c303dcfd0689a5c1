"""Training and evaluation of the learned warm start.

Data: plain-Newton fluid steps on dam-break columns (seeded); every `every`
steps, the features at the state the step solves at (positions advanced by
dt v and clamped, previous weights psi^k, velocities, the change
psi^k - psi^{k-1}) and the converged weights psi^{k+1} of `per_sample` random
sites give samples (x, y = (psi^{k+1} - psi^k - (psi^k - psi^{k-1})) / h^2,
the departure from the linear extrapolation; without psi^{k-1}, and for the
76-input model, the plain change), h = nu^(1/3).

Training: Adam on the mean squared error, shuffled batches, all kernels in
libpot.so (tensor-core forward and back-propagation).  Evaluation: the same
fluid steps started from the MLP prediction and from the previous weights.

Dataset assembly (row sampling, the target difference) uses torch indexing as
plumbing; features, training and solves run in the library.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import pot, scenes


# parameter layout of the model (pot.h: W1 80x128 (row = input), b1, W2
# 128x128, b2, W3 128x128, b3, w4 128, b4 1); inputs 77..79 are padding
_SHAPES = ((80, 128), (128,), (128, 128), (128,), (128, 128), (128,), (128,), (1,))
_N_FEAT = 77


def init_params(seed: int = 0, device="cuda", n_inputs: int = _N_FEAT) -> torch.Tensor:
    """Fresh parameters: He-uniform weights (limit sqrt(6 / fan_in)), zero
    biases, the head scaled by 0.1 so that the first predictions are small,
    zero weights for the padding inputs (from n_inputs on).  FP32 vector on
    `device`."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for k, shp in enumerate(_SHAPES):
        if len(shp) == 2 or k == 6:
            lim = math.sqrt(6.0 / shp[0])
            w = (torch.rand(shp, generator=gen, dtype=torch.float64) * 2.0 - 1.0) * lim
            if k == 0:
                w[n_inputs:, :] = 0.0
            if k == 6:
                w *= 0.1
        else:
            w = torch.zeros(shp, dtype=torch.float64)
        parts.append(w.reshape(-1))
    flat = torch.cat(parts).to(torch.float32)
    assert flat.numel() == pot.Mlp.num_params()
    return flat.to(device)


def _state(sc, dev):
    return (torch.from_numpy(sc.pos).to(dev), torch.from_numpy(sc.vel).to(dev),
            torch.from_numpy(sc.psi).to(dev), torch.from_numpy(sc.nu).to(dev))


def settle(ctx, pos, vel, psi, nu, prm, relax=0):
    """Start state (not a sample): the initial weights converged in place,
    then `relax` rounds of sites moved to their cell centroids."""
    if relax > 0:
        return pot.relax_to_centroids(ctx, pos, psi, nu, relax, params=prm)["solves"][-1]
    return pot.pot_newton_solve(ctx, pos, nu, psi, params=prm, check=False)


def collect(ctx, mlp, scene, steps, every, per_sample, seed, dt, tol=1e-4, eps=0.01, relax=0,
            history=True):
    """Samples from `steps` plain-Newton fluid steps of `scene`; without
    `history` (the 76-input model) no weight change enters the features or
    the target."""
    dev = ctx.device
    pos, vel, psi, nu = _state(scene, dev)
    prm = pot.default_params(dt=dt, tol=tol, eps=eps)
    settle(ctx, pos, vel, psi, nu, prm, relax)
    h2 = torch.pow(nu, 2.0 / 3.0).float()
    gen = torch.Generator(device="cpu").manual_seed(seed)
    xs, ys = [], []
    psi_old = None
    for k in range(steps):
        take = k % every == 0
        psi_prev = psi.clone()
        hist = psi_old if history else None
        if take:
            feat = pot.pot_mlp_features(ctx, mlp, pos, vel, psi, nu, params=prm, psi_old=hist)
        psi_old = psi_prev
        st = pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm, check=False)
        if st["status"] != 0:
            raise RuntimeError(f"fluid step {k} failed: {st}")
        if take:
            idx = torch.randperm(scene.n, generator=gen)[:per_sample].to(dev)
            xs.append(feat[idx])
            # the target: the new weight's departure from the linear
            # extrapolation psi^k + (psi^k - psi^{k-1}) (plain change without
            # history), as the fluid step applies it
            lin = psi_prev if hist is None else 2.0 * psi_prev - hist
            ys.append(((psi - lin) / h2)[idx])
    return torch.cat(xs), torch.cat(ys)


def train(mlp, x, y, epochs, batch=8192, lr=1e-3, seed=0):
    """Adam epochs over (x, y); returns the mean loss of each epoch."""
    n = int(x.shape[0])
    batch = min(batch, (n // 8) * 8)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to(torch.int32).to(x.device)
        acc, nb = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            mlp.train_step(x, y, perm[b0:b0 + batch], lr=lr, loss=loss)
            acc += float(loss.item()) if nb % 64 == 0 else 0.0
            nb += 1
        mlp.check()
        hist.append(acc / max(1, (nb + 63) // 64))
    return hist


def compare(ctx, mlp, scene, steps, dt, warm_steps=0, tol=1e-4, eps=0.01, relax=0,
            modes=((0, "plain"), (2, "extrapolated"), (1, "mlp"))):
    """Run the same fluid steps from the same state with the plain start
    (previous weights), the extrapolated start (warm_start 2) and the MLP
    start; returns per-step stats of each.  The warm-up steps run with the
    extrapolated start, which leaves the weight history of the last one in
    the context (their converged weights are those of the plain start, to
    the tolerance)."""
    dev = ctx.device
    pos, vel, psi, nu = _state(scene, dev)
    prm = pot.default_params(dt=dt, tol=tol, eps=eps, warm_start=2)
    settle(ctx, pos, vel, psi, nu, prm, relax)
    pot.clear_history(ctx)
    psi_old = None
    for _ in range(warm_steps):
        psi_old = psi.clone()
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    state = (pos.clone(), vel.clone(), psi.clone())
    out = {}
    for mode, name in modes:
        pos, vel, psi = (t.clone() for t in state)
        p = pot.default_params(dt=dt, tol=tol, eps=eps, warm_start=mode)
        pot.set_warm_start(ctx, mlp if mode == 1 else None)
        if mode == 1:
            mlp.set_history(psi_old)
        stats = []
        for _ in range(steps):
            stats.append(pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=p, check=False))
        out[name] = stats
    pot.set_warm_start(ctx, None)
    return out


def summarize(stats):
    keys = ("err_start", "newton_iters", "pcg_iters", "halvings", "cell_evals", "ms_total")
    s = {k: float(np.mean([st[k] for st in stats])) for k in keys}
    s["fallback_rate"] = float(np.mean([st["mlp_fallback"] for st in stats]))
    s["used_rate"] = float(np.mean([st["mlp_used"] for st in stats]))
    s["all_converged"] = all(st["status"] == 0 for st in stats)
    s["max_err"] = float(max(st["err_max"] for st in stats))
    return s

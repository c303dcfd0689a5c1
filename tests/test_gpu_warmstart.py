"""Learned warm start end to end on the GPU: features, training and the
MLP-started fluid step against the plain start (previous weights).

The warm start only changes where Newton starts, so correctness is the
converged result (checked in test_gpu_newton.py); what is checked here is
that (a) a model whose output is 0 reproduces the extrapolated start
(psi + (psi - psi_prev)) exactly, and
(b) a model trained on a few dam-break steps needs fewer Newton and PCG
iterations than the start from the previous weights on unseen steps of
another seed, with no fallback and every step converged, and is not worse
than the linear extrapolation it corrects.  (The worst-cell
start error is not the measure: the prediction moves most cells much closer
and a few outliers further.)"""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M
from paper_2601_05765_b300 import pot, scenes
from paper_2601_05765_b300 import warmstart as W

pytestmark = pytest.mark.gpu

DT = 2e-3


def column(seed, nx=12):
    return scenes.dam_break(nx=nx, ny=nx, nz=2 * nx, width=0.15, seed=seed)


@pytest.fixture(scope="module")
def setup():
    sc = column(19)
    ctx = pot.Context(sc.n, 128, 0, fp64=False)
    mlp = pot.Mlp(65536, 0)
    yield ctx, mlp
    pot.set_warm_start(ctx, None)
    mlp.close()
    ctx.close()


def test_zero_model_is_the_extrapolated_start(setup):
    """The network corrects the linear extrapolation: with its output 0 the
    learned start is the extrapolated start (warm_start 2) exactly."""
    ctx, mlp = setup
    mlp.set_params(torch.zeros(pot.Mlp.num_params(), dtype=torch.float32, device=ctx.device))
    res = W.compare(ctx, mlp, column(19), steps=3, dt=DT, warm_steps=2)
    for a, b in zip(res["extrapolated"], res["mlp"]):
        assert a["status"] == 0 and b["status"] == 0
        assert a["mlp_used"] == 1 and b["mlp_used"] == 1 and b["mlp_fallback"] == 0
        assert b["err_start"] == a["err_start"]
        assert b["newton_iters"] == a["newton_iters"]


def test_trained_model_starts_closer(setup):
    ctx, mlp = setup
    dev = ctx.device
    mlp.set_params(torch.as_tensor(M.init_params(0), dtype=torch.float32, device=dev))
    xs, ys = [], []
    for seed in (10, 11, 12):
        x, y = W.collect(ctx, mlp, column(seed), steps=30, every=2, per_sample=2048, seed=seed, dt=DT)
        xs.append(x)
        ys.append(y)
    x, y = torch.cat(xs), torch.cat(ys)
    hist = W.train(mlp, x, y, epochs=120, batch=4096, lr=1e-3)
    assert hist[-1] < 0.1 * hist[0]
    res = W.compare(ctx, mlp, column(19), steps=8, dt=DT, warm_steps=12)
    plain, learned = W.summarize(res["plain"]), W.summarize(res["mlp"])
    extrap = W.summarize(res["extrapolated"])
    print("Newton / PCG iterations per step: plain", plain["newton_iters"], plain["pcg_iters"],
          "extrapolated", extrap["newton_iters"], extrap["pcg_iters"],
          "learned", learned["newton_iters"], learned["pcg_iters"])
    assert plain["all_converged"] and learned["all_converged"] and extrap["all_converged"]
    assert learned["fallback_rate"] == 0.0 and learned["used_rate"] == 1.0
    # the gain over the method without the network (plain Newton from the
    # previous weights) ...
    assert learned["newton_iters"] <= plain["newton_iters"] - 0.5, (learned, plain)
    assert learned["pcg_iters"] < plain["pcg_iters"], (learned, plain)
    # ... and against the free linear extrapolation of the weights, which the
    # network corrects: not worse by more than a quarter of a Newton
    # iteration per step (on these columns the two are close; the splash
    # comparison is in bench.py --mode warmstart)
    assert learned["newton_iters"] <= extrap["newton_iters"] + 0.25, (learned, extrap)


def test_extrapolated_start(setup):
    """warm_start 2: the first step after clear_history starts from the
    previous weights, later ones from psi + (psi - psi_prev); every step
    converges to the tolerance, and in FP64 far below it the weights equal
    the plain start's (the solution does not depend on the start)."""
    ctx, _ = setup
    sc = column(19)
    dev = ctx.device
    res = {}
    for ws in (0, 2):
        ctx64 = pot.Context(sc.n, 128, 0, fp32=False, fp64=True)
        pos, vel, psi, nu = (torch.as_tensor(a, dtype=torch.float64, device=dev)
                             for a in (sc.pos, sc.vel, sc.psi, sc.nu))
        prm = pot.default_params(dt=DT, tol=1e-10, warm_start=ws)
        pot.pot_newton_solve(ctx64, pos, nu, psi, params=prm)
        pot.clear_history(ctx64)
        stats = [pot.pot_fluid_step(ctx64, pos, vel, psi, nu, params=prm) for _ in range(6)]
        assert all(s["status"] == 0 and s["err_max"] <= 1e-10 for s in stats)
        res[ws] = (psi.cpu().numpy(), stats)
        ctx64.close()
    used = [s["mlp_used"] for s in res[2][1]]
    assert used[0] == 0 and all(u == 1 for u in used[1:]), used
    assert sum(s["newton_iters"] for s in res[2][1]) <= sum(s["newton_iters"] for s in res[0][1])
    np.testing.assert_allclose(res[2][0], res[0][0], rtol=0, atol=1e-8 * float(np.max(res[0][0])))


def test_76_input_model(setup):
    """The configuration's 76-input model (no weight-change input; the
    prediction corrects the previous weights): its features leave input 77
    at 0 whatever the history, a zero model is the plain start exactly, and
    a model trained on a few dam-break steps starts no worse than the plain
    start on unseen steps of another seed, every step converged."""
    ctx, _ = setup
    dev = ctx.device
    mlp76 = pot.Mlp(65536, 0)
    try:
        mlp76.set_inputs(76)
        with pytest.raises(pot.PotError):
            mlp76.set_inputs(75)
        sc = column(19)
        pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
        prm = pot.default_params(dt=DT)
        W.settle(ctx, pos, vel, psi, nu, prm)
        old = psi * 0.9  # a history that would give a nonzero change feature
        f76 = pot.pot_mlp_features(ctx, mlp76, pos, vel, psi, nu, params=prm, psi_old=old)
        assert bool(torch.all(f76[:, 76] == 0))
        mlp77 = pot.Mlp(65536, 0)
        f77 = pot.pot_mlp_features(ctx, mlp77, pos, vel, psi, nu, params=prm, psi_old=old)
        mlp77.close()
        assert bool(torch.any(f77[:, 76] != 0))
        assert torch.equal(f76[:, :76], f77[:, :76])
        # zero model: the plain start
        mlp76.set_params(torch.zeros(pot.Mlp.num_params(), dtype=torch.float32, device=dev))
        res = W.compare(ctx, mlp76, column(19), steps=3, dt=DT, warm_steps=2,
                        modes=((0, "plain"), (1, "mlp")))
        for a, b in zip(res["plain"], res["mlp"]):
            assert a["status"] == 0 and b["status"] == 0 and b["mlp_used"] == 1
            assert b["err_start"] == a["err_start"] and b["newton_iters"] == a["newton_iters"]
        # trained
        mlp76.set_params(W.init_params(0, device=dev, n_inputs=76))
        xs, ys = [], []
        for seed in (10, 11, 12):
            x, y = W.collect(ctx, mlp76, column(seed), steps=30, every=2, per_sample=2048,
                             seed=seed, dt=DT, history=False)
            assert bool(torch.all(x[:, 76] == 0))
            xs.append(x)
            ys.append(y)
        hist = W.train(mlp76, torch.cat(xs), torch.cat(ys), epochs=120, batch=4096, lr=1e-3)
        assert hist[-1] < 0.1 * hist[0]
        res = W.compare(ctx, mlp76, column(19), steps=8, dt=DT, warm_steps=12,
                        modes=((0, "plain"), (1, "mlp")))
        plain, learned = W.summarize(res["plain"]), W.summarize(res["mlp"])
        print("76 inputs, Newton / PCG iterations per step: plain", plain["newton_iters"],
              plain["pcg_iters"], "learned", learned["newton_iters"], learned["pcg_iters"])
        assert learned["all_converged"] and learned["fallback_rate"] == 0.0
        assert learned["newton_iters"] <= plain["newton_iters"], (learned, plain)
    finally:
        pot.set_warm_start(ctx, None)
        mlp76.close()

"""The 2M-site two-ball splash (the benchmark's workload) run for its 100
fluid steps, with every quantity checked against the FP64 oracle on a
100k-cell subset (seed 1003): at the start state (sites at their cell
centroids), after step 50 and after step 99 (the balls pressed together
since step ~10), in the launch configuration bench.py times.  The oracle
computes the sampled cells one by one from the same float32 inputs; the GPU
computes all 2M."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import pot, scenes

from _cmp import compare_cells, to_np

pytestmark = pytest.mark.gpu

TOL32 = dict(tol_v=1e-5, tol_h=1e-4, tol_c=1e-4)


def check_subset(ctx, pos, psi, nu, q):
    out = pot.lgc_compute_cells(ctx, pos, psi, nu)
    p32, s32 = to_np(pos), to_np(psi)
    ref = O.cells(p32.astype(np.float64), s32.astype(np.float64), query=q)
    assert np.all(ref["status"] == 0)
    rep = compare_cells(out, ref, s32, to_np(nu), **TOL32)
    # the GPU's converged weights, measured by the oracle: the tolerance
    # plus the FP32 geometry error
    nu_q = to_np(nu)[q]
    rep["oracle_vol_err"] = float(np.max(np.abs(ref["vol"] - nu_q) / nu_q))
    assert rep["oracle_vol_err"] <= 1e-4, rep
    return rep


def test_splash_2m_100_steps_subset_per_quantity():
    sc = scenes.splash()
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    vel = torch.from_numpy(sc.vel).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    q = scenes.random_subset(n, 100000, 1003)
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    relax = pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    assert all(st["status"] == 0 for st in relax["solves"])
    # the moves shrink: the start is near the spring's rest state
    assert relax["moved_max"][-1] < 0.5 * relax["moved_max"][0]
    reports = {0: check_subset(ctx, pos, psi, nu, q)}
    x0 = to_np(pos)[:, 0].copy()
    for k in range(1, 101):
        st = pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
        assert st["status"] == 0 and st["err_max"] <= 1e-4, (k, st)
        if k in (50, 99):
            reports[k] = check_subset(ctx, pos, psi, nu, q)
    for k, rep in reports.items():
        print(f"step {k}:", rep)
    # the balls met: the left ball (+3 m/s at the start, which it keeps in
    # free flight) has passed momentum to the right one (2.80 m/s measured)
    vx = to_np(vel)[:, 0]
    left = x0 < 0.5
    print("mean x-velocity of the left ball after 100 steps:", float(vx[left].mean()))
    assert vx[left].mean() < 2.9
    ctx.close()

"""The 500,094-site dam break (the dam-break recipe: dt 2e-3 per step in 5
substeps, spring s/8, start state at the cells' centroids) in the bench's
launch configuration, every quantity against the FP64 oracle on 20k sampled
cells (seed 1004): at the start state and after 40 steps (the column
collapsing, the front running along the floor).  Every substep must converge
to the tolerance."""
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
    nu_q = to_np(nu)[q]
    rep["oracle_vol_err"] = float(np.max(np.abs(ref["vol"] - nu_q) / nu_q))
    assert rep["oracle_vol_err"] <= 1e-4, rep
    return rep


def test_dam_break_500k_subset_per_quantity():
    sc = scenes.dam_break()
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 1024, 0, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    vel = torch.from_numpy(sc.vel).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    q = scenes.random_subset(n, 20000, 1004)
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"], substeps=sc.extra["substeps"])
    relax = pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    assert all(st["status"] == 0 for st in relax["solves"])
    reports = {0: check_subset(ctx, pos, psi, nu, q)}
    z0 = float(to_np(pos)[:, 2].mean())
    for k in range(1, 41):
        st = pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
        assert st["status"] == 0 and st["err_max"] <= 1e-4 and st["grid_builds"] == 5, (k, st)
    reports[40] = check_subset(ctx, pos, psi, nu, q)
    for k, rep in reports.items():
        print(f"step {k}:", rep)
    # the column has collapsed: its centre of mass went down, its front out
    x = to_np(pos)
    print("centre-of-mass height", z0, "->", float(x[:, 2].mean()), "front", float(np.percentile(x[:, 0], 99.9)))
    assert x[:, 2].mean() < z0 - 0.002
    assert np.percentile(x[:, 0], 99.9) > 0.42
    ctx.close()

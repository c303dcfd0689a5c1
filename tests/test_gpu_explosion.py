"""The robustness case (a ball flying apart into the box walls) at about 14k
sites: all 100 fluid steps converge to the tolerance, and after the wall
impact every cell -- many of them pressed against the walls, with
degenerate wall facets -- matches the FP64 oracle per quantity."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import pot, scenes

from _cmp import compare_cells, to_np

pytestmark = pytest.mark.gpu

TOL32 = dict(tol_v=1e-5, tol_h=1e-4, tol_c=1e-4)


def test_explosion_100_steps_against_oracle():
    sc = scenes.explosion(spacing=0.02)
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 1024, 0, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for k in range(100):
        st = pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
        assert st["status"] == 0 and st["err_max"] <= 1e-4, (k, st)
    x = to_np(pos)
    at_walls = int(np.sum(np.any((x < 1e-5) | (x > 1 - 1e-5), axis=1)))
    assert at_walls >= 20, at_walls  # the shell has reached the walls
    out = pot.lgc_compute_cells(ctx, pos, psi, nu)
    s32 = to_np(psi)
    ref = O.cells(x.astype(np.float64), s32.astype(np.float64))
    assert np.all(ref["status"] == 0)
    rep = compare_cells(out, ref, s32, to_np(nu), **TOL32)
    err = float(np.max(np.abs(ref["vol"] - sc.nu) / sc.nu))
    print(rep, "sites at the walls", at_walls, "oracle-measured volume error", err)
    assert err <= 1e-4
    ctx.close()

"""The 2M-site two-ball splash (the benchmark's workload) against the FP64
oracle, per quantity, on a 100k-cell subset (seed 1003): at the converged
start and after 10 fluid steps (just before the balls touch), in the launch
configuration bench.py times.  The oracle computes the sampled cells one by
one from the same float32 inputs; the GPU computes all 2M."""
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
    return rep, out


def test_splash_2m_subset_per_quantity():
    sc = scenes.splash()
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    vel = torch.from_numpy(sc.vel).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    q = scenes.random_subset(n, 100000, 1003)
    st = pot.pot_newton_solve(ctx, pos, nu, psi)
    assert st["status"] == 0
    rep0, out0 = check_subset(ctx, pos, psi, nu, q)
    # the converged start meets the tolerance in the oracle's volumes too
    v = to_np(out0["volumes"]).astype(np.float64)[q]
    assert np.max(np.abs(v - sc.nu[q]) / sc.nu[q]) <= 1e-4 + 2e-5
    prm = pot.default_params(dt=5e-4)
    for _ in range(10):
        st = pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
        assert st["status"] == 0
    rep10, out10 = check_subset(ctx, pos, psi, nu, q)
    ref = O.cells(to_np(pos).astype(np.float64), to_np(psi).astype(np.float64), query=q)
    err = np.max(np.abs(ref["vol"] - sc.nu[q]) / sc.nu[q])
    # the GPU's converged weights, measured by the oracle: the tolerance
    # plus the FP32 geometry error
    assert err <= 1.5e-4, err
    print("step 0:", rep0)
    print("step 10:", rep10, "oracle-measured volume error", err)
    ctx.close()

"""GPU Newton solve (Algorithm 1, KMT steps, Jacobi-PCG) and fluid step
(Sec. 5) against the FP64 oracle.

The partial-transport weights are unique (psi_0 = 0 fixed, Sec. 2.2), so the
converged psi of GPU and oracle must agree: with both solved far below the
tolerance in FP64 they agree to ~1e-8; the mixed-precision solve at 1e-4 is
checked by recomputing its volumes with the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import pot, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pot.Context(200000, 64, 0)
    yield c
    c.close()


def tens(a, dtype, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def test_block_fp64_matches_oracle(ctx):
    sc = scenes.jittered_block()
    pos = sc.pos.astype(np.float64)
    ref = O.newton(pos, sc.nu, sc.psi.astype(np.float64), tol=1e-11)
    assert ref.status == O.NEWTON_OK
    dev = ctx.device
    psi = tens(sc.psi, torch.float64, dev)
    st = pot.pot_newton_solve(ctx, tens(pos, torch.float64, dev), tens(sc.nu, torch.float64, dev), psi,
                              params=pot.default_params(tol=1e-11))
    assert st["status"] == 0 and st["err_max"] <= 1e-11
    got = psi.cpu().numpy()
    np.testing.assert_allclose(got, ref.psi, rtol=1e-8)
    # the iteration count follows the oracle's (same algorithm, different rounding)
    assert abs(st["newton_iters"] - ref.iters) <= 1


def test_block_mixed_precision(ctx):
    sc = scenes.jittered_block()
    dev = ctx.device
    psi = tens(sc.psi, torch.float32, dev)
    st = pot.pot_newton_solve(ctx, tens(sc.pos, torch.float32, dev), tens(sc.nu, torch.float64, dev), psi)
    assert st["status"] == 0 and st["err_max"] <= 1e-4
    got = psi.cpu().numpy().astype(np.float64)
    v = O.cells(sc.pos.astype(np.float64), got)["vol"]
    err = np.max(np.abs(v - sc.nu) / sc.nu)
    assert err <= 1e-4, err  # the mixed solve stops at 0.9 tol: room for the FP32 error
    ref = O.newton(sc.pos.astype(np.float64), sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    np.testing.assert_allclose(got, ref.psi, rtol=2e-3)


def test_far_start_needs_kmt_halving(ctx):
    sc = scenes.jittered_block(n_side=6, seed=4)
    dev = ctx.device
    far = (0.05 * sc.psi.astype(np.float64))
    psi = tens(far, torch.float64, dev)
    st = pot.pot_newton_solve(ctx, tens(sc.pos.astype(np.float64), torch.float64, dev),
                              tens(sc.nu, torch.float64, dev), psi, params=pot.default_params(tol=1e-8))
    ref = O.newton(sc.pos.astype(np.float64), sc.nu, far, tol=1e-8)
    assert st["status"] == 0 and ref.status == O.NEWTON_OK
    assert st["halvings"] > 0
    np.testing.assert_allclose(psi.cpu().numpy(), ref.psi, rtol=1e-5)


def test_failure_statuses(ctx):
    sc = scenes.jittered_block(n_side=3, seed=4)
    dev = ctx.device
    pos = tens(sc.pos, torch.float32, dev)
    nu = tens(sc.nu, torch.float64, dev)
    bad = sc.psi.copy()
    bad[0] = 0.0
    got = tens(bad, torch.float32, dev)
    st = pot.pot_newton_solve(ctx, pos, nu, got, check=False)
    # an empty cell at the start is repaired, then Newton converges to the
    # unique weights (the oracle with the same repair agrees)
    assert st["status"] == 0 and st["repairs"] >= 1
    ref = O.newton(sc.pos.astype(np.float64), sc.nu, bad.astype(np.float64), tol=1e-10, repair=True)
    np.testing.assert_allclose(got.cpu().numpy(), ref.psi, rtol=2e-3)
    far = tens(0.05 * sc.psi, torch.float32, dev)
    st = pot.pot_newton_solve(ctx, pos, nu, far, params=pot.default_params(max_halvings=0), check=False)
    assert st["status"] == 7  # KMT step not found
    st = pot.pot_newton_solve(ctx, pos, nu, tens(0.05 * sc.psi, torch.float32, dev),
                              params=pot.default_params(max_newton=1), check=False)
    assert st["status"] == 6  # iteration cap


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_fluid_step_matches_oracle(ctx, dtype):
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=2)
    dev = ctx.device
    npdt = np.float64 if dtype == torch.float64 else np.float32
    # converge the start first so that one step is a warm-started solve
    r0 = O.newton(sc.pos.astype(npdt).astype(np.float64), sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    psi0 = r0.psi.astype(npdt)
    vel0 = np.zeros_like(sc.pos, dtype=npdt)
    vel0[:, 0] = 0.5
    pos = tens(sc.pos.astype(npdt), dtype, dev)
    vel = tens(vel0, dtype, dev)
    psi = tens(psi0, dtype, dev)
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    prm = pot.default_params(tol=tol, dt=2e-3)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    assert st["status"] == 0
    x1, v1, nr = O.fluid_step(sc.pos.astype(npdt).astype(np.float64), vel0.astype(np.float64),
                              psi0.astype(np.float64), sc.nu, dt=2e-3, tol=1e-11)
    gx = pos.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gx, x1, rtol=0, atol=1e-15 if dtype == torch.float64 else 1e-7)
    gv = vel.cpu().numpy().astype(np.float64)
    # velocity = dt/eps^2 * centroid offset: centroid error of ~1e-4 r (FP32) or ~1e-9 r (FP64)
    r = math.sqrt(float(psi0.max()))
    atol = 2e-3 / 1e-4 * r * (1e-9 if dtype == torch.float64 else 2e-3)
    np.testing.assert_allclose(gv, v1, rtol=0, atol=atol)


def test_fluid_substeps_match_oracle_steps(ctx):
    """substeps = 3 equals three oracle fluid steps of dt / 3 (FP64, solved
    far below the tolerance), and the stats sum the substeps."""
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=5)
    dev = ctx.device
    r0 = O.newton(sc.pos.astype(np.float64), sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    x = sc.pos.astype(np.float64)
    v = np.zeros_like(x)
    v[:, 0] = 0.5
    psi0 = r0.psi.copy()
    pos, vel, psi = tens(x, torch.float64, dev), tens(v, torch.float64, dev), tens(psi0, torch.float64, dev)
    prm = pot.default_params(tol=1e-10, dt=3e-3, eps=4e-3, substeps=3)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    assert st["status"] == 0 and st["grid_builds"] == 3 and st["err_max"] <= 1e-10
    one = pot.pot_fluid_step(ctx, tens(x, torch.float64, dev), tens(v, torch.float64, dev),
                             tens(psi0, torch.float64, dev), tens(sc.nu, torch.float64, dev),
                             params=pot.default_params(tol=1e-10, dt=1e-3, eps=4e-3))
    assert one["grid_builds"] == 1 and st["newton_iters"] >= one["newton_iters"]
    p = psi0
    for _ in range(3):
        x, v, nr = O.fluid_step(x, v, p, sc.nu, dt=1e-3, eps=4e-3, tol=1e-11)
        p = nr.psi
    # positions take dt times velocities that carry the centroid error
    np.testing.assert_allclose(pos.cpu().numpy(), x, rtol=0, atol=1e-11)
    # velocity = dt/eps^2 * centroid offset, centroids agree to ~1e-9 r
    r = math.sqrt(float(psi0.max()))
    np.testing.assert_allclose(vel.cpu().numpy(), v, rtol=0, atol=3 * 1e-3 / 1.6e-5 * r * 1e-9)
    np.testing.assert_allclose(psi.cpu().numpy(), p, rtol=0, atol=1e-8 * float(np.max(p)))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_viscous_fluid_step_matches_oracle(ctx, dtype):
    """Eq. 4 (viscosity and surface tension over the P1 Laplacian of the
    converged cells) against the oracle's dense solve, one fluid step of a
    dam-break column with a strong coupling (dt mu sum_j w_ij ~ 0.4)."""
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=2)
    dev = ctx.device
    npdt = np.float64 if dtype == torch.float64 else np.float32
    r0 = O.newton(sc.pos.astype(npdt).astype(np.float64), sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    psi0 = r0.psi.astype(npdt)
    rng = np.random.default_rng(4)
    vel0 = (rng.normal(size=sc.pos.shape) * 0.3).astype(npdt)
    pos, vel, psi = tens(sc.pos.astype(npdt), dtype, dev), tens(vel0, dtype, dev), tens(psi0, dtype, dev)
    mu, gamma = 2000.0, 500.0
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    prm = pot.default_params(tol=tol, dt=2e-3, mu=mu, gamma=gamma)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    assert st["status"] == 0 and (st["visc_iters"] > 0)
    x1, v1, nr = O.fluid_step(sc.pos.astype(npdt).astype(np.float64), vel0.astype(np.float64),
                              psi0.astype(np.float64), sc.nu, dt=2e-3, tol=1e-11, mu=mu, gamma=gamma)
    explicit = O.velocity_update(x1, O.advect_and_clamp(sc.pos.astype(npdt).astype(np.float64),
                                                        vel0.astype(np.float64), 2e-3)[1],
                                 nr.res["cen"], 2e-3)
    gv = vel.cpu().numpy().astype(np.float64)
    # the viscous update differs from the explicit one by far more than the tolerance
    assert np.max(np.abs(v1 - explicit)) > 1e-2
    scale = float(np.max(np.abs(v1)))
    atol = 1e-9 * scale if dtype == torch.float64 else 2e-3 * scale
    np.testing.assert_allclose(gv, v1, rtol=0, atol=atol)


def test_viscous_factors_match_oracle(ctx):
    """Two fluids: per-site viscosity factors (mu_ij = mu (f_i + f_j) / 2),
    the lower half of the column 20x more viscous, against the oracle (FP64)."""
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=2)
    dev = ctx.device
    x0 = sc.pos.astype(np.float64)
    r0 = O.newton(x0, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    rng = np.random.default_rng(6)
    vel0 = rng.normal(size=sc.pos.shape) * 0.3
    f = np.where(x0[:, 2] < 0.08, 2.0, 0.1)
    pos, vel, psi = tens(x0, torch.float64, dev), tens(vel0, torch.float64, dev), tens(r0.psi, torch.float64, dev)
    pot.set_viscosity_factors(ctx, torch.as_tensor(f, dtype=torch.float32, device=dev))
    try:
        prm = pot.default_params(tol=1e-10, dt=2e-3, mu=2000.0, gamma=100.0)
        st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    finally:
        pot.set_viscosity_factors(ctx, None)
    assert st["status"] == 0
    x1, v1, _ = O.fluid_step(x0, vel0, r0.psi, sc.nu, dt=2e-3, tol=1e-11, mu=2000.0, gamma=100.0,
                             factors=f.astype(np.float32).astype(np.float64))
    _, v_one, _ = O.fluid_step(x0, vel0, r0.psi, sc.nu, dt=2e-3, tol=1e-11, mu=2000.0, gamma=100.0)
    assert np.max(np.abs(v1 - v_one)) > 1e-2  # the factors matter
    np.testing.assert_allclose(vel.cpu().numpy(), v1, rtol=0, atol=1e-9 * float(np.max(np.abs(v1))))


@pytest.mark.parametrize("dtype,mu", [(torch.float64, 0.0), (torch.float32, 2000.0)])
def test_wall_viscosity_matches_oracle(ctx, dtype, mu):
    """The fluid-boundary term (Sec. 5, walls at rest): mu_wall times the
    walls' P1 Laplacian weight sum_w |B_iw| / (2 h_iw) on the diagonal of
    Eq. 4, alone (the bulk viscosity off) and with the bulk viscosity, against
    the oracle's dense solve on a dam-break column standing in a box corner."""
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=2)
    dev = ctx.device
    npdt = np.float64 if dtype == torch.float64 else np.float32
    x0 = sc.pos.astype(npdt).astype(np.float64)
    r0 = O.newton(x0, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    psi0 = r0.psi.astype(npdt)
    rng = np.random.default_rng(8)
    vel0 = (rng.normal(size=sc.pos.shape) * 0.3).astype(npdt)
    pos, vel, psi = tens(x0, dtype, dev), tens(vel0, dtype, dev), tens(psi0, dtype, dev)
    mu_wall = 1e4
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    prm = pot.default_params(tol=tol, dt=2e-3, mu=mu, gamma=0.0, mu_wall=mu_wall)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    assert st["status"] == 0 and st["visc_iters"] > 0
    args = (x0, vel0.astype(np.float64), psi0.astype(np.float64), sc.nu)
    _, v1, _ = O.fluid_step(*args, dt=2e-3, tol=1e-11, mu=mu, mu_wall=mu_wall)
    _, v_free, _ = O.fluid_step(*args, dt=2e-3, tol=1e-11, mu=mu)
    assert np.max(np.abs(v1 - v_free)) > 1e-2  # the walls matter
    scale = float(np.max(np.abs(v1)))
    atol = 1e-9 * scale if dtype == torch.float64 else 2e-3 * scale
    np.testing.assert_allclose(vel.cpu().numpy().astype(np.float64), v1, rtol=0, atol=atol)


@pytest.mark.parametrize("dtype,mu,gamma", [(torch.float64, 0.0, 0.0), (torch.float32, 0.0, 0.0),
                                            (torch.float32, 2000.0, 500.0)])
def test_wall_tension_matches_oracle(ctx, dtype, mu, gamma):
    """The walls' part of the surface tension (Sec. 5, fluid-boundary
    interaction: each wall facet is the facet to a neighbour cbrt(|V_i|)
    beyond the wall), alone (an explicit update) and with the bulk
    viscosity and surface tension (a semi-implicit solve), against the
    oracle's dense fluid step on a dam-break column standing in a box
    corner."""
    sc = scenes.dam_break(nx=10, ny=10, nz=20, width=0.16, seed=3)
    dev = ctx.device
    npdt = np.float64 if dtype == torch.float64 else np.float32
    x0 = sc.pos.astype(npdt).astype(np.float64)
    r0 = O.newton(x0, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    psi0 = r0.psi.astype(npdt)
    rng = np.random.default_rng(9)
    vel0 = (rng.normal(size=sc.pos.shape) * 0.3).astype(npdt)
    pos, vel, psi = tens(x0, dtype, dev), tens(vel0, dtype, dev), tens(psi0, dtype, dev)
    gamma_wall = 3e4
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    prm = pot.default_params(tol=tol, dt=2e-3, mu=mu, gamma=gamma, gamma_wall=gamma_wall)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tens(sc.nu, torch.float64, dev), params=prm)
    assert st["status"] == 0
    args = (x0, vel0.astype(np.float64), psi0.astype(np.float64), sc.nu)
    _, v1, _ = O.fluid_step(*args, dt=2e-3, tol=1e-11, mu=mu, gamma=gamma, gamma_wall=gamma_wall)
    _, v_free, _ = O.fluid_step(*args, dt=2e-3, tol=1e-11, mu=mu, gamma=gamma)
    assert np.max(np.abs(v1 - v_free)) > 1e-2  # the walls matter
    scale = float(np.max(np.abs(v1)))
    atol = 1e-9 * scale if dtype == torch.float64 else 2e-3 * scale
    got = vel.cpu().numpy().astype(np.float64)
    print("wall tension: max |dv| from the walls", float(np.max(np.abs(v1 - v_free))),
          "GPU error", float(np.max(np.abs(got - v1))), "of scale", scale)
    np.testing.assert_allclose(got, v1, rtol=0, atol=atol)

"""Degenerate inputs of the path: an empty site set (rejected on the host,
nothing launched, the context usable afterwards) and a single site, where
Newton (Algorithm 1) and the fluid step (Sec. 5) reduce to closed forms.

A lone ball inside the box is its own cell (Eq. 1 with no neighbour and no
wall): V = 4/3 pi psi^{3/2}, so the weight that gives it volume nu is
psi = (3 nu / (4 pi))^{2/3}; its centroid is the site, so the pressure
spring vanishes and the step is free fall, v1 = v0 + dt g, x1 = x0 + dt v0.
With no neighbour and no wall facet the Laplacian of Eq. 4 is empty, so the
viscous update is the same free fall."""
import math

import numpy as np
import pytest
import torch

from paper_2601_05765_b300 import pot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pot.Context(1000, 32, 0)
    yield c
    c.close()


def test_empty_input_is_rejected_and_context_survives(ctx):
    dev = ctx.device
    for dt in (torch.float32, torch.float64):
        pos = torch.empty((0, 3), dtype=dt, device=dev)
        vel = torch.empty((0, 3), dtype=dt, device=dev)
        psi = torch.empty(0, dtype=dt, device=dev)
        nu = torch.empty(0, dtype=torch.float64, device=dev)
        out = pot.lgc_compute_cells(ctx, pos, psi, nu, check=False)
        assert out["status"] == pot.POT_ERR_INVALID_ARG
        assert pot.pot_newton_solve(ctx, pos, nu, psi, check=False)["status"] == pot.POT_ERR_INVALID_ARG
        assert pot.pot_fluid_step(ctx, pos, vel, psi, nu, check=False)["status"] == pot.POT_ERR_INVALID_ARG
    with pytest.raises(pot.PotError):
        pot.render_depth(ctx, torch.empty((0, 3), device=dev), torch.empty(0, device=dev),
                         (0.5, -1.0, 0.5), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), 0.8, 16, 16)
    # the context still works
    out = pot.lgc_compute_cells(ctx, torch.tensor([[0.5, 0.5, 0.5]], device=dev),
                                torch.tensor([1e-4], device=dev))
    assert abs(float(out["volumes"][0]) - 4 / 3 * math.pi * 1e-6) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_single_site_newton_closed_form(ctx, dtype):
    dev = ctx.device
    r = 0.05
    nu = 4 / 3 * math.pi * r ** 3
    pos = torch.tensor([[0.3, 0.6, 0.5]], dtype=dtype, device=dev)
    psi = torch.tensor([(0.8 * r) ** 2], dtype=dtype, device=dev)
    tgt = torch.tensor([nu], dtype=torch.float64, device=dev)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    st = pot.pot_newton_solve(ctx, pos, tgt, psi, params=pot.default_params(tol=tol))
    assert st["status"] == 0 and st["err_max"] <= tol
    rel = abs(float(psi[0]) - r * r) / (r * r)
    assert rel <= (1e-11 if dtype == torch.float64 else 2e-5), rel


@pytest.mark.parametrize("mu", [0.0, 500.0])
def test_single_site_fluid_step_is_free_fall(ctx, mu):
    dev = ctx.device
    r = 0.05
    nu = 4 / 3 * math.pi * r ** 3
    x0 = np.array([[0.4, 0.5, 0.6]])
    v0 = np.array([[0.3, -0.2, 0.1]])
    pos = torch.tensor(x0, dtype=torch.float64, device=dev)
    vel = torch.tensor(v0, dtype=torch.float64, device=dev)
    psi = torch.tensor([r * r], dtype=torch.float64, device=dev)
    tgt = torch.tensor([nu], dtype=torch.float64, device=dev)
    dt = 1e-3
    prm = pot.default_params(tol=1e-12, dt=dt, eps=0.01, mu=mu, gamma=0.0)
    for _ in range(3):
        st = pot.pot_fluid_step(ctx, pos, vel, psi, tgt, params=prm)
        assert st["status"] == 0
    g = np.array([0.0, 0.0, -9.81])
    v, x = v0.copy(), x0.copy()
    for _ in range(3):
        x = x + dt * v
        v = v + dt * g
    np.testing.assert_allclose(pos.cpu().numpy(), x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vel.cpu().numpy(), v, rtol=0, atol=1e-9)
    assert abs(float(psi[0]) - r * r) <= 1e-12 * r * r


def test_single_site_in_a_box_edge_with_wall_viscosity(ctx):
    """One ball cut by the floor and the -x wall (two wall facets clipping
    each other), no-slip wall viscosity on: the GPU fluid step against the
    oracle's (Eq. 4 with the walls' Laplacian weight on the diagonal)."""
    from oracle import oracle as O
    dev = ctx.device
    h, r = 0.05, 0.08
    x0 = np.array([[h, 0.5, h]])
    v0 = np.array([[0.2, 0.1, -0.3]])
    nu = O.cells(x0, np.array([r * r]))["vol"]
    pos = torch.tensor(x0, dtype=torch.float64, device=dev)
    vel = torch.tensor(v0, dtype=torch.float64, device=dev)
    psi = torch.tensor([r * r], dtype=torch.float64, device=dev)
    tgt = torch.tensor(nu, dtype=torch.float64, device=dev)
    dt, eps, mu_wall = 1e-3, 0.01, 50.0
    prm = pot.default_params(tol=1e-12, dt=dt, eps=eps, mu_wall=mu_wall)
    st = pot.pot_fluid_step(ctx, pos, vel, psi, tgt, params=prm)
    assert st["status"] == 0 and st["visc_iters"] > 0
    x1, v1, _ = O.fluid_step(x0, v0, np.array([r * r]), nu, dt=dt, eps=eps, tol=1e-12,
                             mu_wall=mu_wall)
    _, v_free, _ = O.fluid_step(x0, v0, np.array([r * r]), nu, dt=dt, eps=eps, tol=1e-12)
    assert np.max(np.abs(v1 - v_free)) > 1e-3  # the walls matter
    np.testing.assert_allclose(pos.cpu().numpy(), x1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vel.cpu().numpy(), v1, rtol=0, atol=1e-9 * float(np.max(np.abs(v1))))

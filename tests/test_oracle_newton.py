"""Pins of the oracle's Newton solve (Algorithm 1 with KMT steps) and fluid step.

Closed forms: an isolated site converges to psi* = (3 nu / 4 pi)^(2/3); two
symmetric sites converge to the root of the spherical-cap volume equation
(found here by bisection, independently of the oracle).  The weights of the
partial transport problem are unique (Sec. 2.2, psi_0 = 0 fixed), so two
different starts must reach the same psi.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_05765_b300 import scenes


def test_isolated_site_closed_form():
    nu = np.array([1e-4])
    r0 = 0.5 * (3 * nu[0] / (4 * math.pi)) ** (1 / 3)
    nr = O.newton([[0.5, 0.5, 0.5]], nu, [r0 * r0], tol=1e-12)
    assert nr.status == O.NEWTON_OK
    assert nr.psi[0] == pytest.approx((3 * nu[0] / (4 * math.pi)) ** (2 / 3), rel=1e-11)


def test_two_symmetric_sites_bisection():
    d = 0.05
    nu = 1e-4

    def vol(r):  # ball minus the cap beyond the mid-plane
        if r <= d / 2:
            return 4 / 3 * math.pi * r ** 3
        t = r - d / 2
        return 4 / 3 * math.pi * r ** 3 - math.pi * t * t * (3 * r - t) / 3

    lo, hi = 1e-4, 0.2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if vol(mid) < nu else (lo, mid)
    r_star = 0.5 * (lo + hi)
    assert r_star > d / 2  # the two cells touch
    pos = [[0.5 - d / 2, 0.5, 0.5], [0.5 + d / 2, 0.5, 0.5]]
    nr = O.newton(pos, [nu, nu], [(0.7 * r_star) ** 2] * 2, tol=1e-12)
    assert nr.status == O.NEWTON_OK
    np.testing.assert_allclose(nr.psi, r_star ** 2, rtol=1e-10)


def test_block_uniqueness_and_tolerance():
    sc = scenes.jittered_block(n_side=4, spacing=0.05, seed=0)
    pos = sc.pos.astype(np.float64)
    a = O.newton(pos, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    b = O.newton(pos, sc.nu, 1.3 * sc.psi.astype(np.float64), tol=1e-10)
    assert a.status == O.NEWTON_OK and b.status == O.NEWTON_OK
    np.testing.assert_allclose(a.psi, b.psi, rtol=1e-8)
    # self-verification: the geometry, recomputed, meets the tolerance
    v = O.cells(pos, a.psi)["vol"]
    assert np.max(np.abs(v - sc.nu) / sc.nu) <= 1e-10
    # the converged cells hold the prescribed total volume
    assert v.sum() == pytest.approx(sc.nu.sum(), rel=1e-9)


def test_kmt_halving_and_failure_codes():
    sc = scenes.jittered_block(n_side=3, spacing=0.05, seed=4)
    pos = sc.pos.astype(np.float64)
    # a far start (tiny balls) needs damped steps
    far = 0.05 * sc.psi.astype(np.float64)
    nr = O.newton(pos, sc.nu, far, tol=1e-8)
    assert nr.status == O.NEWTON_OK
    assert nr.halvings > 0
    # the error history is eventually monotone and quadratic near the end
    h = nr.history
    assert h[-1] <= 1e-8 and h[-2] > h[-1]
    # no halving allowed: the KMT test rejects alpha = 1 and the search fails
    nr0 = O.newton(pos, sc.nu, far, tol=1e-8, max_halvings=0)
    assert nr0.status == O.NEWTON_LINESEARCH_FAILED
    # a start with an empty cell is refused (the KMT bound eps0 would be 0)
    bad = sc.psi.astype(np.float64).copy()
    bad[0] = 0.0
    assert O.newton(pos, sc.nu, bad).status == O.NEWTON_EMPTY_CELL_AT_START
    # the iteration cap is reported
    assert O.newton(pos, sc.nu, far, tol=1e-12, max_newton=2).status == O.NEWTON_NOT_CONVERGED


def test_fluid_step_free_fall_single_site():
    # an isolated cell's centroid is its site: only gravity acts
    nu = np.array([1e-4])
    psi = np.array([(3 * nu[0] / (4 * math.pi)) ** (2 / 3)])
    x1, v1, nr = O.fluid_step([[0.5, 0.5, 0.5]], [[0.1, 0.0, 0.0]], psi, nu, dt=1e-3, tol=1e-10)
    np.testing.assert_allclose(x1[0], [0.5001, 0.5, 0.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(v1[0], [0.1, 0.0, -9.81e-3], rtol=0, atol=1e-9)


def test_fluid_step_wall_clamp_and_spring():
    # a cell cut by the floor: the centroid is above the site, so the spring
    # pushes up against gravity; the site is clamped into the box
    nu = np.array([2e-4])
    x, v = np.array([[0.5, 0.5, 0.002]]), np.array([[0.0, 0.0, -3.0]])
    psi = np.array([(3 * nu[0] / (4 * math.pi)) ** (2 / 3)])
    x1, v1, nr = O.fluid_step(x, v, psi, nu, dt=1e-3, tol=1e-10)
    assert x1[0, 2] == pytest.approx(1e-6)
    cen = nr.res["cen"][0]
    assert cen[2] > x1[0, 2]
    expect = 0.0 + 1e-3 * (-9.81 + (cen[2] - x1[0, 2]) / 1e-4)
    assert v1[0, 2] == pytest.approx(expect, rel=1e-12)


def test_empty_cell_repair_puts_sites_inside_their_cells():
    sc = scenes.jittered_block(n_side=4, seed=0)
    pos = sc.pos.astype(np.float64)
    psi = sc.psi.astype(np.float64).copy()
    # two empty cells: a zero weight, and a ball swallowed by a heavy neighbour
    psi[5] = 0.0
    psi[6] = psi[6] * 0.01
    psi[7] = psi[7] * 6.0
    res = O.cells(pos, psi)
    assert np.sum(res["vol"] <= 0) >= 1
    fixed = O.repair_empty(pos, psi, res["vol"], sc.nu)
    after = O.cells(pos, fixed)
    for i in np.nonzero(res["vol"] <= 0)[0]:
        d = np.linalg.norm(pos - pos[i], axis=1)
        d[i] = np.inf
        h = (d * d + fixed[i] - fixed) / (2 * d)
        assert np.all(h[np.isfinite(d)] > 0)  # the site lies inside its own cell
        assert after["vol"][i] > 0
    # non-empty cells keep their weights; Newton from the repaired start converges
    keep = res["vol"] > 0
    np.testing.assert_array_equal(fixed[keep], psi[keep])
    nr = O.newton(pos, sc.nu, psi, tol=1e-10, repair=True)
    ref = O.newton(pos, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    assert nr.status == O.NEWTON_OK
    np.testing.assert_allclose(nr.psi, ref.psi, rtol=1e-8)


def _viscous_setup(seed=8):
    from paper_2601_05765_b300 import scenes
    sc = scenes.dam_break(nx=6, ny=6, nz=8, width=0.12, seed=seed)
    x = sc.pos.astype(np.float64)
    nr = O.newton(x, sc.nu, sc.psi.astype(np.float64), tol=1e-10)
    assert nr.status == O.NEWTON_OK
    w = O.laplacian_weights(nr.res, nr.psi)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=x.shape)
    return x, v, nr.res["cen"], w


def test_viscous_update_pins():
    """Eq. 4 against what the algebra fixes: the weights are symmetric and
    non-negative; without viscosity and surface tension the solve is the
    explicit update; a uniform velocity field under no force is left
    unchanged; the Laplacian terms conserve momentum (the total velocity
    change is dt times the summed pressure and gravity forces); viscosity
    never adds kinetic energy to the explicit update; surface tension pulls
    a free blob inwards."""
    x, v, cen, w = _viscous_setup()
    n = x.shape[0]
    dt, eps, g = 1e-3, 0.01, np.array([0.0, 0.0, -9.81])
    np.testing.assert_allclose(w, w.T, rtol=1e-9, atol=1e-15)
    assert np.all(w >= 0) and np.all(np.diag(w) == 0) and w.sum() > 0
    explicit = O.velocity_update(x, v, cen, dt, eps=eps, g=g)
    np.testing.assert_allclose(O.viscous_velocity(x, v, cen, w, dt, eps, g, 0.0, 0.0), explicit,
                               rtol=1e-12, atol=1e-12)
    u = np.tile([0.3, -0.2, 0.1], (n, 1))
    np.testing.assert_allclose(O.viscous_velocity(x, u, x, w, dt, eps, 0 * g, 50.0, 0.0), u,
                               rtol=1e-12, atol=1e-12)
    v1 = O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 3.0)
    np.testing.assert_allclose(v1.sum(0), explicit.sum(0), rtol=1e-9, atol=1e-9)
    vv = O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 0.0)
    assert np.sum(vv ** 2) < np.sum(explicit ** 2)
    # surface tension alone, no other force, at rest: the blob contracts
    vt = O.viscous_velocity(x, np.zeros_like(v), x, w, dt, eps, 0 * g, 0.0, 3.0)
    assert np.sum(vt * (x - x.mean(0))) < 0


def test_viscous_update_against_graph_laplacian():
    """L u built site by site from its definition (sum_j w_ij (u_j - u_i))
    equals the matrix form the solve uses, and the solution satisfies the
    system row by row."""
    x, v, cen, w = _viscous_setup(9)
    n = x.shape[0]
    dt, eps, g, mu, gamma = 1e-3, 0.01, np.array([0.0, 0.0, -9.81]), 20.0, 2.0
    v1 = O.viscous_velocity(x, v, cen, w, dt, eps, g, mu, gamma)
    for i in range(0, n, 7):
        lap_v = sum(w[i, j] * (v1[j] - v1[i]) for j in range(n) if w[i, j] > 0)
        lap_x = sum(w[i, j] * (x[j] - x[i]) for j in range(n) if w[i, j] > 0)
        lhs = v1[i] / dt - mu * lap_v
        rhs = v[i] / dt + (cen[i] - x[i]) / eps ** 2 + g + gamma * lap_x
        np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-6)


def test_viscous_factors_pins():
    """Per-site viscosity factors (mu_ij = mu (f_i + f_j) / 2): all ones is
    the single-fluid update; the system stays symmetric with zero row sums
    off the I/dt part, so momentum is conserved; a site of factor 0 among
    factor-0 neighbours moves as without viscosity."""
    x, v, cen, w = _viscous_setup(10)
    n = x.shape[0]
    dt, eps, g = 1e-3, 0.01, np.array([0.0, 0.0, -9.81])
    one = O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 1.0)
    np.testing.assert_allclose(O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 1.0, np.ones(n)),
                               one, rtol=1e-12, atol=1e-12)
    f = np.random.default_rng(3).uniform(0.1, 2.0, n)
    vf = O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 1.0, f)
    explicit = O.velocity_update(x, v, cen, dt, eps=eps, g=g)
    lap_x_sum = (w @ x - w.sum(1)[:, None] * x).sum(0)
    np.testing.assert_allclose(vf.sum(0), explicit.sum(0) + dt * 1.0 * lap_x_sum, rtol=1e-9, atol=1e-9)
    zero = O.viscous_velocity(x, v, cen, w, dt, eps, g, 50.0, 0.0, np.zeros(n))
    np.testing.assert_allclose(zero, explicit, rtol=1e-12, atol=1e-12)


def test_wall_weights_closed_form_and_no_slip():
    """A lone ball cut by the floor at height h: its wall facet is the disk
    of radius sqrt(psi - h^2), weight pi (psi - h^2) / (2 h); a stiff wall
    affinity brings that site's velocity to rest (no-slip) while a site away
    from the walls keeps its explicit update."""
    pos = np.array([[0.5, 0.5, 0.05], [0.5, 0.5, 0.5]])
    psi = np.array([0.08 ** 2, 0.05 ** 2])
    res = O.cells(pos, psi)
    ww = O.wall_weights(res, pos)
    assert abs(ww[0] - math.pi * (psi[0] - 0.05 ** 2) / (2 * 0.05)) < 1e-12
    assert ww[1] == 0.0
    w = O.laplacian_weights(res, psi)
    v = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    out = O.viscous_velocity(pos, v, res["cen"], w, 1e-3, 0.01, np.zeros(3), 0.0, 0.0,
                             wall_w=ww, mu_wall=1e13)
    assert np.max(np.abs(out[0])) < 1e-6
    expl = O.velocity_update(pos, v, res["cen"], 1e-3, eps=0.01, g=(0.0, 0.0, 0.0))
    np.testing.assert_allclose(out[1], expl[1], rtol=1e-12, atol=1e-12)


def test_wall_tension_closed_form():
    """The walls' part of the surface tension (Sec. 5): a lone ball cut by
    the floor at height h is pulled toward the floor by
    pi (psi - h^2) / (2 h) * (h + cbrt(V)), V the ball minus its cap below
    the floor, 4/3 pi r^3 - pi t^2 (3 r - t) / 3 with t = r - h; a ball in
    the edge of the floor and the -x wall is pulled equally toward both; a
    ball away from the walls not at all.  Its velocity update then gains
    dt gamma_wall times that (explicit: no viscosity)."""
    h, r = 0.05, 0.08
    pos = np.array([[0.5, 0.5, h], [0.5, 0.5, 0.5], [h, 0.3, h]])
    psi = np.array([r * r, 0.05 ** 2, r * r])
    res = O.cells(pos, psi)
    t = r - h
    vol = 4.0 / 3.0 * math.pi * r ** 3 - math.pi * t * t * (3 * r - t) / 3.0
    assert abs(res["vol"][0] - vol) < 1e-14
    wt = O.wall_tension(res, pos)
    mag = math.pi * (r * r - h * h) / (2 * h) * (h + vol ** (1.0 / 3.0))
    np.testing.assert_allclose(wt[0], [0.0, 0.0, -mag], rtol=1e-12, atol=1e-15)
    assert np.all(wt[1] == 0.0)
    assert wt[2][0] < 0 and wt[2][2] < 0 and wt[2][1] == 0.0
    assert abs(wt[2][0] - wt[2][2]) < 1e-12 * abs(wt[2][0])
    w = O.laplacian_weights(res, psi)
    v = np.zeros((3, 3))
    dt, gw = 1e-3, 7.0
    out = O.viscous_velocity(pos, v, res["cen"], w, dt, 0.01, np.zeros(3), 0.0, 0.0,
                             wall_t=wt, gamma_wall=gw)
    expl = O.velocity_update(pos, v, res["cen"], dt, eps=0.01, g=(0.0, 0.0, 0.0))
    np.testing.assert_allclose(out, expl + dt * gw * wt, rtol=1e-12, atol=1e-15)


def test_wall_weights_two_walls_clip_each_other():
    """A ball in the edge between the floor and the -x wall, both at distance
    h: each wall's disk (radius rho = sqrt(psi - h^2), centre at distance h
    from the other wall) loses the circular segment beyond the other wall,
    rho^2 acos(h / rho) - h sqrt(rho^2 - h^2); the weight is twice that
    clipped area over 2 h."""
    h, r = 0.05, 0.08
    pos = np.array([[h, 0.5, h]])
    psi = np.array([r * r])
    res = O.cells(pos, psi)
    rho2 = r * r - h * h
    rho = math.sqrt(rho2)
    seg = rho2 * math.acos(h / rho) - h * math.sqrt(rho2 - h * h)
    area = math.pi * rho2 - seg
    np.testing.assert_allclose(res["wall_area"][0, [0, 4]], [area, area], rtol=1e-10)
    assert np.all(res["wall_area"][0, [1, 2, 3, 5]] == 0.0)
    ww = O.wall_weights(res, pos)
    assert abs(ww[0] - 2 * area / (2 * h)) < 1e-10 * ww[0]

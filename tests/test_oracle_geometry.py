"""Pins of the FP64 oracle's cell geometry against things other than itself.

Closed forms (spherical caps, cubic lattices), Monte Carlo estimates drawn
from the plain definition of the cell (Eq. 1: ball, box and power-distance
tests only), finite differences of the volume in the weights (the Hessian
identities of Eq. 2), and invariants (symmetry of facet areas, total volume
below the box volume, brute force vs bucket-grid candidate search).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

LO = np.zeros(3)
HI = np.ones(3)


def cap_volume(r, h):
    """Volume of the part of a ball of radius r beyond a plane at distance h."""
    t = r - h
    return math.pi * t * t * (3 * r - t) / 3.0


def ball_volume(r):
    return 4.0 / 3.0 * math.pi * r ** 3


# --------------------------------------------------------------------------
# closed forms


def test_isolated_ball():
    r = 0.1
    res = O.cells([[0.5, 0.4, 0.6]], [r * r])
    assert res["vol"][0] == pytest.approx(ball_volume(r), rel=1e-14)
    assert res["karea"][0] == pytest.approx(4 * math.pi * r * r, rel=1e-14)
    assert res["nfac"][0] == 0 and res["n_planes"][0] == 0
    np.testing.assert_allclose(res["cen"][0], [0.5, 0.4, 0.6], atol=1e-15)


@pytest.mark.parametrize("psi", [(0.01, 0.01), (0.01, 0.008), (0.006, 0.011)])
def test_two_balls_caps(psi):
    d = 0.12
    pos = [[0.5 - d / 2, 0.5, 0.5], [0.5 + d / 2, 0.5, 0.5]]
    res = O.cells(pos, list(psi))
    for i in range(2):
        ps, pj = psi[i], psi[1 - i]
        r = math.sqrt(ps)
        h = (d * d + ps - pj) / (2 * d)
        assert res["vol"][i] == pytest.approx(ball_volume(r) - cap_volume(r, h), rel=1e-13)
        assert res["fac_area"][i, 0] == pytest.approx(math.pi * (ps - h * h), rel=1e-13)
        assert res["karea"][i] == pytest.approx(2 * math.pi * r * (r + h), rel=1e-13)
        # centroid of a ball minus a cap lies on the axis, shifted away from the cap
        zc = -math.pi * (r * r - h * h) ** 2 / 4.0 / res["vol"][i]  # int over cap of x / V
        sgn = -1.0 if i == 0 else 1.0
        assert res["cen"][i, 0] - pos[i][0] == pytest.approx(-sgn * zc, rel=1e-11)
    # the shared facet has one area seen from both sides
    assert res["fac_area"][0, 0] == pytest.approx(res["fac_area"][1, 0], rel=1e-14)


@pytest.mark.parametrize("axis,side", [(0, 0), (1, 1), (2, 0)])
def test_wall_cap(axis, side):
    r, h = 0.1, 0.04
    p = np.full(3, 0.5)
    p[axis] = h if side == 0 else 1.0 - h
    res = O.cells([p], [r * r])
    assert res["vol"][0] == pytest.approx(ball_volume(r) - cap_volume(r, h), rel=1e-13)
    assert res["wall_area"][0, 2 * axis + side] == pytest.approx(math.pi * (r * r - h * h), rel=1e-13)
    assert res["karea"][0] == pytest.approx(2 * math.pi * r * (r + h), rel=1e-13)
    assert res["nfac"][0] == 0


def test_box_corner_exact_and_offset():
    r = 0.1
    # site exactly on the corner: three planes through the site at once
    res = O.cells([[0.0, 0.0, 0.0]], [r * r])
    assert res["vol"][0] == pytest.approx(ball_volume(r) / 8, rel=1e-10)
    assert res["karea"][0] == pytest.approx(4 * math.pi * r * r / 8, rel=1e-10)
    # offset by 1e-9: the change is the slab volume, about 3 * quarter disk * 1e-9
    res = O.cells([[1e-9, 1e-9, 1e-9]], [r * r])
    expect = ball_volume(r) / 8 + 3 * (math.pi * r * r / 4) * 1e-9
    assert res["vol"][0] == pytest.approx(expect, rel=1e-12)
    # site on one face only
    res = O.cells([[0.0, 0.5, 0.5]], [r * r])
    assert res["vol"][0] == pytest.approx(ball_volume(r) / 2, rel=1e-12)


def test_site_outside_its_ball_side():
    # site behind a wall: h < 0 but > -r, the cell is the cap inside the box
    r = 0.1
    res = O.cells([[-0.03, 0.5, 0.5]], [r * r])
    assert res["inside"][0] == 0
    assert res["vol"][0] == pytest.approx(cap_volume(r, 0.03), rel=1e-12)
    assert res["karea"][0] == pytest.approx(2 * math.pi * r * (r - 0.03), rel=1e-12)
    # fully behind the wall: empty
    res = O.cells([[-0.2, 0.5, 0.5]], [r * r])
    assert res["vol"][0] == 0.0 and res["karea"][0] == 0.0


def test_empty_and_nonpositive_weight():
    res = O.cells([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], [0.0, 0.01])
    assert res["vol"][0] == 0.0
    # a site with psi <= 0 never clips its neighbour
    assert res["vol"][1] == pytest.approx(ball_volume(0.1), rel=1e-14)
    # a ball inside a bigger ball with larger weight is empty
    res = O.cells([[0.5, 0.5, 0.5], [0.51, 0.5, 0.5]], [0.0004, 0.01])
    assert res["vol"][0] == 0.0


def _lattice(n_side, s, r):
    k = np.arange(n_side) - (n_side - 1) / 2
    z, y, x = np.meshgrid(k, k, k, indexing="ij")
    pos = 0.5 + s * np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    psi = np.full(pos.shape[0], r * r)
    return pos, psi


def test_cubic_lattice_separate_caps():
    """s/2 < r < s/sqrt(2): six disjoint caps cut the interior ball."""
    s = 1.0 / 16
    r = 0.6 * s
    pos, psi = _lattice(5, s, r)
    c = 62
    res = O.cells(pos, psi, query=[c])
    assert res["vol"][0] == pytest.approx(ball_volume(r) - 6 * cap_volume(r, s / 2), rel=1e-13)
    assert res["karea"][0] == pytest.approx(4 * math.pi * r * r - 12 * math.pi * r * (r - s / 2), rel=1e-13)
    nf = res["nfac"][0]
    assert nf == 6
    np.testing.assert_allclose(res["fac_area"][0, :nf], math.pi * (r * r - s * s / 4), rtol=1e-13)
    np.testing.assert_allclose(res["cen"][0], pos[c], atol=1e-15)


def test_cubic_lattice_full_cube():
    """r >= (sqrt(3)/2) s: the interior cell is the cube; edge and corner
    neighbours are candidates whose facets have zero area."""
    s = 1.0 / 16
    r = 0.9 * s
    pos, psi = _lattice(5, s, r)
    c = 62
    res = O.cells(pos, psi, query=[c])
    assert res["vol"][0] == pytest.approx(s ** 3, rel=1e-12)
    assert abs(res["karea"][0]) < 1e-12 * r * r
    nf = res["nfac"][0]
    assert nf == 26  # 6 face + 12 edge + 8 corner neighbours cut the ball
    d = res["fac_dist"][0, :nf]
    a = res["fac_area"][0, :nf]
    face = np.isclose(d, s)
    assert face.sum() == 6
    np.testing.assert_allclose(a[face], s * s, rtol=1e-12)
    assert np.all(np.abs(a[~face]) < 1e-12 * s * s)
    diag, rows = O.hessian_entries(res, psi)
    cols, vals = rows[0]
    assert len(cols) == 6
    np.testing.assert_allclose(vals, -s / 2, rtol=1e-12)
    assert diag[0] == pytest.approx(3 * s, rel=1e-12)


# --------------------------------------------------------------------------
# Monte Carlo from the plain definition (Eq. 1)


def _inside_cell(x, i, pos, psi):
    """x (m,3): membership in C_i by direct power-distance tests."""
    pi = pos[i]
    pow_i = np.sum((x - pi) ** 2, 1) - psi[i]
    ok = pow_i <= 0.0
    ok &= np.all((x >= 0.0) & (x <= 1.0), axis=1)
    for j in range(pos.shape[0]):
        if j == i:
            continue
        ok &= pow_i <= np.sum((x - pos[j]) ** 2, 1) - psi[j]
    return ok


def _cluster(seed, n=10):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.02, 0.25, size=(n, 3))
    psi = rng.uniform(0.06, 0.11, size=n) ** 2
    return pos, psi


@pytest.mark.parametrize("seed", [11, 12])
def test_monte_carlo_volume_surface_centroid(seed):
    pos, psi = _cluster(seed)
    res = O.cells(pos, psi)
    rng = np.random.default_rng(100 + seed)
    n_samp = 2_000_000
    checked = 0
    for i in range(pos.shape[0]):
        r = math.sqrt(psi[i])
        hits, tot, csum = 0, 0, np.zeros(3)
        for _ in range(4):
            x = pos[i] + rng.uniform(-r, r, size=(n_samp // 4, 3))
            ok = _inside_cell(x, i, pos, psi)
            hits += ok.sum()
            tot += x.shape[0]
            csum += x[ok].sum(0)
        f = hits / tot
        cube = (2 * r) ** 3
        v_mc = f * cube
        sig = cube * math.sqrt(max(f * (1 - f), 1e-12) / tot)
        assert abs(res["vol"][i] - v_mc) <= 4.5 * sig + 1e-12, (i, res["vol"][i], v_mc, sig)
        if hits > 1000:
            cen = csum / hits
            spread = r / math.sqrt(hits)
            np.testing.assert_allclose(res["cen"][i], cen, atol=5 * spread)
            checked += 1
        # free surface: uniform points on the sphere
        u = rng.normal(size=(n_samp // 2, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        xs = pos[i] + r * u * (1 - 1e-12)
        ok = _inside_cell(xs, i, pos, psi)
        fk = ok.mean()
        k_mc = 4 * math.pi * psi[i] * fk
        sk = 4 * math.pi * psi[i] * math.sqrt(max(fk * (1 - fk), 1e-12) / xs.shape[0])
        assert abs(res["karea"][i] - k_mc) <= 4.5 * sk + 1e-12, (i, res["karea"][i], k_mc, sk)
    assert checked >= 4


def test_monte_carlo_facet_areas():
    pos, psi = _cluster(13)
    res = O.cells(pos, psi)
    rng = np.random.default_rng(7)
    n_samp = 400_000
    tested = 0
    for i in range(pos.shape[0]):
        for k in range(res["nfac"][i]):
            j = res["fac_j"][i, k]
            d = pos[j] - pos[i]
            dist = np.linalg.norm(d)
            n = d / dist
            h = (dist * dist + psi[i] - psi[j]) / (2 * dist)
            rho = math.sqrt(psi[i] - h * h)
            # uniform points in the disk of the bisector plane
            a = rng.uniform(0, 2 * math.pi, n_samp)
            rr = rho * np.sqrt(rng.uniform(0, 1, n_samp))
            e = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
            u = np.cross(n, e)
            u /= np.linalg.norm(u)
            v = np.cross(n, u)
            x = pos[i] + h * n + (rr * np.cos(a))[:, None] * u + (rr * np.sin(a))[:, None] * v
            # on the plane, the i-j test is an equality: test every other site
            pow_i = np.sum((x - pos[i]) ** 2, 1) - psi[i]
            ok = np.all((x >= 0) & (x <= 1), axis=1)
            for jj in range(pos.shape[0]):
                if jj in (i, j):
                    continue
                ok &= pow_i <= np.sum((x - pos[jj]) ** 2, 1) - psi[jj]
            f = ok.mean()
            disk = math.pi * rho * rho
            sig = disk * math.sqrt(max(f * (1 - f), 1e-12) / n_samp)
            assert abs(res["fac_area"][i, k] - f * disk) <= 4.5 * sig + 1e-12
            tested += 1
    assert tested >= 10


# --------------------------------------------------------------------------
# finite differences: dV_i/dpsi_j = -|B_ij|/(2 d_ij), dV_i/dpsi_i = M_ii (Eq. 2)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_finite_difference_hessian(seed):
    pos, psi = _cluster(seed, n=8)
    n = pos.shape[0]
    res = O.cells(pos, psi)
    m = O.hessian_dense(res, psi)
    fd = np.zeros((n, n))
    for j in range(n):
        dlt = 1e-6 * psi[j]
        pp, pm = psi.copy(), psi.copy()
        pp[j] += dlt
        pm[j] -= dlt
        fd[:, j] = (O.cells(pos, pp)["vol"] - O.cells(pos, pm)["vol"]) / (2 * dlt)
    scale = np.abs(np.diag(m)).max()
    np.testing.assert_allclose(fd, m, atol=2e-7 * scale, rtol=1e-6)
    # symmetry of the Hessian (|B_ij| = |B_ji|)
    np.testing.assert_allclose(m, m.T, atol=1e-12 * scale)


def test_finite_difference_position_independent_planes():
    # a wall facet does not move with psi: only the free surface enters M_ii
    r = 0.1
    p = [[0.05, 0.5, 0.5]]
    res = O.cells(p, [r * r])
    dlt = 1e-7
    vp = O.cells(p, [r * r + dlt])["vol"][0]
    vm = O.cells(p, [r * r - dlt])["vol"][0]
    diag, _ = O.hessian_entries(res, [r * r])
    assert (vp - vm) / (2 * dlt) == pytest.approx(diag[0], rel=1e-7)


# --------------------------------------------------------------------------
# invariants


def test_volume_bounds_and_candidate_search():
    rng = np.random.default_rng(5)
    n = 400
    pos = rng.uniform(0, 1, (n, 3))
    psi = (rng.uniform(0.5, 1.6, n) * (3 / (4 * math.pi * n)) ** (1 / 3)) ** 2
    a = O.cells(pos, psi, brute=True)
    b = O.cells(pos, psi, brute=False)
    assert np.all(a["status"] == 0)
    np.testing.assert_array_equal(a["nfac"], b["nfac"])
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-12, atol=0)  # plane order differs
    assert a["vol"].sum() <= 1.0
    assert np.all(a["vol"] <= 4 / 3 * math.pi * psi ** 1.5 * (1 + 1e-14))
    # shared facets: |B_ij| == |B_ji|
    area = {}
    for i in range(n):
        for k in range(a["nfac"][i]):
            area[(i, int(a["fac_j"][i, k]))] = a["fac_area"][i, k]
    for (i, j), v in area.items():
        # an empty cell lists no facets; its shared facets then have zero area
        other = area.get((j, i), 0.0)
        assert abs(v - other) <= 1e-12 * max(psi[i], psi[j])


def test_packed_volume_sum_equals_box():
    """Balls large enough to fill the box: cells tile it (full transport)."""
    rng = np.random.default_rng(9)
    n = 300
    pos = rng.uniform(0, 1, (n, 3))
    psi = np.full(n, 0.5 ** 2)
    res = O.cells(pos, psi, max_facets=n)
    assert np.all(res["status"] == 0)
    assert res["vol"].sum() == pytest.approx(1.0, rel=1e-12)
    assert np.all(res["karea"] < 1e-12)

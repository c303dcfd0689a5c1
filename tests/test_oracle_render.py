"""The oracle's first-hit rendering against closed forms: a ball straight
ahead is hit at distance D - r with the normal facing the camera; rays miss
exactly outside its silhouette (tan of the angle to the centre > r /
sqrt(D^2 - r^2)); a nearer ball occludes a farther one; the box clips the
union of balls; culling by the free-surface area keeps the first hit."""
import math

import numpy as np

from oracle import oracle as O


def test_single_ball_straight_ahead():
    o, f, up = (0.5, 0.5, -1.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)
    p = np.array([[0.5, 0.5, 0.5]])
    r = 0.2
    depth, normal = O.render_depth(p, [r * r], o, f, up, math.radians(30), 41, 31)
    # the centre pixel's ray is the axis: distance 1.5 - 0.2
    assert abs(depth[15, 20] - 1.3) < 1e-12
    np.testing.assert_allclose(normal[15, 20], [0.0, 0.0, -1.0], atol=1e-12)
    d = O.camera_rays(o, f, up, math.radians(30), 41, 31)
    cosang = d[..., 2]
    tan = np.sqrt(1 - cosang ** 2) / cosang
    inside = tan < r / math.sqrt(1.5 ** 2 - r ** 2)
    edge = np.abs(tan - r / math.sqrt(1.5 ** 2 - r ** 2)) < 1e-9
    assert np.all((depth >= 0) == inside | edge)
    # every hit lies on the sphere
    x = np.asarray(o)[None, None, :] + depth[..., None] * d
    rr = np.linalg.norm(x - p[0], axis=2)
    assert np.all(np.abs(rr[depth >= 0] - r) < 1e-12)


def test_occlusion_box_and_culling():
    o, f, up = (0.5, 0.5, -1.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)
    p = np.array([[0.5, 0.5, 0.7], [0.5, 0.5, 0.3]])
    psi = np.array([0.1 ** 2, 0.05 ** 2])
    depth, _ = O.render_depth(p, psi, o, f, up, math.radians(20), 11, 11)
    assert abs(depth[5, 5] - (1.3 - 0.05)) < 1e-12  # the nearer, smaller ball
    # a ball sticking out of the box: the hit is the box face z = 0
    depth, normal = O.render_depth(np.array([[0.5, 0.5, 0.05]]), [0.1 ** 2], o, f, up,
                                   math.radians(10), 5, 5)
    assert abs(depth[2, 2] - 1.0) < 1e-12
    # a ball without free surface hidden inside a bigger one: culling keeps the hit
    p = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.45]])
    psi = np.array([0.2 ** 2, 0.1 ** 2])
    a, _ = O.render_depth(p, psi, o, f, up, math.radians(20), 9, 9)
    b, _ = O.render_depth(p, psi, o, f, up, math.radians(20), 9, 9, karea=[1.0, 0.0])
    np.testing.assert_array_equal(a, b)


def test_volume_closed_forms():
    """The oracle's volume traversal: a lone ball along the axis is crossed
    over its diameter, and off the axis over the chord 2 sqrt(r^2 - b^2)
    (b the ray's distance from the centre); two disjoint balls add their
    chords and the last exit is the far one's; two overlapping balls on the
    axis give the length of their union, r1 + r2 + (their centres' distance);
    a ball cut by the box face is crossed from the face; a ray missing
    everything has no entry."""
    o, f, up = (0.5, 0.5, -1.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)
    r = 0.2
    first, thick, last = O.render_volume(np.array([[0.5, 0.5, 0.5]]), [r * r], o, f, up,
                                         math.radians(30), 41, 31)
    assert abs(first[15, 20] - 1.3) < 1e-12 and abs(thick[15, 20] - 0.4) < 1e-12
    assert abs(last[15, 20] - 1.7) < 1e-12
    d = O.camera_rays(o, f, up, math.radians(30), 41, 31)
    e = np.array([0.5, 0.5, 0.5]) - np.asarray(o)
    bb = d @ e
    b2 = np.sum(e * e) - bb * bb
    hit = b2 < r * r - 1e-12
    np.testing.assert_allclose(thick[hit], 2 * np.sqrt(r * r - b2[hit]), rtol=0, atol=1e-12)
    assert np.all(thick[~hit & (b2 > r * r + 1e-12)] == 0.0)
    assert np.all(first[thick == 0.0] == -1.0)
    # two disjoint balls on the axis
    p = np.array([[0.5, 0.5, 0.3], [0.5, 0.5, 0.75]])
    first, thick, last = O.render_volume(p, [0.1 ** 2, 0.05 ** 2], o, f, up, math.radians(10), 5, 5)
    assert abs(thick[2, 2] - 0.3) < 1e-12 and abs(first[2, 2] - 1.2) < 1e-12
    assert abs(last[2, 2] - 1.8) < 1e-12
    # overlapping balls on the axis: union = r1 + r2 + distance
    p = np.array([[0.5, 0.5, 0.4], [0.5, 0.5, 0.55]])
    _, thick, last = O.render_volume(p, [0.1 ** 2, 0.08 ** 2], o, f, up, math.radians(10), 5, 5)
    assert abs(thick[2, 2] - (0.1 + 0.08 + 0.15)) < 1e-12 and abs(last[2, 2] - 1.63) < 1e-12
    # a ball sticking out of the box face z = 0
    first, thick, _ = O.render_volume(np.array([[0.5, 0.5, 0.05]]), [0.1 ** 2], o, f, up,
                                      math.radians(10), 5, 5)
    assert abs(first[2, 2] - 1.0) < 1e-12 and abs(thick[2, 2] - 0.15) < 1e-12


def test_smooth_single_ball_is_the_ball():
    """One ball has no neighbours: its smoothed surface is its sphere, so
    sphere tracing stops within the hit tolerance of the exact entry, with
    the sphere's normal; rays outside the silhouette miss."""
    o, f, up = (0.5, 0.5, -1.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)
    p = np.array([[0.5, 0.5, 0.5]])
    r, k = 0.2, 0.02
    depth, normal, steps = O.render_smooth(p, [r * r], o, f, up, math.radians(30), 21, 15, k)
    ref, refn = O.render_depth(p, [r * r], o, f, up, math.radians(30), 21, 15)
    hit = ref >= 0
    assert np.array_equal(depth >= 0, hit)
    d = O.camera_rays(o, f, up, math.radians(30), 21, 15)
    cos = -np.sum(d * refn, axis=2)  # ray against the outward normal
    # the march stops where f <= 1e-3 k: before the sphere by at most that / cos
    gap = ref[hit] - depth[hit]
    assert np.all(gap >= -1e-12) and np.all(gap <= O.SMOOTH_HIT * k / cos[hit] + 1e-12)
    np.testing.assert_allclose(normal[hit], refn[hit], atol=2e-3)
    assert steps.max() < O.SMOOTH_MAX_STEPS


def test_smooth_bridge_between_two_balls():
    """Two equal overlapping balls (centres at x = 0.5 -/+ a) are Laguerre
    neighbours.  On their mid plane both distances are D - r (D from either
    centre), so the cubic smooth union is D - r - k/6: a ray in that plane
    meets the surface where D = r + k/6 -- the bridge the smoothing adds
    above the crease of the two spheres (a closed form)."""
    a, r, k = 0.06, 0.1, 0.03
    p = np.array([[0.5 - a, 0.5, 0.5], [0.5 + a, 0.5, 0.5]])
    psi = np.array([r * r, r * r])
    for y0 in (0.0, 0.02, 0.04):
        o = (0.5, 0.5 + y0, 1.5)  # straight down, in the plane x = 0.5
        depth, normal, _ = O.render_smooth(p, psi, o, (0.0, 0.0, -1.0), (0.0, 1.0, 0.0),
                                           math.radians(10), 1, 1, k)
        zc = math.sqrt((r + k / 6) ** 2 - a * a - y0 * y0)
        t_exact = 1.0 - zc
        cos = zc / (r + k / 6)
        assert -1e-12 <= t_exact - depth[0, 0] <= O.SMOOTH_HIT * k / cos + 1e-12
        # the normal is the bisector of the two spheres' normals: no x part
        n_exact = np.array([0.0, y0, zc]) / math.hypot(y0, zc)
        np.testing.assert_allclose(normal[0, 0], n_exact, atol=1e-2)
        # the union of the balls alone (the crease, D = r) lies below
        assert 1.0 - math.sqrt(r * r - a * a - y0 * y0) > t_exact + 0.1 * k


def test_smooth_small_k_is_the_union():
    """As k goes to 0 the smooth union tends to the union of the balls: on
    a random cloud the hits agree with the first-hit oracle."""
    rng = np.random.default_rng(5)
    n = 60
    pos = rng.uniform(0.3, 0.7, (n, 3))
    psi = rng.uniform(0.04, 0.08, n) ** 2
    o, f, up = (0.5, 0.5, -0.5), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)
    k = 1e-5
    depth, _, steps = O.render_smooth(pos, psi, o, f, up, math.radians(30), 24, 18, k)
    ref, _ = O.render_depth(pos, psi, o, f, up, math.radians(30), 24, 18)
    both = (depth >= 0) & (ref >= 0)
    assert np.mean((depth >= 0) == (ref >= 0)) > 0.99
    assert np.max(np.abs(depth[both] - ref[both])) < 1e-4

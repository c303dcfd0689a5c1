"""First hit of camera rays on the fluid (pot_render_depth) against the
oracle's brute force over all balls, on a small splash in the middle of its
impact: hit or miss agree except on grazing rays, depths and normals agree
to FP32 precision, and skipping the balls of cells without free surface
changes nothing."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import pot, scenes

from _cmp import to_np

pytestmark = pytest.mark.gpu


def test_render_matches_oracle():
    sc = scenes.splash(spacing=0.02, seed=3)
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for _ in range(20):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    karea = pot.lgc_compute_cells(ctx, pos, psi, nu, hessian=False)["karea"]
    cam = dict(origin=(0.5, -0.9, 0.8), forward=(0.0, 1.0, -0.55), up=(0.0, 0.0, 1.0),
               fov_y=math.radians(40), width=96, height=72)
    depth, normal = pot.render_depth(ctx, pos, psi, karea=karea, **cam)
    depth_all, _ = pot.render_depth(ctx, pos, psi, **cam)
    x, s = to_np(pos).astype(np.float64), to_np(psi).astype(np.float64)
    ref_d, ref_n = O.render_depth(x, s, **cam)
    gd, gn = to_np(depth).astype(np.float64), to_np(normal).astype(np.float64)
    hit, ref_hit = gd >= 0, ref_d >= 0
    assert ref_hit.mean() > 0.1 and (~ref_hit).mean() > 0.1  # the fluid and the background
    # hit or miss: only grazing rays may differ (FP32 ray-sphere discriminants near 0)
    assert np.mean(hit != ref_hit) < 2e-3, np.mean(hit != ref_hit)
    both = hit & ref_hit
    # depth: FP32 rounding of the offset r^2 - |h|^2 is amplified by its
    # square root on grazing rays
    err = np.abs(gd[both] - ref_d[both]) / float(ref_d.max())
    assert np.percentile(err, 99) < 2e-5 and err.max() < 1e-3, (np.percentile(err, 99), err.max())
    # normals: unit, and equal to the oracle's where the same sphere was hit
    assert np.all(np.abs(np.linalg.norm(gn[both], axis=1) - 1) < 1e-3)
    same = np.sum(gn[both] * ref_n[both], axis=1) > 0.999
    assert same.mean() > 0.99
    # culling by the free-surface area keeps the first hit (up to cells whose
    # sliver of free surface the FP32 evaluation rounds to none)
    ga = to_np(depth_all).astype(np.float64)
    assert np.mean(np.abs(gd - ga) > 1e-6) < 2e-3
    ctx.close()


def test_volume_traversal_matches_oracle():
    """Cell-by-cell traversal of the fluid (pot_render_volume, Sec. 6) on the
    same small splash during its impact against the oracle's union of the
    balls' intervals along each ray: the length inside the fluid, the first
    entry and the last exit agree to FP32 precision except on rays that
    graze a sphere, where an FP32 discriminant near 0 decides hit or miss."""
    sc = scenes.splash(spacing=0.02, seed=3)
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for _ in range(20):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    for cam in (dict(origin=(0.5, -0.9, 0.8), forward=(0.0, 1.0, -0.55), up=(0.0, 0.0, 1.0),
                     fov_y=math.radians(40), width=96, height=72),
                dict(origin=(-0.6, 0.5, 0.5), forward=(1.0, 0.02, 0.01), up=(0.0, 0.0, 1.0),
                     fov_y=math.radians(30), width=80, height=60)):
        first, thick, last, visits = pot.render_volume(ctx, pos, psi, **cam)
        x, s = to_np(pos).astype(np.float64), to_np(psi).astype(np.float64)
        rf, rt, rl = O.render_volume(x, s, **cam)
        gf, gt, gl = (to_np(a).astype(np.float64) for a in (first, thick, last))
        hit, ref_hit = gf >= 0, rf >= 0
        assert ref_hit.mean() > 0.1 and (~ref_hit).mean() > 0.1
        assert np.mean(hit != ref_hit) < 2e-3, np.mean(hit != ref_hit)
        both = hit & ref_hit
        scale = float(rt.max())
        et = np.abs(gt - rt)[both] / scale
        el = np.abs(gl - rl)[both] / float(rl.max())
        print("volume traversal: thickness err / max p50 %.2e p99 %.2e max %.2e; last exit p99 %.2e;"
              " cells per ray max %d mean %.1f" % (np.median(et), np.percentile(et, 99), et.max(),
                                                   np.percentile(el, 99), int(to_np(visits).max()),
                                                   float(to_np(visits)[both].mean())))
        assert np.percentile(et, 99) < 1e-4 and np.percentile(el, 99) < 1e-4
        assert np.mean(et > 1e-3) < 5e-3
        assert int(to_np(visits).max()) < 1 << 15  # no walk ran out of visits
    ctx.close()


def test_volume_traversal_full_size_sampled():
    """The traversal on the 2.0M-site splash after 30 steps (the balls
    pressed together), 320 x 180 rays from bench.py's render camera: no walk
    runs out of visits, and on 200 sampled rays that reach the fluid the
    length inside it, first entry and last exit agree with the oracle's
    union of the balls' intervals over all 2M balls."""
    sc = scenes.splash()
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for _ in range(30):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    cam = dict(origin=(0.5, -0.9, 0.8), forward=(0.0, 1.0, -0.55), up=(0.0, 0.0, 1.0),
               fov_y=math.radians(40), width=320, height=180)
    first, thick, last, visits = pot.render_volume(ctx, pos, psi, **cam)
    gf, gt, gl = (to_np(a).astype(np.float64).ravel() for a in (first, thick, last))
    vis = to_np(visits).ravel()
    assert vis.max() < 1 << 15
    hit = np.nonzero(gf >= 0)[0]
    assert hit.size > 1000
    pix = np.random.default_rng(7).choice(hit, 200, replace=False)
    x, s = to_np(pos).astype(np.float64), to_np(psi).astype(np.float64)
    rf, rt, rl = O.render_volume(x, s, pixels=pix, **cam)
    assert np.all(rf >= 0)
    et = np.abs(gt[pix] - rt) / float(rt.max())
    ef = np.abs(gf[pix] - rf) / float(rl.max())
    el = np.abs(gl[pix] - rl) / float(rl.max())
    print("full-size traversal: thickness err / max p99 %.2e max %.2e; first p99 %.2e; last p99 %.2e;"
          " cells per ray max %d" % (np.percentile(et, 99), et.max(), np.percentile(ef, 99),
                                     np.percentile(el, 99), int(vis.max())))
    assert np.percentile(et, 99) < 1e-4 and np.percentile(el, 99) < 1e-4 and np.percentile(ef, 99) < 1e-5
    ctx.close()


def test_smooth_surface_matches_oracle():
    """Sphere tracing of the smoothed free surface (pot_render_smooth, Sec.
    6) on the small splash during its impact, smoothing radius half a
    spacing, against the oracle's march over all balls with its own FP64
    cells: hit or miss agree except on rays that graze the surface or cross
    where the closest site changes (f jumps there), depths agree to the
    march's stopping tolerance, normals to FP32 precision."""
    sc = scenes.splash(spacing=0.02, seed=3)
    n = sc.n
    dev = torch.device("cuda", 0)
    ctx = pot.Context(n, 246, 0, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for _ in range(20):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    k = 0.5 * 0.02
    cam = dict(origin=(0.5, -0.9, 0.8), forward=(0.0, 1.0, -0.55), up=(0.0, 0.0, 1.0),
               fov_y=math.radians(40), width=64, height=48)
    depth, normal, steps = pot.render_smooth(ctx, pos, psi, k=k, **cam)
    x, s = to_np(pos).astype(np.float64), to_np(psi).astype(np.float64)
    rd, rn, rs = O.render_smooth(x, s, k=k, **cam)
    gd, gn, gs = (to_np(a).astype(np.float64) for a in (depth, normal, steps))
    hit, ref_hit = gd >= 0, rd >= 0
    assert ref_hit.mean() > 0.1 and (~ref_hit).mean() > 0.1
    disagree = np.mean(hit != ref_hit)
    both = hit & ref_hit
    scale = float(rd.max())
    err = np.abs(gd - rd)[both] / scale
    dots = np.sum(gn[both] * rn[both], axis=1)
    print("smooth surface: hit disagreement %.2e; depth err / max p50 %.2e p99 %.2e max %.2e;"
          " normal dot p1 %.5f; steps max %d mean %.1f (oracle %d %.1f)"
          % (disagree, np.median(err), np.percentile(err, 99), err.max(), np.percentile(dots, 1),
             gs.max(), gs.mean(), rs.max(), rs.mean()))
    assert disagree < 1e-2
    # the march stops within 1e-3 k of f = 0 on both sides
    assert np.percentile(err, 99) < 1e-3 * k / scale * 20
    assert np.mean(err > 1e-2) < 1e-2  # a jump of the closest site may move a few hits
    assert np.all(np.abs(np.linalg.norm(gn[both], axis=1) - 1) < 1e-3)
    assert np.mean(dots > 0.99) > 0.98
    assert np.mean(gs >= 1024) < 1e-2
    # the smoothing only adds fluid: every ray that meets the balls meets
    # the smoothed surface no later
    d0, _ = pot.render_depth(ctx, pos, psi, **cam)
    g0 = to_np(d0).astype(np.float64)
    ok = (g0 >= 0) & hit
    assert np.mean(g0 >= 0) <= np.mean(hit) + 1e-3
    assert np.mean(gd[ok] > g0[ok] + 1e-4 * scale) < 1e-2
    ctx.close()

"""Seeded synthetic scenes shared by the oracle tests, the GPU tests and bench.py.

This module only draws inputs: site positions, initial weights psi0, target
volumes nu and velocities.  It holds none of the method's arithmetic (no cell
geometry, no Newton, no fluid update), so both the FP64 CPU oracle and the
CUDA path can consume the same arrays without sharing code.

Every generator draws with numpy ``default_rng(seed)`` (PCG64) in float64 in
a fixed order, then casts positions and weights to float32.  The float32
values are the inputs of record: the oracle widens exactly these float32
numbers to float64, so both sides see bit-identical sites and weights.

The domain is always the unit box [0,1]^3 and gravity points along -z.
The scene shapes restate the paper's workloads synthetically (Sec. 7): a
jittered block solved once, a random cloud of balls for the cell kernel, a
dam-break column and a two-ball splash at the teaser's 2M scale.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DOMAIN_LO = (0.0, 0.0, 0.0)
DOMAIN_HI = (1.0, 1.0, 1.0)
GRAVITY = (0.0, 0.0, -9.81)


@dataclasses.dataclass
class Scene:
    """A set of weighted sites in the unit box.

    pos: (n,3) float32 site positions p_i.
    psi: (n,) float32 weights psi_i (ball radius sqrt(psi_i)).
    nu:  (n,) float64 prescribed volumes nu_i.
    vel: (n,3) float32 velocities (zeros unless the scene moves).
    name: workload name with its sizes.
    """

    pos: np.ndarray
    psi: np.ndarray
    nu: np.ndarray
    vel: np.ndarray
    name: str
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _ball_radius_for_volume(nu: np.ndarray) -> np.ndarray:
    # radius of the ball whose volume is nu: input recipe for psi0 only
    return (3.0 * nu / (4.0 * math.pi)) ** (1.0 / 3.0)


def jittered_block(n_side: int = 10, spacing: float = 0.05, jitter: float = 0.3,
                   seed: int = 0, fill: float = 0.9, r_factor: float = 0.8) -> Scene:
    """Jittered cubic block of n_side^3 sites filling [0, n_side*spacing]^3.

    Lattice index i = ix + n_side*iy + n_side^2*iz; position
    (ix+0.5, iy+0.5, iz+0.5)*spacing + U(-jitter, jitter)^3 * spacing with one
    (n,3) draw from default_rng(seed).  Targets nu_i = fill*spacing^3, initial
    weights psi_i = (r_factor * radius(nu_i))^2.  With the defaults this is the
    1000-site single-solve case (block [0,0.5]^3 in the unit box).
    """
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    iz, iy, ix = np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side), indexing="ij")
    lat = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    jit = rng.uniform(-jitter, jitter, size=(n, 3))
    pos = ((lat + 0.5) + jit) * spacing
    nu = np.full(n, fill * spacing ** 3, dtype=np.float64)
    r = r_factor * _ball_radius_for_volume(nu)
    return Scene(pos=pos.astype(np.float32), psi=(r * r).astype(np.float32), nu=nu,
                 vel=np.zeros((n, 3), np.float32), name=f"jittered_block_{n}")


def uniform_cloud(n: int = 1 << 20, seed: int = 1, subset: int = 10000,
                  subset_seed: int = 1001) -> Scene:
    """n sites uniform in [0,1]^3 with radii r_i = f_i * R0, f_i ~ U(0.4, 1.2).

    R0 = (3/(4 pi n))^(1/3); psi_i = r_i^2 rounded to float32; nu_i = 0.5/n.
    Positions are drawn first, then the factors, from the same generator.
    extra['subset'] holds `subset` distinct indices from default_rng(subset_seed)
    for checks against the oracle.
    """
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n, 3))
    f = rng.uniform(0.4, 1.2, size=n)
    r0 = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r = f * r0
    nu = np.full(n, 0.5 / n, dtype=np.float64)
    sub = np.random.default_rng(subset_seed).choice(n, size=min(subset, n), replace=False)
    return Scene(pos=pos.astype(np.float32), psi=(r * r).astype(np.float32), nu=nu,
                 vel=np.zeros((n, 3), np.float32), name=f"uniform_cloud_{n}",
                 extra={"subset": np.sort(sub).astype(np.int64), "R0": r0})


# Dam break: fluid step dt = 2e-3; spring length eps = s / 8 keeps the
# front (about 2 sqrt(g H) = 5.6 m/s for the 0.8 m column) below the
# spring's signal speed s / eps, and each step is taken as substeps of about
# eps / 2.
DAM_DT = 2e-3
DAM_EPS_PER_SPACING = 1.0 / 8.0
DAM_RELAX_ROUNDS = 3


def dam_break(nx: int = 63, ny: int = 63, nz: int = 126, width: float = 0.4,
              jitter: float = 0.3, seed: int = 2, fill: float = 0.9,
              r_factor: float = 0.8) -> Scene:
    """Jittered column nx*ny*nz of spacing s = width/nx filling
    [0,width]x[0,width*ny/nx]x[0,s*nz] (z up); nu = fill*s^3, psi0 as jittered_block.

    The defaults give 63x63x126 = 500,094 sites in a 0.4 x 0.4 x 0.8 column.
    extra holds the recipe's step dt, spring length eps, substeps per step
    and the rounds that move the sites to their cell centroids first.
    """
    rng = np.random.default_rng(seed)
    s = width / nx
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lat = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    n = lat.shape[0]
    jit = rng.uniform(-jitter, jitter, size=(n, 3))
    pos = ((lat + 0.5) + jit) * s
    nu = np.full(n, fill * s ** 3, dtype=np.float64)
    r = r_factor * _ball_radius_for_volume(nu)
    eps = DAM_EPS_PER_SPACING * s
    return Scene(pos=pos.astype(np.float32), psi=(r * r).astype(np.float32), nu=nu,
                 vel=np.zeros((n, 3), np.float32), name=f"dam_break_{n}",
                 extra={"spacing": s, "dt": DAM_DT, "eps": eps,
                        "substeps": max(1, int(round(DAM_DT / (0.5 * eps)))),
                        "relax_rounds": DAM_RELAX_ROUNDS})


# Spring length and time step of the splash, in units of its lattice spacing
# s: eps = s / 16 puts each ball's 3 m/s at 0.19 of the spring's signal speed
# s / eps, and dt = eps / 2 takes 2 steps per radian of the spring's
# oscillation.  Both scale with s, so every resolution of the recipe sees the
# same number of steps to contact and the same impact relative to the spring.
SPLASH_EPS_PER_SPACING = 1.0 / 16.0
SPLASH_DT_PER_EPS = 0.5
SPLASH_RELAX_ROUNDS = 3


def splash(spacing: float = 3.224e-3, radius: float = 0.2, speed: float = 3.0,
           jitter: float = 0.3, seed: int = 3, fill: float = 0.9,
           r_factor: float = 0.8, gap: float = 2.0, centers=None) -> Scene:
    """Two balls of jittered lattice sites flying at each other along x.

    The balls are centred at (0.5 -/+ (radius + gap*spacing/2), 0.5, 0.5)
    unless `centers` is given: their surfaces start gap spacings apart and,
    closing at 2*speed, touch after about gap*spacing/(2*speed*dt) steps
    (10 with the recipe's dt).  Lattice points (k+0.5)*spacing whose
    unjittered position lies inside a ball of the given radius around each
    centre are kept; then every kept site is jittered by
    U(-jitter, jitter)^3*spacing (one draw, default_rng(seed)).  Ball 0 moves
    with (+speed,0,0), ball 1 with (-speed,0,0).  nu = fill*s^3, psi0 as
    jittered_block.  extra holds the recipe's spring length eps, time step dt
    and the number of rounds that move the sites to their cell centroids
    before the first step (the spring's rest state).  The defaults give about
    2.0M sites.
    """
    rng = np.random.default_rng(seed)
    if centers is None:
        off = radius + 0.5 * gap * spacing
        centers = ((0.5 - off, 0.5, 0.5), (0.5 + off, 0.5, 0.5))
    parts, vels = [], []
    for b, c in enumerate(centers):
        c = np.asarray(c, np.float64)
        lo = np.floor((c - radius) / spacing).astype(int)
        hi = np.ceil((c + radius) / spacing).astype(int)
        axes = [np.arange(lo[k], hi[k] + 1) for k in range(3)]
        gz, gy, gx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        pts = (np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64) + 0.5) * spacing
        keep = np.sum((pts - c) ** 2, axis=1) < radius * radius
        pts = pts[keep]
        parts.append(pts)
        v = np.zeros_like(pts)
        v[:, 0] = speed if b == 0 else -speed
        vels.append(v)
    pos = np.concatenate(parts)
    vel = np.concatenate(vels)
    n = pos.shape[0]
    pos = pos + rng.uniform(-jitter, jitter, size=(n, 3)) * spacing
    nu = np.full(n, fill * spacing ** 3, dtype=np.float64)
    r = r_factor * _ball_radius_for_volume(nu)
    eps = SPLASH_EPS_PER_SPACING * spacing
    return Scene(pos=pos.astype(np.float32), psi=(r * r).astype(np.float32), nu=nu,
                 vel=vel.astype(np.float32), name=f"splash_{n}",
                 extra={"spacing": spacing, "eps": eps, "dt": SPLASH_DT_PER_EPS * eps,
                        "relax_rounds": SPLASH_RELAX_ROUNDS})


def explosion(spacing: float = 8.3e-3, radius: float = 0.3, speed: float = 5.0,
              jitter: float = 0.3, seed: int = 5, fill: float = 0.9,
              r_factor: float = 0.8) -> Scene:
    """A ball of fluid flying apart into the walls (the paper's robustness
    case, Sec. 7: cells start as a sphere with a strong outward velocity and
    hit the domain boundary).

    Lattice points (k+0.5)*spacing inside the ball of the given radius
    around (0.5, 0.5, 0.5), jittered by U(-jitter, jitter)^3*spacing (one
    draw, default_rng(seed)); velocity speed*(x - c)/radius (radial, speed
    at the surface); nu = fill*s^3, psi0 as jittered_block.  extra: spring
    length eps = s/8 (the surface speed is 0.6 of the spring's signal speed
    s/eps = 8 m/s), step dt = eps/2 and 3 rounds of sites moved to their
    cell centroids first.  The surface reaches the walls (0.2 away) near
    step 77 of 100.  The defaults give about 200k sites.
    """
    rng = np.random.default_rng(seed)
    c = np.array([0.5, 0.5, 0.5])
    lo = np.floor((c - radius) / spacing).astype(int)
    hi = np.ceil((c + radius) / spacing).astype(int)
    axes = [np.arange(lo[k], hi[k] + 1) for k in range(3)]
    gz, gy, gx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    pts = (np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64) + 0.5) * spacing
    pts = pts[np.sum((pts - c) ** 2, axis=1) < radius * radius]
    n = pts.shape[0]
    vel = speed * (pts - c) / radius
    pos = pts + rng.uniform(-jitter, jitter, size=(n, 3)) * spacing
    nu = np.full(n, fill * spacing ** 3, dtype=np.float64)
    r = r_factor * _ball_radius_for_volume(nu)
    eps = spacing / 8.0
    return Scene(pos=pos.astype(np.float32), psi=(r * r).astype(np.float32), nu=nu,
                 vel=vel.astype(np.float32), name=f"explosion_{n}",
                 extra={"spacing": spacing, "eps": eps, "dt": 0.5 * eps, "relax_rounds": 3})


def random_subset(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted indices out of n from default_rng(seed)."""
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False)).astype(np.int64)

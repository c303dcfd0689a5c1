"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this module.  It shares no code with the CUDA path (the product
package never imports it).  Everything runs in float64 on the host.

Contents, each citing the paper passage it follows:
  cells()         generalized Laguerre cells: volume, free-surface area,
                  restricted facet areas, centroid (Eq. 1, Sec. 3.2-3.4,
                  Algorithm 2) -- computed by oracle/lgc_oracle.c.
  hessian_dense() the Hessian of Eq. 2 as M = -grad^2 K (sign flipped so that
                  M is symmetric positive definite), dense.
  newton()        Algorithm 1: damped Newton with KMT steps, dense direct solve.
  repair_empty()  raise the weights of empty cells until each site is inside
                  its own cell, before Algorithm 1 (not in the paper: its
                  precondition, no empty cell at the start, made to hold).
  fluid_step()    Gallouet-Merigot step of Sec. 5 (pressure spring, gravity,
                  symplectic update); with viscosity or surface tension the
                  semi-implicit velocity solve of Eq. 4 over the P1
                  Laplacian of Eq. 3 (laplacian_weights, viscous_velocity),
                  with the walls' terms of Sec. 5 (wall_weights,
                  wall_tension).
  render_depth()  first point of each camera ray inside the fluid (the union
                  of the balls inside the box), with the free-surface culling
                  of Sec. 6's first-cell search; brute force over all balls.
  render_volume() the fluid along each camera ray (Sec. 6's volume
                  traversal): first entry, length inside, last exit, from the
                  union of the balls' intervals; brute force.
  render_smooth() sphere tracing of the smoothed free surface (Sec. 6's
                  surface smoothing): the cubic smooth union over the
                  nearest sphere's Laguerre neighbourhood; brute force.
  mlp_*()         FP64 reference of the learned warm-start MLP (not in the
                  paper): forward, backward, Adam, on BF16-rounded operands.

Parity pins: tests/test_oracle_geometry.py, tests/test_oracle_newton.py,
tests/test_oracle_mlp.py, tests/test_oracle_render.py (closed forms, Monte
Carlo, finite differences, invariants).  Functions without such a pin say "parity unpinned" below.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

STATUS_OK = 0
STATUS_TOO_MANY_FACETS = 1
STATUS_COINCIDENT = 2


def build(force: bool = False) -> str:
    """Compile lgc_oracle.c (gcc -O2 -fopenmp, no fast-math) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_cells.restype = ctypes.c_int
        lib.oracle_cells.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64, P, ctypes.c_int,
                                     ctypes.c_int] + [P] * 13 + [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def cells(pos, psi, query=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), brute=False,
          max_facets=128, nthreads=0):
    """Generalized Laguerre cells of the sites `query` (default: all).

    pos (n,3), psi (n,) are widened to float64 exactly.  Returns a dict:
      vol, karea (free-surface |K_i|), omega_sum, inside, n_planes, cen (q,3),
      status, wall_area (q,6), nfac, fac_j, fac_area, fac_dist, fac_h (q,max_facets)
    fac_* list every bisector plane that cuts the ball (area may be 0).
    """
    lib = _load()
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape(-1))
    n = pos.shape[0]
    if query is None:
        query = np.arange(n, dtype=np.int64)
    query = np.ascontiguousarray(np.asarray(query, dtype=np.int64))
    q = query.shape[0]
    lo = np.ascontiguousarray(np.asarray(lo, np.float64))
    hi = np.ascontiguousarray(np.asarray(hi, np.float64))
    out = {
        "vol": np.zeros(q), "karea": np.zeros(q), "omega_sum": np.zeros(q),
        "inside": np.zeros(q, np.int32), "n_planes": np.zeros(q, np.int32),
        "cen": np.zeros((q, 3)), "status": np.zeros(q, np.int32), "wall_area": np.zeros((q, 6)),
        "nfac": np.zeros(q, np.int32), "fac_j": np.full((q, max_facets), -1, np.int64),
        "fac_area": np.zeros((q, max_facets)), "fac_dist": np.zeros((q, max_facets)),
        "fac_h": np.zeros((q, max_facets)),
    }
    lib.oracle_cells(n, _p(pos), _p(psi), _p(lo), _p(hi), q, _p(query), int(brute), int(max_facets),
                     _p(out["vol"]), _p(out["karea"]), _p(out["omega_sum"]), _p(out["inside"]),
                     _p(out["n_planes"]), _p(out["cen"]), _p(out["status"]), _p(out["wall_area"]),
                     _p(out["nfac"]), _p(out["fac_j"]), _p(out["fac_area"]), _p(out["fac_dist"]),
                     _p(out["fac_h"]), int(nthreads))
    out["query"] = query
    return out


def hessian_entries(res, psi, query=None):
    """Rows of M = -grad^2 K (Eq. 2 with the sign flipped):
    M_ij = -|B_ij| / (2 d_ij) for bisector facets with |B_ij| > 0,
    M_ii = sum_j |B_ij| / (2 d_ij) + |K_i| / (2 sqrt(psi_i)).
    Returns (diag (q,), list of (cols int64 ascending, vals float64) per row)."""
    psi = np.asarray(psi, np.float64)
    q = res["vol"].shape[0]
    query = res["query"] if query is None else query
    diag = np.zeros(q)
    rows = []
    for k in range(q):
        nf = int(res["nfac"][k])
        j = res["fac_j"][k, :nf]
        a = res["fac_area"][k, :nf]
        d = res["fac_dist"][k, :nf]
        keep = a > 0.0
        j, a, d = j[keep], a[keep], d[keep]
        off = a / (2.0 * d)
        ps = psi[query[k]]
        kterm = res["karea"][k] / (2.0 * math.sqrt(ps)) if ps > 0 else 0.0
        diag[k] = off.sum() + kterm
        order = np.argsort(j)
        rows.append((j[order], -off[order]))
    return diag, rows


def hessian_dense(res, psi):
    """Dense M (n,n) for a full evaluation (query = all sites)."""
    n = res["vol"].shape[0]
    diag, rows = hessian_entries(res, psi)
    m = np.zeros((n, n))
    for i in range(n):
        m[i, i] = diag[i]
        cols, vals = rows[i]
        m[i, cols] = vals
    return m


class NewtonResult:
    def __init__(self, psi, vol, iters, halvings, status, history, res):
        self.psi = psi
        self.vol = vol
        self.iters = iters
        self.halvings = halvings
        self.status = status
        self.history = history
        self.res = res


NEWTON_OK = 0
NEWTON_NOT_CONVERGED = 1
NEWTON_LINESEARCH_FAILED = 2
NEWTON_EMPTY_CELL_AT_START = 3


def repair_empty(pos, psi, vol, nu):
    """Raise the weight of every empty cell i to
    max(max_j (psi_j - d_ij^2) + 0.25 d*^2, (nu_i^(1/3) / 2)^2), d* the distance
    to the maximising site: then every bisector of i has h_ij > 0, so p_i is
    inside its own (non-empty) cell, and each neighbour j keeps h_ji > 0
    (reading: Algorithm 1 needs a start without empty cells; the paper does
    not say how to get one after a fast step).  Brute force over all sites."""
    pos = np.asarray(pos, np.float64)
    psi = np.asarray(psi, np.float64).copy()
    new = psi.copy()
    for i in np.nonzero(np.asarray(vol) <= 0.0)[0]:
        d2 = np.sum((pos - pos[i]) ** 2, 1)
        v = psi - d2
        v[i] = -np.inf
        j = int(np.argmax(v))
        cand = psi[i]
        if d2[j] > 0 and np.isfinite(v[j]):
            cand = max(cand, v[j] + 0.25 * d2[j])
        new[i] = max(cand, 0.25 * np.cbrt(nu[i]) ** 2)
    return new


def newton(pos, nu, psi0, tol=1e-4, max_newton=100, max_halvings=30,
           lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), nthreads=0, repair=False):
    """Algorithm 1 (damped Newton with KMT steps), dense direct solve.

    Readings (Algorithm 1 is garbled in the paper: its inner loop halves while
    the volumes are large and omits KMT's decrease condition):
      - start from the given psi0 > 0, not psi = 0 (psi = 0 gives empty cells);
      - Newton system M u = nu - V(psi), M = -grad^2 K (Eq. 2);
      - stop when max_i |V_i - nu_i| / nu_i <= tol (relative worst-cell error, Sec. 7);
      - KMT step: alpha = 1, 1/2, ... until min V(psi + alpha u) >= eps0 and
        ||nu - V(psi + alpha u)||_2 <= (1 - alpha/2) ||nu - V(psi)||_2,
        eps0 = 1/2 min(min nu, min V(psi0)); at most max_halvings halvings.
    """
    pos = np.asarray(pos, np.float64)
    nu = np.asarray(nu, np.float64)
    psi = np.asarray(psi0, np.float64).copy()
    res = cells(pos, psi, lo=lo, hi=hi, nthreads=nthreads)
    vol = res["vol"]
    for _ in range(32 if repair else 0):
        if vol.min() > 0.0:
            break
        psi = repair_empty(pos, psi, vol, nu)
        res = cells(pos, psi, lo=lo, hi=hi, nthreads=nthreads)
        vol = res["vol"]
    if vol.min() <= 0.0:
        return NewtonResult(psi, vol, 0, 0, NEWTON_EMPTY_CELL_AT_START, [], res)
    eps0 = 0.5 * min(nu.min(), vol.min())
    history = []
    halv_total = 0
    for it in range(max_newton + 1):
        g = nu - vol
        err = float(np.max(np.abs(g) / nu))
        history.append(err)
        if err <= tol:
            return NewtonResult(psi, vol, it, halv_total, NEWTON_OK, history, res)
        if it == max_newton:
            break
        m = hessian_dense(res, psi)
        u = np.linalg.solve(m, g)
        gnorm = float(np.linalg.norm(g))
        alpha = 1.0
        accepted = False
        for _ in range(max_halvings + 1):
            pt = psi + alpha * u
            rt = cells(pos, pt, lo=lo, hi=hi, nthreads=nthreads)
            vt = rt["vol"]
            # KMT: a sufficient decrease of the l2 norm of the gradient
            if vt.min() >= eps0 and np.linalg.norm(nu - vt) <= (1.0 - 0.5 * alpha) * gnorm:
                accepted = True
                break
            alpha *= 0.5
            halv_total += 1
        if not accepted:
            return NewtonResult(psi, vol, it, halv_total, NEWTON_LINESEARCH_FAILED, history, res)
        psi, res, vol = pt, rt, vt
    return NewtonResult(psi, vol, max_newton, halv_total, NEWTON_NOT_CONVERGED, history, res)


def advect_and_clamp(pos, vel, dt, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), margin=1e-6):
    """First half of the fluid step (Sec. 5, numerical integration):
    x^{k+1} = x^k + dt v^k, then clamp into [lo+margin, hi-margin] and zero the
    velocity component that pointed through the wall (reading: the paper leaves
    wall handling unstated)."""
    x = np.asarray(pos, np.float64) + dt * np.asarray(vel, np.float64)
    v = np.asarray(vel, np.float64).copy()
    lo = np.asarray(lo, np.float64) + margin
    hi = np.asarray(hi, np.float64) - margin
    below = x < lo
    above = x > hi
    x = np.where(below, lo, np.where(above, hi, x))
    v = np.where(below & (v < 0), 0.0, v)
    v = np.where(above & (v > 0), 0.0, v)
    return x, v


def velocity_update(x1, v, cen, dt, eps=0.01, g=(0.0, 0.0, -9.81)):
    """v^{k+1} = v + dt (g + (c_i - x_i)/eps^2): Gallouet-Merigot pressure spring
    F_p = (c_i - p_i)/eps^2 (Sec. 5, incompressibility) with unit mass."""
    return np.asarray(v, np.float64) + dt * (np.asarray(g, np.float64)[None, :]
                                             + (np.asarray(cen, np.float64) - x1) / (eps * eps))


def laplacian_weights(res, psi):
    """Dense weights w_ij = |B_ij| / (2 d_ij) of the P1 Laplacian (Eq. 3) over
    the restricted bisector facets of a full evaluation: the off-diagonal
    of M = -grad^2 K with its sign flipped (walls and the free surface add
    nothing)."""
    n = res["vol"].shape[0]
    _, rows = hessian_entries(res, psi)
    w = np.zeros((n, n))
    for i in range(n):
        cols, vals = rows[i]
        w[i, cols] = -vals
    return w


def wall_weights(res, pos, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Per cell, the walls' P1 Laplacian weight sum_w |B_iw| / (2 h_iw) (Eq. 3
    with the wall as the neighbour, Sec. 5's fluid-boundary term without the
    volume factor): wall facet areas over twice the site's distance to the
    wall (walls in the order -x, +x, -y, +y, -z, +z)."""
    pos = np.asarray(pos, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    h = np.stack([pos[:, 0] - lo[0], hi[0] - pos[:, 0], pos[:, 1] - lo[1], hi[1] - pos[:, 1],
                  pos[:, 2] - lo[2], hi[2] - pos[:, 2]], axis=1)
    a = res["wall_area"]
    return np.sum(np.where(a > 0, a / (2.0 * np.where(h > 0, h, np.inf)), 0.0), axis=1)


def wall_tension(res, pos, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Per cell, the walls' part of the surface-tension Laplacian of the
    positions (Sec. 5, fluid-boundary interaction): each wall facet B_iw acts
    as the facet to a neighbour placed cbrt(|V_i|) beyond the wall plane,
    with the P1 weight |B_iw| / (2 h_iw) of the boundary term (h_iw the
    site's distance to the wall), so it adds
        |B_iw| / (2 h_iw) * (h_iw + cbrt(|V_i|)) * n_w
    (n_w the wall's outward normal; walls -x, +x, -y, +y, -z, +z).  (n, 3)."""
    pos = np.asarray(pos, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    h = np.stack([pos[:, 0] - lo[0], hi[0] - pos[:, 0], pos[:, 1] - lo[1], hi[1] - pos[:, 1],
                  pos[:, 2] - lo[2], hi[2] - pos[:, 2]], axis=1)
    normals = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], float)
    a = res["wall_area"]
    cv = np.cbrt(np.maximum(res["vol"], 0.0))
    mag = np.where(a > 0, a / (2.0 * np.where(h > 0, h, np.inf)) * (h + cv[:, None]), 0.0)
    return mag @ normals


def viscous_velocity(x1, v, cen, w, dt, eps, g, mu, gamma, factors=None, wall_w=None,
                     mu_wall=0.0, wall_t=None, gamma_wall=0.0):
    """Semi-implicit velocity update with viscosity and surface tension
    (Sec. 5, Eq. 4, unit mass):
    (I/dt + (D_mu - W_mu)) v^{k+1} = v^k/dt + F_p + F_g + F_t,
    F_p = (c - x)/eps^2, F_g = g, F_t = gamma L x, (L u)_i = sum_j w_ij (u_j - u_i),
    W_mu = mu_ij w_ij with mu_ij = mu (f_i + f_j) / 2 (per-site factors f for
    several fluids, the per-pair coefficients of Sec. 5; all 1 by default),
    D_mu = diag(sum_j mu_ij w_ij); walls at rest add mu_wall * wall_w to the
    diagonal (no-slip); the walls' part of the surface tension adds
    gamma_wall * wall_t (wall_tension) to F_t; one dense solve for the three
    components."""
    x1 = np.asarray(x1, np.float64)
    n = x1.shape[0]
    f = np.ones(n) if factors is None else np.asarray(factors, np.float64)
    wm = mu * 0.5 * (f[:, None] + f[None, :]) * w
    d = w.sum(axis=1)
    lap_x = w @ x1 - d[:, None] * x1
    b = (np.asarray(v, np.float64) / dt + (np.asarray(cen, np.float64) - x1) / (eps * eps)
         + np.asarray(g, np.float64)[None, :] + gamma * lap_x)
    if wall_t is not None and gamma_wall != 0.0:
        b = b + gamma_wall * np.asarray(wall_t, np.float64)
    dw = np.zeros(n) if wall_w is None else mu_wall * np.asarray(wall_w, np.float64)
    a = np.diag(1.0 / dt + wm.sum(axis=1) + dw) - wm
    return np.linalg.solve(a, b)


def fluid_step(pos, vel, psi, nu, dt, eps=0.01, g=(0.0, 0.0, -9.81), tol=1e-4,
               max_newton=100, nthreads=0, mu=0.0, gamma=0.0, factors=None, mu_wall=0.0,
               gamma_wall=0.0):
    """One fluid step: advect + clamp, Newton at x^{k+1} warm-started from
    psi, centroids of the converged cells, velocity update -- explicit, or
    semi-implicit with viscosity mu and surface tension gamma (Eq. 4) when
    either is non-zero."""
    x1, v = advect_and_clamp(pos, vel, dt)
    nr = newton(x1, nu, psi, tol=tol, max_newton=max_newton, nthreads=nthreads)
    cen = nr.res["cen"]
    if mu == 0.0 and gamma == 0.0 and mu_wall == 0.0 and gamma_wall == 0.0:
        v1 = velocity_update(x1, v, cen, dt, eps=eps, g=g)
    else:
        w = laplacian_weights(nr.res, nr.psi)
        ww = wall_weights(nr.res, x1) if mu_wall > 0.0 else None
        wt = wall_tension(nr.res, x1) if gamma_wall != 0.0 else None
        v1 = viscous_velocity(x1, v, cen, w, dt, eps, g, mu, gamma, factors, ww, mu_wall, wt,
                              gamma_wall)
    return x1, v1, nr


# ---------------------------------------------------------------------------
# first hit of camera rays (Sec. 6, finding the first cell)


def camera_rays(origin, forward, up, fov_y, width, height):
    """Pinhole camera: unit directions (height, width, 3) of the rays through
    the pixel centres; row 0 at the top.  right = forward x up (normalised),
    the image's up = right x forward, tan of the half angles fov_y / 2 and
    that times width / height."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    tv = math.tan(0.5 * fov_y)
    th = tv * width / height
    sx = ((np.arange(width) + 0.5) / width * 2.0 - 1.0) * th
    sy = (1.0 - (np.arange(height) + 0.5) / height * 2.0) * tv
    d = f[None, None, :] + sx[None, :, None] * r[None, None, :] + sy[:, None, None] * u[None, None, :]
    return d / np.linalg.norm(d, axis=2, keepdims=True)


def render_depth(pos, psi, origin, forward, up, fov_y, width, height, karea=None,
                 lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Depth and normal of the first point of each camera ray inside the
    fluid, brute force over all balls.  The fluid (the union of the
    generalized Laguerre cells of Eq. 1) is the union of the balls inside the
    box: a point of ball j lies in the cell of the site of least power
    distance, which is inside that site's own ball.  Its first point along a
    ray lies on a sphere whose cell has a free surface, so with `karea` the
    balls of cells with |K| = 0 are skipped (the paper's free-surface
    impostors).  depth: t of the hit (-1 when none); normal: unit outward
    normal of the hit sphere (0 when none)."""
    pos = np.asarray(pos, np.float64)
    psi = np.asarray(psi, np.float64)
    o = np.asarray(origin, np.float64)
    d = camera_rays(origin, forward, up, fov_y, width, height).reshape(-1, 3)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo[None, :] - o[None, :]) / d
        tb = (hi[None, :] - o[None, :]) / d
    t0 = np.max(np.minimum(ta, tb), axis=1).clip(min=0.0)
    t1 = np.min(np.maximum(ta, tb), axis=1)
    keep = psi > 0
    if karea is not None:
        keep &= np.asarray(karea, np.float64) > 0
    p, r2 = pos[keep], psi[keep]
    best = np.full(d.shape[0], np.inf)
    arg = np.full(d.shape[0], -1)
    for k in range(p.shape[0]):
        b = d @ (p[k] - o)
        c = np.dot(p[k] - o, p[k] - o) - r2[k]
        disc = b * b - c
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t = np.maximum(b - sq, t0)
        hit = ok & (t < np.minimum(b + sq, t1)) & (t < best)
        best = np.where(hit, t, best)
        arg = np.where(hit, k, arg)
    depth = np.where(np.isfinite(best), best, -1.0)
    normal = np.zeros_like(d)
    h = arg >= 0
    x = o[None, :] + best[h, None] * d[h]
    normal[h] = (x - p[arg[h]]) / np.sqrt(r2[arg[h]])[:, None]
    return depth.reshape(height, width), normal.reshape(height, width, 3)


def render_volume(pos, psi, origin, forward, up, fov_y, width, height,
                  lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), pixels=None):
    """Traversal of the fluid volume along camera rays (Sec. 6, volume
    traversal), from its plain definition: the fluid is the union of the
    generalized Laguerre cells of Eq. 1, i.e. the union of the balls inside
    the box, so the part of a ray in the fluid is the union of the ray's
    intervals inside the balls, clipped to the box.  Brute force over all
    balls: every ball's interval, then their union (sorted, merged).
    Returns (first entry t, total length inside the fluid, last exit t),
    each (height, width); -1 / 0 / -1 where the ray misses the fluid.  With
    `pixels` (flat pixel indices), only those rays, each result of their
    length."""
    pos = np.asarray(pos, np.float64)
    psi = np.asarray(psi, np.float64)
    o = np.asarray(origin, np.float64)
    d = camera_rays(origin, forward, up, fov_y, width, height).reshape(-1, 3)
    if pixels is not None:
        d = d[np.asarray(pixels)]
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo[None, :] - o[None, :]) / d
        tb = (hi[None, :] - o[None, :]) / d
    t0 = np.max(np.minimum(ta, tb), axis=1).clip(min=0.0)
    t1 = np.min(np.maximum(ta, tb), axis=1)
    keep = psi > 0
    p, r2 = pos[keep], psi[keep]
    m = d.shape[0]
    first = np.full(m, -1.0)
    thick = np.zeros(m)
    last = np.full(m, -1.0)
    e = p - o[None, :]
    ee = np.sum(e * e, axis=1) - r2
    for k in range(m):
        # every ball's interval along ray k
        bb = e @ d[k]
        disc = bb * bb - ee
        ok = disc > 0
        sq = np.sqrt(disc[ok])
        a = np.maximum(bb[ok] - sq, t0[k])
        b = np.minimum(bb[ok] + sq, t1[k])
        iv = sorted((x, y) for x, y in zip(a, b) if x < y)
        if not iv:
            continue
        total, cur0, cur1 = 0.0, iv[0][0], iv[0][1]
        for x, y in iv[1:]:
            if x > cur1:
                total += cur1 - cur0
                cur0, cur1 = x, y
            else:
                cur1 = max(cur1, y)
        total += cur1 - cur0
        first[k], thick[k], last[k] = iv[0][0], total, cur1
    if pixels is not None:
        return first, thick, last
    return first.reshape(height, width), thick.reshape(height, width), last.reshape(height, width)


# Sphere tracing of the smoothed free surface (Sec. 6, surface smoothing).
# Readings: the signed distance of ball i is d_i(x) = |x - p_i| - r_i; "the
# closest site" is the site whose ball surface is nearest, i = argmin d_i(x);
# its "Laguerre neighbourhood" is the sites sharing a restricted facet with
# it of area above 4e-7 psi_i (the FP32 path's emission threshold); the cubic
# polynomial smooth union joins the two nearest spheres of that set,
# f = smin_k(d_(1), d_(2)) with smin_k(a, b) = min(a, b) - k h^3 / 6,
# h = max(k - |a - b|, 0) / k.  f is 1-Lipschitz within one neighbourhood and
# f >= d_(1) - k/6, so the surface {f = 0} lies within k/6 of the balls: a
# ray point farther than k/6 from every ball jumps to the next entry into
# the balls grown by k/6.  The march stops at f <= SMOOTH_HIT k, steps at
# least SMOOTH_MIN_STEP k, at most SMOOTH_MAX_STEPS evaluations.
SMOOTH_HIT = 1e-3
SMOOTH_MIN_STEP = 1e-4
SMOOTH_MAX_STEPS = 1024
SMOOTH_EMIT = 4e-7


def smooth_min(a, b, k):
    """The cubic polynomial smooth minimum of two distances (smooth union)."""
    h = np.maximum(k - np.abs(a - b), 0.0) / k
    return np.minimum(a, b) - k * h ** 3 / 6.0


def laguerre_neighbours(pos, psi, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Padded array (n, m) of each site's restricted-facet neighbours (area
    above SMOOTH_EMIT psi_i), -1 beyond a site's count."""
    psi = np.asarray(psi, np.float64)
    res = cells(pos, psi, lo=lo, hi=hi)
    n = psi.shape[0]
    rows = []
    for i in range(n):
        nf = int(res["nfac"][i])
        j = res["fac_j"][i, :nf]
        a = res["fac_area"][i, :nf]
        rows.append(np.sort(j[a > SMOOTH_EMIT * psi[i]]))
    m = max(1, max(len(r) for r in rows))
    nb = np.full((n, m), -1, np.int64)
    for i, r in enumerate(rows):
        nb[i, :len(r)] = r
    return nb


def _smooth_march(o, d, t0, t1, pos, r, live, nb, k):
    """The sphere-tracing march of render_smooth for a block of rays."""
    grow = k / 6.0
    m = d.shape[0]
    t = t0.copy()
    depth = np.full(m, -1.0)
    normal = np.zeros((m, 3))
    steps = np.zeros(m, np.int64)
    act = t0 <= t1
    e = pos - o[None, :]
    ee_g = np.sum(e * e, axis=1) - (r + grow) ** 2
    while np.any(act):
        idx = np.nonzero(act)[0]
        steps[idx] += 1
        x = o[None, :] + t[idx, None] * d[idx]
        dist = np.linalg.norm(x[:, None, :] - pos[None, :, :], axis=2)
        db = np.where(live[None, :], dist - r[None, :], np.inf)
        i = np.argmin(db, axis=1)
        d1 = db[np.arange(idx.size), i]
        # outside the grown balls: jump to the next entry into them
        far = d1 > grow
        for q in np.nonzero(far)[0]:
            ray = idx[q]
            bb = e @ d[ray]
            disc = bb * bb - ee_g
            ok = live & (disc > 0)
            sq = np.sqrt(np.where(ok, disc, 0.0))
            tin, tout = bb - sq, bb + sq
            cand = ok & (tout > t[ray])
            te = np.max([np.min(np.where(cand, tin, np.inf)), t[ray]]) if np.any(cand) else np.inf
            if te > t1[ray]:
                act[ray] = False
            elif te > t[ray]:
                t[ray] = te
                far[q] = True
            else:
                far[q] = False  # at the grown surface within rounding: take a step
        go = ~far & act[idx]
        if not np.any(go):
            continue
        sel = np.nonzero(go)[0]
        ray = idx[sel]
        ii = i[sel]
        nbr = nb[ii]
        dn = np.where(nbr >= 0, db[sel[:, None], np.maximum(nbr, 0)], np.inf)
        j2 = np.argmin(dn, axis=1)
        d2 = dn[np.arange(sel.size), j2]
        a = d1[sel]
        f = np.where(np.isfinite(d2), smooth_min(a, np.where(np.isfinite(d2), d2, 0.0), k), a)
        done = f <= SMOOTH_HIT * k
        hit = ray[done]
        depth[hit] = t[hit]
        # normal: the smooth minimum's weights on the two spheres' gradients
        xs = x[sel][done]
        g1 = xs - pos[ii[done]]
        g1 /= np.linalg.norm(g1, axis=1, keepdims=True)
        jn = nbr[done, j2[done]]
        has2 = np.isfinite(d2[done])
        g2 = xs - pos[np.maximum(jn, 0)]
        g2 /= np.maximum(np.linalg.norm(g2, axis=1, keepdims=True), 1e-300)
        aa, b2 = a[done], np.where(has2, d2[done], np.inf)
        hh = np.where(has2, np.maximum(k - np.abs(aa - b2), 0.0) / k, 0.0)
        w_lo = 1.0 - hh ** 2 / 2.0  # weight of the smaller distance
        first_is_min = aa <= b2
        w1 = np.where(first_is_min, w_lo, 1.0 - w_lo)
        n = w1[:, None] * g1 + (1.0 - w1)[:, None] * np.where(has2[:, None], g2, 0.0)
        normal[hit] = n / np.linalg.norm(n, axis=1, keepdims=True)
        act[hit] = False
        rest = ray[~done]
        t[rest] += np.maximum(f[~done], SMOOTH_MIN_STEP * k)
        act[rest] &= (t[rest] <= t1[rest]) & (steps[rest] < SMOOTH_MAX_STEPS)
        act[idx[far]] &= steps[idx[far]] < SMOOTH_MAX_STEPS
    return depth, normal, steps


def render_smooth(pos, psi, origin, forward, up, fov_y, width, height, k,
                  lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), pixels=None, neighbours=None):
    """First hit of each camera ray on the smoothed fluid surface by sphere
    tracing (Sec. 6, surface smoothing; readings above).  Rays march in
    blocks of 256; every step is brute force over all balls.  Returns depth (t
    of the hit, -1 when none), the unit normal there (gradient of f; 0 when
    none) and the evaluations of f taken per ray, each (height, width[, 3]),
    or per pixel of `pixels`.  Parity unpinned beyond the closed forms of
    tests/test_oracle_render.py (one ball; the bridge of two balls)."""
    pos = np.asarray(pos, np.float64)
    psi = np.asarray(psi, np.float64)
    o = np.asarray(origin, np.float64)
    d = camera_rays(origin, forward, up, fov_y, width, height).reshape(-1, 3)
    if pixels is not None:
        d = d[np.asarray(pixels)]
    nb = laguerre_neighbours(pos, psi, lo, hi) if neighbours is None else neighbours
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo[None, :] - o[None, :]) / d
        tb = (hi[None, :] - o[None, :]) / d
    t0 = np.max(np.minimum(ta, tb), axis=1).clip(min=0.0)
    t1 = np.min(np.maximum(ta, tb), axis=1)
    r = np.sqrt(np.maximum(psi, 0.0))
    live = psi > 0
    m = d.shape[0]
    depth = np.full(m, -1.0)
    normal = np.zeros((m, 3))
    steps = np.zeros(m, np.int64)
    for b0 in range(0, m, 256):  # blocks of rays march together
        sl = slice(b0, min(m, b0 + 256))
        depth[sl], normal[sl], steps[sl] = _smooth_march(o, d[sl], t0[sl], t1[sl], pos, r, live,
                                                         nb, k)
    if pixels is not None:
        return depth, normal, steps
    return depth.reshape(height, width), normal.reshape(height, width, 3), steps.reshape(height, width)

"""GPU parity of lgc_compute_cells (FP32 and FP64 entry points) with the FP64
oracle, element by element, plus the edge cases of the cell definition
(Eq. 1, Sec. 3.4: empty cells, full balls, planes through the site, walls)
and the error statuses."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import pot, scenes

from _cmp import compare_cells, to_np

pytestmark = pytest.mark.gpu

TOL32 = dict(tol_v=1e-5, tol_h=1e-4, tol_c=1e-4)
TOL64 = dict(tol_v=1e-10, tol_h=1e-9, tol_c=1e-9)


@pytest.fixture(scope="module")
def ctx():
    c = pot.Context(1 << 20, 64, 0)
    yield c
    c.close()


def run(ctx, pos, psi, nu=None, dtype=torch.float32, **kw):
    dev = ctx.device
    p = torch.as_tensor(np.asarray(pos), dtype=dtype, device=dev).contiguous()
    s = torch.as_tensor(np.asarray(psi), dtype=dtype, device=dev).contiguous()
    t = None if nu is None else torch.as_tensor(np.asarray(nu), dtype=torch.float64, device=dev)
    out = pot.lgc_compute_cells(ctx, p, s, t, **kw)
    torch.cuda.synchronize()
    return out


def oracle_of(pos, psi, query=None):
    # the oracle sees exactly the values the GPU got (float32 widened, or float64)
    return O.cells(np.asarray(pos, np.float64), np.asarray(psi, np.float64), query=query)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_jittered_block_1000(ctx, dtype):
    sc = scenes.jittered_block()
    for scale in (1.0, 1.6):  # initial balls, and balls large enough to pack the block
        psi = (sc.psi.astype(np.float64) * scale).astype(np.float32 if dtype == torch.float32 else np.float64)
        pos = sc.pos if dtype == torch.float32 else sc.pos.astype(np.float64)
        out = run(ctx, pos, psi, sc.nu, dtype)
        ref = oracle_of(pos, psi)
        rep = compare_cells(out, ref, psi, sc.nu, **(TOL32 if dtype == torch.float32 else TOL64))
        assert out["stats"]["n_empty"] == int(np.sum(ref["vol"] <= 0))
        print(scale, rep)


@pytest.mark.parametrize("n", [30011, 1 << 20])
def test_uniform_cloud(ctx, n):
    """Random balls (r = U(0.4,1.2) R0).  30011 sites: every cell against the
    oracle (several CTA tiles and a ragged tail); 2^20 sites: the benchmark's
    launch, 10k sampled cells."""
    sc = scenes.uniform_cloud(n=n, seed=1)
    out = run(ctx, sc.pos, sc.psi, sc.nu)
    q = None if n < 100000 else sc.extra["subset"]
    ref = oracle_of(sc.pos, sc.psi, query=q)
    rep = compare_cells(out, ref, sc.psi, sc.nu, **TOL32)
    print(rep, out["stats"])
    # invariants at any size
    v = to_np(out["volumes"]).astype(np.float64)
    r = np.sqrt(sc.psi.astype(np.float64))
    assert v.sum() <= 1.0 and np.all(v <= 4 / 3 * math.pi * r ** 3 * (1 + 1e-6))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_graded_weights_cloud(ctx, dtype):
    """Ball radii doubling across the box (r = U(0.7,1.0) R0 (1 + x)):
    the largest weight near most sites is below the global one, so the
    candidate search reaches only as far as the nearby weights allow.  Every
    cell against the oracle: exact topology, volumes, gradient, Hessian."""
    n = 30011
    rng = np.random.default_rng(17)
    pos = rng.uniform(0.0, 1.0, (n, 3))
    r0 = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r = rng.uniform(0.7, 1.0, n) * r0 * (1.0 + pos[:, 0])
    ft = np.float32 if dtype == torch.float32 else np.float64
    pos, psi = pos.astype(ft), (r * r).astype(ft)
    nu = np.full(n, 0.5 / n)
    out = run(ctx, pos, psi, nu, dtype)
    ref = oracle_of(pos, psi)
    rep = compare_cells(out, ref, psi, nu, **(TOL32 if dtype == torch.float32 else TOL64))
    # cells emptied by a plane at h = -r within rounding are decided either
    # way: every cell of zero GPU volume has an oracle volume within the
    # volume floor (1e-9 of its ball in FP32, 1e-14 in FP64; the converse is
    # part of compare_cells)
    n_empty_ref = int(np.sum(ref["vol"] <= 0))
    v = to_np(out["volumes"]).astype(np.float64)
    ball = 4.0 / 3.0 * math.pi * psi.astype(np.float64) ** 1.5
    floor = 1e-9 if dtype == torch.float32 else 1e-14
    assert np.all(ref["vol"][v <= 0] <= floor * ball[v <= 0])
    print(rep, out["stats"], "oracle empty", n_empty_ref)


def test_graded_weights_cloud_large_sampled():
    """The same construction at 300,007 sites with radii growing 2.5-fold
    across the box (r = U(0.7,1.0) R0 (1 + 1.5x)), FP32, 10k sampled cells
    against the oracle (cells of up to about 100 cutting bisectors: a
    context with k_max 246)."""
    n = 300007
    rng = np.random.default_rng(29)
    pos = rng.uniform(0.0, 1.0, (n, 3))
    r0 = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r = rng.uniform(0.7, 1.0, n) * r0 * (1.0 + 1.5 * pos[:, 0])
    pos, psi = pos.astype(np.float32), (r * r).astype(np.float32)
    nu = np.full(n, 0.5 / n)
    with pot.Context(n, 246, 0) as big:
        out = run(big, pos, psi, nu)
        q = np.random.default_rng(30).choice(n, 10000, replace=False)
        rep = compare_cells(out, oracle_of(pos, psi, query=q), psi, nu, **TOL32)
    print(rep, out["stats"])


@pytest.mark.parametrize("jitter", [1e-2, 3e-2])
def test_nearly_regular_lattice(ctx, jitter):
    """Sites of a 30^3 cubic lattice of spacing s jittered by U(-j, j) s and
    balls of radius 0.9 s that contain the cube corners: every face facet
    is bounded by nearly coincident lines (its side neighbour's trace and
    its edge neighbours'), whose vertices the facet tasks must share.  Every
    cell against the oracle in FP32."""
    m = 30
    s = 1.0 / m
    rng = np.random.default_rng(7)
    g = (np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
         .reshape(-1, 3) + 0.5) * s
    pos = (g + rng.uniform(-jitter, jitter, g.shape) * s).astype(np.float32)
    n = pos.shape[0]
    psi = np.full(n, (0.9 * s) ** 2, np.float32)
    nu = np.full(n, 0.9 * s ** 3)
    out = run(ctx, pos, psi, nu)
    rep = compare_cells(out, oracle_of(pos, psi), psi, nu, **TOL32)
    print(rep)


def test_uniform_cloud_fp64(ctx):
    sc = scenes.uniform_cloud(n=20000, seed=5)
    pos, psi = sc.pos.astype(np.float64), sc.psi.astype(np.float64)
    out = run(ctx, pos, psi, sc.nu, torch.float64)
    rep = compare_cells(out, oracle_of(pos, psi), psi, sc.nu, **TOL64)
    print(rep)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_closed_forms_and_planes_through_site(ctx, dtype):
    r = 0.1
    d = 0.12
    cases = [
        ([[0.5, 0.4, 0.6]], [r * r]),                                 # isolated ball
        ([[0.5 - d / 2, 0.5, 0.5], [0.5 + d / 2, 0.5, 0.5]], [0.01, 0.008]),  # two caps
        ([[0.04, 0.5, 0.5]], [r * r]),                                # wall cap
        ([[0.0, 0.0, 0.0]], [r * r]),                                 # site on a box corner
        ([[0.0, 0.5, 0.5]], [r * r]),                                 # site on a face
        ([[-0.03, 0.5, 0.5]], [r * r]),                               # site behind a wall
        ([[-0.2, 0.5, 0.5]], [r * r]),                                # ball outside the box
        ([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], [0.0, 0.01]),          # psi = 0
        ([[0.5, 0.5, 0.5], [0.51, 0.5, 0.5]], [0.0004, 0.01]),       # ball inside a heavier ball
        ([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5]], [0.01, 0.01 + 0.01]),   # bisector through site 0
    ]
    tol = TOL32 if dtype == torch.float32 else TOL64
    for pos, psi in cases:
        out = run(ctx, pos, psi, None, dtype)
        ref = oracle_of(np.asarray(pos, np.float32 if dtype == torch.float32 else np.float64),
                        np.asarray(psi, np.float32 if dtype == torch.float32 else np.float64))
        compare_cells(out, ref, np.asarray(psi, np.float64), None, **tol)


def test_big_cells_take_the_whole_warp(ctx):
    """A heavy site surrounded by 48 light ones: its cell has > 32 cutting
    planes and runs on the multi-round path of the cell kernel."""
    rng = np.random.default_rng(3)
    u = rng.normal(size=(48, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    pos = np.concatenate([[[0.5, 0.5, 0.5]], 0.5 + 0.05 * u]).astype(np.float32)
    psi = np.concatenate([[0.06 ** 2], np.full(48, 0.03 ** 2)]).astype(np.float32)
    out = run(ctx, pos, psi)
    ref = oracle_of(pos, psi)
    assert ref["n_planes"][0] > 32
    compare_cells(out, ref, psi, None, **TOL32)


def test_cubic_lattice_zero_area_facets(ctx):
    s = 1.0 / 16
    k = np.arange(5) - 2
    z, y, x = np.meshgrid(k, k, k, indexing="ij")
    pos = (0.5 + s * np.stack([x.ravel(), y.ravel(), z.ravel()], 1)).astype(np.float32)
    for rf in (0.6, 0.9):
        psi = np.full(125, (rf * s) ** 2, np.float32)
        out = run(ctx, pos, psi)
        ref = oracle_of(pos, psi, query=[62])
        compare_cells(out, ref, psi, None, **TOL32)
        rp = to_np(out["row_ptr"])
        assert rp[63] - rp[62] == 7  # diagonal + 6 face neighbours


def test_error_statuses(ctx):
    # coincident sites cutting each other's ball
    out = run(ctx, [[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]], [0.01, 0.01], check=False)
    assert out["status"] == 4 and out["stats"]["error_site"] in (0, 1)
    # more cutting bisectors than k_max
    small = pot.Context(1000, 4, 0, fp64=False)
    rng = np.random.default_rng(1)
    pos = rng.uniform(0.45, 0.55, size=(50, 3)).astype(np.float32)
    out = run(small, pos, np.full(50, 0.02 ** 2, np.float32), check=False)
    assert out["status"] == 3
    # the context still works afterwards
    out = run(small, [[0.5, 0.5, 0.5]], [0.01])
    assert abs(float(out["volumes"][0]) - 4 / 3 * math.pi * 1e-3) < 1e-9
    # more sites than the context holds
    with pytest.raises(pot.PotError):
        run(small, np.full((1001, 3), 0.5, np.float32), np.full(1001, 1e-4, np.float32))
    # CSR capacity too small: status and the needed nnz are reported
    sc = scenes.jittered_block(n_side=4)
    out = run(ctx, sc.pos, sc.psi * 2, csr_cap=10, check=False)
    assert out["status"] == 9 and out["nnz"] > 10
    small.close()


def test_deterministic(ctx):
    sc = scenes.uniform_cloud(n=50000, seed=7)
    a = run(ctx, sc.pos, sc.psi, sc.nu)
    b = run(ctx, sc.pos, sc.psi, sc.nu)
    for key in ("volumes", "grad", "centroids", "karea", "row_ptr", "cols", "vals"):
        assert torch.equal(a[key], b[key]), key


def test_cell_diagnostics_invariants(ctx):
    """After an evaluation every cell lies inside its security ball (extent
    below the radius, or the radius covers the site's ball), standalone
    evaluations centre the ball on the site, and a cell is built from at
    least as many planes as it has Hessian entries."""
    sc = scenes.jittered_block(n_side=10, seed=2)
    out = run(ctx, sc.pos, sc.psi, sc.nu)
    dg = pot.cell_diagnostics(ctx, sc.n)
    ext = to_np(dg["extent"]).astype(np.float64)
    rad = to_np(dg["radius"]).astype(np.float64)
    off = to_np(dg["center_offset"]).astype(np.float64)
    planes = to_np(dg["planes"])
    r = np.sqrt(sc.psi.astype(np.float64))
    assert np.all(off == 0.0)
    assert np.all((ext < rad * (1 - 1e-5)) | (rad >= r * (1 - 1e-6)))
    rp = to_np(out["row_ptr"]).astype(np.int64)
    assert np.all(planes >= np.diff(rp) - 1)


def test_big_cells_against_oracle():
    """A cell that needs more planes than the cell kernel's shared window
    (252): in a jittered 14^3 lattice with balls 2.5 spacings wide, one site
    whose weight exceeds its neighbours' by 12.5 s^2 owns a cell about 3.5
    spacings wide, bounded by the bisectors of the shell of sites between
    about 2.3 and 5.5 spacings -- several hundred planes, so it goes through
    the big-cell kernel.  The central 5^3 cells (the big one, the swallowed
    empty ones, the shell) against the oracle."""
    n_side, s = 14, 0.04
    rng = np.random.default_rng(12)
    g = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((g + 0.5 + rng.uniform(-0.2, 0.2, g.shape)) * s + 0.2).astype(np.float32)
    n = pos.shape[0]
    psi = np.full(n, (2.5 * s) ** 2, np.float32)
    c = int(np.nonzero(np.all(g == n_side // 2, axis=1))[0][0])
    psi[c] = np.float32(3 * (2.5 * s) ** 2)
    nu = np.full(n, s ** 3)
    big = pot.Context(n, 1024, 0, fp64=False)
    out = run(big, pos, psi, nu)
    planes = to_np(pot.cell_diagnostics(big, n)["planes"])
    assert planes[c] > 252, planes[c]
    q = np.nonzero(np.all(np.abs(g - n_side // 2) <= 2, axis=1))[0]
    ref = O.cells(pos.astype(np.float64), psi.astype(np.float64), query=q, max_facets=4096)
    assert np.all(ref["status"] == 0)
    rep = compare_cells(out, ref, psi, nu, **TOL32)
    print(rep, int(planes[c]), float(ref["vol"][np.nonzero(q == c)[0][0]] / s ** 3))
    big.close()

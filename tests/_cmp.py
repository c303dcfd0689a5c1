"""Element-by-element comparison of GPU cell outputs with the FP64 oracle.

Tolerance bases:
  volumes    |V_gpu - V_ref| <= tol_v * V_ref + tol_floor * 4/3 pi r^3
  gradient   |g_gpu - (nu - V_ref)| <= tol_v * max(nu, V_ref) + tol_floor * 4/3 pi r^3
             (nu is exact, so the gradient's error is the volume's; relative
             to nu rather than to g, which goes to 0 near convergence)
The floor comes from the arithmetic: V contains r |K| / 3 with
|K| = psi (4 pi [inside] - sum_f Omega_f), and the solid-angle sum carries an
absolute rounding error dOmega (a few ulp of 4 pi), so |dV| <= r psi dOmega / 3
of the ball volume for any cell.  In FP64 that is about 1e-14 of the ball
(tol_floor 1e-14).  The FP32 path recomputes in FP64 every cell where its
own rounding (about 2e-7 of the ball) could reach 1e-5 of the volume (ball
above 20 V, or a diagonal below 0.1 r, with a spherical part or the site
outside its polytope), so its floor is 1e-9 of the ball, far below either.
For cells above a few percent of their ball the floor is negligible and the
test is the plain relative one; it only matters for sliver cells.
  |K|        |K_gpu - K_ref| <= tol_v * 4 pi psi
  centroid   |c_gpu - c_ref| <= tol_c * r   (cells with V_ref > 1e-3 ball)
  Hessian    |M_gpu - M_ref| <= tol_h * max(|M_ii,ref|, floor_h r_i) for every entry of row i
The Hessian floor also comes from the arithmetic: M_ij = |B_ij| / (2 d_ij)
(Eq. 2) and a facet near the rim of the ball has |B| = pi (psi - h^2), so the
rounding of the plane offset h_ij (a few ulp of r in FP32) moves M_ij by about
pi r eps = 2e-7 r whatever the cell, and the diagonal carries r times the
solid-angle rounding; a sliver cell (a cap far from its site, M_ii << r)
would reach that, but the FP32 path recomputes every cell with M_ii < 0.1 r
in FP64.  floor_h = 1e-3 (FP32 and FP64).
Topology: a bisector facet with oracle area > 1e-6 psi_i must be in the GPU
row; a GPU entry must be a facet with oracle area > 0; facets in between are
ambiguous (counted, not compared).
"""
import math

import numpy as np

from oracle import oracle as O


def to_np(t):
    return None if t is None else t.detach().cpu().numpy()


def compare_cells(out, ref, psi, nu, tol_v, tol_h, tol_c=None, tol_floor=None,
                  check_hessian=True):
    q = ref["query"]
    psi = np.asarray(psi, np.float64)
    ps = psi[q]
    r = np.sqrt(np.maximum(ps, 0))
    ball = 4.0 / 3.0 * math.pi * r ** 3
    if tol_floor is None:
        tol_floor = 1e-9 if tol_v >= 1e-7 else 1e-14
    v_gpu = to_np(out["volumes"]).astype(np.float64)[q]
    base = ref["vol"] + (tol_floor / tol_v) * ball
    base = np.where(base > 0, base, 1.0)
    ev = np.abs(v_gpu - ref["vol"]) / base
    worst = int(np.argmax(ev))
    assert ev.max() <= tol_v, f"volume rel err {ev.max():.3e} at site {q[worst]}"
    # cells that pass only because of the floor: the plain relative test
    # |dV| <= tol_v V_ref would fail them
    plain = np.abs(v_gpu - ref["vol"]) > tol_v * ref["vol"]
    # of those, cells of non-negligible volume (above 1e-6 of the ball); the
    # others are cells of next to no volume, whose relative error is noise
    sized = ref["vol"] > 1e-6 * ball
    report = {"cells": int(q.shape[0]), "vol_max_rel": float(ev.max()),
              "vol_floor_cells": int(np.sum(plain)),
              "vol_floor_cells_sized": int(np.sum(plain & sized))}
    if nu is not None:
        g = to_np(out["grad"])[q]
        nb = np.maximum(np.asarray(nu)[q], ref["vol"]) + (tol_floor / tol_v) * ball
        eg = np.abs(g - (np.asarray(nu)[q] - ref["vol"])) / nb
        assert eg.max() <= tol_v, f"grad rel err {eg.max():.3e}"
        report["grad_max_rel"] = float(eg.max())
    if out.get("karea") is not None:
        k = to_np(out["karea"]).astype(np.float64)[q]
        kb = np.where(ps > 0, 4 * math.pi * ps, 1.0)
        ek = np.abs(k - ref["karea"]) / kb
        assert ek.max() <= tol_v, f"karea rel err {ek.max():.3e}"
        report["karea_max_rel"] = float(ek.max())
    if tol_c is not None and out.get("centroids") is not None:
        c = to_np(out["centroids"]).astype(np.float64)[q]
        ok = ref["vol"] > 1e-3 * ball
        ec = np.linalg.norm(c - ref["cen"], axis=1)[ok] / r[ok]
        if ec.size:
            assert ec.max() <= tol_c, f"centroid err {ec.max():.3e} r"
            report["cen_max_rel"] = float(ec.max())
    if check_hessian:
        report.update(compare_hessian(out, ref, psi, tol_h, floor_h=1e-3))
    return report


def compare_hessian(out, ref, psi, tol_h, floor_h=1e-3):
    q = ref["query"]
    rp = to_np(out["row_ptr"]).astype(np.int64)
    cols = to_np(out["cols"]).astype(np.int64)
    vals = to_np(out["vals"]).astype(np.float64)
    diag_ref, rows_ref = O.hessian_entries(ref, psi)
    amb = 0
    worst = 0.0
    floor_rows = 0  # rows that pass only because of the floor (|M_ii| < floor_h r_i)
    floor_rows_sized = 0  # of those, rows with |M_ii| above 1e-6 r_i
    for k, i in enumerate(q):
        gc = cols[rp[i]:rp[i + 1]]
        gv = vals[rp[i]:rp[i + 1]]
        assert np.all(np.diff(gc) > 0), f"row {i} columns not ascending"
        assert i in gc, f"row {i} has no diagonal"
        d_gpu = gv[gc == i][0]
        # entries scale like r (an isolated ball has M_ii = 2 pi r); a sliver
        # or empty cell has M_ii << r, so the base has the floor of the header
        ri = math.sqrt(psi[i]) if psi[i] > 0 else 0.0
        scale = max(abs(diag_ref[k]), floor_h * ri)
        off = gc != i
        gcols = set(gc[off].tolist())
        nf = int(ref["nfac"][k])
        fj = ref["fac_j"][k, :nf]
        fa = ref["fac_area"][k, :nf]
        strong = set(fj[fa > 1e-6 * psi[i]].tolist())
        positive = set(fj[fa > 0].tolist())
        missing = strong - gcols
        assert not missing, f"row {i}: facets {sorted(missing)} missing on the GPU"
        extra = gcols - positive
        assert not extra, f"row {i}: GPU facets {sorted(extra)} have zero oracle area"
        amb += len(positive - strong)
        if scale == 0:
            assert abs(d_gpu) <= 1e-30 and not gcols
            continue
        e = abs(d_gpu - diag_ref[k]) / scale
        rc, rv = rows_ref[k]
        rmap = dict(zip(rc.tolist(), rv.tolist()))
        for c, v in zip(gc[off].tolist(), gv[off].tolist()):
            e = max(e, abs(v - rmap[c]) / scale)
        worst = max(worst, e)
        assert e <= tol_h, f"row {i}: Hessian rel err {e:.3e}"
        if scale > abs(diag_ref[k]) and e * scale > tol_h * abs(diag_ref[k]):
            floor_rows += 1
            floor_rows_sized += int(abs(diag_ref[k]) > 1e-6 * ri)
    return {"hess_max_rel": worst, "ambiguous_facets": amb, "hess_floor_rows": floor_rows,
            "hess_floor_rows_sized": floor_rows_sized}

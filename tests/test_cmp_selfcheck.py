"""The GPU-parity comparison helper, checked on the CPU: the oracle's own
results, laid out as the library returns them (volumes, gradient, caller-order
CSR with the diagonal, centroids, free-surface areas), must pass every check,
and a planted error in one Hessian entry or one volume must fail."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_05765_b300 import scenes
from _cmp import compare_cells


def as_gpu_output(ref, psi, nu):
    n = ref["vol"].shape[0]
    diag, rows = O.hessian_entries(ref, psi)
    row_ptr, cols, vals = [0], [], []
    for i in range(n):
        c, v = rows[i]
        c = np.append(c, i)
        v = np.append(v, diag[i])
        order = np.argsort(c)
        cols += c[order].tolist()
        vals += v[order].tolist()
        row_ptr.append(len(cols))
    t = lambda a, dt=torch.float64: torch.as_tensor(np.asarray(a), dtype=dt)
    return {"volumes": t(ref["vol"]), "grad": t(nu - ref["vol"]), "karea": t(ref["karea"]),
            "centroids": t(ref["cen"]), "row_ptr": t(row_ptr, torch.int64),
            "cols": t(cols, torch.int64), "vals": t(vals)}


@pytest.fixture(scope="module")
def block():
    sc = scenes.jittered_block(n_side=5, seed=3)
    pos, psi = sc.pos.astype(np.float64), sc.psi.astype(np.float64)
    ref = O.cells(pos, psi)
    return ref, psi, sc.nu


def test_oracle_against_itself_passes(block):
    ref, psi, nu = block
    out = as_gpu_output(ref, psi, nu)
    rep = compare_cells(out, ref, psi, nu, tol_v=1e-5, tol_h=1e-4, tol_c=1e-4)
    assert rep["karea_max_rel"] == 0.0


def test_planted_errors_fail(block):
    ref, psi, nu = block
    out = as_gpu_output(ref, psi, nu)
    k = int(np.argmax(ref["vol"]))
    out["volumes"][k] *= 1.0 + 3e-5
    with pytest.raises(AssertionError):
        compare_cells(out, ref, psi, nu, tol_v=1e-5, tol_h=1e-4)
    out = as_gpu_output(ref, psi, nu)
    rp = out["row_ptr"].numpy()
    cols = out["cols"].numpy()
    vals = out["vals"].numpy()
    i = int(np.argmax(np.diff(rp)))
    seg = np.arange(rp[i], rp[i + 1])
    off = seg[cols[seg] != i]
    j = int(off[np.argmax(np.abs(vals[off]))])  # the row's largest bisector entry
    out["vals"][j] *= 1.0 + 1e-2
    with pytest.raises(AssertionError):
        compare_cells(out, ref, psi, nu, tol_v=1e-5, tol_h=1e-4)

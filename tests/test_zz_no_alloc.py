"""lgc_compute_cells_noalloc: the cell evaluation for callers that cannot
allocate device memory (a plugin inside a host application that owns every
device allocation, a real-time loop that cannot afford a cudaMalloc stall).
Its scratch is a fixed array inside libpot.so, so two calls in a row must
each match the ordinary entry point (which uses a context's workspace), and
the second must not see leftovers of the first.  The file is named to be
collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_05765_b300 import pot, scenes

pytestmark = pytest.mark.gpu

MAX_SITES = 8192


def noalloc_fn():
    f = pot.lib().lgc_compute_cells_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.POINTER(pot.Domain), P, P, P, P,
                  ctypes.POINTER(pot.CellStats)]
    f.restype = ctypes.c_int
    return f


def outputs(n, dev):
    return {"volumes": torch.empty(n, dtype=torch.float32, device=dev),
            "grad": torch.empty(n, dtype=torch.float64, device=dev),
            "centroids": torch.empty((n, 3), dtype=torch.float32, device=dev),
            "karea": torch.empty(n, dtype=torch.float32, device=dev)}


def call_noalloc(pos, psi, nu, out=None):
    n = pos.shape[0]
    if out is None:
        out = outputs(n, pos.device)
    st = pot.CellStats()
    dom = pot._domain(pot.UNIT_BOX)
    code = noalloc_fn()(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), n,
                        ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                        ctypes.c_void_p(nu.data_ptr()), ctypes.byref(dom),
                        ctypes.c_void_p(out["volumes"].data_ptr()), ctypes.c_void_p(out["grad"].data_ptr()),
                        ctypes.c_void_p(out["centroids"].data_ptr()),
                        ctypes.c_void_p(out["karea"].data_ptr()), ctypes.byref(st))
    torch.cuda.synchronize()
    return code, out, st


def close(a, b, nu, psi):
    """Same tolerance as the parity tests: 1e-5 relative plus a floor of
    1e-9 of the ball volume."""
    ball = 4.0 / 3.0 * np.pi * np.maximum(psi, 0.0) ** 1.5
    va, vb = a["volumes"].double().cpu().numpy(), b["volumes"].double().cpu().numpy()
    assert np.all(np.abs(va - vb) <= 1e-5 * np.abs(vb) + 1e-9 * ball)
    ga, gb = a["grad"].cpu().numpy(), b["grad"].cpu().numpy()
    assert np.all(np.abs(ga - gb) <= 1e-5 * nu + 1e-9 * ball)
    ka, kb = a["karea"].double().cpu().numpy(), b["karea"].double().cpu().numpy()
    assert np.all(np.abs(ka - kb) <= 1e-5 * 4 * np.pi * psi)
    ca, cb = a["centroids"].double().cpu().numpy(), b["centroids"].double().cpu().numpy()
    assert np.all(np.linalg.norm(ca - cb, axis=1) <= 1e-4 * np.sqrt(psi))


def test_noalloc_matches_context_entry_point_twice():
    dev = torch.device("cuda", 0)
    ctx = pot.Context(MAX_SITES, 64, 0, fp64=False)
    # a large call, then a smaller one: the second must not read leftovers
    for sc in (scenes.uniform_cloud(n=MAX_SITES, seed=21), scenes.jittered_block(n_side=10)):
        pos = torch.from_numpy(sc.pos).to(dev)
        psi = torch.from_numpy(sc.psi).to(dev)
        nu = torch.from_numpy(sc.nu).to(dev)
        code, got, st = call_noalloc(pos, psi, nu)
        assert code == 0, pot.STATUS.get(code)
        ref = pot.lgc_compute_cells(ctx, pos, psi, nu, hessian=False)
        close(got, ref, sc.nu, sc.psi.astype(np.float64))
        assert st.n_empty == ref["stats"]["n_empty"]
        assert st.max_planes == ref["stats"]["max_planes"]
    ctx.close()


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the array's address), a call
    leaves the device's free memory unchanged: torch's own counters would
    not see a cudaMalloc inside the library, the driver's free count does."""
    dev = torch.device("cuda", 0)
    sc = scenes.uniform_cloud(n=MAX_SITES, seed=22)
    pos = torch.from_numpy(sc.pos).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    out = outputs(sc.n, dev)
    code, _, _ = call_noalloc(pos, psi, nu, out)
    assert code == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    code, _, _ = call_noalloc(pos, psi, nu, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert code == 0
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_too_many_sites():
    dev = torch.device("cuda", 0)
    n = MAX_SITES + 1
    pos = torch.full((n, 3), 0.5, dtype=torch.float32, device=dev)
    psi = torch.full((n,), 1e-4, dtype=torch.float32, device=dev)
    nu = torch.full((n,), 1e-6, dtype=torch.float64, device=dev)
    code, _, _ = call_noalloc(pos, psi, nu)
    assert code == 11  # POT_ERR_TOO_LARGE

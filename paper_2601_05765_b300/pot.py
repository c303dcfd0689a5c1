"""Thin ctypes binding of libpot.so (C ABI in include/pot.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libpot.so.  Tensors are torch CUDA tensors (PyTorch provides
device memory and streams); float32 inputs select the mixed-precision entry
points, float64 inputs the *_f64 ones.  Nothing here falls back to the CPU:
if libpot.so is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpot.so")

POT_OK = 0
POT_ERR_INVALID_ARG = 1
STATUS = {
    0: "POT_OK", 1: "POT_ERR_INVALID_ARG", 2: "POT_ERR_CUDA", 3: "POT_ERR_NEIGHBOUR_OVERFLOW",
    4: "POT_ERR_COINCIDENT_SITES", 5: "POT_ERR_EMPTY_CELL_AT_START", 6: "POT_ERR_NOT_CONVERGED",
    7: "POT_ERR_LINESEARCH_FAILED", 8: "POT_ERR_POLYGON_OVERFLOW", 9: "POT_ERR_CAPACITY",
    10: "POT_ERR_PCG_BREAKDOWN", 11: "POT_ERR_TOO_LARGE",
}
UNIT_BOX = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


class PotError(RuntimeError):
    def __init__(self, code, where, stats=None):
        self.code = code
        self.stats = stats
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class Domain(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class Csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("cols", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("cap", ctypes.c_int64), ("nnz", ctypes.c_int64)]


class CellStats(ctypes.Structure):
    _fields_ = [("n_empty", ctypes.c_int64), ("n_planes", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("error_site", ctypes.c_int64), ("max_planes", ctypes.c_int32),
                ("ms_grid", ctypes.c_float), ("ms_cells", ctypes.c_float), ("ms_csr", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_newton", ctypes.c_int32),
                ("max_halvings", ctypes.c_int32), ("max_pcg", ctypes.c_int32),
                ("pcg_chunk", ctypes.c_int32), ("pcg_rtol", ctypes.c_double),
                ("dt", ctypes.c_double), ("eps", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("wall_margin", ctypes.c_double), ("warm_start", ctypes.c_int32),
                ("substeps", ctypes.c_int32), ("mu", ctypes.c_double), ("gamma", ctypes.c_double),
                ("mu_wall", ctypes.c_double), ("gamma_wall", ctypes.c_double),
                ("pcg_host_loop", ctypes.c_int32), ("reserved_params", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("pcg_iters", ctypes.c_int32), ("halvings", ctypes.c_int32),
                ("cell_evals", ctypes.c_int32), ("grid_builds", ctypes.c_int32),
                ("err_max", ctypes.c_double), ("err_l2", ctypes.c_double),
                ("err_start", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_cells", ctypes.c_double), ("ms_pcg", ctypes.c_double),
                ("nnz", ctypes.c_int64), ("mlp_used", ctypes.c_int32),
                ("mlp_fallback", ctypes.c_int32), ("repairs", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("error_site", ctypes.c_int64),
                ("visc_iters", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms_visc", ctypes.c_double)]


class Camera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("forward", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fov_y", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


def _as_dict(st):
    return {name: getattr(st, name) for name, _ in st._fields_}


_lib = None


def lib():
    """Load libpot.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpot.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.pot_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, I64, I32, I32]
        L.pot_destroy.argtypes = [P]
        L.pot_status_string.restype = ctypes.c_char_p
        L.pot_status_string.argtypes = [ctypes.c_int]
        L.pot_default_params.argtypes = [ctypes.POINTER(Params)]
        L.pot_default_params.restype = None
        L.pot_kernel_launches.argtypes = []
        L.pot_kernel_launches.restype = I64
        for name in ("lgc_compute_cells", "lgc_compute_cells_f64"):
            f = getattr(L, name)
            f.argtypes = [P, P, I64, P, P, P, ctypes.POINTER(Domain), P, P, ctypes.POINTER(Csr), P, P,
                          ctypes.POINTER(CellStats)]
        for name in ("pot_newton_solve", "pot_newton_solve_f64"):
            f = getattr(L, name)
            f.argtypes = [P, P, I64, P, P, P, ctypes.POINTER(Domain), ctypes.POINTER(Params),
                          ctypes.POINTER(SolveStats)]
        for name in ("pot_fluid_step", "pot_fluid_step_f64"):
            f = getattr(L, name)
            f.argtypes = [P, P, I64, P, P, P, P, ctypes.POINTER(Domain), ctypes.POINTER(Params),
                          ctypes.POINTER(SolveStats)]
        L.pot_mlp_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, I64]
        L.pot_mlp_destroy.argtypes = [P]
        L.pot_mlp_num_params.argtypes = []
        L.pot_mlp_set_params.argtypes = [P, P, P]
        L.pot_mlp_get_params.argtypes = [P, P, P]
        L.pot_mlp_forward.argtypes = [P, P, I64, P, P]
        L.pot_mlp_gradients.argtypes = [P, P, I64, P, P, P, I64, P, P]
        L.pot_mlp_train_step.argtypes = [P, P, I64, P, P, P, I64, ctypes.c_float, P]
        L.pot_mlp_check.argtypes = [P, P]
        L.pot_mlp_features.argtypes = [P, P, P, I64, P, P, P, P, P, ctypes.POINTER(Domain),
                                       ctypes.POINTER(Params), P]
        L.pot_mlp_set_history.argtypes = [P, P, I64, P]
        L.pot_set_warm_start.argtypes = [P, P]
        L.pot_cell_kernel_time.argtypes = [P, ctypes.c_int, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                           ctypes.POINTER(ctypes.c_double)]
        L.pot_cell_kernel_time.restype = ctypes.c_int
        L.pot_cell_diagnostics.argtypes = [P, P, I64, P, P, P, P]
        L.pot_cell_diagnostics.restype = ctypes.c_int
        L.pot_clear_history.argtypes = [P]
        L.pot_clear_history.restype = ctypes.c_int
        L.pot_set_viscosity_factors.argtypes = [P, I64, P]
        L.pot_set_viscosity_factors.restype = ctypes.c_int
        L.pot_render_depth.argtypes = [P, P, I64, P, P, P, ctypes.POINTER(Domain),
                                       ctypes.POINTER(Camera), P, P]
        L.pot_render_depth.restype = ctypes.c_int
        L.pot_render_volume.argtypes = [P, P, I64, P, P, ctypes.POINTER(Domain),
                                        ctypes.POINTER(Camera), P, P, P, P]
        L.pot_render_volume.restype = ctypes.c_int
        L.pot_render_smooth.argtypes = [P, P, I64, P, P, ctypes.POINTER(Domain),
                                        ctypes.POINTER(Camera), ctypes.c_float, P, P, P]
        L.pot_render_smooth.restype = ctypes.c_int
        L.pot_mlp_set_inputs.argtypes = [P, ctypes.c_int32]
        L.pot_mlp_set_inputs.restype = ctypes.c_int
        L.pot_measure_fp32_peak.argtypes = [P, P, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
        L.pot_measure_fp32_peak.restype = ctypes.c_int
        for f in (L.pot_mlp_create, L.pot_mlp_destroy, L.pot_mlp_num_params, L.pot_mlp_set_params,
                  L.pot_mlp_get_params, L.pot_mlp_forward, L.pot_mlp_gradients, L.pot_mlp_train_step,
                  L.pot_mlp_check, L.pot_mlp_features, L.pot_mlp_set_history,
                  L.pot_set_warm_start):
            f.restype = ctypes.c_int
        for f in (L.pot_create, L.pot_destroy, L.lgc_compute_cells, L.lgc_compute_cells_f64,
                  L.pot_newton_solve, L.pot_newton_solve_f64, L.pot_fluid_step, L.pot_fluid_step_f64):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernel launches issued by libpot.so so far in this process."""
    return int(lib().pot_kernel_launches())


def measure_fp32_peak(device=None, stream=None) -> dict:
    """FP32 FMA throughput of the current device (TFLOP/s), measured by the
    library's FMA-chain kernel (best of five launches)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sm * 8, dtype=torch.float32, device=dev)
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    code = lib().pot_measure_fp32_peak(_stream(stream), _ptr(sink), ctypes.byref(tf), ctypes.byref(ms))
    if code != POT_OK:
        raise PotError(code, "pot_measure_fp32_peak")
    return {"tflops": float(tf.value), "ms": float(ms.value)}


def cell_diagnostics(ctx: "Context", n: int, stream=None) -> dict:
    """Security ball (centre offset, radius), cell extent from its centre and
    plane count of every site after the last FP32 cell evaluation of `ctx`
    (caller order of that evaluation)."""
    dev = ctx.device
    out = {"center_offset": torch.empty((n, 3), dtype=torch.float32, device=dev),
           "radius": torch.empty(n, dtype=torch.float32, device=dev),
           "extent": torch.empty(n, dtype=torch.float32, device=dev),
           "planes": torch.empty(n, dtype=torch.int32, device=dev)}
    code = lib().pot_cell_diagnostics(ctx.handle, _stream(stream), n, _ptr(out["center_offset"]),
                                      _ptr(out["radius"]), _ptr(out["extent"]), _ptr(out["planes"]))
    if code != POT_OK:
        raise PotError(code, "pot_cell_diagnostics")
    return out


def cell_kernel_time(ctx: "Context", reset: bool = False) -> dict:
    """Cell-kernel launches, cells processed and device ms accumulated in
    `ctx` (CUDA events around each launch); reset clears them after reading."""
    la, ce, ms = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
    code = lib().pot_cell_kernel_time(ctx.handle, int(reset), ctypes.byref(la), ctypes.byref(ce),
                                      ctypes.byref(ms))
    if code != POT_OK:
        raise PotError(code, "pot_cell_kernel_time")
    return {"launches": int(la.value), "cells": int(ce.value), "ms": float(ms.value)}


def default_params(**kw) -> Params:
    p = Params()
    lib().pot_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "gravity":
            for i in range(3):
                p.gravity[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def _domain(dom) -> Domain:
    d = Domain()
    for k in range(3):
        d.lo[k] = float(dom[0][k])
        d.hi[k] = float(dom[1][k])
    return d


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, shape, name, device):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, context on {device}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


class Context:
    """A libpot context (workspace for up to n_max sites) on one device."""

    def __init__(self, n_max: int, k_max: int = 246, device: int = 0, fp32: bool = True,
                 fp64: bool = True):
        self._h = ctypes.c_void_p()
        self.device = torch.device("cuda", device)
        self.n_max = int(n_max)
        self.k_max = int(k_max)
        mask = (1 if fp32 else 0) | (2 if fp64 else 0)
        with torch.cuda.device(device):
            code = lib().pot_create(ctypes.byref(self._h), device, self.n_max, self.k_max, mask)
        if code != POT_OK:
            raise PotError(code, "pot_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().pot_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def lgc_compute_cells(ctx: Context, pos, psi, targets=None, domain=UNIT_BOX, hessian=True,
                      centroids=True, karea=True, csr_cap=None, stream=None, check=True):
    """Generalized Laguerre cells (Eq. 1): volumes, gradient nu - V, CSR of
    M = -grad^2 K (Eq. 2), centroids, free-surface areas.  Returns a dict of
    CUDA tensors plus 'stats' and 'status'."""
    dt = pos.dtype
    if dt not in (torch.float32, torch.float64):
        raise TypeError("pos must be float32 or float64")
    n = int(pos.shape[0])
    dev = ctx.device
    pos = _dev(pos, dt, (n, 3), "pos", dev)
    psi = _dev(psi, dt, (n,), "psi", dev)
    if targets is not None:
        targets = _dev(targets, torch.float64, (n,), "targets", dev)
    out = {"volumes": torch.empty(n, dtype=dt, device=dev),
           "grad": torch.empty(n, dtype=torch.float64, device=dev)}
    out["centroids"] = torch.empty((n, 3), dtype=dt, device=dev) if centroids else None
    out["karea"] = torch.empty(n, dtype=dt, device=dev) if karea else None
    csr = None
    if hessian:
        cap = int(csr_cap) if csr_cap is not None else n * (ctx.k_max + 1)
        out["row_ptr"] = torch.empty(n + 1, dtype=torch.int32, device=dev)
        out["cols"] = torch.empty(cap, dtype=torch.int32, device=dev)
        out["vals"] = torch.empty(cap, dtype=dt, device=dev)
        csr = Csr(out["row_ptr"].data_ptr(), out["cols"].data_ptr(), out["vals"].data_ptr(), cap, 0)
    st = CellStats()
    f = lib().lgc_compute_cells if dt == torch.float32 else lib().lgc_compute_cells_f64
    dom = _domain(domain)
    code = f(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(psi), _ptr(targets), ctypes.byref(dom),
             _ptr(out["volumes"]), _ptr(out["grad"]), ctypes.byref(csr) if csr else None,
             _ptr(out["centroids"]), _ptr(out["karea"]), ctypes.byref(st))
    out["stats"] = _as_dict(st)
    out["status"] = code
    if hessian:
        out["nnz"] = int(csr.nnz)
        if code == POT_OK:
            out["cols"] = out["cols"][: csr.nnz]
            out["vals"] = out["vals"][: csr.nnz]
    if check and code != POT_OK:
        raise PotError(code, "lgc_compute_cells", out["stats"])
    return out


def pot_newton_solve(ctx: Context, pos, targets, psi, domain=UNIT_BOX, params=None, stream=None,
                     check=True):
    """Damped Newton with KMT steps (Algorithm 1); psi is updated in place.
    Returns the stats dict (status included)."""
    dt = pos.dtype
    n = int(pos.shape[0])
    dev = ctx.device
    pos = _dev(pos, dt, (n, 3), "pos", dev)
    targets = _dev(targets, torch.float64, (n,), "targets", dev)
    if not (psi.is_cuda and psi.is_contiguous() and psi.dtype == dt and psi.shape == (n,)):
        raise ValueError("psi must be a contiguous CUDA tensor of shape (n,) and pos's dtype")
    p = params if params is not None else default_params()
    st = SolveStats()
    f = lib().pot_newton_solve if dt == torch.float32 else lib().pot_newton_solve_f64
    dom = _domain(domain)
    code = f(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(targets), _ptr(psi), ctypes.byref(dom),
             ctypes.byref(p), ctypes.byref(st))
    s = _as_dict(st)
    s["status"] = code
    if check and code != POT_OK:
        raise PotError(code, "pot_newton_solve", s)
    return s


def pot_fluid_step(ctx: Context, pos, vel, psi, targets, domain=UNIT_BOX, params=None, stream=None,
                   check=True):
    """One fluid step (Sec. 5); pos, vel, psi updated in place.  Returns stats."""
    dt = pos.dtype
    n = int(pos.shape[0])
    for name, t, shape in (("pos", pos, (n, 3)), ("vel", vel, (n, 3)), ("psi", psi, (n,))):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt and tuple(t.shape) == shape):
            raise ValueError(f"{name} must be a contiguous CUDA tensor {shape} of pos's dtype")
    targets = _dev(targets, torch.float64, (n,), "targets", ctx.device)
    p = params if params is not None else default_params()
    st = SolveStats()
    f = lib().pot_fluid_step if dt == torch.float32 else lib().pot_fluid_step_f64
    dom = _domain(domain)
    code = f(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(vel), _ptr(psi), _ptr(targets),
             ctypes.byref(dom), ctypes.byref(p), ctypes.byref(st))
    s = _as_dict(st)
    s["status"] = code
    if check and code != POT_OK:
        raise PotError(code, "pot_fluid_step", s)
    return s


def render_depth(ctx: Context, pos, psi, origin, forward, up, fov_y, width, height, karea=None,
                 domain=UNIT_BOX, normals=True, stream=None):
    """First point of each camera ray inside the fluid (pot_render_depth):
    depth (height, width) with -1 for a miss, and unit normals
    (height, width, 3) when `normals`."""
    n = int(pos.shape[0])
    dev = ctx.device
    pos = _dev(pos, torch.float32, (n, 3), "pos", dev)
    psi = _dev(psi, torch.float32, (n,), "psi", dev)
    if karea is not None:
        karea = _dev(karea, torch.float32, (n,), "karea", dev)
    cam = Camera()
    for k in range(3):
        cam.origin[k], cam.forward[k], cam.up[k] = float(origin[k]), float(forward[k]), float(up[k])
    cam.fov_y, cam.width, cam.height = float(fov_y), int(width), int(height)
    depth = torch.empty((height, width), dtype=torch.float32, device=dev)
    normal = torch.empty((height, width, 3), dtype=torch.float32, device=dev) if normals else None
    code = lib().pot_render_depth(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(psi), _ptr(karea),
                                  ctypes.byref(_domain(domain)), ctypes.byref(cam), _ptr(depth),
                                  _ptr(normal))
    if code != POT_OK:
        raise PotError(code, "pot_render_depth")
    return depth, normal


def render_volume(ctx: Context, pos, psi, origin, forward, up, fov_y, width, height,
                  domain=UNIT_BOX, stream=None, visits=True):
    """Walk camera rays through the fluid cell by cell (pot_render_volume):
    returns (first entry t, thickness, last exit t, cells visited or None),
    each (height, width) on the device."""
    dev = ctx.device
    n = int(pos.shape[0])
    pos = _dev(pos, torch.float32, (n, 3), "pos", dev)
    psi = _dev(psi, torch.float32, (n,), "psi", dev)
    first = torch.empty((height, width), dtype=torch.float32, device=dev)
    thick = torch.empty((height, width), dtype=torch.float32, device=dev)
    last = torch.empty((height, width), dtype=torch.float32, device=dev)
    vis = torch.empty((height, width), dtype=torch.int32, device=dev) if visits else None
    cam = Camera()
    for k in range(3):
        cam.origin[k], cam.forward[k], cam.up[k] = float(origin[k]), float(forward[k]), float(up[k])
    cam.fov_y, cam.width, cam.height = float(fov_y), int(width), int(height)
    code = lib().pot_render_volume(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(psi),
                                   ctypes.byref(_domain(domain)), ctypes.byref(cam), _ptr(first),
                                   _ptr(thick), _ptr(last), _ptr(vis))
    if code != POT_OK:
        raise PotError(code, "pot_render_volume")
    return first, thick, last, vis


def render_smooth(ctx: Context, pos, psi, origin, forward, up, fov_y, width, height, k,
                  domain=UNIT_BOX, stream=None, normals=True, steps=True):
    """Sphere-trace camera rays to the smoothed free surface with smoothing
    radius k (pot_render_smooth): returns (depth, normal or None, steps or
    None), (height, width[, 3]) on the device."""
    dev = ctx.device
    n = int(pos.shape[0])
    pos = _dev(pos, torch.float32, (n, 3), "pos", dev)
    psi = _dev(psi, torch.float32, (n,), "psi", dev)
    depth = torch.empty((height, width), dtype=torch.float32, device=dev)
    nrm = torch.empty((height, width, 3), dtype=torch.float32, device=dev) if normals else None
    st = torch.empty((height, width), dtype=torch.int32, device=dev) if steps else None
    cam = Camera()
    for c in range(3):
        cam.origin[c], cam.forward[c], cam.up[c] = float(origin[c]), float(forward[c]), float(up[c])
    cam.fov_y, cam.width, cam.height = float(fov_y), int(width), int(height)
    code = lib().pot_render_smooth(ctx.handle, _stream(stream), n, _ptr(pos), _ptr(psi),
                                   ctypes.byref(_domain(domain)), ctypes.byref(cam), float(k),
                                   _ptr(depth), _ptr(nrm), _ptr(st))
    if code != POT_OK:
        raise PotError(code, "pot_render_smooth")
    return depth, nrm, st


def set_viscosity_factors(ctx: Context, factors):
    """Per-site viscosity factors (mu_ij = mu (f_i + f_j) / 2) for later
    viscous fluid steps; None clears them.  The tensor must stay alive while
    they are in use (the library keeps its pointer)."""
    if factors is None:
        code = lib().pot_set_viscosity_factors(ctx.handle, 0, None)
        ctx._visc_factors = None
    else:
        n = int(factors.shape[0])
        factors = _dev(factors, torch.float32, (n,), "factors", ctx.device)
        ctx._visc_factors = factors
        code = lib().pot_set_viscosity_factors(ctx.handle, n, _ptr(factors))
    if code != POT_OK:
        raise PotError(code, "pot_set_viscosity_factors")


def clear_history(ctx: Context):
    """Forget the weight history of the extrapolated start (warm_start = 2)."""
    code = lib().pot_clear_history(ctx.handle)
    if code != POT_OK:
        raise PotError(code, "pot_clear_history")


def relax_to_centroids(ctx: Context, pos, psi, targets, rounds: int, domain=UNIT_BOX, params=None):
    """Start state of a fluid run at rest under the pressure spring of Sec. 5
    (F_p = (c_i - x_i) / eps^2): solve, then `rounds` times move every site to
    its cell's centroid and solve again (Lloyd steps of the volume-constrained
    diagram).  pos and psi are updated in place; returns the solves' stats and
    the mean and max site-to-centroid distance before each move."""
    out = {"solves": [pot_newton_solve(ctx, pos, targets, psi, domain=domain, params=params)],
           "moved_mean": [], "moved_max": []}
    for _ in range(rounds):
        cells = lgc_compute_cells(ctx, pos, psi, targets, domain=domain, hessian=False, karea=False)
        d = (cells["centroids"] - pos).norm(dim=1)
        out["moved_mean"].append(float(d.mean()))
        out["moved_max"].append(float(d.max()))
        pos.copy_(cells["centroids"])
        out["solves"].append(pot_newton_solve(ctx, pos, targets, psi, domain=domain, params=params))
    return out


# ---------------------------------------------------------------------------
# learned warm start


class Mlp:
    """The warm-start MLP (80 -> 128 -> 128 -> 128 -> 1, BF16 on tensor cores)."""

    N_IN = 80

    def __init__(self, max_rows: int, device: int = 0):
        self._h = ctypes.c_void_p()
        self.device = torch.device("cuda", device)
        self.max_rows = int(max_rows)
        with torch.cuda.device(device):
            code = lib().pot_mlp_create(ctypes.byref(self._h), device, self.max_rows)
        if code != POT_OK:
            raise PotError(code, "pot_mlp_create")

    @staticmethod
    def num_params() -> int:
        return int(lib().pot_mlp_num_params())

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().pot_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code, where):
        if code != POT_OK:
            raise PotError(code, where)

    def set_params(self, params, stream=None):
        p = _dev(params, torch.float32, (self.num_params(),), "params", self.device)
        self._check(lib().pot_mlp_set_params(self._h, _stream(stream), _ptr(p)), "pot_mlp_set_params")

    def get_params(self, stream=None):
        p = torch.empty(self.num_params(), dtype=torch.float32, device=self.device)
        self._check(lib().pot_mlp_get_params(self._h, _stream(stream), _ptr(p)), "pot_mlp_get_params")
        return p

    def forward(self, x, stream=None):
        rows = int(x.shape[0])
        x = _dev(x, torch.bfloat16, (rows, self.N_IN), "x", self.device)
        out = torch.empty(rows, dtype=torch.float32, device=self.device)
        self._check(lib().pot_mlp_forward(self._h, _stream(stream), rows, _ptr(x), _ptr(out)),
                    "pot_mlp_forward")
        return out

    def gradients(self, x_all, y_all, idx, stream=None):
        n_all, batch = int(x_all.shape[0]), int(idx.shape[0])
        x_all = _dev(x_all, torch.bfloat16, (n_all, self.N_IN), "x_all", self.device)
        y_all = _dev(y_all, torch.float32, (n_all,), "y_all", self.device)
        idx = _dev(idx, torch.int32, (batch,), "idx", self.device)
        g = torch.empty(self.num_params(), dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        self._check(lib().pot_mlp_gradients(self._h, _stream(stream), n_all, _ptr(x_all), _ptr(y_all),
                                            _ptr(idx), batch, _ptr(g), _ptr(loss)), "pot_mlp_gradients")
        return g, loss

    def train_step(self, x_all, y_all, idx, lr=1e-3, loss=None, stream=None):
        """One Adam step on rows idx; the batch loss lands in `loss` (device)."""
        n_all, batch = int(x_all.shape[0]), int(idx.shape[0])
        self._check(lib().pot_mlp_train_step(self._h, _stream(stream), n_all, _ptr(x_all), _ptr(y_all),
                                             _ptr(idx), batch, ctypes.c_float(lr), _ptr(loss)),
                    "pot_mlp_train_step")

    def check(self, stream=None):
        self._check(lib().pot_mlp_check(self._h, _stream(stream)), "pot_mlp_check")

    def set_history(self, psi_old, stream=None):
        """Seed (psi_old: n weights, caller order) or clear (None) the weight
        history the next warm-started fluid step reads."""
        if psi_old is None:
            self._check(lib().pot_mlp_set_history(self._h, _stream(stream), 0, None),
                        "pot_mlp_set_history")
            return
        n = int(psi_old.shape[0])
        psi_old = _dev(psi_old, torch.float32, (n,), "psi_old", self.device)
        self._check(lib().pot_mlp_set_history(self._h, _stream(stream), n, _ptr(psi_old)),
                    "pot_mlp_set_history")

    def set_inputs(self, n_inputs):
        """77 inputs (with the previous weight change; the default) or 76
        (without it: the prediction corrects the previous weights)."""
        self._check(lib().pot_mlp_set_inputs(self._h, int(n_inputs)), "pot_mlp_set_inputs")


def pot_mlp_features(ctx: Context, mlp: Mlp, pos, vel, psi, targets, domain=UNIT_BOX, params=None,
                     stream=None, psi_old=None):
    """Warm-start features (n x 80 BF16, caller order) at the state the next
    fluid step solves at; psi_old: the weights one step before psi (None: no
    history)."""
    n = int(pos.shape[0])
    dev = ctx.device
    pos = _dev(pos, torch.float32, (n, 3), "pos", dev)
    vel = _dev(vel, torch.float32, (n, 3), "vel", dev)
    psi = _dev(psi, torch.float32, (n,), "psi", dev)
    if psi_old is not None:
        psi_old = _dev(psi_old, torch.float32, (n,), "psi_old", dev)
    targets = _dev(targets, torch.float64, (n,), "targets", dev)
    p = params if params is not None else default_params()
    feat = torch.empty((n, Mlp.N_IN), dtype=torch.bfloat16, device=dev)
    dom = _domain(domain)
    code = lib().pot_mlp_features(ctx.handle, mlp.handle, _stream(stream), n, _ptr(pos), _ptr(vel),
                                  _ptr(psi), _ptr(psi_old) if psi_old is not None else None,
                                  _ptr(targets), ctypes.byref(dom), ctypes.byref(p), _ptr(feat))
    if code != POT_OK:
        raise PotError(code, "pot_mlp_features")
    return feat


def set_warm_start(ctx: Context, mlp):
    code = lib().pot_set_warm_start(ctx.handle, mlp.handle if mlp is not None else None)
    if code != POT_OK:
        raise PotError(code, "pot_set_warm_start")

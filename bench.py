#!/usr/bin/env python
"""Benchmark: partial-OT fluid steps on the two-ball splash at ~2M sites.

One step = one complete fluid step (Sec. 5): advect, grid build, Newton solve
to 1e-4 worst-cell relative volume error (Algorithm 1: cell geometry, CSR
Hessian, Jacobi-PCG, KMT line search), centroids, velocity update.  Inputs
are resident in HBM when the timed region starts; the working set (sites,
CSR Hessian, candidate lists) is larger than the 126 MB L2, so no flush is
needed between steps.

value  = cells/s: sites whose generalized Laguerre cell is solved to 1e-4 per
         second (N x steps / device time), summed over ranks.
extras = Newton solve ms (median, p90), geometry throughput (cell
         evaluations per second of the cell kernels), iteration counts.
e2e    = the same metric through the public API with host buffers: every step
         copies the state from pinned host memory and reads it back.
--gpus N runs N independent replicas (one process per GPU, different seeds);
the path has no exchange step of its own.

--impl reference times the FP64 CPU oracle (its Newton with a dense solve)
on the same splash recipe scaled to ~2000 sites, one oracle fluid step per
step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPLASH_DT = 5e-4
SMALL_SPACING = 0.032  # ~2000 sites with the splash recipe


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="step", choices=["step", "cells"],
                    help="step: fluid steps on the splash; cells: lgc_compute_cells alone on the "
                         "2^20-site random cloud")
    ap.add_argument("--spacing", type=float, default=3.224e-3, help="splash lattice spacing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: barrier and max/sum over ranks)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_timing(seconds: float, units: float, world: int, device=None):
    """Whole-job timing: max seconds over ranks, total units over ranks."""
    if world <= 1:
        return seconds, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# oracle fluid steps (reference arm and cpu_baseline)


def oracle_steps(seconds_budget: float, max_steps: int, seed: int = 3):
    """Run oracle fluid steps on the small splash until the budget or step
    count is reached; returns (cells/s, steps, sites, cores, seconds)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2601_05765_b300 import scenes
    sc = scenes.splash(spacing=SMALL_SPACING, seed=seed)
    n = sc.n
    cores = O.max_threads()
    x = sc.pos.astype(np.float64)
    v = sc.vel.astype(np.float64)
    psi = sc.psi.astype(np.float64)
    # converge the start once (not timed): steps are then warm-started solves
    psi = O.newton(x, sc.nu, psi, tol=1e-4).psi
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (time.perf_counter() - t0) < seconds_budget:
        x, v, nr = O.fluid_step(x, v, psi, sc.nu, dt=SPLASH_DT, tol=1e-4)
        psi = nr.psi
        steps += 1
    dt = time.perf_counter() - t0
    return n * steps / dt, steps, n, cores, dt


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    # warm-up steps, then timed steps, each one oracle fluid step
    oracle_steps(1e9, max(args.warmup, 0))
    val, steps, n, cores, dt = oracle_steps(1e9, args.steps)
    line = {
        "impl": "reference", "metric": "generalized Laguerre cells/s (cells solved to 1e-4 per second)",
        "value": val, "unit": "cells/s", "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"two-ball splash, {n} sites (spacing {SMALL_SPACING}), dt {SPLASH_DT}",
                   "tol": 1e-4},
        "cpu_baseline": {"value": val, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"oracle fluid steps (dense-LU Newton, KMT, tol 1e-4) on the splash "
                                   f"recipe at {n} sites"},
        "e2e": {"value": val, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


def run_ours(args):
    import numpy as np
    import torch

    from paper_2601_05765_b300 import pot, scenes

    rank, world, local = dist_env()
    dist_init(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.splash(spacing=args.spacing, seed=3 + rank)
    n = sc.n
    ctx = pot.Context(n, 256, local, fp32=True, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    vel = torch.from_numpy(sc.vel).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    prm = pot.default_params(dt=SPLASH_DT)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)

    # ---- device-timed region
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    sampler = ClockSampler(gpu_index)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    l0 = pot.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        stats.append(pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm))
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pot.kernel_launches() - l0
    barrier(world)
    clocks = sampler.stop()
    t_dev = e0.elapsed_time(e1) / 1e3
    T, units = reduce_timing(t_dev, n * args.steps, world, dev)
    value = units / T

    # ---- end to end through the public API with host buffers
    h_pos = pos.cpu().pin_memory()
    h_vel = vel.cpu().pin_memory()
    h_psi = psi.cpu().pin_memory()
    h_nu = nu.cpu().pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        pos.copy_(h_pos, non_blocking=True)
        vel.copy_(h_vel, non_blocking=True)
        psi.copy_(h_psi, non_blocking=True)
        nu.copy_(h_nu, non_blocking=True)
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
        h_pos.copy_(pos, non_blocking=True)
        h_vel.copy_(vel, non_blocking=True)
        h_psi.copy_(psi, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    T_e2e, units_e2e = reduce_timing(f0.elapsed_time(f1) / 1e3, n * args.steps, world, dev)
    h2d = n * (12 + 12 + 4 + 8)
    d2h = n * (12 + 12 + 4)

    # ---- per-phase numbers from the library's CUDA-event timers
    solve_ms = sorted(s["ms_total"] for s in stats)
    evals = sum(s["cell_evals"] for s in stats)
    ms_cells = sum(s["ms_cells"] for s in stats)
    ms_pcg = sum(s["ms_pcg"] for s in stats)
    pcg_iters = sum(s["pcg_iters"] for s in stats)
    nnz = statistics.mean(s["nnz"] for s in stats)
    # PCG iteration (k_spmv + k_update), algorithmic bytes in FP32:
    #   spmv: 8 B per off-diagonal entry (value + column) + row_ptr, diag,
    #         z, p_old reads and p_new, q writes (6 x 4 B per row);
    #   update: diag, x, r, p, q reads and x, r, z writes (8 x 4 B per row)
    nnz_off = nnz - n
    bytes_per_iter = 8.0 * nnz_off + 4.0 * (6 + 8) * n
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_iter * pcg_iters / (ms_pcg / 1e3) / 1e9 if ms_pcg > 0 else None
    line = {
        "metric": "generalized Laguerre cells/s (cells solved to 1e-4 per second)",
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry, f64 reductions", "data": "synthetic",
        "config": {"workload": f"two-ball splash (configs[3] recipe), {n} sites per GPU, 1e-4 Newton per step",
                   "sites_per_gpu": n, "dt": SPLASH_DT, "tol": 1e-4, "parallelism": f"replicas x{world}",
                   "l2": "working set > 126 MB L2, no flush"},
        "newton_solve_ms": {"median": solve_ms[len(solve_ms) // 2],
                            "p90": solve_ms[min(len(solve_ms) - 1, int(0.9 * len(solve_ms)))]},
        "cell_eval_cells_per_s": n * evals / (ms_cells / 1e3) if ms_cells > 0 else None,
        "newton_iters_per_step": statistics.mean(s["newton_iters"] for s in stats),
        "pcg_iters_per_step": pcg_iters / args.steps,
        "cell_evals_per_step": evals / args.steps,
        "ms_cells_per_step": ms_cells / args.steps,
        "ms_pcg_per_step": ms_pcg / args.steps,
        "nnz": nnz,
        "max_err": max(s["err_max"] for s in stats),
        "status": sorted({s["status"] for s in stats}),
        "roofline": {"kernel": "PCG iteration (k_spmv + k_update)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "peak_kind": peak_kind, "bytes_per_iter": bytes_per_iter},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": units_e2e / T_e2e, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, steps, nsm, cores, dt = oracle_steps(args.cpu_seconds, 1000)
        line["cpu_baseline"] = {"value": val, "unit": "cells/s", "cores": cores, "kind": "oracle",
                                "sample": f"{steps} oracle fluid steps (dense-LU Newton, KMT, tol 1e-4) "
                                          f"on the splash recipe at {nsm} sites, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def run_cells(args):
    """lgc_compute_cells (grid, candidates, cell geometry, CSR) on the 2^20-site
    random cloud: generalized Laguerre cells per second of the cell path."""
    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    sc = scenes.uniform_cloud(n=1 << 20, seed=1)
    n = sc.n
    ctx = pot.Context(n, 128, 0, fp32=True, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    for _ in range(args.warmup):
        pot.lgc_compute_cells(ctx, pos, psi, nu)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = []
    l0 = pot.kernel_launches()
    e0.record(stream)
    for _ in range(args.steps):
        st.append(pot.lgc_compute_cells(ctx, pos, psi, nu)["stats"])
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    ms = {k: statistics.mean(s[k] for s in st) for k in ("ms_grid", "ms_cells", "ms_csr")}
    print(json.dumps({"metric": "generalized Laguerre cells/s (lgc_compute_cells, 2^20-site random cloud)",
                      "value": n / t, "unit": "cells/s", "ms_per_call": 1e3 * t, **ms,
                      "nnz": st[-1]["nnz"], "gpu_launches": pot.kernel_launches() - l0,
                      "geometry_cells_per_s": n / (ms["ms_cells"] / 1e3)}))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "cells":
        run_cells(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

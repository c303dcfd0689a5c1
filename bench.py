#!/usr/bin/env python
"""Benchmark: partial-OT fluid steps on the two-ball splash at ~2M sites.

One step = one complete fluid step (Sec. 5): advect, grid build, Newton solve
to 1e-4 worst-cell relative volume error (Algorithm 1: cell geometry, CSR
Hessian, Jacobi-PCG, KMT line search), centroids, velocity update.  The
timed steps are steps 0..K-1 of the run (default K = 100: the balls touch
near step 10 and are pressed together until the end), from the recipe's
start state (sites at their cell centroids); the warm-up steps run from the
same state, which is restored before the timed region.  Inputs are resident
in HBM when the timed region starts; the working set (sites, CSR Hessian,
candidate lists) is larger than the 126 MB L2, so no flush is needed between
steps.

value  = cells/s: sites whose generalized Laguerre cell is solved to 1e-4 per
         second (N x steps / device time), summed over ranks.
extras = Newton solve ms (median, p90), geometry throughput (cell
         evaluations per second of the cell kernels), iteration counts.
e2e    = the same metric through the public API with host buffers: the same
         steps are run again from a pinned-host snapshot of the state the
         timed region started from; every step copies the state in from
         pinned host memory and the new state back out.
roofline = the dominant kernel, k_cells (clipping, restriction, analytic
         quantities), against the FP32 ALU peak: FLOP per processed cell
         from ncu x cells per launch / the launch's event-timed duration
         (the library times every k_cells launch with CUDA events).
         roofline_pcg: the PCG iteration against the measured HBM copy
         bandwidth.
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

SMALL_SPACING = 0.032  # ~2000 sites with the splash recipe
# Per cell processed by k_cells, from an ncu capture of one launch on the
# splash recipe at 536k sites, step 30 (the bench's run in miniature;
# profiles/k_cells_splash_536k_step30.md): FP32 FLOP executed (fadd + fmul +
# 2 ffma of the instruction mix), warp instructions issued, and DRAM bytes
# (cold caches: ncu flushes them before the launch).
K_CELLS_FLOP_PER_CELL = 5505.7
K_CELLS_WARP_INST_PER_CELL = 823.8
K_CELLS_DRAM_BYTES_PER_CELL = 383.1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="step",
                    choices=["step", "cells", "warmstart", "dam", "solve", "robust", "render"],
                    help="step: fluid steps on the splash; cells: lgc_compute_cells alone; "
                         "warmstart: train the warm-start MLP on dam-break columns, then run the "
                         "same splash steps from the plain and the learned start; dam: the 500k "
                         "dam break in mixed precision and in FP64; solve: the 1000-site single "
                         "Newton solve")
    ap.add_argument("--scene", default="cloud", choices=["cloud", "splash"],
                    help="cells mode: the 2^20-site random cloud, or the splash at converged weights")
    ap.add_argument("--spacing", type=float, default=3.224e-3, help="splash lattice spacing")
    ap.add_argument("--mu", type=float, default=0.0, help="dam mode: viscosity (Eq. 4)")
    ap.add_argument("--gamma", type=float, default=0.0, help="dam mode: surface tension")
    ap.add_argument("--mu-wall", type=float, default=0.0, help="dam mode: no-slip wall viscosity")
    ap.add_argument("--advance", type=int, default=0,
                    help="cells mode, splash: fluid steps taken from the recipe's start state "
                         "before the timed calls")
    ap.add_argument("--train-splash", action="store_true",
                    help="warmstart mode: add free-flight samples (small splashes before contact, "
                         "other seeds) to the dam-break training set")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads' numbers (FP32 peak, 2^20 cloud, 1000-site solve)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--pcg-host-loop", action="store_true",
                    help="step mode: host-driven PCG launches instead of the device-side loop "
                         "(slower; lets a profiler see every PCG kernel)")
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
    # the recipe's start state (not timed): converged weights, sites moved
    # to their cell centroids, converged again
    psi = O.newton(x, sc.nu, psi, tol=1e-4).psi
    for _ in range(sc.extra["relax_rounds"]):
        x = O.cells(x, psi)["cen"].copy()
        psi = O.newton(x, sc.nu, psi, tol=1e-4).psi
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (time.perf_counter() - t0) < seconds_budget:
        x, v, nr = O.fluid_step(x, v, psi, sc.nu, dt=sc.extra["dt"], eps=sc.extra["eps"], tol=1e-4)
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
        "config": {"workload": f"two-ball splash (radius 0.2, \u00b13 m/s), {n} sites "
                               f"(spacing {SMALL_SPACING}), steps 0..{steps - 1}",
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


def k_cells_roofline(kc, clocks, sm_count, fp32_peak=None):
    """ALU roofline of the cell kernel from its live event timings.

    Work per cell = FP32 FLOP executed per processed cell (fadd + fmul +
    2 ffma) counted by ncu on the splash at converged weights; peak = the
    FP32 FMA throughput measured on this GPU by the library's FMA-chain
    kernel (else SMs x 128 FP32 lanes x 2 FLOP x the median SM clock sampled
    during the timed region).  The kernel is mostly control, shuffles and
    shared-memory traffic around its FP32 math, so the instruction issue
    rate is given too: warp instructions per cell from the same capture
    against 4 issue slots per SM per clock.  Traffic per launch = DRAM bytes
    per processed cell from the same capture x cells per launch."""
    if not kc["launches"] or kc["ms"] <= 0:
        return None
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2032.0
    if fp32_peak:
        peak = fp32_peak
        kind = "measured: FP32 FMA chains on this GPU (pot_measure_fp32_peak, best of 5)"
    else:
        peak = sm_count * 128 * 2 * mhz * 1e6 / 1e12
        kind = f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (median under load)"
    cells_per_launch = kc["cells"] / kc["launches"]
    launch_ms = kc["ms"] / kc["launches"]
    out = {"kernel": "k_cells", "bound": "alu", "unit": "TFLOP/s", "peak": peak,
           "peak_kind": kind,
           "cells_per_launch": cells_per_launch, "launch_ms": launch_ms, "launches": kc["launches"],
           "flop_per_cell": K_CELLS_FLOP_PER_CELL, "achieved": None, "frac": None, "traffic": None}
    if K_CELLS_FLOP_PER_CELL:
        out["achieved"] = K_CELLS_FLOP_PER_CELL * cells_per_launch / (launch_ms / 1e3) / 1e12
        out["frac"] = out["achieved"] / peak
    if K_CELLS_DRAM_BYTES_PER_CELL:
        out["traffic"] = K_CELLS_DRAM_BYTES_PER_CELL * cells_per_launch
    issue_peak = sm_count * 4 * mhz * 1e6 / 1e9
    issue = K_CELLS_WARP_INST_PER_CELL * cells_per_launch / (launch_ms / 1e3) / 1e9
    out["issue"] = {"achieved": issue, "peak": issue_peak, "unit": "G warp instructions/s",
                    "frac": issue / issue_peak,
                    "peak_kind": f"{sm_count} SMs x 4 issue slots x {mhz:.0f} MHz"}
    return out


def secondary(dev, cpu_baseline=True):
    """The other workloads' headline numbers, each within a few seconds:
    the FP32 FMA peak; lgc_compute_cells on the 2^20-site random cloud
    (median of 20 calls after 3 warm-ups, grid build reported separately);
    the 1000-site jittered block solved to 1e-4 from psi0 in mixed precision
    and in FP64 (median of 5 after 1 warm-up); and the oracle on the cloud's
    10k-cell subset, single-threaded and on all host cores."""
    import numpy as np
    import torch

    from paper_2601_05765_b300 import pot, scenes
    out = {"fp32_peak_tflops": pot.measure_fp32_peak(dev)["tflops"]}
    stream = torch.cuda.current_stream()
    sc = scenes.uniform_cloud(n=1 << 20, seed=1)
    ctx = pot.Context(sc.n, 128, dev.index, fp32=True, fp64=False)
    pos, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.psi, sc.nu))
    for _ in range(3):
        pot.lgc_compute_cells(ctx, pos, psi, nu)
    times, st = [], []
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.append(pot.lgc_compute_cells(ctx, pos, psi, nu)["stats"])
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.close()
    times.sort()
    med = times[len(times) // 2]
    out["cells_per_s_cloud"] = {
        "value": sc.n / (med / 1e3), "unit": "cells/s", "ms_per_call_median": med,
        "ms_grid": statistics.mean(x["ms_grid"] for x in st),
        "ms_cells": statistics.mean(x["ms_cells"] for x in st),
        "ms_csr": statistics.mean(x["ms_csr"] for x in st),
        "workload": "lgc_compute_cells (grid, candidates, cells, CSR Hessian) on the 2^20-site "
                    "random cloud (positions U(0,1)^3 seed 1, r = U(0.4,1.2) (3/(4 pi N))^(1/3)), "
                    "median of 20 calls"}
    blk = scenes.jittered_block()
    solve = {}
    for prec, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
        ctx = pot.Context(blk.n, 246, dev.index, fp32=dt == torch.float32, fp64=dt == torch.float64)
        p = torch.as_tensor(blk.pos, dtype=dt, device=dev)
        n_ = torch.as_tensor(blk.nu, dtype=torch.float64, device=dev)
        ts, it = [], None
        for k in range(6):
            ps = torch.as_tensor(blk.psi, dtype=dt, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it = pot.pot_newton_solve(ctx, p, n_, ps)
            torch.cuda.synchronize()
            if k:
                ts.append(1e3 * (time.perf_counter() - t0))
        ctx.close()
        ts.sort()
        solve[prec] = {"ms": ts[len(ts) // 2], "newton_iters": it["newton_iters"],
                       "pcg_iters": it["pcg_iters"], "err_max": it["err_max"]}
    out["solve_1000_ms"] = {**solve, "workload": "jittered 10x10x10 block (spacing 0.05, seed 0), "
                                                 "psi0 = (0.8 r_nu)^2, Newton to 1e-4, host wall time"}
    if cpu_baseline:
        from oracle import oracle as O
        q = sc.extra["subset"]
        res = {}
        for name, nt in (("1_thread", 1), ("all_cores", 0)):
            t0 = time.perf_counter()
            O.cells(sc.pos.astype(np.float64), sc.psi.astype(np.float64), query=q, nthreads=nt)
            res[name] = len(q) / (time.perf_counter() - t0)
        out["cpu_baseline_cloud"] = {"unit": "cells/s", "kind": "oracle", "cores_all": O.max_threads(),
                                     **res, "sample": f"oracle cells of the cloud's {len(q)}-cell "
                                                      f"subset (seed 1001)"}
    return out


def run_ours(args):
    import torch

    from paper_2601_05765_b300 import pot, scenes

    rank, world, local = dist_env()
    dist_init(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.splash(spacing=args.spacing, seed=3 + rank)
    n = sc.n
    ctx = pot.Context(n, 246, local, fp32=True, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    vel = torch.from_numpy(sc.vel).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"],
                             pcg_host_loop=1 if args.pcg_host_loop else 0)
    stream = torch.cuda.current_stream()

    # the recipe's start state (untimed): sites at their cell centroids
    relax = pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    # the state the timed steps start from (step 0 of the run), kept on the
    # device for the restore after the warm-up and in pinned host memory for
    # the end-to-end run below, which repeats the same steps from it
    d0 = [t.clone() for t in (pos, vel, psi)]
    h0 = [t.cpu().pin_memory() for t in (pos, vel, psi)]
    for _ in range(args.warmup):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    for t, t0 in zip((pos, vel, psi), d0):
        t.copy_(t0)
    del d0

    # ---- device-timed region
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    sampler = ClockSampler(gpu_index)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    pot.cell_kernel_time(ctx, reset=True)
    l0 = pot.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        stats.append(pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm))
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pot.kernel_launches() - l0
    kc = pot.cell_kernel_time(ctx, reset=True)
    barrier(world)
    clocks = sampler.stop()
    t_dev = e0.elapsed_time(e1) / 1e3
    T, units = reduce_timing(t_dev, n * args.steps, world, dev)
    value = units / T

    # ---- end to end through the public API with host buffers: the same
    # steps, each one copying the state in from pinned host memory and the
    # new state back out.  The copies run on two side streams, array by
    # array: each array goes back in as soon as it has come out (the two
    # directions of the bus run at once), and the targets of the next step,
    # which no step changes, go into a second device buffer while the
    # current step computes.
    h_pos, h_vel, h_psi = (t.clone().pin_memory() for t in h0)
    h_nu = nu.cpu().pin_memory()
    nu_buf = [nu, torch.empty_like(nu)]
    s_out, s_in = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def event(s):
        e = torch.cuda.Event()
        e.record(s)
        return e

    barrier(world)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s_in.wait_event(f0)
    with torch.cuda.stream(s_in):
        for t, h in ((pos, h_pos), (vel, h_vel), (psi, h_psi), (nu_buf[0], h_nu)):
            t.copy_(h, non_blocking=True)
    ready = event(s_in)
    prev_done = f0
    for k in range(args.steps):
        stream.wait_event(ready)
        pot.pot_fluid_step(ctx, pos, vel, psi, nu_buf[k % 2], params=prm)
        done = event(stream)
        if k + 1 < args.steps:
            # the other targets buffer was last read by the previous step
            s_in.wait_event(prev_done)
            with torch.cuda.stream(s_in):
                nu_buf[(k + 1) % 2].copy_(h_nu, non_blocking=True)
        s_out.wait_event(done)
        outs = []
        with torch.cuda.stream(s_out):
            for t, h in ((pos, h_pos), (vel, h_vel), (psi, h_psi)):
                h.copy_(t, non_blocking=True)
                outs.append(event(s_out))
        if k + 1 < args.steps:
            with torch.cuda.stream(s_in):
                for (t, h), e in zip(((pos, h_pos), (vel, h_vel), (psi, h_psi)), outs):
                    s_in.wait_event(e)
                    t.copy_(h, non_blocking=True)
            ready = event(s_in)
        prev_done = done
    stream.wait_event(outs[-1])
    stream.wait_event(ready)
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
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    line = {
        "metric": "generalized Laguerre cells/s (cells solved to 1e-4 per second)",
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 geometry, f64 reductions", "data": "synthetic",
        "config": {"workload": f"two-ball splash (radius 0.2, \u00b13 m/s), {n} sites per GPU, "
                               f"1e-4 Newton per step",
                   "sites_per_gpu": n, "dt": prm.dt, "eps": prm.eps, "tol": 1e-4,
                   "timed_steps": f"0..{args.steps - 1} of the run (the warm-up steps are run "
                                  f"from the same start state, which is then restored)",
                   "start": f"{sc.extra['relax_rounds']} rounds of sites moved to their cell "
                            f"centroids (last move: mean {relax['moved_mean'][-1]:.2e}, max "
                            f"{relax['moved_max'][-1]:.2e})",
                   "recipe": f"splash: two balls of radius 0.2 centred at (0.5 -/+ (0.2 + s), 0.5, 0.5), "
                             f"+/-3 m/s along x, lattice spacing s = {args.spacing:g} jittered by 0.3 s "
                             f"(seed {3 + rank}), nu = 0.9 s^3, spring eps = s/16, dt = eps/2",
                   "parallelism": f"replicas x{world}",
                   "pcg": ("host-driven launches (profiling run)" if args.pcg_host_loop
                           else "device-side loop"),
                   "l2": "working set > 126 MB L2, no flush"},
        "newton_solve_ms": {"median": solve_ms[len(solve_ms) // 2],
                            "p90": solve_ms[min(len(solve_ms) - 1, int(0.9 * len(solve_ms)))]},
        "cell_eval_cells_per_s": n * evals / (ms_cells / 1e3) if ms_cells > 0 else None,
        "newton_iters_per_step": statistics.mean(s["newton_iters"] for s in stats),
        "pcg_iters_per_step": pcg_iters / args.steps,
        "cell_evals_per_step": evals / args.steps,
        "passes_per_step": sum(s["passes"] for s in stats) / args.steps,
        "ms_cells_per_step": ms_cells / args.steps,
        "ms_pcg_per_step": ms_pcg / args.steps,
        "nnz": nnz,
        "max_err": max(s["err_max"] for s in stats),
        "status": sorted({s["status"] for s in stats}),
        "roofline": None,
        "roofline_pcg": {"kernel": "PCG iteration (k_spmv + k_update)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_kind": peak_kind, "bytes_per_iter": bytes_per_iter},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": units_e2e / T_e2e, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": "the same steps as the device-timed region",
                "copies": "pinned host buffers; out and back in array by array on two side "
                          "streams, the next step's targets into a second buffer during the step"},
    }
    ctx.close()
    # the other workloads (rank 0 only; untimed for `value`)
    fp32_peak = None
    if rank == 0 and not args.no_extras:
        sec = secondary(dev, cpu_baseline=world == 1 and not args.no_cpu_baseline)
        fp32_peak = sec["fp32_peak_tflops"]
        line.update(sec)
    line["roofline"] = k_cells_roofline(kc, clocks, sm_count, fp32_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, steps, nsm, cores, dt = oracle_steps(args.cpu_seconds, 100)
        line["cpu_baseline"] = {"value": val, "unit": "cells/s", "cores": cores, "kind": "oracle",
                                "sample": f"oracle fluid steps 0..{steps - 1} (dense-LU Newton, KMT, "
                                          f"tol 1e-4) of the splash recipe at {nsm} sites, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line))


def run_cells(args):
    """lgc_compute_cells (grid, candidates, cell geometry, CSR) alone:
    generalized Laguerre cells per second of the cell path, on the 2^20-site
    random cloud or on the splash at converged weights: the recipe's start
    state (untimed), then `advance` untimed fluid steps."""
    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    if args.scene == "splash":
        sc = scenes.splash(spacing=args.spacing, seed=3)
        label = f"two-ball splash at converged weights, {sc.n} sites, step {args.advance}"
    else:
        sc = scenes.uniform_cloud(n=1 << 20, seed=1)
        label = "2^20-site random cloud"
    n = sc.n
    ctx = pot.Context(n, 246 if args.scene == "splash" else 128, 0, fp32=True, fp64=False)
    pos = torch.from_numpy(sc.pos).to(dev)
    psi = torch.from_numpy(sc.psi).to(dev)
    nu = torch.from_numpy(sc.nu).to(dev)
    if args.scene == "splash":
        prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
        pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
        vel = torch.from_numpy(sc.vel).to(dev)
        for _ in range(args.advance):
            pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    for _ in range(args.warmup):
        pot.lgc_compute_cells(ctx, pos, psi, nu)
    torch.cuda.synchronize()
    before = pot.cell_kernel_time(ctx, reset=True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    st = []
    l0 = pot.kernel_launches()
    for e0, e1 in ev:
        e0.record(stream)
        st.append(pot.lgc_compute_cells(ctx, pos, psi, nu)["stats"])
        e1.record(stream)
    torch.cuda.synchronize()
    kc = pot.cell_kernel_time(ctx, reset=True)
    times = sorted(e0.elapsed_time(e1) / 1e3 for e0, e1 in ev)
    t = times[len(times) // 2]
    ms = {k: statistics.mean(s[k] for s in st) for k in ("ms_grid", "ms_cells", "ms_csr")}
    line = {"metric": f"generalized Laguerre cells/s (lgc_compute_cells, {label})",
            "value": n / t, "unit": "cells/s", "ms_per_call_median": 1e3 * t,
            "ms_per_call_mean": 1e3 * statistics.mean(times), "calls": len(times), **ms,
            "nnz": st[-1]["nnz"], "max_planes": st[-1]["max_planes"],
            "gpu_launches": pot.kernel_launches() - l0,
            "geometry_cells_per_s": n / (ms["ms_cells"] / 1e3),
            "k_cells": kc, "k_cells_launches_before_timed": before["launches"]}
    if args.scene == "cloud" and not args.no_cpu_baseline:
        import numpy as np

        from oracle import oracle as O
        q = sc.extra["subset"]
        t0 = time.perf_counter()
        O.cells(sc.pos.astype(np.float64), sc.psi.astype(np.float64), query=q)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(q) / dt, "unit": "cells/s", "cores": O.max_threads(),
                                "kind": "oracle", "sample": f"oracle cells of the {len(q)}-cell subset "
                                                            f"(seed 1001), {dt:.1f} s"}
    print(json.dumps(line))
    ctx.close()


def run_warmstart(args):
    """Learned warm start against the plain start on the splash.

    Training: plain-Newton fluid substeps on dam-break columns (the
    dam-break recipe at spacing 0.4/24, 24 x 24 x 48 sites, seeds 10-19:
    spring s/8, its 2e-3 steps as substeps, the first 40 steps, every 2nd
    substep 4096 sampled sites), Adam on the library's tensor-core kernels.
    Every sample is one substep: the model predicts the weights of the next
    solve, which is what the fluid step asks it for.  Evaluation: after
    `warmup` plain steps, the same `steps` splash steps from the same state
    with the plain start (previous weights) and with the MLP start (its
    history seeded with the weights one step earlier), both FP32 geometry
    with FP64 reductions at tol 1e-4; the same comparison over substeps of a
    dam-break column of an unseen seed (in the training distribution) is
    reported beside it."""
    import torch

    from paper_2601_05765_b300 import pot, scenes
    from paper_2601_05765_b300 import warmstart as W
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    cols = [scenes.dam_break(nx=24, ny=24, nz=48, width=0.4, seed=s) for s in range(10, 20)]
    sc = scenes.splash(spacing=args.spacing, seed=3)
    ctx_t = pot.Context(cols[0].n, 246, 0, fp32=True, fp64=False)
    mlp = pot.Mlp(max(sc.n, 65536), 0)
    mlp.set_params(W.init_params(0, device=dev))
    xs, ys = [], []
    def sub(scene):
        e = scene.extra
        return e["dt"] / e["substeps"], e["eps"], e["substeps"], e["relax_rounds"]

    # the 76-input model of the configuration (no weight-change input; it
    # corrects the previous weights), trained on the same runs
    mlp76 = pot.Mlp(max(sc.n, 65536), 0)
    mlp76.set_inputs(76)
    mlp76.set_params(W.init_params(0, device=dev, n_inputs=76))
    xs76, ys76 = [], []
    for k, col in enumerate(cols):
        dts, eps, nsub, relax = sub(col)
        x, y = W.collect(ctx_t, mlp, col, steps=40 * nsub, every=2, per_sample=4096, seed=10 + k,
                         dt=dts, eps=eps, relax=relax)
        xs.append(x)
        ys.append(y)
        x, y = W.collect(ctx_t, mlp76, col, steps=40 * nsub, every=2, per_sample=4096, seed=10 + k,
                         dt=dts, eps=eps, relax=relax, history=False)
        xs76.append(x)
        ys76.append(y)
    ctx_t.close()
    extra = "none"
    if args.train_splash:
        # smaller splashes of the same recipe (spacing 0.01, about 65k
        # sites), seeds 40-43, the first 40 steps (contact near step 10)
        for k in range(4):
            sm = scenes.splash(spacing=0.01, seed=40 + k)
            ctx_s = pot.Context(sm.n, 246, 0, fp32=True, fp64=False)
            x, y = W.collect(ctx_s, mlp, sm, steps=40, every=2, per_sample=8192, seed=40 + k,
                             dt=sm.extra["dt"], eps=sm.extra["eps"], relax=sm.extra["relax_rounds"])
            xs.append(x)
            ys.append(y)
            ctx_s.close()
        extra = "small splashes (spacing 0.01, seeds 40-43, steps 0-39, every 2nd)"
    x, y = torch.cat(xs), torch.cat(ys)
    t1 = time.perf_counter()
    hist = W.train(mlp, x, y, epochs=60, batch=8192, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    hist76 = W.train(mlp76, torch.cat(xs76), torch.cat(ys76), epochs=60, batch=8192, lr=1e-3)

    def both(ctx, scene, dt, warm, eps=0.01, relax=0):
        res = W.compare(ctx, mlp, scene, steps=args.steps, dt=dt, warm_steps=warm, eps=eps,
                        relax=relax)
        res["mlp76"] = W.compare(ctx, mlp76, scene, steps=args.steps, dt=dt, warm_steps=warm,
                                 eps=eps, relax=relax, modes=((1, "mlp"),))["mlp"]
        out = {}
        for k in ("plain", "extrapolated", "mlp", "mlp76"):
            out[k] = W.summarize(res[k])
            ms = sorted(st["ms_total"] for st in res[k])
            out[k]["ms_total_median"] = ms[len(ms) // 2]
        return out

    # in distribution: a dam-break column of an unseen seed, 3x the sites
    dam = scenes.dam_break(nx=36, ny=36, nz=72, width=0.4, seed=20)
    ctx_d = pot.Context(dam.n, 246, 0, fp32=True, fp64=False)
    dts, eps_d, nsub_d, relax_d = sub(dam)
    held = both(ctx_d, dam, dts, 12 * nsub_d, eps_d, relax_d)
    pot.set_warm_start(ctx_d, None)
    ctx_d.close()
    ctx = pot.Context(sc.n, 246, 0, fp32=True, fp64=False)
    spl = both(ctx, sc, sc.extra["dt"], args.warmup, sc.extra["eps"], sc.extra["relax_rounds"])
    plain, learned = spl["plain"], spl["mlp"]
    print(json.dumps({
        "metric": "Newton iterations and ms per fluid-step solve, learned vs plain start",
        "workload": f"two-ball splash, {sc.n} sites, steps {args.warmup}..{args.warmup + args.steps - 1}, "
                    f"dt {sc.extra['dt']:.4g}, eps {sc.extra['eps']:.4g}, tol 1e-4, FP32 geometry with "
                    f"FP64 reductions",
        "training": {"samples": int(x.shape[0]), "epochs": len(hist), "loss_first": hist[0],
                     "loss_last": hist[-1], "collect_s": t1 - t0, "train_s": t2 - t1,
                     "scenes": "dam-break columns 24x24x48, seeds 10-19, the substeps of their "
                               "first 40 steps of 2e-3",
                     "extra_scenes": extra},
        "training_76": {"loss_first": hist76[0], "loss_last": hist76[-1],
                        "inputs": "24 neighbour offsets, previous weight, velocity (76); the "
                                  "prediction corrects the previous weights"},
        "plain": plain, "extrapolated": spl["extrapolated"], "mlp": learned, "mlp76": spl["mlp76"],
        "newton_iters_saved": plain["newton_iters"] - learned["newton_iters"],
        "ms_saved_per_solve": plain["ms_total"] - learned["ms_total"],
        "holdout_dam_break": {"workload": f"dam-break column 36x36x72 ({dam.n} sites), seed 20, "
                                          f"substeps {12 * nsub_d}..{12 * nsub_d + args.steps - 1} "
                                          f"of {dts:.3g}, eps {eps_d:.3g}",
                              "plain": held["plain"], "extrapolated": held["extrapolated"],
                              "mlp": held["mlp"], "mlp76": held["mlp76"],
                              "newton_iters_saved": held["plain"]["newton_iters"] - held["mlp"]["newton_iters"],
                              "ms_saved_per_solve": held["plain"]["ms_total"] - held["mlp"]["ms_total"]}}))
    pot.set_warm_start(ctx, None)
    ctx.close()
    mlp.close()
    mlp76.close()


def _pcts(v):
    v = sorted(v)
    return {"median": v[len(v) // 2], "p90": v[min(len(v) - 1, int(0.9 * len(v)))], "max": v[-1]}


def run_dam(args):
    """The 500,094-site dam break (dt 2e-3 in substeps, the recipe's spring),
    stepped `steps` times from the recipe's start state in mixed precision
    (FP32 geometry, FP64 reductions) and in FP64: per-step Newton iterations
    (summed over the substeps), step ms and worst volume error, and the
    distance between the two trajectories."""
    import numpy as np
    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    sc = scenes.dam_break()
    n = sc.n
    marks = sorted({k for k in (args.steps // 4, args.steps // 2, 3 * args.steps // 4, args.steps) if k > 0})
    out, snaps = {}, {}
    for prec, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
        ctx = pot.Context(n, 1024, 0, fp32=dt == torch.float32, fp64=dt == torch.float64)
        pos = torch.as_tensor(sc.pos, dtype=dt, device=dev)
        vel = torch.as_tensor(sc.vel, dtype=dt, device=dev)
        psi = torch.as_tensor(sc.psi, dtype=dt, device=dev)
        nu = torch.as_tensor(sc.nu, dtype=torch.float64, device=dev)
        prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"],
                                 substeps=sc.extra["substeps"], mu=args.mu, gamma=args.gamma,
                                 mu_wall=args.mu_wall)
        pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
        stats, snaps[prec] = [], {}
        for k in range(1, args.steps + 1):
            stats.append(pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm, check=False))
            if stats[-1]["status"] != 0:
                break
            if k in marks:
                snaps[prec][k] = pos.double().cpu().numpy()
        out[prec] = {"steps_done": len(stats), "all_converged": all(st["status"] == 0 for st in stats),
                     "newton_iters_mean": float(np.mean([st["newton_iters"] for st in stats])),
                     "pcg_iters_mean": float(np.mean([st["pcg_iters"] for st in stats])),
                     "step_ms": _pcts([st["ms_total"] for st in stats]),
                     "viscosity_ms": _pcts([st["ms_visc"] for st in stats]),
                     "viscosity_pcg_iters_mean": float(np.mean([st["visc_iters"] for st in stats])),
                     "err_max_per_step": _pcts([st["err_max"] for st in stats]),
                     "newton_iters_per_step": [st["newton_iters"] for st in stats]}
        ctx.close()
    s = 0.4 / 63
    drift = {}
    for k in marks:
        if k in snaps["mixed"] and k in snaps["fp64"]:
            a, b = snaps["mixed"][k], snaps["fp64"][k]
            d = np.linalg.norm(a - b, axis=1) / s
            drift[str(k)] = {"median": float(np.median(d)), "p99": float(np.percentile(d, 99)),
                             "max": float(d.max()),
                             "centre_of_mass": float(np.linalg.norm(a.mean(0) - b.mean(0)) / s),
                             "front_x_p999": [float(np.percentile(a[:, 0], 99.9)),
                                              float(np.percentile(b[:, 0], 99.9))]}
    print(json.dumps({"metric": "dam break, mixed precision against FP64 on the GPU",
                      "workload": f"dam-break column 63x63x126 ({n} sites), dt 2e-3 as "
                                  f"{sc.extra['substeps']} substeps, eps {sc.extra['eps']:.3g}, "
                                  f"viscosity {args.mu:g}, surface tension {args.gamma:g}, wall viscosity {args.mu_wall:g}, "
                                  f"{args.steps} steps, tol 1e-4",
                      "mixed": out["mixed"], "fp64": out["fp64"],
                      "speedup_mixed_over_fp64": out["fp64"]["step_ms"]["median"] / out["mixed"]["step_ms"]["median"],
                      "trajectory_distance_in_spacings": drift}))


def run_robust(args):
    """The robustness case: a ball of about 200k sites flying apart at up to
    5 m/s into the box walls (near step 77), `steps` fluid steps in mixed
    precision from the recipe's start state; counts the steps whose solve
    converged to 1e-4 (a failed step is not retried and the run goes on
    from its state)."""
    import numpy as np
    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    sc = scenes.explosion()
    n = sc.n
    ctx = pot.Context(n, 1024, 0, fp32=True, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    stats = []
    for _ in range(args.steps):
        stats.append(pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm, check=False))
    x = pos.cpu().numpy()
    ok = [s["status"] == 0 and s["err_max"] <= 1e-4 for s in stats]
    print(json.dumps({
        "metric": "converged fluid steps (worst cell within 1e-4 of its volume), robustness case",
        "workload": f"ball of {n} sites (radius 0.3, up to 5 m/s outward) into the box walls, "
                    f"dt {prm.dt:.3g}, eps {prm.eps:.3g}, FP32 geometry with FP64 reductions",
        "converged": int(sum(ok)), "steps": len(stats),
        "statuses": sorted({s["status"] for s in stats}),
        "newton_iters_mean": float(np.mean([s["newton_iters"] for s in stats])),
        "halvings_total": int(sum(s["halvings"] for s in stats)),
        "repairs_total": int(sum(s["repairs"] for s in stats)),
        "step_ms": _pcts([s["ms_total"] for s in stats]),
        "err_max_per_step": _pcts([s["err_max"] for s in stats]),
        "sites_at_walls": int(np.sum(np.any((x < 1e-5) | (x > 1 - 1e-5), axis=1))),
        "max_planes_last": int(pot.cell_diagnostics(ctx, n)["planes"].max())}))
    ctx.close()


def run_render(args):
    """First hit of camera rays (pot_render_depth) on the 2M splash after
    `advance` fluid steps from the recipe's start state: a 1920 x 1080 depth
    and normal image, median of `steps` frames after `warmup`, with the
    balls of cells without free surface skipped and without; then the
    volume traversal and the sphere tracing of the smoothed surface over
    the same frame."""
    import math

    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    sc = scenes.splash(spacing=args.spacing, seed=3)
    n = sc.n
    ctx = pot.Context(n, 246, 0, fp32=True, fp64=False)
    pos, vel, psi, nu = (torch.from_numpy(a).to(dev) for a in (sc.pos, sc.vel, sc.psi, sc.nu))
    prm = pot.default_params(dt=sc.extra["dt"], eps=sc.extra["eps"])
    pot.relax_to_centroids(ctx, pos, psi, nu, sc.extra["relax_rounds"], params=prm)
    for _ in range(args.advance):
        pot.pot_fluid_step(ctx, pos, vel, psi, nu, params=prm)
    karea = pot.lgc_compute_cells(ctx, pos, psi, nu, hessian=False)["karea"]
    cam = dict(origin=(0.5, -0.9, 0.8), forward=(0.0, 1.0, -0.55), up=(0.0, 0.0, 1.0),
               fov_y=math.radians(40), width=1920, height=1080)
    out = {}
    for name, ka in (("culled", karea), ("all_balls", None)):
        for _ in range(args.warmup):
            pot.render_depth(ctx, pos, psi, karea=ka, **cam)
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            depth, _ = pot.render_depth(ctx, pos, psi, karea=ka, **cam)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        ms = times[len(times) // 2]
        out[name] = {"ms_per_frame": ms, "rays_per_s": 1920 * 1080 / (ms / 1e3),
                     "hit_fraction": float((depth >= 0).float().mean())}
    # the volume traversal (cell evaluation included)
    for _ in range(args.warmup):
        pot.render_volume(ctx, pos, psi, **cam)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        first, thick, _, visits = pot.render_volume(ctx, pos, psi, **cam)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    hit = first >= 0
    out["volume"] = {"ms_per_frame": ms, "rays_per_s": 1920 * 1080 / (ms / 1e3),
                     "hit_fraction": float(hit.float().mean()),
                     "cells_per_ray_mean": float(visits[hit].float().mean()),
                     "cells_per_ray_max": int(visits.max()),
                     "note": "includes the cell evaluation at these weights"}
    # sphere tracing of the smoothed surface, smoothing radius half a spacing
    ks = 0.5 * args.spacing
    for _ in range(args.warmup):
        pot.render_smooth(ctx, pos, psi, k=ks, **cam)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sd, _, sst = pot.render_smooth(ctx, pos, psi, k=ks, **cam)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    hit = sd >= 0
    out["smooth"] = {"ms_per_frame": ms, "rays_per_s": 1920 * 1080 / (ms / 1e3),
                     "k": ks, "hit_fraction": float(hit.float().mean()),
                     "steps_per_ray_mean": float(sst.float().mean()),
                     "steps_per_ray_max": int(sst.max()),
                     "note": "includes the cell evaluation at these weights"}
    print(json.dumps({"metric": "camera rays per second, first hit on the fluid (pot_render_depth), "
                                "volume traversal (pot_render_volume) and sphere tracing of the "
                                "smoothed surface (pot_render_smooth)",
                      "workload": f"two-ball splash, {n} sites, step {args.advance}, 1920 x 1080, "
                                  f"grid build included",
                      "free_surface_cells": int((karea > 0).sum()), **out}))
    ctx.close()


def run_solve(args):
    """The 1000-site jittered block solved to 1e-4 from psi0 (single Newton
    solve), FP64 and mixed precision on the GPU; the FP64 oracle's Newton
    (dense direct solve) timed on the host beside it."""
    import torch

    from paper_2601_05765_b300 import pot, scenes
    dev = torch.device("cuda", 0)
    sc = scenes.jittered_block()
    res = {}
    for prec, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        ctx = pot.Context(sc.n, 246, 0, fp32=dt == torch.float32, fp64=dt == torch.float64)
        pos = torch.as_tensor(sc.pos, dtype=dt, device=dev)
        nu = torch.as_tensor(sc.nu, dtype=torch.float64, device=dev)
        times, st = [], None
        for k in range(args.warmup + args.steps):
            psi = torch.as_tensor(sc.psi, dtype=dt, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = pot.pot_newton_solve(ctx, pos, nu, psi)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(1e3 * (time.perf_counter() - t0))
        res[prec] = {"ms_per_solve": _pcts(times), "newton_iters": st["newton_iters"],
                     "halvings": st["halvings"], "pcg_iters": st["pcg_iters"], "err_max": st["err_max"]}
        ctx.close()
    line = {"metric": "Newton solve ms to 1e-4, 1000-site jittered block",
            "workload": "jittered 10x10x10 block, spacing 0.05, psi0 = (0.8 r_nu)^2, tol 1e-4",
            "fp64": res["fp64"], "mixed": res["mixed"]}
    if not args.no_cpu_baseline:
        import numpy as np

        from oracle import oracle as O
        x = sc.pos.astype(np.float64)
        t0 = time.perf_counter()
        reps = 0
        while reps < 3 or time.perf_counter() - t0 < 2.0:
            r = O.newton(x, sc.nu, sc.psi.astype(np.float64), tol=1e-4)
            reps += 1
        line["cpu_baseline"] = {"value": 1e3 * (time.perf_counter() - t0) / reps, "unit": "ms per solve",
                                "cores": O.max_threads(), "kind": "oracle",
                                "sample": f"{reps} oracle Newton solves (dense LU, KMT), {r.iters} iterations"}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "cells":
        run_cells(args)
    elif args.mode == "warmstart":
        run_warmstart(args)
    elif args.mode == "dam":
        run_dam(args)
    elif args.mode == "robust":
        run_robust(args)
    elif args.mode == "render":
        run_render(args)
    elif args.mode == "solve":
        run_solve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

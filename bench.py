"""Benchmark of the axion-coupled Yee step on GB300.

Workload: the 2D weak-pulse conversion run -- 4096 x 2048 cells, dx = dy =
lambda/32, CFL 0.95, Gaussian E_z pulse a0 = 0.01 (waist 4 lambda, FWHM 8
lambda/c), B_ext along z, g = 1e-4, massless axion, PML on every edge (20
cells, sigma_max dt = 0.2).  One bench step = one full time step of every
coupled field on the whole grid.  Metric: cell-updates/s (one cell advanced
one full step with all fields).  Inputs: synthetic (analytic pulse), all
arrays far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Multi-GPU: every rank runs its own replica of the workload (replicas only,
weak scaling, no data-path collective); value = all ranks' cell-updates / max
rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 2048
METRIC = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="axp", choices=["axp", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-scan", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-1d", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-bc", action="store_true")
    ap.add_argument("--no-window", action="store_true")
    ap.add_argument("--no-group", action="store_true")
    ap.add_argument("--no-plasma", action="store_true",
                    help="leave out the magnetised-plasma (perturbed-particle current) measurement")
    ap.add_argument("--group-members", type=int, default=40,
                    help="2D requests of the seeded serving stream in the group measurement")
    ap.add_argument("--scan-tiling", default=None,
                    help="block_steps,segment_cells,threads for the scan instead of the autotuner's choice")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-open-requests", type=int, default=200)
    ap.add_argument("--n3d", type=int, default=512, help="edge of the 3D axion box")
    ap.add_argument("--tm2d-form", default="auto", choices=["auto", "grid", "list"],
                    help="launch form of the 2D kernel on the headline grid: the planner's choice, the uniform "
                         "grid of strips by chunks, or the balanced work lists (FP64)")
    return ap.parse_args()


def workload(args, precision):
    from paper_2406_16796_gb300 import workloads as W

    w = W.pulse_2d(nx=args.nx, ny=args.ny, precision=precision)
    return w


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values of x (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------

def oracle_rate(w, steps, rows=None):
    """cell-updates/s of the CPU oracle on the workload (optionally a strip of `rows` rows)."""
    import oracle

    grid = w.grid
    if rows is not None and rows < grid.n[1]:
        grid = grid.replace(n=(grid.n[0], rows, 1))
    og = oracle.OracleGrid(grid)
    for L in w.lasers:
        og.inject_laser(L)
    t0 = time.perf_counter()
    og.step(steps)
    dt = time.perf_counter() - t0
    return grid.cells * steps / dt, dt, grid


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else the machine type)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.machine()


def oracle_rate_one_thread(args, rows=64, steps=2):
    """The oracle's rate on one thread: a fresh process with OMP_NUM_THREADS=1 (the
    OpenMP runtime reads it once, at load) steps a strip of the bench grid."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "from paper_2406_16796_gb300 import workloads as W; "
            "w = W.pulse_2d(nx=%d, ny=%d, precision='fp64'); "
            "r, s, g = bench.oracle_rate(w, %d, rows=%d); print(json.dumps([r, s, g.n[0], g.n[1]]))"
            % (os.path.dirname(os.path.abspath(__file__)), args.nx, args.ny, steps, rows))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        rate, sec, nx, ny = json.loads(out.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": rate, "unit": "cell-updates/s", "cores": 1,
            "sample": "%d oracle steps of a %dx%d strip of the grid (%.1f s)" % (steps, nx, ny, sec)}


def reference_arm(args):
    rank, world, local = dist_env()
    from paper_2406_16796_gb300 import workloads as W

    w = workload(args, "fp64")
    if rank != 0:
        return 0
    # each step: one oracle step on a 16-row strip of the 4096-wide grid (same
    # boundaries and pulse), so the whole run stays within a few minutes
    rows = 16
    import oracle

    grid = w.grid.replace(n=(w.grid.n[0], rows, 1))
    og = oracle.OracleGrid(grid)
    for L in w.lasers:
        og.inject_laser(L)
    og.step(args.warmup)
    t0 = time.perf_counter()
    og.step(args.steps)
    el = time.perf_counter() - t0
    value = grid.cells * args.steps / el
    sample = "%d oracle steps of a %dx%d strip of the %dx%d grid" % (args.steps, grid.n[0], rows, w.grid.n[0],
                                                                      w.grid.n[1])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": w.grid.cells, "precision": "fp64", "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# Algorithmic work of one cell-update of the 2D pulse workload (E0z, B0x, B0y
# laser; all six order-1 components; axion):
#  * HBM bytes: every active array read once and written once: 9 field arrays
#    plus the axion (FP64: phi^{n+1/2}, phi^{n-1/2} read, phi^{n+3/2} written;
#    FP32 split: phi and its increment read and written).
#  * FP64 operations: 77 adds, multiplies and fused multiply-adds per
#    cell-update, 33 of them FMAs, so 110 FLOPs (FMA = 2), counted from the
#    operations of the fused scheme for this component set (B update 22 ops /
#    33 FLOPs, axion + E0 16 / 22, axion current 13 / 17, E update 26 / 38).
#    Every one of them occupies the FP64 pipe for the same issue slot, so the
#    FP64 roofline is in pipe operations.  (The 2D kernel executes 50 of them per
#    cell-update: it folds each pair of half-steps into one multiply-add per
#    difference, forms E0z's second half-step from its first, and folds
#    constants.  The roofline counts the scheme's 77; `executed_frac` is the
#    kernel's own 50 against the same peak.)
ACTIVE_ARRAYS = 9
FLOPS_PER_CELL = 110
FP64_OPS_PER_CELL = 77
EXECUTED_FP64_OPS_PER_CELL = 50


def bytes_per_cell(prec):
    e = 8 if prec == "fp64" else 4
    phi_words = 3 if prec == "fp64" else 4
    return (2 * ACTIVE_ARRAYS + phi_words) * e


# DRAM bytes (read + write) per launch of the timed kernel at the bench's full
# size, from ncu captures of a smaller case scaled by cells (the traffic of a
# one-pass stencil grows with the cells); None until a capture of the kernel as
# it stands exists.  Sources are summarised under profiles/.
TRAFFIC = {
    # k_tm2d_list (FP64, work lists), captured at this size (one-pass metrics): 773.5 + 628.6 MB
    ("k_tm2d_list (one launch per step)", "fp64"): 1402.0e6,
    # k_tm2d (FP64, uniform grid), 2048 x 2048 capture: 689.2 MB per launch
    ("k_tm2d (one launch per step)", "fp64"): 689.2e6 * (4096 * 2048) / (2048 * 2048),
    # k_tm2d_x2 (FP32 split, two columns per thread), captured at this size (one-pass
    # metrics): 395.6 + 322.0 MB per launch
    ("k_tm2d_x2 (one launch per step)", "fp32"): 717.5e6,
}
# k_ax3d_x2 (3D, no order-0 fields, two x cells per thread, evict-first stores),
# 256^3 capture (one-pass metrics): 574.7 + 488.5 MB per launch
TRAFFIC_3D_PER_CELL = 1063.2e6 / 256 ** 3


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# FP64 pipe of GB300, read from ncu on the 2D kernel (profiles/
# k_tm2d_fp64_pipe_2d_pulse_2048x2048.md): sm__inst_executed_pipe_fp64 peaks at
# 1/16 warp instruction per cycle per SM, i.e. 2 FP64 thread operations (add,
# multiply or FMA) per cycle per SM; the SM count and the SM clock are read
# live (device properties; nvidia-smi samples over the timed region).
FP64_PIPE_WARP_INST_PER_CYCLE_PER_SM = 1.0 / 16.0
# FP64-pipe warp instructions the 2D kernel executes per cell-update, by launch
# form (ncu, sm__inst_executed_pipe_fp64.sum over one launch): on work lists
# 13,976,291 on the 4096 x 2048 pulse grid itself (53.3 thread-operation slots
# per cell); on the uniform grid 7,468,742 on the 2048 x 2048 grid (57.0; per
# cell about the same at 4096 x 2048, to the share of halo columns and layer cells)
FP64_PIPE_WARP_INST_PER_CELL = {"k_tm2d_list (one launch per step)": 13976291 / 8388608,
                                "k_tm2d (one launch per step)": 7468742 / 4194304}


def fp64_pipe_peak_gops(sm_count, sm_mhz):
    """FP64 thread operations per second the pipe sustains at this clock (Gop/s)."""
    return FP64_PIPE_WARP_INST_PER_CYCLE_PER_SM * 32 * sm_count * sm_mhz * 1e6 / 1e9


def timed_run(g, steps, warmup, stream):
    import torch

    g.step(warmup)
    g.synchronize()
    torch.cuda.synchronize()
    l0 = g.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / 1e3, g.launches() - l0


# 3D axion box: active arrays E1 (3), B1 (3) and the axion; FP32 split stores
# phi and its increment (read and written); every field array read once and
# written once per cell-update.
BYTES_3D_FP32 = (2 * 6 + 4) * 4


def axion3d_measurement(steps, warmup, hbm_peak, hbm_src, world, n=512):
    """n^3 (512^3) periodic box seeded with an axion plane wave, B_ext along y,
    FP32 split (no laser: the order-0 arrays are identically zero and are
    skipped)."""
    import torch

    from paper_2406_16796_gb300 import axp, workloads as W

    w = W.axion_3d(n=n)
    g = axp.Grid(w.grid)
    for a in w.axions:
        g.inject_axion(a)
    el, launches = timed_run(g, steps, warmup, g.stream)
    cells = w.grid.cells
    per = el / max(1, launches)
    ach = BYTES_3D_FP32 * cells / per / 1e9
    out = {"workload": w.name, "cells": cells, "precision": "fp32_split", "steps": steps,
           "value": cells * steps * world / el, "unit": "cell-updates/s", "ms_per_step": el / steps * 1e3,
           "kernel_path": g.kernel_path(), "gpu_launches": launches,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                        "peak_source": hbm_src, "algorithmic_bytes_per_cell": BYTES_3D_FP32,
                        "traffic": (TRAFFIC_3D_PER_CELL * cells if TRAFFIC_3D_PER_CELL is not None
                                    and g.kernel_path() == axp.AXP_KERNEL_AX3D else None)},
           # FP32 split on an even-width box takes the two-cell form of the axion-box kernel
           "kernel": {axp.AXP_KERNEL_AX3D: "k_ax3d_x2" if n % 2 == 0 else "k_ax3d",
                      axp.AXP_KERNEL_FUSED: "k_fused"}.get(g.kernel_path(), "general")}
    g.close()
    torch.cuda.synchronize()
    return out


def vacuum1d_measurement(world):
    """The 1D conversion run in FP64: Nx = 4096, 20000 steps, periodic.  The state
    (8 arrays x 4096 x 8 B) stays in L2, so the bound is per-step launch and
    synchronisation latency: reported as microseconds per step."""
    from paper_2406_16796_gb300 import axp, workloads as W

    w = W.vacuum_1d()
    g = axp.Grid(w.grid)
    g.inject_laser(w.lasers[0])
    el, launches = timed_run(g, w.steps, 100, g.stream)
    d = g.diagnostics()
    out = {"workload": w.name, "cells": w.grid.cells, "precision": "fp64", "steps": w.steps,
           "value": w.grid.cells * w.steps * world / el, "unit": "cell-updates/s", "us_per_step": el / w.steps * 1e6,
           "kernel_path": g.kernel_path(), "gpu_launches": launches, "P_g2a": d["P_g2a"]}
    g.close()
    return out


def fp64_sequential_sample(reqs, served, sample=8, seed=20240628):
    """The requests run one after another as single-grid FP64 runs, timed in full
    (every step, device time) on a seeded sample, and extrapolated to the whole
    set by cell-updates, per class (1D and 2D run at different rates).  The
    same sample gives the served FP32-split conversion probabilities' error
    against FP64."""
    import numpy as np
    import torch

    from paper_2406_16796_gb300 import axp, workloads as W

    rng = np.random.default_rng(seed)
    by_class = {nd: [i for i, r in enumerate(reqs) if r.ndim == nd] for nd in (1, 2)}
    # the sample keeps the stream's class mix (at least one of each class present)
    n2 = max(1 if by_class[2] else 0, round(sample * len(by_class[2]) / max(1, len(reqs))))
    pick = {1: sorted(rng.choice(by_class[1], min(sample - n2, len(by_class[1])), replace=False).tolist()),
            2: sorted(rng.choice(by_class[2], min(n2, len(by_class[2])), replace=False).tolist()) if n2 else []}
    rate, errs, secs = {}, [], 0.0
    for nd, idx in pick.items():
        t_tot, cu_tot = 0.0, 0
        for i in idx:
            r = reqs[i]
            w = W.request_workload(r, precision="fp64")
            g = axp.Grid(w.grid)
            g.inject_laser(w.lasers[0])
            g.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(g.stream)
            g.step(r.steps)
            ev1.record(g.stream)
            ev1.synchronize()
            t_tot += ev0.elapsed_time(ev1) / 1e3
            cu_tot += r.n[0] * r.n[1] * r.steps
            d = g.diagnostics()
            g.close()
            if served.get(i) is not None and d["P_g2a"] > 0:
                errs.append(abs(served[i] - d["P_g2a"]) / d["P_g2a"])
        secs += t_tot
        if cu_tot:
            rate[nd] = cu_tot / t_tot
    total = sum(r.n[0] * r.n[1] * r.steps / rate[r.ndim] for r in reqs if r.ndim in rate)
    return {"seconds_extrapolated": total, "sims_per_s": len(reqs) / total,
            "sample": "%d seeded requests (%d 1D, %d 2D) run one after another in FP64, every step timed (%.1f s)"
                      % (len(pick[1]) + len(pick[2]), len(pick[1]), len(pick[2]), secs),
            "cell_updates_per_s_1d": rate.get(1), "cell_updates_per_s_2d": rate.get(2),
            "max_rel_err_P_served_vs_fp64": max(errs) if errs else None}


# k_tm2d_group on the first 40 2D requests of the seeded stream (21,932,100 cells),
# one-pass ncu capture of one launch: 1054.2 + 919.8 MB
TRAFFIC_GROUP40 = 1974.2e6


def group_measurement(members, steps, hbm_peak, hbm_src):
    """The serving path's 2D kernel alone: the first `members` 2D requests of the
    seeded stream (FP32 split, beam set-up) admitted into one group and advanced
    together, one persistent launch per step, timed with CUDA events on the
    group's stream."""
    import torch
    from paper_2406_16796_gb300 import axp, group as G, workloads as W

    reqs = [r for r in W.serve_requests(count=20 * members) if r.ndim == 2][:members]
    grp = G.Group(max(64, members), 65536)
    grids, cells = [], 0
    for r in reqs:
        w = W.request_workload(r, precision="fp32")
        g = axp.Grid(w.grid)
        g.inject_laser(w.lasers[0])
        grp.add(g, 10 ** 6)
        grids.append(g)
        cells += w.grid.cells
    grp.run(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(grp.stream)
    grp.run(steps)
    e1.record(grp.stream)
    e1.synchronize()
    per = e0.elapsed_time(e1) / 1e3 / steps
    ach = bytes_per_cell("fp32") * cells / per / 1e9
    out = {"workload": "serve_2d_group_%d" % len(grids), "members": len(grids), "cells": cells, "steps": steps,
           "ms_per_step": per * 1e3, "value": cells / per, "unit": "cell-updates/s", "kernel": "k_tm2d_group",
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                        "peak_source": hbm_src, "algorithmic_bytes_per_cell": bytes_per_cell("fp32"),
                        "traffic": TRAFFIC_GROUP40 if len(grids) == 40 else None}}
    grp.close()
    for g in grids:
        g.close()
    return out


# one push of a macroparticle reads its weight, positions and momenta of both
# orders (13 doubles) and writes the positions and momenta back (12 doubles)
BYTES_PER_PARTICLE = (13 + 12) * 8
# k_particles_push on the magnetised plasma (4.8M particles, 2D), one-pass ncu
# capture of one launch: FP64-pipe warp instructions and DRAM bytes
PUSH_FP64_WARP_INST_PER_PARTICLE = 110118800 / 4800000
PUSH_TRAFFIC_PER_PARTICLE = (843438848 + 531257856) / 4800000


def plasma_oracle_rate(nx=1200, steps=2):
    """The CPU oracle on a sample of the magnetised plasma: the same box and
    particle density on nx x 100 cells (4 particles per cell), `steps` coupled
    steps; particle-steps/s.  The oracle's field passes use OpenMP, its particle
    loop one thread."""
    import oracle

    from paper_2406_16796_gb300 import workloads as W

    grid, plasma, fields = W.magnetised_plasma_2d(nx=nx)
    og = oracle.OracleGrid(grid)
    og.load(fields)
    og.attach_particles(plasma.q, plasma.m, plasma.w, plasma.x0, plasma.u0, plasma.x1, plasma.u1)
    t0 = time.perf_counter()
    og.step(steps)
    el = time.perf_counter() - t0
    return {"value": plasma.count * steps / el, "unit": "particle-steps/s", "cores": omp_threads(), "kind": "oracle",
            "sample": "%d x %d cells, %d particles, %d steps (the particle loop runs on one thread)"
                      % (grid.n[0], grid.n[1], plasma.count, steps)}


def plasma_measurement(steps, warmup, hbm_peak, hbm_src, world, cpu=False):
    """Weak laser in a magnetised plasma (perturbed-particle current): 12000 x
    100 cells, 4 electrons per cell (4.8M), the laser in the first-order fields;
    FP64, one grid per GPU.  Each step is the general field kernels plus one
    particle push that gathers, kicks, drifts and deposits both orders."""
    import torch

    from paper_2406_16796_gb300 import axp, workloads as W

    grid, plasma, fields = W.magnetised_plasma_2d()
    g = axp.Grid(grid)
    for k, v in fields.items():
        g.write(k, v)
    g.attach_particles(plasma.q, plasma.m, plasma.w, plasma.x0, plasma.u0, plasma.x1, plasma.u1)
    cs = ClockSampler(torch.cuda.current_device())
    cs.start()
    el, launches = timed_run(g, steps, warmup, g.stream)
    clk = cs.stop().get("sm_mhz")
    per = el / steps
    ach = BYTES_PER_PARTICLE * plasma.count / per / 1e9
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk if clk else 2070.0
    fp64_peak = 2.0 * sms * mhz * 1e6 / 1e9  # Gop/s: 1/16 warp instruction per cycle per SM
    fp64_ach = PUSH_FP64_WARP_INST_PER_PARTICLE * 32 * plasma.count / per / 1e9
    out = {"workload": "magnetised_plasma_2d_%dx%d_ppc4" % (grid.n[0], grid.n[1]), "cells": grid.cells,
           "particles": plasma.count, "precision": "fp64", "steps": steps, "ms_per_step": per * 1e3,
           "value": plasma.count * steps * world / el, "unit": "particle-steps/s",
           "cell_updates_per_s": grid.cells * steps * world / el, "gpu_launches": launches,
           "kernel": "k_particles_push and the general field kernels",
           "roofline": {"bound": "alu", "achieved": fp64_ach, "peak": fp64_peak, "unit": "Gop/s (FP64 pipe)",
                        "frac": fp64_ach / fp64_peak, "kernel": "k_particles_push",
                        "executed_fp64_ops_per_particle": PUSH_FP64_WARP_INST_PER_PARTICLE * 32,
                        "what": "the push kernel's executed FP64 operations (ncu count per particle) over the whole "
                                "step's time, so a lower bound of the kernel's own fraction",
                        "peak_source": "1/16 warp instruction per cycle per SM x %d SMs x %.0f MHz sampled"
                                       % (sms, mhz),
                        "traffic": PUSH_TRAFFIC_PER_PARTICLE * plasma.count,
                        "hbm": {"achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                                "peak_source": hbm_src, "algorithmic_bytes_per_particle": BYTES_PER_PARTICLE}}}
    g.close()
    torch.cuda.synchronize()
    if cpu:
        out["cpu_baseline"] = plasma_oracle_rate()
    return out


def serve_measurement(count, rank, world, open_count=200):
    """The serving loop on the first `count` requests of the seeded stream (80%
    1D Nx log-uniform in [1024, 65536], 20% 2D Nx log-uniform in [256, 2048]
    with Ny = Nx/2, scan parameters, 5000-40000 steps).  Capacity is measured
    closed-loop (every request present at t = 0) on all of them; then the first
    `open_count` arrive as a Poisson stream at 0.5, 0.9 and 1.2 x that
    capacity.  Latency percentiles are reported overall and per class.  Each
    rank serves its own share (replicas).  The comparator is the same requests
    run one after another as single-grid FP64 runs, timed in full on a seeded
    sample."""
    from paper_2406_16796_gb300 import serve, workloads as W

    stream = W.serve_requests(count=count)
    base = W.shard(stream, rank, world)
    fields = ("ndim", "n", "m", "g", "B0", "steps")
    closed = [W.Request(0.0, *[getattr(r, f) for f in fields]) for r in base]

    def job_rate(summary, n_local, n_all):
        # all ranks' requests over the slowest rank's span (latencies are rank 0's)
        return n_all / max_over_ranks(n_local / summary["sims_per_s"], world)

    srv = serve.Server()
    cstats = srv.serve(closed)
    cap = cstats.summary()
    cap["sims_per_s"] = job_rate(cap, len(base), count)
    served = {k: rec.P_g2a for k, rec in enumerate(cstats.records)}
    levels = []
    n_open = min(open_count, count)
    for f in (0.5, 0.9, 1.2):
        rate = f * cap["sims_per_s"]
        reqs = W.shard(W.serve_requests(count=n_open, rate_per_s=rate), rank, world)
        s = srv.serve(reqs).summary()
        s["sims_per_s"] = job_rate(s, len(reqs), n_open)
        s["offered_load"] = f
        s["offered_rate_per_s"] = rate
        levels.append(s)
    srv.close()
    seq = fp64_sequential_sample(base, served)
    seq_s = max_over_ranks(seq["seconds_extrapolated"], world)
    cu = sum(r.n[0] * r.n[1] * r.steps for r in stream)
    return {"workload": "serve_%d_requests" % count, "requests": count, "cell_updates": cu,
            "sample": "closed loop: the first %d of the 10000-request seeded stream; open loop: its first %d"
                      % (count, n_open),
            "capacity": cap, "load": levels,
            "fp64_sequential": dict(seq, sims_per_s=count / seq_s),
            "speedup_vs_fp64_sequential": cap["sims_per_s"] / (count / seq_s)}


def boundary_measurement():
    """The Sec. 3.1 boundary benchmark on the paper's grid (400 x 400 cells over
    [-20, 20]^2 lambda0, pulse w = 5 lambda0, m = 1 meV, t = 30 lambda0 / c),
    FP64, for the PML and the outflow axion boundary; the paper reports about
    1% reflectivity for both."""
    from paper_2406_16796_gb300 import bccheck

    out = {"workload": "bc_check_400x400", "paper_reflectivity": 0.01}
    for bc in ("pml", "outflow"):
        r = bccheck.reflectivity(bc, n=400)
        out[bc] = {k: r[k] for k in ("energy", "amplitude", "steps", "seconds", "cell_updates_per_s", "kernel")}
    return out


def window_measurement(steps=400, shifts=(16, 64)):
    """Cost of the moving window on the 2D pulse grid in FP32 split: ms/step with
    the window moving at c in shifts of each size, against the fixed box.  A
    shift also brings the state to integer time and back (the general kernels),
    so larger shifts amortise it."""
    import torch

    from paper_2406_16796_gb300 import axp, workloads as W

    w = W.pulse_2d(precision="fp32")
    out = {"workload": w.name, "precision": "fp32_split", "steps": steps}
    for cells in (0,) + tuple(shifts):
        g = axp.Grid(w.grid)
        g.inject_laser(w.lasers[0])
        if cells:
            g.set_moving_window(0, 1.0, cells, 0)
        g.step(20)
        g.synchronize()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        g.synchronize()
        ms = (time.perf_counter() - t0) / steps * 1e3
        if cells == 0:
            out["ms_per_step_fixed"] = ms
        else:
            out["shift_%d" % cells] = {"ms_per_step": ms, "overhead": ms / out["ms_per_step_fixed"] - 1.0,
                                       "shifts": g.window_offset() // cells}
        g.close()
    return out


def scan_measurement(rank, world, fp64_sample=6, tiling=None):
    """The batched parameter scan: 512 seeded 1D instances (Nx log-uniform in
    [1024, 65536], m/omega0 in [1e-3, 2], g in [1e-6, 1e-3], B0 in [0.1, 10],
    5000-40000 steps), FP32 split, one persistent kernel per block of steps,
    CUDA-graph replay and autotuned tiling (the tuner's probe steps are inside
    the timing).  Each rank runs its own share of the instances (replicas).
    The comparator is sequential single-instance FP64 runs of a seeded sample
    of the same instances through the grid API, extrapolated by cell-updates;
    the sample also gives the FP32 batch's conversion-probability error."""
    import numpy as np
    import torch

    from paper_2406_16796_gb300 import axp, batch as B, workloads as W

    insts = W.shard(W.scan_instances(), rank, world)
    cu = sum(i.nx * i.steps for i in insts)
    phases = {}
    res, el, tiling = B.run_scan([B.scan_instance(i) for i in insts], tiling=tiling, phases=phases)
    el = max_over_ranks(el, world)
    every = W.scan_instances()
    cu_all = sum(i.nx * i.steps for i in every)
    out = {"workload": "scan_512x1d", "instances": len(every), "cell_updates": cu_all, "seconds": el,
           "sims_per_s": len(every) / el, "cell_updates_per_s": cu_all / el, "tiling": list(tiling),
           "graphs": True, "precision": "fp32_split", "phases_rank0": phases}
    if rank != 0:
        return out
    rng = np.random.default_rng(20240624)
    idx = sorted(rng.choice(len(insts), min(fp64_sample, len(insts)), replace=False).tolist())
    t_tot, cu_tot, errs = 0.0, 0, []
    for j in idx:
        i = insts[j]
        w = W.scan_workload(i, precision="fp64")
        g = axp.Grid(w.grid)
        g.inject_laser(w.lasers[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(i.steps)
        d = g.diagnostics()
        t_tot += time.perf_counter() - t0
        cu_tot += i.nx * i.steps
        errs.append(abs(res[j]["P_g2a"] - d["P_g2a"]) / abs(d["P_g2a"]))
        g.close()
    fp64_cu_rate = cu_tot / t_tot
    fp64_sims = fp64_cu_rate / (cu / len(insts))
    out["fp64_per_instance"] = {"sims_per_s": fp64_sims, "cell_updates_per_s": fp64_cu_rate,
                                "sample": "%d seeded instances run one after another in FP64, full steps" % len(idx)}
    out["speedup_vs_fp64_per_instance"] = out["sims_per_s"] / fp64_sims
    out["max_rel_err_P_vs_fp64"] = max(errs)
    return out


def gpu_arm(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2406_16796_gb300 import axp

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    prec = args.precision
    w = workload(args, prec)
    g = axp.Grid(w.grid)
    if args.tm2d_form != "auto":
        g.set_kernel(axp.AXP_KERNEL_TM2D if args.tm2d_form == "grid" else axp.AXP_KERNEL_TM2D_LIST)
    for L in w.lasers:
        g.inject_laser(L)
    cells = w.grid.cells
    path = g.kernel_path()

    # headline: K steps of the requested precision, clocks sampled meanwhile
    g.step(args.warmup)
    g.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    el, launches = timed_run(g, args.steps, 0, g.stream)
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = max_over_ranks(el, world)
    value = cells * args.steps * world / el
    ms = el / args.steps * 1e3
    per_launch = el / max(1, launches)  # the fused path launches one kernel per step

    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    bpc = bytes_per_cell(prec)
    hbm_achieved = bpc * cells / per_launch / 1e9
    hbm = {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
           "peak_source": hbm_src, "algorithmic_bytes_per_cell": bpc}
    kern = {axp.AXP_KERNEL_TM2D: "k_tm2d (one launch per step)",
            axp.AXP_KERNEL_TM2D_LIST: "k_tm2d_list (one launch per step)",
            axp.AXP_KERNEL_FUSED: "k_fused (one launch per step)"}.get(path, "general kernels (8 launches per step)")
    if prec == "fp64":
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = fp64_pipe_peak_gops(sm_count, sm_mhz)
        # executed: the kernel's FP64-pipe issue (ncu count per cell) at the live rate
        inst_per_cell = FP64_PIPE_WARP_INST_PER_CELL.get(kern)
        executed = inst_per_cell * 32 * cells / per_launch / 1e9 if inst_per_cell else None
        # algorithmic: the scheme's 77 operations per cell-update at the same rate
        algorithmic = FP64_OPS_PER_CELL * cells / per_launch / 1e9
        flops = FLOPS_PER_CELL * cells / per_launch / 1e12
        roofline = {"bound": "alu", "achieved": executed, "peak": peak, "unit": "Gop/s (FP64 pipe)",
                    "frac": executed / peak if executed else None,
                    "traffic": TRAFFIC.get((kern, prec)) if cells == NX * NY else None, "kernel": kern,
                    "peak_source": "measured: ncu sm__inst_executed_pipe_fp64 peak 1/16 warp instruction per cycle "
                                   "per SM (2 FP64 ops/cycle/SM) x %d SMs x %.0f MHz sampled" % (sm_count, sm_mhz),
                    "executed_fp64_ops_per_cell": inst_per_cell * 32 if inst_per_cell else None,
                    "algorithmic_fp64_ops_per_cell": FP64_OPS_PER_CELL,
                    "algorithmic_equivalent": {"achieved": algorithmic, "frac": algorithmic / peak,
                                               "what": "the scheme's 77 operations per cell-update at the measured "
                                                       "rate; the kernel folds them into fewer"},
                    "flops": {"achieved": flops, "peak": 2 * peak / 1e3, "unit": "TFLOP/s",
                              "frac": flops / (2 * peak / 1e3), "algorithmic_flops_per_cell": FLOPS_PER_CELL},
                    "hbm": hbm}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": TRAFFIC.get((kern, prec)) if cells == NX * NY else None,
                    "kernel": kern,
                    "peak_source": hbm_src, "algorithmic_bytes_per_cell": bpc}

    # e2e through the C ABI with pinned host buffers, the way a user resumes the
    # workload from a checkpoint: upload the state image, run the steps with the
    # diagnostics recorded every 100 steps (the workload's cadence) into the
    # grid's ring, read the records back, download the final image
    e2e = None
    if not args.no_e2e:
        ge = axp.Grid(w.grid, diag_every=100, diag_capacity=64)
        for L in w.lasers:
            ge.inject_laser(L)
        nbytes = axp.axp_state_bytes(ge.h)
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        axp.axp_save_state(ge.h, host.data_ptr(), nbytes)
        ge.step(args.warmup)
        ge.synchronize()
        k = max(100, args.steps)
        # one untimed pass of the whole sequence first (pinned pages, first copies)
        axp.axp_load_state(ge.h, host.data_ptr(), nbytes)
        ge.step(k)
        ge.read_diagnostics()
        axp.axp_save_state(ge.h, host.data_ptr(), nbytes)
        axp.axp_load_state(ge.h, host.data_ptr(), nbytes)
        ge.synchronize()
        axp.axp_save_state(ge.h, host.data_ptr(), nbytes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        axp.axp_load_state(ge.h, host.data_ptr(), nbytes)
        ge.step(k)
        recs = ge.read_diagnostics()
        axp.axp_save_state(ge.h, host.data_ptr(), nbytes)
        t1 = time.perf_counter()
        diag_bytes = 88 * len(recs)
        e2e = {"value": cells * k * world / (t1 - t0), "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes / k,
               "d2h_bytes_per_step": (nbytes + diag_bytes) / k, "steps": k, "diagnostics_records": len(recs),
               "what": "checkpoint image of the running simulation uploaded from pinned host, k steps with "
                       "FP64 diagnostics every 100 steps, diagnostics read-back, checkpoint image downloaded"}
        ge.close()
    g.close()

    # the FP32 split storage on the same workload, as a second measurement
    other = None
    if prec == "fp64" and not args.no_fp32:
        w32 = workload(args, "fp32")
        g32 = axp.Grid(w32.grid)
        for L in w32.lasers:
            g32.inject_laser(L)
        k32 = 4 * args.steps
        el32, l32 = timed_run(g32, k32, args.warmup, g32.stream)
        per32 = el32 / max(1, l32)
        ach = bytes_per_cell("fp32") * cells / per32 / 1e9
        # FP32 split on an even-width grid takes the two-column form of the 2D kernel
        path32 = g32.kernel_path()
        kern32 = ("k_tm2d_x2 (one launch per step)" if (path32 == axp.AXP_KERNEL_TM2D and args.nx % 2 == 0)
                  else "k_tm2d (one launch per step)" if path32 == axp.AXP_KERNEL_TM2D
                  else "k_fused (one launch per step)" if path32 == axp.AXP_KERNEL_FUSED
                  else "general kernels (8 launches per step)")
        other = {"precision": "fp32_split", "value": cells * k32 * world / el32, "unit": "cell-updates/s",
                 "steps": k32, "ms_per_step": el32 / k32 * 1e3, "kernel": kern32,
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                              "frac": ach / hbm_peak, "peak_source": hbm_src,
                              "traffic": TRAFFIC.get((kern32, "fp32")) if args.nx * args.ny == NX * NY else None,
                              "algorithmic_bytes_per_cell": bytes_per_cell("fp32")}}
        g32.close()

    scan = None
    if not args.no_scan:
        tl = tuple(int(x) for x in args.scan_tiling.split(",")) if args.scan_tiling else None
        scan = scan_measurement(rank, world, tiling=tl)
    srv = None
    if not args.no_serve:
        srv = serve_measurement(args.serve_requests, rank, world, open_count=args.serve_open_requests)
    plasma = None
    if not args.no_plasma:
        plasma = plasma_measurement(20, 3, hbm_peak, hbm_src, world,
                                    cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    grp = None
    if not args.no_group:
        grp = group_measurement(args.group_members, 50, hbm_peak, hbm_src)
    bcm = None
    if not args.no_bc and rank == 0:
        bcm = boundary_measurement()
    win = None
    if not args.no_window and rank == 0:
        win = window_measurement()
    ax3 = None
    if not args.no_3d:
        ax3 = axion3d_measurement(max(20, args.steps // 3), args.warmup, hbm_peak, hbm_src, world, n=args.n3d)
    v1 = None
    if not args.no_1d:
        v1 = vacuum1d_measurement(world)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # about 10 s of the oracle on every host core, then about 5 s on one
        wb = workload(args, "fp64")
        csteps = 10
        rate, sec, gsp = oracle_rate(wb, steps=csteps)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": omp_threads(), "kind": "oracle",
               "sample": "%d oracle steps of the full %dx%d grid (%.1f s)" % (csteps, gsp.n[0], gsp.n[1], sec),
               "cpu_model": cpu_model(), "single_thread": oracle_rate_one_thread(args, rows=64, steps=10)}
    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": w.name, "cells": cells, "precision": prec, "parallelism": "replicas",
                       "l2": "inputs larger than L2"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    if other:
        line["fp32_split"] = other
    if scan:
        line["scan"] = scan
    if srv:
        line["serve"] = srv
    if grp:
        line["serve_2d_group"] = grp
    if plasma:
        line["magnetised_plasma"] = plasma
    if ax3:
        line["axion_3d"] = ax3
    if bcm:
        line["boundary"] = bcm
    if win:
        line["moving_window"] = win
    if v1:
        line["vacuum_1d"] = v1
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())

"""The axion boundary benchmark of Sec. 3.1 as a product feature.

A left-moving Gaussian axion pulse (w = 5 lambda0, m = 1 meV against an
800 nm wave) starts in the middle of a [-20, 20]^2 lambda0 box of 400 x 400
cells and leaves it through an absorbing side (PML, N = 20, sigma_max dt =
0.2, or the outflow condition).  What stays in the box measures the
boundary's reflectivity, which the paper puts at about 1%:

* energy reflectivity: H_phi left in the box / H_phi at the start;
* amplitude reflectivity: max |phi| inside the box (outside the layers) /
  max |phi| at the start.

The run goes through the grid C ABI (the general kernels for outflow, the 2D
kernel for PML); only the read-out of phi for the amplitude is on the host.
"""
from __future__ import annotations

import time

import numpy as np

from . import axp as _axp
from . import workloads as W


def reflectivity(bc="pml", precision="fp64", n=400, t_end=30.0):
    """Run the Sec. 3.1 set-up with axion boundary `bc` ("pml" or "outflow") until
    t_end (lambda0 / c) and return the reflectivities and the run's timing."""
    import torch

    w = W.bc_check_2d(bc, n=n)
    grid = w.grid.replace(precision=precision)
    g = _axp.Grid(grid)
    g.inject_axion(w.axions[0])
    a0 = float(np.abs(g.read("phi_cur")).max())
    H0 = g.diagnostics()["H_phi"]
    steps = int(round(t_end / grid.dt))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(steps)
    g.synchronize()
    el = time.perf_counter() - t0
    H1 = g.diagnostics()["H_phi"]
    N = grid.pml_cells if bc == "pml" else 0
    phi = g.read("phi_cur")
    amp = float(np.abs(phi[0, N:grid.n[1] - N, N:grid.n[0] - N]).max()) / a0
    path = g.kernel_path()
    g.close()
    return {"bc": bc, "precision": precision, "cells": grid.cells, "steps": steps, "energy": H1 / H0,
            "amplitude": amp, "seconds": el, "cell_updates_per_s": grid.cells * steps / el,
            "kernel": {_axp.AXP_KERNEL_TM2D: "k_tm2d", _axp.AXP_KERNEL_FUSED: "k_fused"}.get(path, "general")}

"""Diagnostics of a grid the single-pass kernels are stepping: E^n is formed
from the two E levels the last step left (E^{n-1/2} in the other field set,
E^{n+1/2} in the present one; their mean outside the absorbing layers, the
layer's one-half-step weights inside).  The records equal, to rounding, those
computed after the general kernels' backward half-step, and the oracle's."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "W", "sum_xB1z2", "sum_B1z2", "gauss_l2")


def grid_of(n, d, prec, bc, pml=8, B=(0.0, 0.0, 1.1)):
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    b = W._bcs(*[bc if n[a] > 1 else "periodic" for a in range(3)])
    return W.GridSpec(n=n, d=d, dt=dt, m=0.9, g=0.7, B_ext=B, axion_bc=b, em_bc=b, pml_cells=pml, precision=prec)


TM = ["E0z", "B0x", "B0y"] + [k for k in W.FIELD_NAMES if k[1] == "1"]
CASES = {
    # name: (grid, active arrays, kernel)
    "tm2d_pml_fp64": (grid_of((300, 140, 1), (0.05, 0.05, 0.05), "fp64", "pml"), TM, "TM2D"),
    "tm2d_list_pml_fp64": (grid_of((520, 130, 1), (0.05, 0.05, 0.05), "fp64", "pml"), TM, "TM2D_LIST"),
    "tm2d_pml_fp32": (grid_of((300, 140, 1), (0.05, 0.05, 0.05), "fp32", "pml"), TM, "TM2D"),
    "tm2d_periodic_fp64": (grid_of((200, 90, 1), (0.05, 0.07, 0.05), "fp64", "periodic", B=(0.2, -0.3, 1.0)), TM,
                           "TM2D"),
    "fused_2d_all_fp64": (grid_of((96, 64, 1), (0.05, 0.06, 0.05), "fp64", "pml", B=(0.3, 0.2, 0.9)), None, "FUSED"),
    "ax3d_fp32": (grid_of((40, 36, 30), (0.06, 0.06, 0.06), "fp32", "periodic", B=(0.1, 1.0, -0.2)),
                  [k for k in W.FIELD_NAMES if k[1] == "1"], "AX3D"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_diagnostics_from_the_two_levels(case):
    from paper_2406_16796_gb300 import axp

    grid, active, kern = CASES[case]
    st = W.random_state(grid, seed=808, active=active)
    recs = []
    for via_levels in (True, False):
        g = axp.Grid(grid)
        g.set_kernel(getattr(axp, "AXP_KERNEL_" + kern))
        g.load(st)
        g.step(11)
        assert g.kernel_path() == getattr(axp, "AXP_KERNEL_" + kern)
        if not via_levels:
            g.read("E1x")  # back to integer time: the record then needs no reconstruction
        n0 = axp.axp_get_launch_count(g.h)
        recs.append(g.diagnostics())
        launches = axp.axp_get_launch_count(g.h) - n0
        if via_levels:
            assert launches == 3, launches  # the level kernel and the two reduction stages
        g.close()
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(st)
    og.step(11)
    ref = og.diagnostics()
    fp64 = grid.precision == "fp64"
    for key in KEYS:
        assert recs[0][key] == pytest.approx(recs[1][key], rel=1e-12 if fp64 else 1e-5, abs=1e-300), key
        assert recs[0][key] == pytest.approx(ref[key], rel=1e-10 if fp64 else 1e-3, abs=1e-300), key


def test_a_second_record_at_the_same_step_takes_the_backward_half_step():
    """After a record the other field set holds E^n, no longer E^{n-1/2}: a second
    record at the same step rebuilds E^n from the present level instead, and
    agrees."""
    from paper_2406_16796_gb300 import axp

    grid, active, kern = CASES["tm2d_pml_fp64"]
    g = axp.Grid(grid)
    g.load(W.random_state(grid, seed=809, active=active))
    g.step(7)
    a = g.diagnostics()
    n0 = axp.axp_get_launch_count(g.h)
    b = g.diagnostics()
    assert axp.axp_get_launch_count(g.h) - n0 > 3
    for key in KEYS:
        assert a[key] == pytest.approx(b[key], rel=1e-12, abs=1e-300), key
    g.step(3)  # and the next step makes the two levels available again
    n0 = axp.axp_get_launch_count(g.h)
    g.diagnostics()
    assert axp.axp_get_launch_count(g.h) - n0 == 3
    g.close()

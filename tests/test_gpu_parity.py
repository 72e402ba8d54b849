"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances:
  * general FP64 kernels (one pass per stage, no multiply-add contraction,
    the oracle's operation order): bit-identical fields;
  * fused FP64 kernels: normwise relative <= 1e-12 after N steps;
  * FP32 split: normwise relative <= 1e-4 on the fields and <= 1e-3 on the
    conversion probability;
  * diagnostics (different summation order): relative <= 1e-12 in FP64.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]


def axp_mod():
    from paper_2406_16796_gb300 import axp

    return axp


def periodic_grid(n, d=(0.05, 0.07, 0.06), cfl=0.5, **kw):
    nd = [a for a in range(3) if n[a] > 1]
    dt = cfl / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    return W.GridSpec(n=tuple(n), d=tuple(d), dt=dt, **kw)


def make_pair(grid, state, ghosts=None, kernel=None):
    axp = axp_mod()
    og = oracle.OracleGrid(grid)
    og.load(state)
    g = axp.Grid(grid)
    if kernel is not None:
        g.set_kernel(kernel)
    g.load(state)
    if ghosts:
        for (a, s), (cur, old) in ghosts.items():
            og.set_ghost(a, s, cur, old)
            g.write_ghost(a, s, 0, cur)
            g.write_ghost(a, s, 1, old)
    return og, g


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_ghosts(grid, seed):
    rng = np.random.default_rng(seed)
    out = {}
    for a in range(3):
        for s in range(2):
            if grid.axion_bc[a][s] == "outflow":
                shape = oracle.plane_shape(grid, a)
                out[(a, s)] = (rng.uniform(-1e-2, 1e-2, shape), rng.uniform(-1e-2, 1e-2, shape))
    return out


CASES = {
    "1d_periodic": dict(n=(64, 1, 1), B_ext=(0.0, 1.0, 0.2)),
    "2d_periodic": dict(n=(40, 24, 1), B_ext=(0.3, 0.0, 1.0)),
    "3d_periodic": dict(n=(12, 10, 8), B_ext=(0.2, -0.5, 0.7), E_ext=(0.05, 0.0, -0.1)),
    "2d_pml": dict(n=(48, 40, 1), B_ext=(0.0, 0.0, 1.0), axion_bc=W._bcs("pml", "pml"),
                   em_bc=W._bcs("pml", "pml"), pml_cells=6),
    "2d_outflow_reflect": dict(n=(36, 30, 1), B_ext=(0.0, 0.4, 1.0), axion_bc=W._bcs("outflow", ("reflect", "pml")),
                               em_bc=W._bcs("pml", ("reflect", "pml")), pml_cells=5),
    "3d_mixed": dict(n=(14, 12, 10), B_ext=(0.5, 0.2, 0.3), axion_bc=W._bcs("outflow", "periodic", "pml"),
                     em_bc=W._bcs("pml", "periodic", "reflect"), pml_cells=3),
    # power-of-two cell sizes: the general kernels multiply by the exact reciprocals
    # instead of dividing, which must leave every bit as the oracle's divisions give it
    "2d_pml_pow2": dict(n=(48, 40, 1), d=(1 / 32, 1 / 32, 1 / 32), B_ext=(0.0, 0.0, 1.0),
                        axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"), pml_cells=6),
    "3d_mixed_pow2": dict(n=(14, 12, 10), d=(0.0625, 0.125, 0.03125), B_ext=(0.5, 0.2, 0.3),
                          E_ext=(0.05, 0.0, -0.1), axion_bc=W._bcs("outflow", "periodic", "pml"),
                          em_bc=W._bcs("pml", "periodic", "reflect"), pml_cells=3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_general_fp64_bitwise_vs_oracle(case):
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, **CASES[case])
    st = W.random_state(grid, seed=101)
    og, g = make_pair(grid, st, random_ghosts(grid, 7), kernel=axp.AXP_KERNEL_GENERAL)
    og.step(6)
    g.step(6)
    ref = og.fields()
    got = g.fields()
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), (case, k, rel(got[k], ref[k]))
    for (a, s) in random_ghosts(grid, 7):
        assert np.array_equal(g.read_ghost(a, s, 0).reshape(og.ghost[a][s][0].shape), og.ghost[a][s][0])
    d, dr = g.diagnostics(), og.diagnostics()
    for key in ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "W", "sum_xB1z2", "sum_B1z2", "gauss_l2"):
        assert d[key] == pytest.approx(dr[key], rel=1e-11, abs=1e-300), key
    g.close()


@pytest.mark.parametrize("case", ["1d_periodic", "2d_pml", "3d_mixed", "3d_mixed_pow2"])
def test_fp32_split_vs_oracle(case):
    grid = periodic_grid(g=0.7, m=1.1, **CASES[case])
    st = W.random_state(grid, seed=102)
    og = oracle.OracleGrid(grid)
    og.load(st)
    for (a, s), (cur, old) in random_ghosts(grid, 8).items():
        og.set_ghost(a, s, cur, old)
    g32 = axp_mod().Grid(grid.replace(precision="fp32"))
    g32.load(st)
    for (a, s), (cur, old) in random_ghosts(grid, 8).items():
        g32.write_ghost(a, s, 0, cur)
        g32.write_ghost(a, s, 1, old)
    og.step(10)
    g32.step(10)
    ref, got = og.fields(), g32.fields()
    for k in NAMES:
        assert rel(got[k], ref[k]) < 1e-4, (case, k, rel(got[k], ref[k]))
    g32.close()


def test_inject_laser_and_axion_match_oracle():
    w = W.pulse_2d(nx=128, ny=64, m=0.3)
    grid = w.grid.replace(pml_cells=8, axion_bc=W._bcs("outflow", "pml"))
    og = oracle.OracleGrid(grid)
    g = axp_mod().Grid(grid)
    L = w.lasers[0]
    A = W.AxionSpec(amplitude=0.3, k=(-W.K0, 0.5, 0.0), centre=(1.0, 0.2, 0.0), waist=0.8, length=0.6, speed=0.9,
                    phase=0.4)
    for x in (og, g):
        x.inject_laser(L)
        x.inject_axion(A)
    ref, got = og.fields(), g.fields()
    for k in ("E0z", "B0x", "B0y", "phi_cur", "phi_old"):
        assert rel(got[k], ref[k]) < 1e-13, k
    for s in range(2):
        for lev in range(2):
            gg = g.read_ghost(0, s, lev).reshape(og.ghost[0][s][lev].shape)
            assert rel(gg, og.ghost[0][s][lev]) < 1e-13
    g.close()


def test_1d_conversion_run_matches_oracle_fp64_and_fp32():
    """The 1D photon->axion workload (Nx = 4096, dx = lambda/32, CFL 0.95, g = 1e-4,
    B0 = 1, amplitude 1e-3) for 2000 steps."""
    w = W.vacuum_1d(nx=4096)
    og = oracle.run_workload(w, steps=2000)
    ref = og.fields()
    P_ref = og.diagnostics()["P_g2a"]
    for prec in ("fp64", "fp32"):
        g = axp_mod().Grid(w.grid.replace(precision=prec))
        g.inject_laser(w.lasers[0])
        g.step(2000)
        got = g.fields()
        P = g.diagnostics()["P_g2a"]
        ftol = 1e-12 if prec == "fp64" else 1e-3
        for k in ("E0y", "B0z", "E1y", "E1z", "B1y", "B1z", "phi_cur"):
            assert rel(got[k], ref[k]) < ftol, (prec, k, rel(got[k], ref[k]))
        assert abs(P / P_ref - 1) < (1e-12 if prec == "fp64" else 1e-3), (prec, P, P_ref)
        g.close()


def test_diagnostics_ring_records_every_k_steps():
    axp = axp_mod()
    w = W.vacuum_1d(nx=256)
    g = axp.Grid(w.grid, diag_every=10, diag_capacity=8)
    g.inject_laser(w.lasers[0])
    g.step(50)
    recs = g.read_diagnostics()
    assert [r["step"] for r in recs] == [10, 20, 30, 40, 50]
    og = oracle.OracleGrid(w.grid)
    og.inject_laser(w.lasers[0])
    og.step(50)
    assert recs[-1]["P_g2a"] == pytest.approx(og.diagnostics()["P_g2a"], rel=1e-10)
    g.step(100)  # ring of 8 overwrites; the 8 newest survive
    recs = g.read_diagnostics()
    assert [r["step"] for r in recs] == list(range(80, 151, 10))
    g.close()


def test_checkpoint_resume_is_bitwise():
    w = W.pulse_2d(nx=96, ny=48, m=0.5 * W.K0, g=1e-2)
    grid = w.grid.replace(pml_cells=8)
    for prec in ("fp64", "fp32"):
        gs = grid.replace(precision=prec)
        a = axp_mod().Grid(gs)
        a.inject_laser(w.lasers[0])
        a.step(30)
        img = a.save_state()
        a.step(30)
        ref = a.fields()
        b = axp_mod().Grid(gs)
        b.load_state(img)
        b.step(30)
        got = b.fields()
        # and both equal a run never saved: the image of a stepping grid keeps its
        # leapfrog-staggered form, so neither the save nor the load converted it
        c = axp_mod().Grid(gs)
        c.inject_laser(w.lasers[0])
        c.step(30)
        c.step(30)
        once = c.fields()
        for k in NAMES:
            assert np.array_equal(got[k], ref[k]), (prec, k)
            assert np.array_equal(once[k], ref[k]), (prec, k)
        assert b.step_count == 60
        a.close()
        b.close()
        c.close()


def test_zero_steps_and_empty_work_are_noops():
    w = W.vacuum_1d(nx=64)
    g = axp_mod().Grid(w.grid)
    g.inject_laser(w.lasers[0])
    before = g.fields()
    g.step(0)
    after = g.fields()
    for k in NAMES:
        assert np.array_equal(before[k], after[k])
    g.close()


FUSED_CASES = {
    "1d_periodic": dict(n=(300, 1, 1), B_ext=(0.0, 1.0, 0.2)),
    "2d_periodic": dict(n=(300, 40, 1), B_ext=(0.3, 0.0, 1.0)),
    "2d_pml": dict(n=(260, 70, 1), B_ext=(0.0, 0.0, 1.0), axion_bc=W._bcs("pml", "pml"),
                   em_bc=W._bcs("pml", "pml"), pml_cells=6),
    "2d_reflect_pml": dict(n=(140, 90, 1), B_ext=(0.0, 0.4, 1.0), axion_bc=W._bcs("reflect", ("pml", "reflect")),
                           em_bc=W._bcs("reflect", ("pml", "reflect")), pml_cells=5),
    "3d_periodic": dict(n=(40, 30, 20), B_ext=(0.2, -0.5, 0.7)),
    "3d_pml_reflect": dict(n=(36, 24, 22), B_ext=(0.5, 0.2, 0.3), axion_bc=W._bcs("reflect", "periodic", "pml"),
                           em_bc=W._bcs("reflect", "periodic", "pml"), pml_cells=4),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(FUSED_CASES))
def test_fused_vs_oracle(case, prec):
    """The single-pass kernel against the oracle on random states (several tiles
    and march chunks with ragged tails), all fields after 12 steps."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, **FUSED_CASES[case]).replace(precision=prec)
    # 3D: order-1 fields and the axion in a uniform background (the 3D workload's
    # case).  In 3D any order-0 laser component couples to all six through the
    # curls, and that ring does not fit in shared memory; nor does any 3D FP64
    # ring.  Those grids run on the general kernels (checked below).
    active = None
    if case.startswith("3d"):
        active = [n for n in W.FIELD_NAMES if n[1] == "1"]
    st = W.random_state(grid, seed=303, active=active)
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(st)
    g = axp.Grid(grid)
    g.set_kernel(axp.AXP_KERNEL_AUTO)
    g.load(st)
    if case == "3d_periodic":
        expect = axp.AXP_KERNEL_AX3D  # periodic 3D without laser fields: the specialised kernel
    elif case.startswith("3d") and prec == "fp64":
        expect = axp.AXP_KERNEL_GENERAL
    elif case.startswith("1d") and prec == "fp64":
        expect = axp.AXP_KERNEL_BLOCK1D  # periodic FP64 line: the time-blocked kernel
    else:
        expect = axp.AXP_KERNEL_FUSED
    assert g.kernel_path() == expect
    if case.startswith("1d"):
        g.set_kernel(axp.AXP_KERNEL_FUSED)  # the single-pass kernel is what this test checks
        assert g.kernel_path() == axp.AXP_KERNEL_FUSED
    og.step(12)
    g.step(12)
    ref, got = og.fields(), g.fields()
    tol = 1e-12 if prec == "fp64" else 1e-4
    for k in NAMES:
        assert rel(got[k], ref[k]) < tol, (case, prec, k, rel(got[k], ref[k]))
    d, dr = g.diagnostics(), og.diagnostics()
    for key in ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "sum_xB1z2", "sum_B1z2"):
        assert d[key] == pytest.approx(dr[key], rel=1e-10 if prec == "fp64" else 1e-4), key
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_matches_general_over_many_steps(prec):
    """2D pulse through B_ext with PML: fused and general paths agree after 300 steps,
    including the in-step diagnostics ring."""
    axp = axp_mod()
    w = W.pulse_2d(nx=384, ny=160, m=0.5 * W.K0, g=1e-2, precision=prec)
    grid = w.grid.replace(pml_cells=10)
    out = {}
    for kern in (axp.AXP_KERNEL_GENERAL, axp.AXP_KERNEL_FUSED):
        g = axp.Grid(grid, diag_every=50, diag_capacity=16)
        g.set_kernel(kern)
        g.inject_laser(w.lasers[0])
        g.step(300)
        out[kern] = (g.fields(), g.read_diagnostics())
        g.close()
    (fa, da), (fb, db) = out[axp.AXP_KERNEL_GENERAL], out[axp.AXP_KERNEL_FUSED]
    tol = 1e-12 if prec == "fp64" else 2e-4
    for k in NAMES:
        assert rel(fb[k], fa[k]) < tol, (prec, k, rel(fb[k], fa[k]))
    assert [r["step"] for r in da] == [r["step"] for r in db] == [50, 100, 150, 200, 250, 300]
    for ra, rb in zip(da, db):
        assert rb["P_g2a"] == pytest.approx(ra["P_g2a"], rel=1e-10 if prec == "fp64" else 1e-3)


TM2D_CASES = {
    "periodic": dict(n=(600, 90, 1), B_ext=(0.2, -0.4, 1.0)),
    "pml": dict(n=(520, 130, 1), B_ext=(0.1, 0.3, 1.0), axion_bc=W._bcs("pml", "pml"),
                em_bc=W._bcs("pml", "pml"), pml_cells=8),
    "periodic_x_pml_y": dict(n=(560, 100, 1), B_ext=(0.0, 0.0, 1.0), axion_bc=W._bcs("periodic", "pml"),
                             em_bc=W._bcs("periodic", "pml"), pml_cells=6),
    # square cells and B_ext along z only: the FP64 kernel's folded form of the current
    "pml_square_cells": dict(n=(520, 130, 1), d=(0.05, 0.05, 0.05), B_ext=(0.0, 0.0, 1.3),
                             axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"), pml_cells=8),
    "periodic_square_cells": dict(n=(600, 90, 1), d=(0.04, 0.04, 0.04), B_ext=(0.0, 0.0, -0.8)),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(TM2D_CASES))
def test_tm2d_kernel_vs_oracle(case, prec):
    """The 2D kernel specialised for the (E0z; B0x, B0y) laser against the oracle on
    random states: several x tiles, march chunks with ragged tails, PML layers and
    periodic wrap, all fields after 12 steps."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, **TM2D_CASES[case]).replace(precision=prec)
    active = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
    st = W.random_state(grid, seed=404, active=active)
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(st)
    g = axp.Grid(grid)
    g.set_kernel(axp.AXP_KERNEL_TM2D)
    g.load(st)
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D
    og.step(12)
    g.step(12)
    ref, got = og.fields(), g.fields()
    tol = 1e-12 if prec == "fp64" else 1e-4
    for k in NAMES:
        assert rel(got[k], ref[k]) < tol, (case, prec, k, rel(got[k], ref[k]))
    g.close()


def test_tm2d_refuses_unsupported_grids():
    """Forcing the specialised kernel on a grid it does not support is an error, not a fallback."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, n=(64, 40, 1), axion_bc=W._bcs("reflect", "pml"),
                         em_bc=W._bcs("reflect", "pml"), pml_cells=4)
    g = axp.Grid(grid)
    g.set_kernel(axp.AXP_KERNEL_TM2D)
    assert g.kernel_path() == axp.AXP_KERNEL_GENERAL
    with pytest.raises(axp.AxpError) as e:
        g.step(1)
    assert e.value.status == axp.AXP_E_STATE
    g.close()


AX3D_CASES = {
    "ragged": dict(n=(70, 37, 45), B_ext=(0.2, -0.5, 0.7), d=(0.05, 0.07, 0.06)),
    "cube": dict(n=(40, 40, 40), B_ext=(0.0, 1.0, 0.0), d=(0.06, 0.06, 0.06)),
    "thin_z": dict(n=(33, 20, 3), B_ext=(1.0, 0.5, -0.2), d=(0.05, 0.05, 0.08)),
}


@pytest.mark.parametrize("case", sorted(TM2D_CASES))
def test_tm2d_work_lists_equal_the_uniform_grid_and_the_oracle(case):
    """The 2D kernel's work-list form (tiles of about equal cost, two short ones
    sharing a block) computes every cell with the same operations as the uniform
    launch grid: the fields are bit for bit those of the grid form, and within
    1e-12 of the oracle, after 12 steps."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, **TM2D_CASES[case])
    active = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
    st = W.random_state(grid, seed=405, active=active)
    out = {}
    for kernel in (axp.AXP_KERNEL_TM2D, axp.AXP_KERNEL_TM2D_LIST):
        g = axp.Grid(grid)
        g.set_kernel(kernel)
        g.load(st)
        assert g.kernel_path() == kernel
        g.step(5)
        g.step(7)
        out[kernel] = g.fields()
        g.close()
    og = oracle.OracleGrid(grid)
    og.load(st)
    og.step(12)
    ref = og.fields()
    for k in NAMES:
        assert np.array_equal(out[axp.AXP_KERNEL_TM2D_LIST][k], out[axp.AXP_KERNEL_TM2D][k]), (case, k)
        assert rel(out[axp.AXP_KERNEL_TM2D_LIST][k], ref[k]) < 1e-12, (case, k)


@pytest.mark.parametrize("n", [(300, 40, 1), (1000, 17, 1), (130, 700, 1), (260, 3, 1)])
def test_tm2d_work_lists_on_ragged_shapes(n):
    """Work lists on shapes whose strips end in a few columns (the last strip's
    warps beyond the grid keep the closure's zeros without computing them), whose
    strips outnumber or are outnumbered by the resident blocks, and one only three
    planes high: bit for bit the uniform grid's fields."""
    axp = axp_mod()
    grid = periodic_grid(g=0.9, m=0.7, n=n, d=(0.05, 0.05, 0.05), B_ext=(0.0, 0.0, 1.1),
                         axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"), pml_cells=min(6, n[1] // 2))
    if n[1] < 8:
        grid = grid.replace(axion_bc=W._bcs("pml", "periodic"), em_bc=W._bcs("pml", "periodic"))
    active = ["E0z", "B0x", "B0y"] + [k for k in W.FIELD_NAMES if k[1] == "1"]
    st = W.random_state(grid, seed=406, active=active)
    out = {}
    for kernel in (axp.AXP_KERNEL_TM2D, axp.AXP_KERNEL_TM2D_LIST, axp.AXP_KERNEL_GENERAL):
        g = axp.Grid(grid)
        g.set_kernel(kernel)
        g.load(st)
        g.step(9)
        out[kernel] = g.fields()
        g.close()
    for k in NAMES:
        assert np.array_equal(out[axp.AXP_KERNEL_TM2D_LIST][k], out[axp.AXP_KERNEL_TM2D][k]), (n, k)
        assert rel(out[axp.AXP_KERNEL_TM2D_LIST][k], out[axp.AXP_KERNEL_GENERAL][k]) < 1e-12, (n, k)


def test_tm2d_work_lists_refuse_fp32_and_soft_sources():
    """The work-list form takes FP64 grids without a soft source; forcing it on
    others is an error, not a fallback."""
    axp = axp_mod()
    kw = dict(n=(200, 60, 1), B_ext=(0.0, 0.0, 1.0), axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"),
              pml_cells=6)
    g = axp.Grid(periodic_grid(g=0.7, m=1.1, precision="fp32", **kw))
    g.set_kernel(axp.AXP_KERNEL_TM2D_LIST)
    assert g.kernel_path() == axp.AXP_KERNEL_GENERAL
    with pytest.raises(axp.AxpError) as e:
        g.step(1)
    assert e.value.status == axp.AXP_E_STATE
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(AX3D_CASES))
def test_ax3d_kernel_vs_oracle_and_generic(case, prec):
    """The 3D kernel specialised for an axion box (periodic, order-1 fields, phi,
    uniform B) against the oracle on random states: several x/y tiles with
    ragged tails and many short z chunks, all fields after 12 steps; in FP32
    also against the generic single-pass kernel to FP32 rounding."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, **AX3D_CASES[case]).replace(precision=prec)
    st = W.random_state(grid, seed=505, active=[n for n in W.FIELD_NAMES if n[1] == "1"])
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(st)
    g = axp.Grid(grid)
    g.set_kernel(axp.AXP_KERNEL_AX3D)
    g.load(st)
    assert g.kernel_path() == axp.AXP_KERNEL_AX3D
    og.step(12)
    g.step(12)
    ref, got = og.fields(), g.fields()
    tol = 1e-12 if prec == "fp64" else 1e-4
    for k in NAMES:
        assert rel(got[k], ref[k]) < tol, (case, prec, k, rel(got[k], ref[k]))
    if prec == "fp32":
        f = axp.Grid(grid)
        f.set_kernel(axp.AXP_KERNEL_FUSED)
        f.load(st)
        assert f.kernel_path() == axp.AXP_KERNEL_FUSED
        f.step(12)
        gen = f.fields()
        for k in NAMES:
            assert rel(got[k], gen[k]) < 2e-6, (case, k, rel(got[k], gen[k]))
        f.close()
    g.close()


def test_ax3d_refuses_grids_with_laser_fields_or_absorbing_sides():
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, n=(20, 18, 16), B_ext=(0.0, 1.0, 0.0)).replace(precision="fp32")
    g = axp.Grid(grid)
    g.write("E0y", W.random_state(grid, seed=1)["E0y"])  # an order-0 field makes the set non-empty
    g.set_kernel(axp.AXP_KERNEL_AX3D)
    assert g.kernel_path() == axp.AXP_KERNEL_GENERAL
    with pytest.raises(axp.AxpError) as e:
        g.step(1)
    assert e.value.status == axp.AXP_E_STATE
    g.close()
    pml = periodic_grid(g=0.7, m=1.1, n=(20, 18, 16), B_ext=(0.0, 1.0, 0.0), axion_bc=W._bcs("periodic", "periodic", "pml"),
                        em_bc=W._bcs("periodic", "periodic", "pml"), pml_cells=3).replace(precision="fp32")
    h = axp.Grid(pml)
    h.set_kernel(axp.AXP_KERNEL_AX3D)
    assert h.kernel_path() == axp.AXP_KERNEL_GENERAL
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_1d_graph_replay_matches_single_launches(prec):
    """Runs of 1D steps replay from CUDA graphs of 48 launches; the states equal
    those of the same steps launched one by one, also across a field write
    between runs (which must invalidate the captured parameters)."""
    axp = axp_mod()
    grid = periodic_grid(g=0.7, m=1.1, n=(500, 1, 1), B_ext=(0.0, 1.0, 0.3)).replace(precision=prec)
    st = W.random_state(grid, seed=606, active=["E0y", "B0z"] + [n for n in W.FIELD_NAMES if n[1] == "1"])
    a, b = axp.Grid(grid), axp.Grid(grid)
    for x in (a, b):
        x.set_kernel(axp.AXP_KERNEL_FUSED)
        x.load(st)
    a.step(100)  # two graph replays and four single launches
    for _ in range(100):
        b.step(1)
    fa, fb = a.fields(), b.fields()
    for k in NAMES:
        assert np.array_equal(fa[k], fb[k]), k
    kick = W.random_state(grid, seed=607)["B1y"]
    for x in (a, b):
        x.write("B1y", kick)
    a.step(97)
    for _ in range(97):
        b.step(1)
    fa, fb = a.fields(), b.fields()
    for k in NAMES:
        assert np.array_equal(fa[k], fb[k]), k
    assert a.step_count == b.step_count == 197
    a.close()
    b.close()


@pytest.mark.parametrize("steps", [1, 3, 7])
def test_fused_odd_step_counts_keep_inactive_arrays_zero(steps):
    """After an odd number of fused steps the state lives in the second field set;
    the arrays the step does not touch (here E0x, E0y, B0z of the TM set) must
    still be zero there, and the fields equal the oracle's."""
    axp = axp_mod()
    grid = periodic_grid(g=1.3, m=2.0, n=(64, 90, 1), B_ext=(0.1, -0.2, -1.0), axion_bc=W._bcs("periodic", "pml"),
                         em_bc=W._bcs("periodic", "pml"), pml_cells=6)
    active = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
    st = W.random_state(grid, seed=77, active=active)
    og = oracle.OracleGrid(grid)
    og.load(st)
    og.step(steps)
    g = axp.Grid(grid)
    g.load(st)
    g.step(steps)
    assert g.kernel_path() in (axp.AXP_KERNEL_TM2D, axp.AXP_KERNEL_TM2D_LIST)
    got, ref = g.fields(), og.fields()
    for k in ("E0x", "E0y", "B0z"):
        assert not got[k].any(), k
    for k in NAMES:
        assert rel(got[k], ref[k]) < 1e-12, (steps, k, rel(got[k], ref[k]))
    g.close()


TM_ACTIVE = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
BOX_ACTIVE = [n for n in W.FIELD_NAMES if n[1] == "1"]
TINY = {
    # name: (n, boundary on each active axis, pml cells, active arrays or None for all,
    #        the kernel the automatic choice takes in FP64 and in FP32)
    "1d_2": ((2, 1, 1), "periodic", 0, None, ("FUSED", "FUSED")),
    "1d_7_pml": ((7, 1, 1), "pml", 2, None, ("FUSED", "FUSED")),
    "2d_5x3_tm": ((5, 3, 1), "periodic", 0, TM_ACTIVE, ("TM2D", "TM2D")),
    "2d_8x16_tm_pml": ((8, 16, 1), "pml", 2, TM_ACTIVE, ("TM2D", "TM2D")),
    "2d_3x4_all": ((3, 4, 1), "periodic", 0, None, ("FUSED", "FUSED")),
    "3d_3_box": ((3, 3, 3), "periodic", 0, BOX_ACTIVE, ("AX3D", "AX3D")),
    "3d_2x3x4_box": ((2, 3, 4), "periodic", 0, BOX_ACTIVE, ("AX3D", "AX3D")),
    "3d_4_all": ((4, 4, 4), "periodic", 0, None, ("GENERAL", "GENERAL")),  # rings too large: general
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(TINY))
def test_tiny_grids_match_the_oracle(case, prec):
    """Degenerate sizes: grids of 2 to 16 cells per axis, far narrower than a tile,
    whose halos wrap more than once around a periodic axis, on whichever kernel the
    automatic choice takes and on the general path, against the oracle."""
    axp = axp_mod()
    n, bc, pml, active, paths = TINY[case]
    b = W._bcs(*[bc if n[a] > 1 else "periodic" for a in range(3)])
    grid = periodic_grid(n, B_ext=(0.3, -0.2, 0.9), m=1.3, g=0.6, axion_bc=b, em_bc=b, pml_cells=pml,
                         precision=prec)
    st = W.random_state(grid, seed=4321, active=active)
    tol = 1e-12 if prec == "fp64" else 1e-4
    for kernel in (axp.AXP_KERNEL_AUTO, axp.AXP_KERNEL_GENERAL):
        g = axp.Grid(grid)
        g.set_kernel(kernel)
        g.load(st)
        og = oracle.OracleGrid(grid.replace(precision="fp64"))
        og.load(st)
        g.step(5)
        og.step(5)
        if kernel == axp.AXP_KERNEL_AUTO:
            want = paths[0 if prec == "fp64" else 1]
            ok = {getattr(axp, "AXP_KERNEL_" + want)}
            if want == "TM2D" and prec == "fp64":
                ok.add(axp.AXP_KERNEL_TM2D_LIST)  # (the 2D kernel's work-list form, where the planner prefers it)
            assert g.kernel_path() in ok, (case, g.kernel_path(), want)
        got, ref = g.fields(), og.fields()
        for k in list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]:
            assert rel(got[k], ref[k]) <= tol, (case, kernel, k, rel(got[k], ref[k]))
        g.close()

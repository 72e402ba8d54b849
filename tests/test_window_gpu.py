"""Moving window (Sec. 3.2): the state shifts by whole cells along the window
axis, vacuum entering at the leading edge.  A shift is compared with the same
shift of the arrays in numpy (bit for bit), and windowed runs with the oracle
stepped on the same schedule with its arrays shifted the same way (general
path bit for bit in FP64; fused paths at their tolerances)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]
AXIS_DIM = {0: 2, 1: 1, 2: 0}  # array dimension of each grid axis (arrays are (nz, ny, nx))


def axp_mod():
    from paper_2406_16796_gb300 import axp

    return axp


def shifted(a, axis, s):
    d = AXIS_DIM[axis]
    out = np.zeros_like(a)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    src[d] = slice(s, None)
    dst[d] = slice(0, a.shape[d] - s)
    out[tuple(dst)] = a[tuple(src)]
    return out


def pml_grid(n, prec, cfl=0.5, d=(0.05, 0.07, 0.06), pml=5, **kw):
    nd = [a for a in range(3) if n[a] > 1]
    dt = cfl / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    bc = W._bcs(*["pml" if n[a] > 1 else "periodic" for a in range(3)])
    return W.GridSpec(n=tuple(n), d=tuple(d), dt=dt, m=1.1, g=0.7, B_ext=(0.1, -0.3, 0.8), axion_bc=bc, em_bc=bc,
                      pml_cells=pml, precision=prec, **kw)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,axis,s", [((90, 40, 1), 0, 7), ((60, 50, 1), 1, 13), ((20, 18, 16), 2, 3)])
def test_shift_is_the_array_shift(prec, n, axis, s):
    axp = axp_mod()
    grid = pml_grid(n, prec)
    g = axp.Grid(grid)
    g.load(W.random_state(grid, seed=808))
    before = g.fields()
    g.shift_window(axis, s)
    after = g.fields()
    for k in NAMES:
        assert np.array_equal(after[k], shifted(before[k], axis, s)), k
    assert g.window_offset() == s
    g.close()


def windowed_pair(prec, kernel, steps, v=1.0, cells=4, start=6, n=(160, 60, 1)):
    """Run the pulse set-up with a moving window on the GPU one step at a time and
    the oracle alongside, shifting the oracle's arrays whenever the GPU window moved."""
    axp = axp_mod()
    w = W.pulse_2d(nx=n[0], ny=n[1], m=0.5 * W.K0, g=1e-2, precision=prec)
    grid = w.grid.replace(pml_cells=8)
    L = W.LaserSpec(amplitude=0.01, k=(W.K0, 0.0, 0.0), pol=(0.0, 0.0, 1.0), centre=(1.5, 0.0, 0.0), waist=0.4,
                    duration=0.8)
    g = axp.Grid(grid)
    g.set_kernel(kernel)
    g.inject_laser(L)
    g.set_moving_window(0, v, cells, start)
    # the oracle starts from the GPU's injected state (the two injections agree
    # to rounding of their sin/cos, not bit for bit)
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(g.fields())
    shifts = []
    off = 0
    for i in range(steps):
        g.step(1)
        og.step(1)
        now = g.window_offset()
        if now != off:
            st = og.fields()
            og.load({k: shifted(st[k], 0, now - off) for k in NAMES})
            shifts.append((i + 1, now - off))
            off = now
    return g, og, shifts, grid


def test_windowed_run_general_path_matches_oracle_bitwise():
    axp = axp_mod()
    g, og, shifts, grid = windowed_pair("fp64", axp.AXP_KERNEL_GENERAL, 60)
    u = grid.dt / grid.d[0]
    # the window starts at step 6 and moves u cells per step in 4-cell shifts
    assert [s for _, s in shifts] == [4] * int((60 - 6) * u / 4)
    assert shifts[0][0] == 6 + math.ceil(4 / u - 1e-9)
    got, ref = g.fields(), og.fields()
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), k
    assert g.step_count == 60
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_windowed_run_fused_path_matches_oracle(prec):
    axp = axp_mod()
    g, og, shifts, grid = windowed_pair(prec, axp.AXP_KERNEL_AUTO, 60)
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D and len(shifts) >= 5
    got, ref = g.fields(), og.fields()
    tol = 1e-12 if prec == "fp64" else 1e-4
    for k in NAMES:
        nb = np.linalg.norm(ref[k])
        assert np.linalg.norm(got[k] - ref[k]) <= tol * (nb if nb > 0 else 1.0), k
    d, dr = g.diagnostics(), og.diagnostics()
    assert d["H_g0"] == pytest.approx(dr["H_g0"], rel=1e-10 if prec == "fp64" else 1e-4)
    g.close()


def test_window_keeps_the_pulse_in_view_and_survives_checkpoints():
    """The window moving at c keeps the laser's energy in the box (a fixed box loses
    it through the absorbing side), and a checkpoint restores the window state."""
    axp = axp_mod()
    w = W.pulse_2d(nx=128, ny=32, m=0.0, g=1e-3, precision="fp64")
    # absorbing along x, periodic along y, a pulse that is plane across y (no diffraction)
    grid = w.grid.replace(pml_cells=8, axion_bc=W._bcs("pml", "periodic"), em_bc=W._bcs("pml", "periodic"))
    L = W.LaserSpec(amplitude=0.01, k=(W.K0, 0.0, 0.0), pol=(0.0, 0.0, 1.0), centre=(2.0, 0.0, 0.0), duration=0.8)
    fixed, moving = axp.Grid(grid), axp.Grid(grid)
    for x in (fixed, moving):
        x.inject_laser(L)
    moving.set_moving_window(0, 1.0, 2, 0)
    e0 = fixed.diagnostics()["H_g0"]
    fixed.step(300)
    moving.step(150)
    blob = moving.save_state()
    moving.step(150)
    ref = moving.fields()
    assert fixed.diagnostics()["H_g0"] < 0.05 * e0
    assert moving.diagnostics()["H_g0"] > 0.8 * e0
    moving.load_state(blob)
    moving.step(150)
    again = moving.fields()
    for k in NAMES:
        assert np.array_equal(again[k], ref[k]), k
    for x in (fixed, moving):
        x.close()


def test_window_refuses_periodic_axes_outflow_and_bad_speeds():
    axp = axp_mod()
    per = W.GridSpec(n=(64, 32, 1), d=(0.05, 0.05, 0.05), dt=0.02, precision="fp64")
    g = axp.Grid(per)
    for call in (lambda: g.shift_window(0, 3), lambda: g.set_moving_window(0, 1.0, 1, 0)):
        with pytest.raises(axp.AxpError) as e:
            call()
        assert e.value.status == axp.AXP_E_INVAL
    g.close()
    grid = pml_grid((64, 32, 1), "fp64")
    h = axp.Grid(grid)
    for args in ((0, 1.5, 1, 0), (0, 1.0, 0, 0), (0, 1.0, 64, 0), (2, 1.0, 1, 0)):
        with pytest.raises(axp.AxpError):
            h.set_moving_window(*args)
    h.shift_window(0, 2)
    with pytest.raises(axp.AxpError):  # one window axis per grid
        h.shift_window(1, 2)
    h.close()
    out = pml_grid((64, 32, 1), "fp64").replace(axion_bc=W._bcs("outflow", "pml"))
    o = axp.Grid(out)
    with pytest.raises(axp.AxpError):
        o.shift_window(0, 1)
    o.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("axis,s", [(0, 4), (0, 16), (1, 7)])
def test_staggered_shift_matches_the_integer_time_shift(prec, axis, s):
    """A shift of a grid held in the fused path's staggered state takes only the
    bands at the ends of the window axis through integer time; it gives the state
    of the same shift done in integer time (the grid converted as a whole first),
    to rounding, and the runs that follow stay together."""
    axp = axp_mod()
    w = W.pulse_2d(nx=300, ny=160, m=0.5 * W.K0, g=1e-2, precision=prec)
    grid = w.grid.replace(pml_cells=10)
    L = W.LaserSpec(amplitude=0.01, k=(W.K0, 0.0, 0.0), pol=(0.0, 0.0, 1.0), centre=(4.0, 0.0, 0.0), waist=0.8,
                    duration=1.0)
    a, b = axp.Grid(grid), axp.Grid(grid)
    for x in (a, b):
        x.inject_laser(L)
        x.step(25)
    assert a.kernel_path() == axp.AXP_KERNEL_TM2D
    n0 = a.launches()
    a.shift_window(axis, s)                # staggered: banded
    banded = a.launches() - n0
    axp.axp_set_background_field(b.h, grid.B_ext, grid.E_ext)  # converts the whole grid to integer time
    n1 = b.launches()
    b.shift_window(axis, s)
    # a whole-grid conversion before the shift would add 4 launches; the two bands'
    # round trips add 14
    assert banded - (b.launches() - n1) > 4
    tol = 1e-12 if prec == "fp64" else 1e-5
    for steps in (0, 20):
        a.step(steps)
        b.step(steps)
        fa, fb = a.fields(), b.fields()
        for k in NAMES:
            nb = np.linalg.norm(fb[k])
            assert np.linalg.norm(fa[k] - fb[k]) <= tol * (nb if nb > 0 else 1.0), (steps, k)
    for x in (a, b):
        x.close()

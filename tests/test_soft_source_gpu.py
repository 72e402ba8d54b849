"""Soft-source laser injection through an x-plane (Sec. 3.2 injects the laser
into the box) on the GPU against the oracle: the general path bit for bit in
FP64, the 2D TM kernel at the fused FP64 tolerance (1e-12) and at the FP32
split tolerance (fields 1e-4, conversion probability 1e-3), with the axion
coupled, on grids of several tiles with a ragged last strip."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]
DX = 1.0 / 32
K0 = 2 * math.pi


def axp_mod():
    from paper_2406_16796_gb300 import axp

    return axp


def grid2d(nx, ny, prec, ybc="pml", m=1.1, g=0.7, pml=12):
    dt = 0.95 * DX / math.sqrt(2)
    bc = W._bcs("pml", ybc)
    return W.GridSpec(n=(nx, ny, 1), d=(DX, DX, DX), dt=dt, m=m, g=g, B_ext=(0.0, 0.2, 1.0), axion_bc=bc, em_bc=bc,
                      pml_cells=pml, precision=prec)


def grid1d(nx, prec, m=0.9, g=0.5):
    bc = W._bcs("pml")
    return W.GridSpec(n=(nx, 1, 1), d=(DX, DX, DX), dt=0.95 * DX, m=m, g=g, B_ext=(0.0, 1.0, 0.3), axion_bc=bc,
                      em_bc=bc, pml_cells=10, precision=prec)


def beam(ny, pol=(0.0, 0.0, 1.0), plane=30):
    return W.SourceSpec(amplitude=0.05, k=K0, pol=pol, plane=plane, centre=(plane * DX, ny * DX * 0.45, 0.0),
                        waist=0.9, duration=1.5, t_centre=1.2, phase=0.4)


def pair(grid, src, steps, kernel):
    axp = axp_mod()
    g = axp.Grid(grid)
    g.set_kernel(kernel)
    g.set_soft_source(src)
    g.step(steps)
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.set_soft_source(src)
    og.step(steps)
    return g, og


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("case", ["1d", "2d"])
def test_general_path_is_bitwise_the_oracle(case):
    axp = axp_mod()
    if case == "1d":
        grid, src = grid1d(500, "fp64"), W.SourceSpec(amplitude=0.05, k=K0, pol=(0.0, 0.6, -0.8), plane=40,
                                                      centre=(40 * DX, 0, 0), duration=1.0, t_centre=1.0, phase=0.2)
    else:
        grid, src = grid2d(130, 60, "fp64"), beam(60, pol=(0.0, 0.6, 0.8), plane=20)
    g, og = pair(grid, src, 90, axp.AXP_KERNEL_GENERAL)
    got, ref = g.fields(), og.fields()
    assert np.max(np.abs(ref["E0y"] if case == "1d" else ref["E0z"])) > 1e-3 * src.amplitude
    assert np.max(np.abs(ref["phi_cur"])) > 0
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), k
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tm2d_kernel_matches_the_oracle(prec):
    axp = axp_mod()
    grid, src = grid2d(600, 150, prec), beam(150)
    g, og = pair(grid, src, 120, axp.AXP_KERNEL_AUTO)
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D
    got, ref = g.fields(), og.fields()
    assert np.max(np.abs(ref["E0z"])) > 1e-2 * src.amplitude
    tol = 1e-12 if prec == "fp64" else 1e-4
    for k in NAMES:
        assert rel(got[k], ref[k]) <= tol, (k, rel(got[k], ref[k]))
    d, dr = g.diagnostics(), og.diagnostics()
    assert d["P_g2a"] == pytest.approx(dr["P_g2a"], rel=1e-10 if prec == "fp64" else 1e-3)
    assert d["H_g0"] == pytest.approx(dr["H_g0"], rel=1e-10 if prec == "fp64" else 1e-4)
    g.close()


def test_tm2d_periodic_y_and_source_switched_mid_run():
    """The source set while the fused path holds its staggered state (which was
    formed without it), later switched off: the grid goes back to integer time
    before each change, as the oracle's run does."""
    axp = axp_mod()
    grid = grid2d(300, 64, "fp64", ybc="periodic")
    src = beam(64, plane=40)
    g = axp.Grid(grid)
    og = oracle.OracleGrid(grid)
    g.step(7)
    og.step(7)
    g.set_soft_source(src)
    og.set_soft_source(src)
    g.step(60)
    og.step(60)
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D
    g.set_soft_source(None)
    og.set_soft_source(None)
    g.step(25)
    og.step(25)
    got, ref = g.fields(), og.fields()
    for k in NAMES:
        assert rel(got[k], ref[k]) <= 1e-12, k
    g.close()


def test_path_selection_and_refusals():
    axp = axp_mod()
    from paper_2406_16796_gb300 import group

    # E_y polarisation in 2D is outside the TM kernel's field set: general path
    g = axp.Grid(grid2d(200, 40, "fp64"))
    g.set_soft_source(beam(40, pol=(0.0, 1.0, 0.0)))
    assert g.kernel_path() == axp.AXP_KERNEL_GENERAL
    g.close()
    # 1D with a source: the generic fused kernel takes none; a forced choice is refused
    h = axp.Grid(grid1d(300, "fp64"))
    h.set_soft_source(W.SourceSpec(amplitude=0.1, k=K0, pol=(0.0, 1.0, 0.0), plane=50))
    assert h.kernel_path() == axp.AXP_KERNEL_GENERAL
    h.set_kernel(axp.AXP_KERNEL_FUSED)
    with pytest.raises(axp.AxpError) as e:
        h.step(1)
    assert e.value.status == axp.AXP_E_STATE
    h.set_kernel(axp.AXP_KERNEL_AUTO)
    # invalid sheets: inside the x layer, at the edge, polarisation along x, k <= 0
    for bad in (dict(plane=5), dict(plane=0), dict(plane=300), dict(pol=(0.6, 0.8, 0.0)), dict(k=-1.0)):
        kw = dict(amplitude=0.1, k=K0, pol=(0.0, 1.0, 0.0), plane=50)
        kw.update(bad)
        with pytest.raises(axp.AxpError) as e:
            h.set_soft_source(W.SourceSpec(**kw))
        assert e.value.status == axp.AXP_E_INVAL
    h.close()
    # a group does not take a grid with a source
    G = group.Group(2, 100)
    s = axp.Grid(grid2d(256, 128, "fp32", ybc="periodic"))
    s.set_soft_source(beam(128))
    with pytest.raises(axp.AxpError) as e:
        G.add(s, 10)
    assert e.value.status == axp.AXP_E_INVAL
    s.close()
    G.close()


def test_injected_pulse_converts_like_the_closed_form():
    """Massless axion, 2D plane pulse entering through the plane on the TM kernel
    (FP64): the conversion probability grows as (g B0 l / 2)^2 with l the distance
    travelled since entry (the closed form of Sec. 3.2 at kappa = 0), with the
    Yee factor sec^2(theta/2) of the discrete energies."""
    axp = axp_mod()
    nx, ny = 1400, 16
    dt = 0.95 * DX / math.sqrt(2)
    bc = W._bcs("pml", "periodic")
    g_c, B0 = 1e-3, 1.0
    grid = W.GridSpec(n=(nx, ny, 1), d=(DX, DX, DX), dt=dt, m=0.0, g=g_c, B_ext=(0.0, 0.0, B0), axion_bc=bc,
                      em_bc=bc, pml_cells=20, precision="fp64")
    dur = 2.0
    tc = 3.5
    src = W.SourceSpec(amplitude=0.01, k=K0, pol=(0.0, 0.0, 1.0), plane=40, centre=(40 * DX, 0.0, 0.0),
                       duration=dur, t_centre=tc)
    g = axp.Grid(grid)
    g.set_soft_source(src)
    steps = int(round(30.0 / dt))
    g.step(steps)
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D
    d = g.diagnostics()
    t = steps * dt
    l = t - tc  # the pulse centre crossed the plane at t_centre
    w = 2 / dt * math.asin(dt / DX * math.sin(K0 * DX / 2))
    theta = w * dt
    want = (g_c * B0 * l / 2) ** 2 / math.cos(theta / 2) ** 2
    assert d["P_g2a"] == pytest.approx(want, rel=0.05)
    g.close()


def test_checkpoints_with_a_soft_source_are_taken_at_integer_time():
    """A grid with a soft source saves its integer-time state (its staggered E
    carries the sheet terms), which a grid with the same source resumes bit for
    bit; the staggered image of a grid without a source is refused by a grid
    that has one."""
    axp = axp_mod()
    grid = grid2d(160, 64, "fp64")
    src = beam(64)
    a = axp.Grid(grid)
    a.set_soft_source(src)
    a.step(20)
    img = a.save_state()
    a.step(15)
    ref = a.fields()
    b = axp.Grid(grid)
    b.set_soft_source(src)
    b.load_state(img)
    b.step(15)
    got = b.fields()
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), k
    plain = axp.Grid(grid)
    plain.step(5)
    staggered_img = plain.save_state()
    with pytest.raises(axp.AxpError) as e:
        b.load_state(staggered_img)
    assert e.value.status == axp.AXP_E_STATE
    for g in (a, b, plain):
        g.close()

"""Pins of the oracle's soft source: a laser entering through an x-plane as an
electric and a magnetic current sheet (Sec. 3.2 injects the laser into the
box; the sheets are the reading of that injection).

The pins do not restate the sheet terms.  They check what the sheets must
achieve: with a CW incident wave that is an exact discrete plane wave of the
Yee scheme (frequency from the Yee dispersion, pinned separately), a state
holding that wave on the +x side of the plane and nothing on the other side
stays exactly so; a pulse enters with the incident wave's shape and leaves
nothing behind the plane; a Gaussian beam stays mirror-symmetric about its
axis; a 2D run with a plane wave equals the 1D run row by row.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

DX = 1.0 / 32
DT = 0.95 * DX
K0 = 2 * math.pi


def yee_omega(k, dx, dt):
    """Yee dispersion of a wave along x: sin(w dt/2)/dt = sin(k dx/2)/dx."""
    return 2.0 / dt * math.asin(dt / dx * math.sin(k * dx / 2))


def line_grid(nx, pml=10, ny=1, ybc="periodic", d=(DX, DX, DX), dt=DT):
    bc = W._bcs(("pml", "pml"), ybc if ny > 1 else "periodic")
    return W.GridSpec(n=(nx, ny, 1), d=d, dt=dt, axion_bc=bc, em_bc=bc, pml_cells=pml)


def plane_wave_state(grid, src, t):
    """The incident CW wave at integer time t in the scheme's state variables on
    cells i >= plane (zero below): B on the faces x = (i+1) dx, and E^n = cos(w dt/2)
    times the incident E at the cell centres (E^n is E^{n+1/2} taken back half a
    step with the curl of B^n, which for the discrete plane wave is this factor)."""
    nx = grid.n[0]
    w = yee_omega(src.k, grid.d[0], grid.dt)
    xc = grid.lo[0] + (np.arange(nx) + 0.5) * grid.d[0]
    xf = grid.lo[0] + (np.arange(nx) + 1.0) * grid.d[0]
    psi_c = src.k * (xc - src.centre[0]) - w * (t - src.t_centre) + src.phase
    psi_f = src.k * (xf - src.centre[0]) - w * (t - src.t_centre) + src.phase
    tf = np.arange(nx) >= src.plane
    E = src.amplitude * math.cos(w * grid.dt / 2) * np.cos(psi_c) * tf
    B = src.amplitude * np.cos(psi_f) * tf
    shape = (grid.n[2], grid.n[1], nx)
    st = {k: np.zeros(shape) for k in W.FIELD_NAMES}
    py, pz = src.pol[1], src.pol[2]
    st["E0y"][...] = py * E
    st["E0z"][...] = pz * E
    st["B0z"][...] = py * B   # B_inc = xhat x E_inc: B_z = E_y, B_y = -E_z
    st["B0y"][...] = -pz * B
    return st


@pytest.mark.parametrize("pol", [(0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.0, 0.6, -0.8)])
def test_cw_plane_wave_is_kept_exactly(pol):
    """Total field / scattered field: the discrete plane wave on the +x side stays
    the discrete plane wave, and nothing appears on the -x side."""
    grid = line_grid(600)
    src = W.SourceSpec(amplitude=1e-3, k=K0, pol=pol, plane=100, centre=(1.3, 0, 0), t_centre=0.4, phase=0.3)
    og = oracle.OracleGrid(grid)
    og.load(plane_wave_state(grid, src, 0.0))
    og.set_soft_source(src)
    N = 100
    og.step(N)
    want = plane_wave_state(grid, src, N * grid.dt)
    got = og.fields()
    # cells the absorbing layer on the right cannot have reached (2 cells per step)
    hi = 600 - 10 - 2 * N - 5
    for name in ("E0y", "E0z", "B0y", "B0z"):
        a, b = got[name][0, 0], want[name][0, 0]
        assert np.max(np.abs(a[:100])) <= 1e-11 * src.amplitude, name   # behind the plane
        assert np.max(np.abs(a[100:hi] - b[100:hi])) <= 1e-11 * src.amplitude, name
    for name in ("E0x", "B0x", "E1x", "E1y", "E1z", "B1x", "B1y", "B1z"):
        assert not np.any(got[name]), name


def test_cw_wave_with_the_wrong_frequency_leaks():
    """Control for the test above: the same state with the continuum frequency
    (w = k) in place of the Yee one is not kept, so the pin is sensitive to the
    dispersion the sheets use."""
    grid = line_grid(600)
    src = W.SourceSpec(amplitude=1e-3, k=K0, pol=(0.0, 0.0, 1.0), plane=100)
    st = plane_wave_state(grid, src, 0.0)
    og = oracle.OracleGrid(grid)
    # a wave whose spatial period differs from what the sheets drive at the Yee frequency
    k_wrong = yee_omega(K0, DX, DT)
    og.load(plane_wave_state(grid, W.SourceSpec(amplitude=1e-3, k=k_wrong, pol=(0.0, 0.0, 1.0), plane=100), 0.0))
    og.set_soft_source(src)
    og.step(100)
    assert np.max(np.abs(og.fields()["E0z"][0, 0, :100])) > 1e-6 * src.amplitude
    assert np.any(st["E0z"])


def test_pulse_enters_with_the_incident_shape_and_leaves_nothing_behind():
    """A pulse switched on from nothing: after it has crossed the plane, the fields
    past the plane follow the incident wave (up to the envelope's small lag at the
    discrete group velocity) and the region behind the plane holds a negligible
    fraction of its energy."""
    grid = line_grid(1400)
    dur = 3.0
    src = W.SourceSpec(amplitude=1e-2, k=K0, pol=(0.0, 1.0, 0.0), plane=60, centre=(60 * DX, 0, 0),
                       duration=dur, t_centre=12.0, phase=0.2)
    og = oracle.OracleGrid(grid)
    og.set_soft_source(src)
    N = int(round(26.0 / DT))
    og.step(N)
    t = N * DT
    f = og.fields()
    w = yee_omega(K0, DX, DT)
    L = dur / math.sqrt(2 * math.log(2))
    xc = (np.arange(1400) + 0.5) * DX
    u = (t - src.t_centre) - (xc - src.centre[0])
    E_inc = src.amplitude * np.exp(-(u * u) / L**2) * np.cos(K0 * (xc - src.centre[0]) - w * (t - src.t_centre)
                                                             + src.phase)
    Ey = f["E0y"][0, 0]
    sl = slice(src.plane, 1400 - 10)
    err = np.linalg.norm(Ey[sl] - math.cos(w * DT / 2) * E_inc[sl]) / np.linalg.norm(E_inc[sl])
    assert err < 2e-2
    behind = np.sum(f["E0y"][0, 0, :src.plane] ** 2 + f["B0z"][0, 0, :src.plane] ** 2)
    ahead = np.sum(f["E0y"][0, 0] ** 2 + f["B0z"][0, 0] ** 2)
    assert behind < 1e-8 * ahead
    # the pulse energy matches the incident pulse's: 1/2 (E^2 + B^2) over the line,
    # with <cos^2> = 1/2, is A^2/2 int exp(-2 u^2/L^2) du = A^2 L sqrt(pi/2)/2 per unit
    # transverse area (the diagnostics integrate over the cells' dy dz as well)
    H = og.diagnostics()["H_g0"] / (DX * DX)
    want = src.amplitude**2 * L * math.sqrt(math.pi / 2) / 2
    assert H == pytest.approx(want, rel=2e-2)


def test_gaussian_beam_is_mirror_symmetric_about_its_axis():
    """2D beam centred on the box's mid-plane in y, periodic in y: E0z and B0y are
    mirror-symmetric and B0x antisymmetric, bit for bit.  (Absorbing y edges would
    break the symmetry: the layer's damping is taken per cell for every component,
    and the B_x faces of a cell are not the mirror images of each other.)"""
    ny = 48
    grid = line_grid(160, ny=ny, d=(DX, DX, DX), dt=0.95 * DX / math.sqrt(2))
    src = W.SourceSpec(amplitude=1e-2, k=K0, pol=(0.0, 0.0, 1.0), plane=20, centre=(0.0, ny * DX / 2, 0.0),
                       waist=0.4, duration=2.0, t_centre=4.0)
    og = oracle.OracleGrid(grid)
    og.set_soft_source(src)
    og.step(300)
    f = og.fields()
    Ez, Bx, By = f["E0z"][0], f["B0x"][0], f["B0y"][0]
    assert np.max(np.abs(Ez)) > 1e-3 * src.amplitude
    assert np.array_equal(Ez, Ez[::-1, :])
    assert np.array_equal(By, By[::-1, :])
    # B_x sits on the y faces (j+1) dy: its mirror image is face ny-2-j (mod ny), sign flipped
    assert np.array_equal(Bx, -Bx[(ny - 2 - np.arange(ny)) % ny, :])


def test_plane_wave_in_2d_equals_the_1d_run_row_by_row():
    nx, ny = 300, 6
    src = W.SourceSpec(amplitude=1e-2, k=K0, pol=(0.0, 0.6, 0.8), plane=30, duration=2.0, t_centre=3.0, phase=0.1)
    g1 = line_grid(nx)
    g2 = line_grid(nx, ny=ny)
    a, b = oracle.OracleGrid(g1), oracle.OracleGrid(g2)
    for og in (a, b):
        og.set_soft_source(src)
        og.step(200)
    fa, fb = a.fields(), b.fields()
    for name in W.FIELD_NAMES:
        for j in range(ny):
            assert np.array_equal(fb[name][0, j], fa[name][0, 0]), name


def test_invalid_sources_are_refused():
    og = oracle.OracleGrid(line_grid(100))
    for bad in (dict(plane=0), dict(plane=100), dict(pol=(1.0, 0.0, 0.0)), dict(k=0.0)):
        kw = dict(amplitude=1.0, k=K0, pol=(0.0, 1.0, 0.0), plane=10)
        kw.update(bad)
        with pytest.raises(ValueError):
            og.set_soft_source(W.SourceSpec(**kw))

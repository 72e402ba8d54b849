"""Perturbed-particle current (Sec. 2.2) on the GPU against the oracle.

Fields, particle states and currents after coupled runs of fields and
macroparticles, through the C ABI, element by element.  The particle push is
the same arithmetic in the same order on both sides; the currents are summed
with atomic adds on the GPU, so they (and the fields they drive) agree to
rounding, not bit for bit: the bound is 1e-12 of each quantity's scale."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_16796_gb300 import workloads as W
from paper_2406_16796_gb300.workloads import GridSpec

pytestmark = pytest.mark.gpu

TOL = 1e-12


def close(a, b, tol=TOL):
    scale = max(np.max(np.abs(b)), 1e-300)
    err = np.max(np.abs(a - b))
    assert err <= tol * scale, (err, scale)


def wrapped_close(a, b, L, tol=1e-12):
    d = (a - b + L / 2) % L - L / 2
    assert np.max(np.abs(d)) <= tol * L, np.max(np.abs(d))


def run_pair(grid, plasma, fields, steps, laser=None):
    from paper_2406_16796_gb300 import axp

    og = O.OracleGrid(grid)
    g = axp.Grid(grid)
    if laser is not None:
        og.inject_laser(laser)
        g.inject_laser(laser)
    og.load(fields)
    g.load(fields)
    og.attach_particles(plasma.q, plasma.m, plasma.w, plasma.x0, plasma.u0, plasma.x1, plasma.u1)
    g.attach_particles(plasma.q, plasma.m, plasma.w, plasma.x0, plasma.u0, plasma.x1, plasma.u1)
    og.step(steps)
    g.step(steps)
    return og, g


def compare(og, g, grid):
    from paper_2406_16796_gb300 import axp

    got = g.fields()
    for k, v in og.fields().items():
        close(got[k], v)
    st = og.particles_now()
    gp = g.read_particles()
    for a in range(3):
        if grid.n[a] > 1:
            wrapped_close(gp["x0"][a], st["x0"][a], grid.n[a] * grid.d[a])
        close(gp["x1"][a], st["x1"][a])
        close(gp["u0"][a], st["u0"][a])
        close(gp["u1"][a], st["u1"][a])
    close(g.particle_current(0), st["j0"])
    close(g.particle_current(1), st["j1"])
    assert g.kernel_path() == axp.AXP_KERNEL_GENERAL


CASES = {
    # 1D: laser (order 0) through a warm magnetised plasma, axion coupling on
    "1d_warm": dict(n=(64, 1, 1), ppc=5, B=(0.0, 0.4, 0.9), g=0.05, m=0.3, steps=25),
    # 2D with a ragged cell count, a perturbed plasma and random first-order fields
    "2d_ragged": dict(n=(37, 19, 1), ppc=3, B=(0.2, 0.0, 0.7), g=0.0, m=0.0, steps=12),
    # 3D, small
    "3d": dict(n=(9, 8, 7), ppc=2, B=(0.3, 0.5, 0.6), g=0.02, m=0.0, steps=6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_coupled_run_matches_the_oracle(name):
    c = CASES[name]
    d = 0.125
    n = c["n"]
    ndim = sum(1 for x in n if x > 1)
    dt = 0.9 * d / math.sqrt(ndim)
    grid = GridSpec(n=n, d=(d, d, d), dt=dt, m=c["m"], g=c["g"], B_ext=c["B"])
    plasma = W.plasma_particles(grid, c["ppc"], density=2.0, seed=W.SEED_BASE + 40 + len(name), u0_spread=0.3,
                                x1_spread=0.01, u1_spread=0.05)
    rs = W.random_state(grid, seed=W.SEED_BASE + 50 + len(name), scale0=0.2, scale1=0.01, scale_phi=0.01)
    fields = {k: v for k, v in rs.items()}
    og, g = run_pair(grid, plasma, fields, c["steps"])
    compare(og, g, grid)
    g.close()


def test_positions_round_trip_and_edge_particles():
    """Positions written at t_n read back at t_n; particles exactly on nodes, on
    the periodic seam and at the top edge of the box take valid nodes."""
    from paper_2406_16796_gb300 import axp

    grid = GridSpec(n=(16, 6, 1), d=(0.25, 0.25, 0.25), dt=0.1, B_ext=(0.0, 0.0, 0.5))
    Lx, Ly = 4.0, 1.5
    x = np.array([0.0, 0.25, 0.125, Lx - 1e-15, Lx - 0.25, 2.0, 3.999999, 1.0])
    y = np.array([0.0, 0.125, Ly - 1e-15, 0.75, 0.0, 1.25, 0.3, 1.4999])
    n = x.size
    X = np.zeros((3, n))
    X[0], X[1] = x, y
    U = np.zeros((3, n))
    U[0] = 0.5
    U[1] = -0.3
    w = np.full(n, 0.1)
    plasma = W.PlasmaSpec(-1.0, 1.0, w, X, U, np.zeros((3, n)), np.full((3, n), 0.01))
    g = axp.Grid(grid)
    g.attach_particles(plasma.q, plasma.m, plasma.w, plasma.x0, plasma.u0, plasma.x1, plasma.u1)
    r = g.read_particles()
    wrapped_close(r["x0"][0], x, Lx, 1e-15)
    wrapped_close(r["x0"][1], y, Ly, 1e-15)
    og, g2 = run_pair(grid, plasma, {}, 7)
    compare(og, g2, grid)
    g.close()
    g2.close()


def test_empty_particle_set_leaves_the_fields_alone():
    """Zero particles: the run equals the run without particles bit for bit
    (general path both)."""
    from paper_2406_16796_gb300 import axp

    grid = GridSpec(n=(32, 8, 1), d=(0.125,) * 3, dt=0.08, g=0.01, B_ext=(0.0, 0.0, 1.0))
    rs = W.random_state(grid, seed=W.SEED_BASE + 61)
    a = axp.Grid(grid)
    b = axp.Grid(grid)
    a.load(rs)
    b.load(rs)
    b.set_kernel(axp.AXP_KERNEL_GENERAL)
    a.attach_particles(-1.0, 1.0, np.zeros(0), np.zeros((3, 0)), np.zeros((3, 0)))
    a.step(5)
    b.step(5)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()


def test_refusals_and_detach():
    from paper_2406_16796_gb300 import axp

    # FP32 grid and absorbing axis: refused
    g32 = axp.Grid(GridSpec(n=(16, 1, 1), d=(0.25,) * 3, dt=0.1, precision="fp32"))
    with pytest.raises(axp.AxpError) as e:
        g32.attach_particles(-1.0, 1.0, np.ones(1), np.zeros((3, 1)), np.zeros((3, 1)))
    assert e.value.status == axp.AXP_E_INVAL
    g32.close()
    pml = W._bcs("pml")
    gp = axp.Grid(GridSpec(n=(64, 1, 1), d=(0.25,) * 3, dt=0.1, pml_cells=8, em_bc=pml, axion_bc=pml))
    with pytest.raises(axp.AxpError) as e:
        gp.attach_particles(-1.0, 1.0, np.ones(1), np.zeros((3, 1)), np.zeros((3, 1)))
    assert e.value.status == axp.AXP_E_INVAL
    gp.close()
    grid = GridSpec(n=(16, 1, 1), d=(0.25,) * 3, dt=0.1)
    g = axp.Grid(grid)
    X = np.zeros((3, 2))
    g.attach_particles(-1.0, 1.0, np.ones(2), X, np.zeros((3, 2)))
    # non-finite input refused, state kept
    rows = np.zeros((13, 2))
    rows[4, 1] = np.nan
    with pytest.raises(axp.AxpError) as e:
        g.write_particles(rows)
    assert e.value.status == axp.AXP_E_NONFINITE
    # a forced single-pass kernel cannot step particles
    g.set_kernel(axp.AXP_KERNEL_BLOCK1D)
    with pytest.raises(axp.AxpError) as e:
        g.step(1)
    assert e.value.status == axp.AXP_E_STATE
    g.set_kernel(axp.AXP_KERNEL_AUTO)
    g.step(2)
    g.detach_particles()
    g.step(2)
    assert g.step_count == 4
    g.close()


def test_cold_plasma_oscillation_on_the_gpu():
    """k = 0 cold-plasma response through the C ABI: the one-step map of
    (u1x, E1x) has determinant 1 and trace 2 - (w_p dt)^2."""
    from paper_2406_16796_gb300 import axp

    grid = GridSpec(n=(8, 1, 1), d=(0.5,) * 3, dt=0.2)
    ppc, density = 4, 3.0
    n = grid.n[0] * ppc
    X = np.zeros((3, n))
    X[0] = (np.arange(n) + 0.5) * grid.d[0] / ppc
    w = np.full(n, density * grid.d[0] ** 3 / ppc)
    M = np.zeros((2, 2))
    for col in range(2):
        g = axp.Grid(grid)
        U1 = np.zeros((3, n))
        if col == 0:
            U1[0] = 1.0
        else:
            g.write("E1x", np.ones((1, 1, 8)))
        g.attach_particles(-1.0, 1.0, w, X, np.zeros((3, n)), None, U1)
        g.step(1)
        M[0, col] = g.read_particles()["u1"][0].mean()
        M[1, col] = g.read("E1x").mean()
        g.close()
    assert abs(np.linalg.det(M) - 1.0) < 1e-13
    assert abs(np.trace(M) - (2.0 - density * grid.dt ** 2)) < 1e-13


def test_magnetised_plasma_full_size_matches_the_oracle():
    """The weak laser in a magnetised plasma at its full size (12000 x 100 cells,
    4 particles per cell, the bench's launch): two coupled steps against the
    oracle, all fields, and particle states on a sample."""
    from paper_2406_16796_gb300 import axp

    grid, plasma, fields = W.magnetised_plasma_2d()
    og, g = run_pair(grid, plasma, fields, 2)
    got = g.fields()
    for k, v in og.fields().items():
        close(got[k], v)
    st = og.particles_now()
    gp = g.read_particles()
    rng = np.random.default_rng(7)
    idx = rng.choice(plasma.count, 20000, replace=False)
    for a in range(2):
        wrapped_close(gp["x0"][a][idx], st["x0"][a][idx], grid.n[a] * grid.d[a])
    for k in ("u0", "u1", "x1"):
        close(gp[k][:, idx], st[k][:, idx])
    # the first-order laser drove a first-order current in the plasma
    assert np.max(np.abs(st["j1"])) > 0 and np.max(np.abs(got["E1y"])) > 0
    g.close()

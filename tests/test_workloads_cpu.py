"""The seeded synthetic inputs against the configurations they stand in for: the
1D CW run, the 2D pulse, the 3D axion box, the 512-instance parameter scan and
the serving stream (sizes, cell sizes and time steps, boundary conditions,
parameter distributions, stability of every draw, determinism of the seeds)."""
import math

import numpy as np

from paper_2406_16796_gb300 import workloads as W


def test_grid_workloads_have_the_stated_sizes_steps_and_boundaries():
    v = W.vacuum_1d()
    assert v.grid.n == (4096, 1, 1) and v.grid.d[0] == 1 / 32 and v.steps == 20000
    assert math.isclose(v.grid.dt, 0.95 / 32, rel_tol=1e-15) and v.grid.B_ext == (0.0, 1.0, 0.0)
    assert v.grid.em_bc[0] == ("periodic", "periodic") and v.grid.g == 1e-4 and v.grid.m == 0.0
    p = W.pulse_2d()
    assert p.grid.n == (4096, 2048, 1) and p.grid.d[:2] == (1 / 32, 1 / 32) and p.steps == 16000
    assert math.isclose(p.grid.dt, 0.95 / 32 / math.sqrt(2), rel_tol=1e-15) and p.grid.B_ext == (0.0, 0.0, 1.0)
    assert p.grid.em_bc[:2] == (("pml", "pml"), ("pml", "pml")) and p.grid.pml_cells == 20
    L = p.lasers[0]
    assert L.amplitude == 0.01 and L.pol == (0.0, 0.0, 1.0) and L.waist == 4.0 and L.duration == 8.0
    assert L.centre[0] == 16.0 and L.k == (W.K0, 0.0, 0.0)
    a = W.axion_3d()
    assert a.grid.n == (512, 512, 512) and a.grid.d == (1 / 16,) * 3 and a.steps == 2000
    assert math.isclose(a.grid.dt, 0.95 / 16 / math.sqrt(3), rel_tol=1e-15) and a.grid.B_ext == (0.0, 1.0, 0.0)
    assert a.grid.precision == "fp32" and a.axions[0].amplitude == 1e-2
    # 32 whole wavelengths across the box
    assert math.isclose(a.axions[0].k[0] * 512 / 16, 2 * math.pi * 32, rel_tol=1e-14)


def test_every_grid_workload_is_within_the_stability_bounds():
    for w in (W.vacuum_1d(), W.pulse_2d(), W.axion_3d(), W.pulse_2d(m=math.pi)):
        g = w.grid
        inv2 = sum(1.0 / g.d[a] ** 2 for a in range(3) if g.n[a] > 1)
        assert g.dt * math.sqrt(inv2) <= 1.0  # Yee CFL
        assert g.dt ** 2 * (4.0 * inv2 + g.m ** 2) <= 4.0  # axion leapfrog


def test_scan_draws_follow_their_distributions_and_are_stable():
    s = W.scan_instances()
    assert len(s) == 512 and s == W.scan_instances()  # seeded: the same draws every time
    nx = np.array([i.nx for i in s])
    steps = np.array([i.steps for i in s])
    m = np.array([i.m for i in s]) / W.K0
    g = np.array([i.g for i in s])
    B0 = np.array([i.B0 for i in s])
    assert nx.min() >= 1024 and nx.max() <= 65536 and steps.min() >= 5000 and steps.max() <= 40000
    assert m.min() >= 1e-3 and m.max() <= 2.0 and g.min() >= 1e-6 and g.max() <= 1e-3
    assert B0.min() >= 0.1 and B0.max() <= 10.0
    # log-uniform draws: their logs spread evenly (mean at the centre of the log range)
    for x, lo, hi in ((nx, 1024, 65536), (m, 1e-3, 2.0), (g, 1e-6, 1e-3), (B0, 0.1, 10.0)):
        centre = 0.5 * (math.log(lo) + math.log(hi))
        assert abs(np.mean(np.log(x)) - centre) < 0.1 * (math.log(hi) - math.log(lo))
    # the scan's size: about 7.9 M cells and 1.7e11 cell-updates in all
    assert 6e6 < nx.sum() < 1e7 and 1.4e11 < np.sum(nx * steps) < 2.2e11
    dt = 0.95 / 32
    assert np.all((m * W.K0 * dt) ** 2 + 0.95 ** 2 * 4 < 4.0)


def test_serving_stream_mix_and_arrivals():
    r = W.serve_requests()
    assert len(r) == 10000 and [x.arrival for x in r[:50]] == [x.arrival for x in W.serve_requests(count=50)]
    one = [x for x in r if x.ndim == 1]
    two = [x for x in r if x.ndim == 2]
    assert abs(len(one) / len(r) - 0.8) < 0.02
    assert all(256 <= x.n[0] <= 2048 and x.n[0] % 2 == 0 and x.n[1] == x.n[0] // 2 for x in two)
    assert all(1024 <= x.n[0] <= 65536 and x.n[1:] == (1, 1) for x in one)
    gaps = np.diff([0.0] + [x.arrival for x in r])
    assert np.all(gaps > 0) and abs(np.mean(gaps) - 1 / 100.0) < 0.05 / 100.0  # Poisson at 100 per second


def test_magnetised_plasma_has_the_papers_parameters():
    """Sec. 3.4: a 40 x 100 wavelength box on 12000 x 100 cells, n0 = 3e-3 n_c,
    B_ext = m w_p/|q| along z, laser B amplitude 1e-20 B_ext in the first-order
    fields; 4 particles per cell inside their own cells; seeded."""
    import json
    import os

    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
    ref = golden["magnetised_plasma"]
    grid, plasma, fields = W.magnetised_plasma_2d()
    assert grid.n[:2] == tuple(ref["cells"]) and grid.n[2] == 1
    bx, by = ref["box_lambda"]["x"], ref["box_lambda"]["y"]
    assert math.isclose(grid.lo[0], bx[0]) and math.isclose(grid.lo[1], by[0])
    assert math.isclose(grid.n[0] * grid.d[0], bx[1] - bx[0], rel_tol=1e-14)
    assert math.isclose(grid.n[1] * grid.d[1], by[1] - by[0], rel_tol=1e-14)
    inv2 = 1.0 / grid.d[0] ** 2 + 1.0 / grid.d[1] ** 2
    assert grid.dt * math.sqrt(inv2) <= 0.95 + 1e-12
    nc = plasma.m * W.K0 ** 2 / plasma.q ** 2
    dV = grid.d[0] * grid.d[1] * grid.d[2]
    density = plasma.w.sum() / (grid.cells * dV)
    assert math.isclose(density / nc, ref["n0_over_nc"], rel_tol=1e-12)
    wp = math.sqrt(density * plasma.q ** 2 / plasma.m)
    assert grid.B_ext[:2] == (0.0, 0.0) and math.isclose(grid.B_ext[2], plasma.m * wp / abs(plasma.q), rel_tol=1e-12)
    assert plasma.q == -1.0 and plasma.count == 4 * grid.cells
    assert np.all(plasma.u0 == 0) and np.all(plasma.u1 == 0) and np.all(plasma.x1 == 0)
    # every particle lies inside the cell it was drawn for
    cell = np.repeat(np.arange(grid.cells), 4)
    ix = np.floor((plasma.x0[0] - grid.lo[0]) / grid.d[0]).astype(np.int64)
    iy = np.floor((plasma.x0[1] - grid.lo[1]) / grid.d[1]).astype(np.int64)
    assert np.array_equal(ix, cell % grid.n[0]) and np.array_equal(iy, cell // grid.n[0])
    # the laser is first order, at 1e-20 of the background field
    Bz = fields["B1z"]
    assert set(fields) == {"E1y", "B1z"}
    ratio = ref["laser_B_over_B_ext"]
    assert 0.9 * ratio < np.max(np.abs(Bz)) / grid.B_ext[2] <= ratio
    # seeded
    _, again, _ = W.magnetised_plasma_2d()
    assert np.array_equal(again.x0, plasma.x0)

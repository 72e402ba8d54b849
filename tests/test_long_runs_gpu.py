"""The CUDA path against the oracle over the workloads' own run lengths, and
the conversion and centroid diagnostics against the oracle on the GPU.

* 1D conversion run (Nx = 4096, dx = lambda/32, CFL 0.95, g = 1e-4, B0 = 1):
  all 20000 steps, FP64 fields <= 1e-12 and P <= 1e-12 against the oracle, P
  against the closed form (g B0 t / 2)^2 sec^2(th/2) of Sec. 3.2; FP32 split
  P <= 1e-3.
* 3D axion box (dx = lambda/16, CFL 0.95, axion plane wave 1e-2 along x, B_ext
  along y, periodic): all 2000 steps on a 32^3 box (two wavelengths per axis,
  with a weak oblique second wave so that every axis varies), FP32 split on
  the 3D axion-box kernel against the FP64 oracle: order-1 fields (as a group)
  and phi <= 1e-4, P_a2g <= 1e-3.
* 2D pulse (dx = lambda/32, CFL 0.95/sqrt(2), E_z Gaussian pulse, B_ext along z,
  PML along y): 4000 steps on 320 x 160 cells, periodic along x so that the
  pulse stays in the box for the whole run, m in {0, pi}, FP32 split on the 2D
  kernel against the FP64 oracle: P_g2a <= 1e-3.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur"]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rel_group(got, ref, names):
    """Normwise relative error of a group of fields taken together (a component
    that is zero in exact arithmetic holds only rounding noise of each side, so
    it is measured against its group)."""
    num = math.sqrt(sum(np.linalg.norm(got[k] - ref[k]) ** 2 for k in names))
    den = math.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in names))
    return num / den


def yee_theta(k, d, dt):
    """th = w dt of the Yee (and massless Klein-Gordon) dispersion
    sin(w dt/2)/dt = sqrt(sum_d sin^2(k_d d_d/2)/d_d^2)."""
    s = math.sqrt(sum((math.sin(k[a] * d[a] / 2.0) / d[a]) ** 2 for a in range(3)))
    return 2.0 * math.asin(dt * s)


def test_1d_conversion_full_run_matches_oracle_and_closed_form():
    """All 20000 steps.  The fields are compared from the same initial bits (the
    oracle's injected laser loaded into the grid): the run is sensitive enough
    that the last-bit differences of the two sides' injections (checked to 1e-13
    on their own) grow to about 1e-12 over it.  P is also compared for the
    grid's own injection."""
    from paper_2406_16796_gb300 import axp

    w = W.vacuum_1d(nx=4096)
    assert w.steps == 20000
    og = oracle.OracleGrid(w.grid)
    og.inject_laser(w.lasers[0])
    start = og.fields()
    og.step(w.steps)
    ref = og.fields()
    dr = og.diagnostics()
    th = yee_theta(w.lasers[0].k, w.grid.d, w.grid.dt)
    closed = (w.grid.g * w.grid.B_ext[1] * dr["t"] / 2.0) ** 2 / math.cos(th / 2.0) ** 2
    assert dr["t"] == pytest.approx(593.75)
    assert abs(dr["P_g2a"] / closed - 1.0) < 5e-3
    for prec in ("fp64", "fp32"):
        for own_injection in (False, True):
            g = axp.Grid(w.grid.replace(precision=prec))
            if own_injection:
                g.inject_laser(w.lasers[0])
            else:
                g.load(start)
            # FP64: the time-blocked 1D kernel
            assert g.kernel_path() == (axp.AXP_KERNEL_BLOCK1D if prec == "fp64" else axp.AXP_KERNEL_FUSED)
            g.step(w.steps)
            d = g.diagnostics()
            assert d["step"] == 20000
            if prec == "fp64" and not own_injection:
                got = g.fields()
                for k in ("E0y", "B0z", "E1y", "E1z", "B1y", "B1z", "phi_cur", "phi_old"):
                    assert rel(got[k], ref[k]) < 1e-12, (k, rel(got[k], ref[k]))
                # and the one-launch-per-step single-pass kernel over the same run
                f = axp.Grid(w.grid)
                f.set_kernel(axp.AXP_KERNEL_FUSED)
                f.load(start)
                f.step(w.steps)
                gotf = f.fields()
                f.close()
                # (its differently ordered roundings drift to 1.3e-12 over the 20000 steps)
                for k in ("E0y", "B0z", "E1y", "E1z", "B1y", "B1z", "phi_cur", "phi_old"):
                    assert rel(gotf[k], ref[k]) < 2e-12, ("fused", k, rel(gotf[k], ref[k]))
            tolP = 1e-10 if prec == "fp64" else 1e-3
            assert abs(d["P_g2a"] / dr["P_g2a"] - 1.0) < tolP, (prec, own_injection, d["P_g2a"], dr["P_g2a"])
            assert abs(d["P_g2a"] / closed - 1.0) < 5e-3
            g.close()


def axion_box_32():
    w = W.axion_3d(n=32)
    assert w.grid.d[0] == 1 / 16 and w.axions[0].k == (2 * math.pi, 0.0, 0.0)
    oblique = W.AxionSpec(amplitude=1e-3, k=(math.pi, 2 * math.pi, math.pi), phase=0.3)
    return w, (w.axions[0], oblique)


def test_3d_axion_box_full_run_fp32_matches_oracle():
    from paper_2406_16796_gb300 import axp

    w, axions = axion_box_32()
    assert w.steps == 2000
    og = oracle.OracleGrid(w.grid.replace(precision="fp64"))
    for a in axions:
        og.inject_axion(a)
    og.step(w.steps)
    ref, dr = og.fields(), og.diagnostics()
    g = axp.Grid(w.grid.replace(precision="fp32"))
    for a in axions:
        g.inject_axion(a)
    assert g.kernel_path() == axp.AXP_KERNEL_AX3D
    g.step(w.steps)
    got, d = g.fields(), g.diagnostics()
    g.close()
    order1 = ("E1x", "E1y", "E1z", "B1x", "B1y", "B1z")
    assert rel_group(got, ref, order1) < 1e-4, rel_group(got, ref, order1)
    assert rel(got["phi_cur"], ref["phi_cur"]) < 1e-4, rel(got["phi_cur"], ref["phi_cur"])
    assert abs(d["P_a2g"] / dr["P_a2g"] - 1.0) < 1e-3, (d["P_a2g"], dr["P_a2g"])
    assert dr["P_a2g"] > 0


@pytest.mark.parametrize("m", [0.0, math.pi])
def test_2d_pulse_long_run_fp32_matches_oracle(m):
    from paper_2406_16796_gb300 import axp

    w = W.pulse_2d(nx=320, ny=160, m=m)
    grid = w.grid.replace(axion_bc=W._bcs("periodic", "pml"), em_bc=W._bcs("periodic", "pml"))
    og = oracle.OracleGrid(grid)
    og.inject_laser(w.lasers[0])
    g = axp.Grid(grid.replace(precision="fp32"), diag_every=1000, diag_capacity=8)
    g.inject_laser(w.lasers[0])
    assert g.kernel_path() == axp.AXP_KERNEL_TM2D
    refs = []
    for _ in range(4):
        og.step(1000)
        refs.append(og.diagnostics())
    g.step(4000)
    recs = g.read_diagnostics()
    assert [r["step"] for r in recs] == [1000, 2000, 3000, 4000]
    for r, dr in zip(recs, refs):
        assert dr["P_g2a"] > 0
        assert abs(r["P_g2a"] / dr["P_g2a"] - 1.0) < 1e-3, (r["step"], r["P_g2a"], dr["P_g2a"])
    got, ref = g.fields(), og.fields()
    g.close()
    for k in ("E0z", "B0x", "B0y", "E1z", "phi_cur"):
        assert rel(got[k], ref[k]) < 1e-3, (k, rel(got[k], ref[k]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_axion_to_photon_ratio_on_the_gpu(prec):
    """A massless axion plane wave converting to photons in a 16 x 2 x 2 periodic
    box (the 3D axion-box set-up, dx = lambda/16): P_a2g = H_g1/H_phi against
    the oracle and the closed form (g B t/2)^2 sec^2(th/2)."""
    from paper_2406_16796_gb300 import axp

    d = (1 / 16,) * 3
    grid = W.GridSpec(n=(16, 2, 2), d=d, dt=0.95 * d[0] / math.sqrt(3), g=1e-4, B_ext=(0.0, 1.0, 0.0))
    A = W.AxionSpec(amplitude=1e-2, k=(W.K0, 0.0, 0.0))
    og = oracle.OracleGrid(grid)
    og.inject_axion(A)
    g = axp.Grid(grid.replace(precision=prec))
    g.inject_axion(A)
    assert g.kernel_path() == axp.AXP_KERNEL_AX3D
    th = yee_theta(A.k, d, grid.dt)
    for _ in range(3):
        og.step(1000)
        g.step(1000)
        dg, dr = g.diagnostics(), og.diagnostics()
        tol = 1e-10 if prec == "fp64" else 1e-3
        for key in ("P_a2g", "H_g1", "H_phi"):
            assert abs(dg[key] / dr[key] - 1.0) < tol, (key, dg[key], dr[key])
        closed = (grid.g * dg["t"] / 2.0) ** 2 / math.cos(th / 2.0) ** 2
        assert abs(dg["P_a2g"] / closed - 1.0) < 1e-3
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_b1z_centroid_on_the_gpu(prec):
    """A weak order-1 packet moving at the Yee group velocity (8 cells per
    wavelength, CFL 0.5, v_g = 0.941): the GPU's B1z^2-weighted centroid
    against the oracle's and the group velocity, on a grid whose lower corner
    is not at the origin."""
    from paper_2406_16796_gb300 import axp

    dx = 1 / 8
    grid = W.GridSpec(n=(640, 1, 1), d=(dx,) * 3, dt=0.5 * dx, lo=(-7.25, 0.0, 0.0), g=1e-3,
                      B_ext=(0.0, 1.0, 0.0))
    x0 = grid.lo[0] + 160 * dx
    n = grid.n[0]
    xf = grid.lo[0] + (np.arange(n) + 1.0) * dx
    B = 1e-3 * np.exp(-((xf - x0) ** 2) / 32.0) * np.cos(W.K0 * (xf - x0))
    k = 2 * np.pi * np.fft.fftfreq(n, d=dx)
    thk = 2 * np.arcsin(grid.dt / dx * np.abs(np.sin(k * dx / 2)))
    E = np.fft.ifft(np.fft.fft(B) * np.cos(thk / 2) * np.exp(-1j * k * dx / 2)).real
    st = {name: np.zeros((1, 1, n)) for name in list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]}
    st["B1z"], st["E1y"] = B.reshape(1, 1, n), E.reshape(1, 1, n)
    og = oracle.OracleGrid(grid)
    og.load(st)
    g = axp.Grid(grid.replace(precision=prec))
    g.load(st)
    th = yee_theta((W.K0, 0, 0), grid.d, grid.dt)
    vg = math.cos(W.K0 * dx / 2) / math.cos(th / 2)
    for _ in range(3):
        og.step(240)
        g.step(240)
        dg, dr = g.diagnostics(), og.diagnostics()
        X, Xr = dg["sum_xB1z2"] / dg["sum_B1z2"], dr["sum_xB1z2"] / dr["sum_B1z2"]
        assert abs(X - Xr) < (1e-10 if prec == "fp64" else 1e-4) * dx, (X, Xr)
        assert abs((X - x0) / (vg * dg["t"]) - 1.0) < 1e-3
    g.close()

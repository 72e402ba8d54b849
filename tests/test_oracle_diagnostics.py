"""The oracle's diagnostics (Sec. 3.2-3.4 energies and ratios, Sec. 2.2 cross
energy, the Gauss residual) against an independent vectorised transcription of
their definitions, on random states of periodic and absorbing-layer grids.

Definitions (the energy reading the oracle follows): at integer time n,
D_t phi = (phi^{n+1/2} - phi^{n-1/2}) / dt and phi^n is the mean of the two
levels; |grad phi|^2 sums the squared forward differences of phi^n per axis;
H_phi = 1/2 sum [(D_t phi)^2 + |grad phi|^2 + m^2 (phi^n)^2] dV,
H_g0 = 1/2 sum (E0^2 + B0^2) dV (laser fields only), H_g1 = 1/2 sum (E1^2 + B1^2) dV,
W = H_phi + sum [(E0 + E_ext) . E1 + (B0 + B_ext) . B1] dV, the B1z-weighted
centroid sums x B1z^2 dV at B1z's x-position, and the Gauss residual
R = div E1 + g Bbar0 . grad_c phi^n at the cell centres, summed as R^2 dV.  Sums
run over the cells outside the absorbing layers."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

AX = {0: 2, 1: 1, 2: 0}  # array dimension of each grid axis (arrays are (nz, ny, nx))


def shift(F, a, s):
    """F at index + s along grid axis a (periodic wrap; wrapped values are used
    only outside the summed region of an absorbing axis)."""
    return np.roll(F, -s, axis=AX[a])


def transcribed(grid, st):
    d, dt, m, g = grid.d, grid.dt, grid.m, grid.g
    dV = d[0] * d[1] * d[2]
    cur, old = st["phi_cur"], st["phi_old"]
    Dt = (cur - old) / dt
    ph = 0.5 * (cur + old)
    g2 = sum(((shift(ph, a, 1) - ph) / d[a]) ** 2 for a in range(3))
    E0 = [st["E0" + c] for c in "xyz"]
    B0 = [st["B0" + c] for c in "xyz"]
    E1 = [st["E1" + c] for c in "xyz"]
    B1 = [st["B1" + c] for c in "xyz"]
    # the summed region: every cell but those of the absorbing layers
    mask = np.ones(cur.shape, dtype=bool)
    for a in range(3):
        if grid.n[a] == 1 or grid.em_bc[a][0] == "periodic":
            continue
        L = grid.pml_cells
        idx = np.arange(grid.n[a])
        keep = np.ones(grid.n[a], dtype=bool)
        if "pml" in (grid.em_bc[a][0], grid.axion_bc[a][0]):
            keep &= idx >= L
        if "pml" in (grid.em_bc[a][1], grid.axion_bc[a][1]):
            keep &= idx < grid.n[a] - L
        shape = [1, 1, 1]
        shape[AX[a]] = grid.n[a]
        mask &= keep.reshape(shape)
    Hphi = 0.5 * np.sum(((Dt * Dt + g2) + m * m * ph * ph)[mask]) * dV
    Hg0 = 0.5 * np.sum(sum(E0[a] ** 2 + B0[a] ** 2 for a in range(3))[mask]) * dV
    Hg1 = 0.5 * np.sum(sum(E1[a] ** 2 + B1[a] ** 2 for a in range(3))[mask]) * dV
    X = np.sum(sum((E0[a] + grid.E_ext[a]) * E1[a] + (B0[a] + grid.B_ext[a]) * B1[a] for a in range(3))[mask]) * dV
    # B1z sits at (i + 1/2, j + 1/2) of cell (i, j): x = lo + (i + 1) dx
    xb = grid.lo[0] + (np.arange(grid.n[0]) + 1.0) * d[0]
    bz2 = B1[2] ** 2 * dV
    sxb = np.sum((xb.reshape(1, 1, -1) * bz2)[mask])
    sb = np.sum(bz2[mask])
    # Gauss residual: backward-difference divergence of E1 at the centre, plus g Bbar0 . grad_c phi
    div = sum((E1[a] - shift(E1[a], a, -1)) / d[a] for a in range(3))
    bbar = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        F = B0[a]
        bbar.append(0.25 * (F + shift(F, c, -1) + shift(F, b, -1) + shift(shift(F, b, -1), c, -1)) + grid.B_ext[a])
    grad = [(shift(ph, a, 1) - shift(ph, a, -1)) / (2 * d[a]) for a in range(3)]
    R = div + g * sum(bbar[a] * grad[a] for a in range(3))
    gl2 = np.sum((R * R)[mask]) * dV
    return {"H_phi": Hphi, "H_g0": Hg0, "H_g1": Hg1, "P_g2a": Hphi / Hg0, "P_a2g": Hg1 / Hphi, "W": Hphi + X,
            "sum_xB1z2": sxb, "sum_B1z2": sb, "gauss_l2": gl2}


@pytest.mark.parametrize("n,sides", [((12, 10, 1), ("periodic", "periodic", "periodic")),
                                     ((9, 8, 7), ("periodic", "periodic", "periodic")),
                                     ((14, 12, 1), ("pml", "pml", "periodic")),
                                     ((11, 9, 10), ("pml", "periodic", "pml"))])
def test_diagnostics_match_their_definitions(n, sides):
    d = (0.05, 0.07, 0.06)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    bc = W._bcs(*sides)
    grid = W.GridSpec(n=n, d=d, dt=dt, lo=(-0.3, 0.1, 0.0), m=1.1, g=0.7, B_ext=(0.3, -0.5, 0.7),
                      E_ext=(0.05, 0.02, -0.1), axion_bc=bc, em_bc=bc, pml_cells=3)
    st = W.random_state(grid, seed=2121, scale1=0.3)
    og = oracle.OracleGrid(grid)
    og.load(st)
    got = og.diagnostics()
    want = transcribed(grid, st)
    for key, v in want.items():
        assert got[key] == pytest.approx(v, rel=1e-12), (key, got[key], v)


def test_the_region_leaves_out_the_layers():
    """Control: on the absorbing-layer grid, the same sums over every cell differ."""
    n, sides = (14, 12, 1), ("pml", "pml", "periodic")
    d = (0.05, 0.07, 0.06)
    dt = 0.5 / math.sqrt(1 / d[0] ** 2 + 1 / d[1] ** 2)
    bc = W._bcs(*sides)
    grid = W.GridSpec(n=n, d=d, dt=dt, m=1.1, g=0.7, axion_bc=bc, em_bc=bc, pml_cells=3)
    st = W.random_state(grid, seed=2122)
    og = oracle.OracleGrid(grid)
    og.load(st)
    periodic = grid.replace(axion_bc=W._bcs(), em_bc=W._bcs())
    whole = transcribed(periodic, st)
    assert og.diagnostics()["H_g0"] < 0.9 * whole["H_g0"]

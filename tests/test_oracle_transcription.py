"""A second, independent transcription of one time step (arXiv 2406.16796,
Sec. 2.3 update equations, on the staggered grid of that section), per cell in
the paper's index notation, against the oracle on tiny periodic grids with
random fields and every coupling term active.

It shares nothing with the oracle but the seeded inputs: plain Python loops
over cells (i, j, k), periodic indices, and the step in the paper's order
(current, first half-steps of E and B, axion, second half-steps, current at the
new time, E1's second half).  Agreement to 1e-14 normwise after five steps pins
every term of the oracle's step, including the 3D-only parts of the cross term
E0 x grad phi and the four-point average of B0.  A second set of cases puts
absorbing layers on some sides and pins the oracle's boundary rules there (the
readings of Sec. 2.4 the oracle follows)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]


class Step:
    """The coupled scheme on a grid of n = (nx, ny, nz) cells, each axis periodic
    or absorbing on both sides."""

    def __init__(self, grid):
        self.nx, self.ny, self.nz = grid.n
        self.dx, self.dy, self.dz = grid.d
        self.dt, self.m, self.g = grid.dt, grid.m, grid.g
        self.Bext, self.Eext = grid.B_ext, grid.E_ext
        # each axis is periodic or absorbing (PML) on both sides, for E/B and the axion alike
        self.per = [grid.em_bc[a][0] == "periodic" for a in range(3)]
        N, smax = grid.pml_cells, grid.pml_sigma_max_dt / grid.dt

        def profile(n, a):
            """sigma per cell along axis a: (1 - q/N)^3 sigma_max, q cells from the outer edge"""
            if self.per[a]:
                return [0.0] * n
            out = []
            for c in range(n):
                q = min(c, n - 1 - c)
                out.append((1.0 - q / N) ** 3 * smax if q < N else 0.0)
            return out

        self.sig = [profile(self.nx, 0), profile(self.ny, 1), profile(self.nz, 2)]

    def sigma(self, i, j, k):
        """the layer's sigma in cell (i, j, k): the largest of the axes' (a corner takes the largest)"""
        return max(self.sig[0][i], self.sig[1][j], self.sig[2][k])

    # field access: periodic indices wrap; beyond an absorbing side every field and
    # the axion are zero (the zero closure and the layer's Dirichlet ghost)
    def at(self, F, i, j, k):
        idx = []
        for c, n, per in ((i, self.nx, self.per[0]), (j, self.ny, self.per[1]), (k, self.nz, self.per[2])):
            if per:
                c %= n
            elif c < 0 or c >= n:
                return 0.0
            idx.append(c)
        return F[idx[2]][idx[1]][idx[0]]

    def cells(self):
        for k in range(self.nz):
            for j in range(self.ny):
                for i in range(self.nx):
                    yield i, j, k

    # E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2)
    # B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2), B_z at (i+1/2, j+1/2, k)
    def curlB(self, Bx, By, Bz, i, j, k):
        """(curl B) at the three E locations of cell (i, j, k)."""
        cx = (self.at(Bz, i, j, k) - self.at(Bz, i, j - 1, k)) / self.dy - \
             (self.at(By, i, j, k) - self.at(By, i, j, k - 1)) / self.dz
        cy = (self.at(Bx, i, j, k) - self.at(Bx, i, j, k - 1)) / self.dz - \
             (self.at(Bz, i, j, k) - self.at(Bz, i - 1, j, k)) / self.dx
        cz = (self.at(By, i, j, k) - self.at(By, i - 1, j, k)) / self.dx - \
             (self.at(Bx, i, j, k) - self.at(Bx, i, j - 1, k)) / self.dy
        return cx, cy, cz

    def curlE(self, Ex, Ey, Ez, i, j, k):
        """(curl E) at the three B locations of cell (i, j, k)."""
        cx = (self.at(Ez, i, j + 1, k) - self.at(Ez, i, j, k)) / self.dy - \
             (self.at(Ey, i, j, k + 1) - self.at(Ey, i, j, k)) / self.dz
        cy = (self.at(Ex, i, j, k + 1) - self.at(Ex, i, j, k)) / self.dz - \
             (self.at(Ez, i + 1, j, k) - self.at(Ez, i, j, k)) / self.dx
        cz = (self.at(Ey, i + 1, j, k) - self.at(Ey, i, j, k)) / self.dx - \
             (self.at(Ex, i, j + 1, k) - self.at(Ex, i, j, k)) / self.dy
        return cx, cy, cz

    def e_centre(self, E, i, j, k):
        """E0 at the cell centre: mean of the two faces along each component's axis, plus E_ext."""
        Ex, Ey, Ez = E
        return (0.5 * (self.at(Ex, i, j, k) + self.at(Ex, i - 1, j, k)) + self.Eext[0],
                0.5 * (self.at(Ey, i, j, k) + self.at(Ey, i, j - 1, k)) + self.Eext[1],
                0.5 * (self.at(Ez, i, j, k) + self.at(Ez, i, j, k - 1)) + self.Eext[2])

    def b_centre(self, B, i, j, k):
        """B0 at the cell centre: mean of the four edges around it, plus B_ext."""
        Bx, By, Bz = B
        bx = 0.25 * (self.at(Bx, i, j, k) + self.at(Bx, i, j - 1, k) + self.at(Bx, i, j, k - 1)
                     + self.at(Bx, i, j - 1, k - 1)) + self.Bext[0]
        by = 0.25 * (self.at(By, i, j, k) + self.at(By, i - 1, j, k) + self.at(By, i, j, k - 1)
                     + self.at(By, i - 1, j, k - 1)) + self.Bext[1]
        bz = 0.25 * (self.at(Bz, i, j, k) + self.at(Bz, i - 1, j, k) + self.at(Bz, i, j - 1, k)
                     + self.at(Bz, i - 1, j - 1, k)) + self.Bext[2]
        return bx, by, bz

    def current(self, E0, B0, hi, lo):
        """J (without g) at the E locations from the axion levels hi = phi^{m+1/2},
        lo = phi^{m-1/2}: P = (D_t phi) Bbar0 - Ebar0 x grad_c phi at the centres,
        then J_a(c + a/2) = (P_a(c) + P_a(c + a)) / 2."""
        def mid(a, b, c):
            return 0.5 * (self.at(hi, a, b, c) + self.at(lo, a, b, c))

        def P(i, j, k):
            """P at the centre of cell (i, j, k), which may lie beyond an absorbing side"""
            Dt = (self.at(hi, i, j, k) - self.at(lo, i, j, k)) / self.dt
            gx = (mid(i + 1, j, k) - mid(i - 1, j, k)) / (2 * self.dx)
            gy = (mid(i, j + 1, k) - mid(i, j - 1, k)) / (2 * self.dy)
            gz = (mid(i, j, k + 1) - mid(i, j, k - 1)) / (2 * self.dz)
            ex, ey, ez = self.e_centre(E0, i, j, k)
            bx, by, bz = self.b_centre(B0, i, j, k)
            return (Dt * bx - (ey * gz - ez * gy), Dt * by - (ez * gx - ex * gz), Dt * bz - (ex * gy - ey * gx))

        J = np.zeros((3, self.nz, self.ny, self.nx))
        for i, j, k in self.cells():
            p = P(i, j, k)
            J[0][k][j][i] = 0.5 * (p[0] + P(i + 1, j, k)[0])
            J[1][k][j][i] = 0.5 * (p[1] + P(i, j + 1, k)[1])
            J[2][k][j][i] = 0.5 * (p[2] + P(i, j, k + 1)[2])
        return J

    def e_half(self, E, B, J):
        """E <- E + (dt/2)(curl B - g J) at every E location (J = None: no current)."""
        h = self.dt / 2
        out = [F.copy() for F in E]
        for i, j, k in self.cells():
            c = self.curlB(*B, i, j, k)
            sg = self.sigma(i, j, k)
            for a in range(3):
                s = c[a] if J is None else c[a] - self.g * J[a][k][j][i]
                out[a][k][j][i] = self.damped(E[a][k][j][i], s, sg, h)
        return out

    @staticmethod
    def damped(F, X, sg, h):
        """dF/dt = X - sigma F over h, trapezoidal in time (plain where sigma = 0)"""
        if sg == 0.0:
            return F + h * X
        return ((1 - sg * h / 2) * F + h * X) / (1 + sg * h / 2)

    def b_half(self, B, E):
        """B <- B - (dt/2) curl E at every B location."""
        h = self.dt / 2
        out = [F.copy() for F in B]
        for i, j, k in self.cells():
            c = self.curlE(*E, i, j, k)
            sg = self.sigma(i, j, k)
            for a in range(3):
                out[a][k][j][i] = self.damped(B[a][k][j][i], -c[a], sg, h)
        return out

    def axion(self, phi, old, E0, B0):
        """phi^{n+3/2} = 2 phi^{n+1/2} - phi^{n-1/2} + dt^2 [L phi - m^2 phi + S], S = g Ebar0 . Bbar0."""
        new = np.zeros_like(phi)
        for i, j, k in self.cells():
            p = phi[k][j][i]
            lap = (self.at(phi, i + 1, j, k) + self.at(phi, i - 1, j, k) - 2 * p) / self.dx ** 2 + \
                  (self.at(phi, i, j + 1, k) + self.at(phi, i, j - 1, k) - 2 * p) / self.dy ** 2 + \
                  (self.at(phi, i, j, k + 1) + self.at(phi, i, j, k - 1) - 2 * p) / self.dz ** 2
            e = self.e_centre(E0, i, j, k)
            b = self.b_centre(B0, i, j, k)
            S = self.g * (e[0] * b[0] + e[1] * b[1] + e[2] * b[2])
            sg = self.sigma(i, j, k)
            dt, po = self.dt, old[k][j][i]
            # in the layer: (1 + s dt) phi^{n+1} = dt^2 [S - m^2 phi + L phi - s^2 phi] + s dt phi^{n-1}
            #               + 2 phi^n - phi^{n-1}   (Sec. 2.4, the PML form of the leapfrog)
            new[k][j][i] = (2 * p - po + dt ** 2 * (lap - self.m ** 2 * p + S) if sg == 0.0 else
                            (dt ** 2 * (S - self.m ** 2 * p + lap - sg * sg * p) + sg * dt * po + 2 * p - po)
                            / (1 + sg * dt))
        return new

    def step(self, s):
        E0 = [s["E0x"], s["E0y"], s["E0z"]]
        B0 = [s["B0x"], s["B0y"], s["B0z"]]
        E1 = [s["E1x"], s["E1y"], s["E1z"]]
        B1 = [s["B1x"], s["B1y"], s["B1z"]]
        phi, old = s["phi_cur"], s["phi_old"]
        J = self.current(E0, B0, phi, old)               # J^n
        E0 = self.e_half(E0, B0, None)                   # E0^{n+1/2}
        E1 = self.e_half(E1, B1, J)                      # E1^{n+1/2}
        B0 = self.b_half(B0, E0)                         # B0^{n+1/2}
        B1 = self.b_half(B1, E1)                         # B1^{n+1/2}
        new = self.axion(phi, old, E0, B0)               # phi^{n+3/2}, source at n+1/2
        B0 = self.b_half(B0, E0)                         # B0^{n+1}
        B1 = self.b_half(B1, E1)                         # B1^{n+1}
        E0 = self.e_half(E0, B0, None)                   # E0^{n+1}
        J = self.current(E0, B0, new, phi)               # J^{n+1}
        E1 = self.e_half(E1, B1, J)                      # E1^{n+1}
        out = {}
        for name, F in zip(W.FIELD_NAMES, E0 + B0 + E1 + B1):
            out[name] = F
        out["phi_cur"], out["phi_old"] = new, phi
        return out


@pytest.mark.parametrize("n", [(3, 3, 1), (4, 4, 4), (5, 5, 5), (7, 4, 3)])
def test_independent_transcription_matches_the_oracle(n):
    d = (0.05, 0.07, 0.06)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    grid = W.GridSpec(n=n, d=d, dt=dt, m=1.1, g=0.7, B_ext=(0.3, -0.5, 0.7), E_ext=(0.05, 0.02, -0.1))
    start = W.random_state(grid, seed=1313, scale1=0.3)
    og = oracle.OracleGrid(grid)
    og.load(start)
    og.step(5)
    ref = og.fields()
    T = Step(grid)
    s = {k: v.copy() for k, v in start.items()}
    for _ in range(5):
        s = T.step(s)
    for name in NAMES:
        nr = np.linalg.norm(ref[name])
        assert nr > 0, name
        assert np.linalg.norm(s[name] - ref[name]) <= 1e-14 * nr, (n, name, np.linalg.norm(s[name] - ref[name]) / nr)


def test_the_transcription_sees_a_flipped_cross_term():
    """Control: the same transcription with the sign of the E0 arrays' part of the
    cross term flipped disagrees with the oracle far beyond rounding."""
    n = (4, 4, 4)
    d = (0.05, 0.07, 0.06)
    dt = 0.5 / math.sqrt(sum(1.0 / x ** 2 for x in d))
    grid = W.GridSpec(n=n, d=d, dt=dt, m=1.1, g=0.7, B_ext=(0.3, -0.5, 0.7), E_ext=(0.05, 0.02, -0.1))
    start = W.random_state(grid, seed=1314, scale1=0.3)
    og = oracle.OracleGrid(grid)
    og.load(start)
    og.step(3)
    ref = og.fields()

    class Flipped(Step):
        def current(self, E0, B0, hi, lo):
            # the current with E0's arrays zero keeps (D_t phi) Bbar0 and the E_ext cross
            # term; twice it minus the full current flips the sign of the E0 arrays' cross term
            Ez = [np.zeros_like(F) for F in E0]
            J_b = Step.current(self, Ez, B0, hi, lo)
            J_full = Step.current(self, E0, B0, hi, lo)
            return 2 * J_b - J_full

    T = Flipped(grid)
    s = {k: v.copy() for k, v in start.items()}
    for _ in range(3):
        s = T.step(s)
    worst = max(np.linalg.norm(s[k] - ref[k]) / np.linalg.norm(ref[k]) for k in ("E1x", "E1y", "E1z"))
    assert worst > 1e-6


@pytest.mark.parametrize("n,sides", [((8, 7, 9), ("pml", "pml", "pml")), ((9, 4, 3), ("pml", "periodic", "periodic")),
                                     ((6, 9, 1), ("periodic", "pml", "periodic"))])
def test_independent_transcription_matches_the_oracle_with_absorbing_layers(n, sides):
    """The same transcription with absorbing layers (2 cells) on some sides: zero
    fields beyond them, the axion's Dirichlet ghost, the layer's sigma per cell
    (the largest of the axes' at a corner), the trapezoidal damped half-steps and
    the paper's damped leapfrog for the axion."""
    d = (0.05, 0.07, 0.06)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    bc = W._bcs(*sides)
    grid = W.GridSpec(n=n, d=d, dt=dt, m=1.1, g=0.7, B_ext=(0.3, -0.5, 0.7), E_ext=(0.05, 0.02, -0.1),
                      axion_bc=bc, em_bc=bc, pml_cells=2)
    start = W.random_state(grid, seed=1315, scale1=0.3)
    og = oracle.OracleGrid(grid)
    og.load(start)
    og.step(5)
    ref = og.fields()
    T = Step(grid)
    assert any(T.sigma(i, j, k) > 0 for i, j, k in T.cells())
    s = {k: v.copy() for k, v in start.items()}
    for _ in range(5):
        s = T.step(s)
    for name in NAMES:
        nr = np.linalg.norm(ref[name])
        assert nr > 0, name
        assert np.linalg.norm(s[name] - ref[name]) <= 1e-14 * nr, (n, name, np.linalg.norm(s[name] - ref[name]) / nr)

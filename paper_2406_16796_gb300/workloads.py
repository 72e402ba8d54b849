"""Workload descriptions and seeded synthetic inputs.

This module holds parameters and random-number draws only: no step of the
field update, no operator, no dispersion relation.  It is the one module that
both the CUDA path's tests/bench and the CPU oracle read their inputs from.

Units are the natural units of arXiv 2406.16796 Sec. 2.1 with the laser
wavelength as the length unit (lambda0 = 1, so k0 = omega0 = 2 pi).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

SEED_BASE = 20240624  # seeds are SEED_BASE + workload index

BC_NAMES = ("periodic", "reflect", "outflow", "pml")
BC_CODE = {name: i for i, name in enumerate(BC_NAMES)}

K0 = 2.0 * math.pi


def _bcs(x="periodic", y="periodic", z="periodic"):
    def pair(v):
        return (v, v) if isinstance(v, str) else tuple(v)

    return (pair(x), pair(y), pair(z))


@dataclass
class GridSpec:
    """One simulation box.  n = cells per axis (invariant axes have n = 1)."""

    n: Tuple[int, int, int]
    d: Tuple[float, float, float]
    dt: float
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    m: float = 0.0
    g: float = 0.0
    B_ext: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    E_ext: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    axion_bc: tuple = field(default_factory=_bcs)
    em_bc: tuple = field(default_factory=_bcs)
    pml_cells: int = 20
    pml_sigma_max_dt: float = 0.2
    precision: str = "fp64"  # "fp64" or "fp32" (FP32 split storage)

    @property
    def ndim(self) -> int:
        return 3 if self.n[2] > 1 else (2 if self.n[1] > 1 else 1)

    @property
    def cells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def replace(self, **kw) -> "GridSpec":
        return dataclasses.replace(self, **kw)


@dataclass
class LaserSpec:
    amplitude: float
    k: Tuple[float, float, float]
    pol: Tuple[float, float, float]
    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    waist: float = 0.0  # transverse 1/e field radius, 0 = plane
    duration: float = 0.0  # intensity FWHM in time, 0 = CW
    phase: float = 0.0


@dataclass
class SourceSpec:
    """A laser entering through the x-plane lo + plane*dx (a soft source): E =
    amplitude pol f(y, z) env(t - t_centre - (x - centre[0])) cos(k (x - centre[0])
    - w (t - t_centre) + phase), moving towards +x."""
    amplitude: float
    k: float
    pol: Tuple[float, float, float]
    plane: int
    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    waist: float = 0.0  # transverse 1/e field radius, 0 = plane
    duration: float = 0.0  # intensity FWHM in time, 0 = CW
    t_centre: float = 0.0
    phase: float = 0.0


@dataclass
class AxionSpec:
    amplitude: float
    k: Tuple[float, float, float]
    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    waist: float = 0.0
    length: float = 0.0
    speed: float = 1.0
    phase: float = 0.0


@dataclass
class Workload:
    name: str
    grid: GridSpec
    lasers: tuple = ()
    axions: tuple = ()
    steps: int = 0
    diag_every: int = 0


# ---------------------------------------------------------------------------
# The five workloads.  Each states its sizes; the step counts are those of the
# full runs (tests and the bench take prefixes of them).
# ---------------------------------------------------------------------------


def vacuum_1d(nx=4096, steps=20000, g=1e-4, B0=1.0, amplitude=1e-3, m=0.0, cfl=0.95,
              precision="fp64") -> Workload:
    """1D photon->axion conversion: CW E_y wave along x, static B_ext along y."""
    dx = 1.0 / 32.0
    grid = GridSpec(n=(nx, 1, 1), d=(dx, dx, dx), dt=cfl * dx, m=m, g=g, B_ext=(0.0, B0, 0.0),
                    precision=precision)
    waves = round(nx * dx)  # whole wavelengths in the box
    k = 2.0 * math.pi * waves / (nx * dx)
    laser = LaserSpec(amplitude=amplitude, k=(k, 0.0, 0.0), pol=(0.0, 1.0, 0.0))
    return Workload("1d_vacuum_nx%d" % nx, grid, lasers=(laser,), steps=steps, diag_every=100)


def pulse_2d(nx=4096, ny=2048, steps=16000, m=0.0, g=1e-4, a0=0.01, precision="fp64",
             cfl=0.95) -> Workload:
    """2D Gaussian pulse (E_z) through B_ext along z, absorbing boundaries on all edges."""
    dx = 1.0 / 32.0
    dt = cfl * dx / math.sqrt(2.0)
    Lx, Ly = nx * dx, ny * dx
    grid = GridSpec(n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, lo=(0.0, -Ly / 2.0, 0.0), m=m, g=g,
                    B_ext=(0.0, 0.0, 1.0), axion_bc=_bcs("pml", "pml"), em_bc=_bcs("pml", "pml"),
                    precision=precision)
    laser = LaserSpec(amplitude=a0, k=(K0, 0.0, 0.0), pol=(0.0, 0.0, 1.0),
                      centre=(min(16.0, Lx / 2.0), 0.0, 0.0), waist=min(4.0, Ly / 8.0),
                      duration=min(8.0, Lx / 8.0))
    return Workload("2d_pulse_%dx%d" % (nx, ny), grid, lasers=(laser,), steps=steps, diag_every=100)


def axion_3d(n=512, steps=2000, g=1e-4, amplitude=1e-2, m=0.0, precision="fp32") -> Workload:
    """3D periodic box seeded with an axion plane wave along x, static B_ext along y."""
    dx = 1.0 / 16.0
    dt = 0.95 * dx / math.sqrt(3.0)
    grid = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=dt, m=m, g=g, B_ext=(0.0, 1.0, 0.0),
                    precision=precision)
    waves = max(1, round(n * dx))
    ax = AxionSpec(amplitude=amplitude, k=(2.0 * math.pi * waves / (n * dx), 0.0, 0.0))
    return Workload("3d_axion_%d" % n, grid, axions=(ax,), steps=steps, diag_every=100)


def bc_check_2d(bc="pml", n=400, m_over_k=6.5e-4) -> Workload:
    """Sec. 3.1 boundary test: left-moving Gaussian axion pulse, box [-20, 20]^2 in lambda0."""
    L = 40.0
    dx = L / n
    dt = 0.95 * dx / math.sqrt(2.0)
    grid = GridSpec(n=(n, n, 1), d=(dx, dx, dx), dt=dt, lo=(-20.0, -20.0, 0.0), m=m_over_k * K0,
                    g=0.0, axion_bc=_bcs(bc, bc), em_bc=_bcs("pml", "pml"), pml_cells=20,
                    pml_sigma_max_dt=0.2)
    # phi = exp(-(eta^2 + y^2)/w^2) sin(k0 eta), eta = x + t: a wave moving along -x
    ax = AxionSpec(amplitude=1.0, k=(-K0, 0.0, 0.0), centre=(0.0, 0.0, 0.0), waist=5.0, length=5.0,
                   speed=1.0, phase=math.pi)
    return Workload("bc_check_%s" % bc, grid, axions=(ax,), steps=int(round(45.0 / dt)))


# ---------------------------------------------------------------------------
# Batched scan and serving draws
# ---------------------------------------------------------------------------


@dataclass
class ScanInstance:
    nx: int
    m: float
    g: float
    B0: float
    steps: int


def scan_instances(count=512, seed=SEED_BASE + 3, nx_range=(1024, 65536), steps_range=(5000, 40000)):
    """Parameter-scan draws: Nx log-uniform, m/omega0 log-uniform in [1e-3, 2],
    g log-uniform in [1e-6, 1e-3], B0 log-uniform in [0.1, 10], steps uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(nx_range[0]), math.log(nx_range[1])))))
        m = K0 * math.exp(rng.uniform(math.log(1e-3), math.log(2.0)))
        g = math.exp(rng.uniform(math.log(1e-6), math.log(1e-3)))
        B0 = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(ScanInstance(nx, m, g, B0, steps))
    return out


def scan_workload(inst: ScanInstance, precision="fp32", amplitude=1e-3) -> Workload:
    w = vacuum_1d(nx=inst.nx, steps=inst.steps, g=inst.g, B0=inst.B0, amplitude=amplitude, m=inst.m,
                  precision=precision)
    return w


def shard(items, rank, world):
    """The share of a list of independent problems that rank `rank` of `world`
    runs: items rank, rank + world, rank + 2 world, ... (replicas, no exchange)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    return list(items)[rank::world]


@dataclass
class Request:
    arrival: float  # seconds after the start
    ndim: int
    n: Tuple[int, int, int]
    m: float
    g: float
    B0: float
    steps: int


def serve_requests(count=10000, rate_per_s=100.0, seed=SEED_BASE + 4, frac_1d=0.8,
                   steps_range=(5000, 40000)):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        m = K0 * math.exp(rng.uniform(math.log(1e-3), math.log(2.0)))
        g = math.exp(rng.uniform(math.log(1e-6), math.log(1e-3)))
        B0 = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if rng.uniform() < frac_1d:
            nx = int(round(math.exp(rng.uniform(math.log(1024), math.log(65536)))))
            out.append(Request(t, 1, (nx, 1, 1), m, g, B0, steps))
        else:
            nx = int(round(math.exp(rng.uniform(math.log(256), math.log(2048)))))
            nx -= nx % 2
            out.append(Request(t, 2, (nx, nx // 2, 1), m, g, B0, steps))
    return out


def beam_2d(nx, ny, steps=0, m=0.0, g=1e-4, B0=1.0, amplitude=1e-3, precision="fp32", pml_cells=20) -> Workload:
    """2D conversion request: a box periodic along x and absorbing along y
    (PML on E/B and phi), a CW E_z beam along x (waist Ly/8, a whole number of
    wavelengths in the box), B_ext along z."""
    dx = 1.0 / 32.0
    dt = 0.95 * dx / math.sqrt(2.0)
    Lx, Ly = nx * dx, ny * dx
    grid = GridSpec(n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, lo=(0.0, -Ly / 2.0, 0.0), m=m, g=g,
                    B_ext=(0.0, 0.0, B0), axion_bc=_bcs("periodic", "pml"), em_bc=_bcs("periodic", "pml"),
                    pml_cells=pml_cells, precision=precision)
    waves = max(1, round(Lx))
    laser = LaserSpec(amplitude=amplitude, k=(2.0 * math.pi * waves / Lx, 0.0, 0.0), pol=(0.0, 0.0, 1.0),
                      centre=(0.0, 0.0, 0.0), waist=Ly / 8.0)
    return Workload("2d_beam_%dx%d" % (nx, ny), grid, lasers=(laser,), steps=steps)


def request_workload(r: Request, precision="fp32") -> Workload:
    if r.ndim == 1:
        return vacuum_1d(nx=r.n[0], steps=r.steps, g=r.g, B0=r.B0, m=r.m, precision=precision)
    return beam_2d(r.n[0], r.n[1], steps=r.steps, m=r.m, g=r.g, B0=r.B0, precision=precision)


# ---------------------------------------------------------------------------
# Random states for element-wise parity tests
# ---------------------------------------------------------------------------

FIELD_NAMES = ("E0x", "E0y", "E0z", "B0x", "B0y", "B0z",
               "E1x", "E1y", "E1z", "B1x", "B1y", "B1z")


def random_state(grid: GridSpec, seed: int, scale0=1.0, scale1=1e-3, scale_phi=1e-2,
                 active=None):
    """Seeded uniform random fields in [-scale, scale) for every array.

    Returns a dict of float64 arrays of shape (nz, ny, nx) keyed by FIELD_NAMES
    plus "phi_cur" (phi^{n+1/2}) and "phi_old" (phi^{n-1/2}).  Arrays not in
    `active` (when given) are zero."""
    rng = np.random.default_rng(seed)
    shape = (grid.n[2], grid.n[1], grid.n[0])
    out = {}
    for name in FIELD_NAMES:
        s = scale0 if name[1] == "0" else scale1
        a = rng.uniform(-s, s, size=shape)
        if active is not None and name not in active:
            a[...] = 0.0
        out[name] = a
    out["phi_cur"] = rng.uniform(-scale_phi, scale_phi, size=shape)
    out["phi_old"] = out["phi_cur"] + rng.uniform(-scale_phi, scale_phi, size=shape) * 0.1
    return out


# ---------------------------------------------------------------------------
# Macroparticles for the perturbed-particle current (Sec. 2.2) and the weak
# laser in a magnetised plasma (Sec. 3.4).
# ---------------------------------------------------------------------------


@dataclass
class PlasmaSpec:
    """One species of macroparticles: charge q, mass m, weights w (count,) and
    positions/momenta (3, count) of both orders at t = 0 (u = gamma v)."""

    q: float
    m: float
    w: np.ndarray
    x0: np.ndarray
    u0: np.ndarray
    x1: np.ndarray
    u1: np.ndarray

    @property
    def count(self) -> int:
        return int(self.w.shape[0])


def plasma_particles(grid: GridSpec, ppc: int, density: float, seed: int, q=-1.0, m=1.0, u0_spread=0.0,
                     x1_spread=0.0, u1_spread=0.0) -> PlasmaSpec:
    """ppc particles in every cell at seeded uniform positions inside the cell,
    weights giving the number density `density`, Gaussian momenta of spread
    u0_spread (order 0) and u1_spread, and displacements of spread x1_spread
    (first order; zero for a plasma that only the fields perturb)."""
    rng = np.random.default_rng(seed)
    n = grid.cells * ppc
    cell = np.repeat(np.arange(grid.cells, dtype=np.int64), ppc)
    idx = (cell % grid.n[0], (cell // grid.n[0]) % grid.n[1], cell // (grid.n[0] * grid.n[1]))
    x0 = np.zeros((3, n))
    for a in range(3):
        if grid.n[a] > 1:
            x0[a] = grid.lo[a] + (idx[a] + rng.uniform(0.0, 1.0, n)) * grid.d[a]
        else:
            x0[a] = grid.lo[a] + 0.5 * grid.d[a]
    dV = grid.d[0] * grid.d[1] * grid.d[2]
    w = np.full(n, density * dV / ppc)
    u0 = rng.normal(size=(3, n)) * u0_spread
    x1 = rng.normal(size=(3, n)) * x1_spread
    for a in range(3):
        if grid.n[a] == 1:
            x1[a] = 0.0
    u1 = rng.normal(size=(3, n)) * u1_spread
    return PlasmaSpec(q, m, w, x0, u0, x1, u1)


def magnetised_plasma_2d(nx=12000, ny=100, ppc=4, n_over_nc=3e-3, amplitude_over_Bc=1e-20, cfl=0.95,
                         seed=SEED_BASE + 5):
    """Weak laser in a transversely magnetised plasma (Sec. 3.4): a box of
    40 x 100 wavelengths on 12000 x 100 cells (finer along the propagation
    axis x), electrons of density n0 = 3e-3 n_c at rest, B_ext = m w_p/|q| along
    z, and a laser pulse of B amplitude 1e-20 B_ext in the first-order fields
    (E1_y, B1_z, propagating along +x).  Both axes periodic (the particles'
    boundary).  n_c = m w0^2/q^2 in these units (eps0 = 1, w0 = 2 pi).

    Returns (grid, plasma, fields): fields maps E1y and B1z to their arrays."""
    Lx, Ly = 40.0, 100.0
    dx, dy = Lx / nx, Ly / ny
    dt = cfl / math.sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy))
    n0 = n_over_nc * K0 * K0
    wp = math.sqrt(n0)
    Bc = wp
    grid = GridSpec(n=(nx, ny, 1), d=(dx, dy, dy), dt=dt, lo=(-Lx / 2.0, -Ly / 2.0, 0.0), m=0.0, g=0.0,
                    B_ext=(0.0, 0.0, Bc))
    plasma = plasma_particles(grid, ppc, n0, seed)
    A = amplitude_over_Bc * Bc
    xc, L, waist = -10.0, 3.0, 20.0
    # E_y at (x_i + dx/2, y_j + dy), B_z at (x_i + dx, y_j + dy) relative to the low faces
    xs_e = grid.lo[0] + (np.arange(nx) + 0.5) * dx
    xs_b = grid.lo[0] + (np.arange(nx) + 1.0) * dx
    ys = grid.lo[1] + (np.arange(ny) + 1.0) * dy

    def pulse(x):
        return A * np.exp(-((x - xc) / L) ** 2) * np.cos(K0 * (x - xc))

    trans = np.exp(-(ys / waist) ** 2)
    fields = {"E1y": (trans[:, None] * pulse(xs_e)[None, :])[None],
              "B1z": (trans[:, None] * pulse(xs_b)[None, :])[None]}
    return grid, plasma, fields

"""SI front-end: the paper's physical parameters in the normalised units of the
solver, and back (arXiv 2406.16796 Sec. 2.1 SI equations, Sec. 2.2 estimate,
Sec. 3.2 parameter set).

The solver works in units where c = 1, lengths are in laser wavelengths
lambda0 (so k0 = omega0 = 2 pi), times in lambda0 / c, and the electric field
in E_u = m_e omega0 c / e (so a laser's normalised amplitude is its a0).  With
B_u = E_u / c the normalised Maxwell equations have no constants, and the SI
axion equation of Sec. 2.1,

    (d_t^2 / c^2 - laplacian + m_a^2 c^2 / hbar^2) phi = g / (hbar mu0) E . B,

with phi in 1/s and g in seconds, becomes the solver's
(d_t^2 - laplacian + m^2) phi~ = g~ E~ . B~ with

    phi_u = E_u lambda0 sqrt(eps0 c / hbar),     g~ = g phi_u,
    m~ = m_a c^2 lambda0 / (hbar c).

The same g~ then multiplies the axion current in the normalised curl-B
equation, and energy densities in both parts share the factor eps0 E_u^2:
  (eps0 E^2 + B^2 / mu0) / 2 = eps0 E_u^2 (E~^2 + B~^2) / 2,
  hbar / (2c) (phi_t^2 / c^2 + |grad phi|^2 + m^2 c^2 / hbar^2 phi^2)
      = eps0 E_u^2 (phi~_t^2 + |grad phi~|^2 + m~^2 phi~^2) / 2,
so the conversion probability (an energy ratio) is the same number in both
systems.  Nothing here is on the compute path: it converts inputs and outputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

# CODATA 2018 (c, e, h exact)
C = 299792458.0                 # m/s
E_CHARGE = 1.602176634e-19      # C
H_PLANCK = 6.62607015e-34       # J s
HBAR = H_PLANCK / (2.0 * math.pi)
M_E = 9.1093837015e-31          # kg
EPS0 = 8.8541878128e-12         # F/m
MU0 = 1.0 / (EPS0 * C * C)      # H/m
ALPHA = E_CHARGE ** 2 / (4.0 * math.pi * EPS0 * HBAR * C)
EV = E_CHARGE                   # J
GEV = 1.0e9 * EV                # J


@dataclass(frozen=True)
class Units:
    """Normalisation for a laser of wavelength lambda0 (metres)."""

    lambda0: float = 8.0e-7

    @property
    def omega0(self):
        return 2.0 * math.pi * C / self.lambda0

    @property
    def length(self):  # metres per unit length
        return self.lambda0

    @property
    def time(self):  # seconds per unit time
        return self.lambda0 / C

    @property
    def E_u(self):  # V/m per unit field (a0 = 1)
        return M_E * self.omega0 * C / E_CHARGE

    @property
    def B_u(self):  # T per unit field
        return self.E_u / C

    @property
    def phi_u(self):  # 1/s per unit axion field
        return self.E_u * self.lambda0 * math.sqrt(EPS0 * C / HBAR)

    @property
    def energy_density(self):  # J/m^3 per unit energy density
        return EPS0 * self.E_u ** 2

    # -- SI -> normalised ------------------------------------------------------
    def E(self, volts_per_m):
        return volts_per_m / self.E_u

    def B(self, tesla):
        return tesla / self.B_u

    def phi(self, per_s):
        return per_s / self.phi_u

    def coupling(self, g_seconds):
        """g (SI, in seconds, as in the Sec. 2.1 equations) -> g~."""
        return g_seconds * self.phi_u

    def mass(self, m_eV):
        """Axion rest energy m_a c^2 in eV -> m~ (the Klein-Gordon mass, per unit length)."""
        return m_eV * EV * self.lambda0 / (HBAR * C)

    def distance(self, metres):
        return metres / self.lambda0

    def duration(self, seconds):
        return seconds / self.time

    # -- normalised -> SI ------------------------------------------------------
    def E_si(self, e):
        return e * self.E_u

    def B_si(self, b):
        return b * self.B_u

    def phi_si(self, p):
        return p * self.phi_u

    def coupling_si(self, g):
        return g / self.phi_u

    def mass_eV(self, m):
        return m * HBAR * C / (self.lambda0 * EV)


def g_seconds(g_per_GeV):
    """A coupling quoted as g hbar / GeV (e.g. 2.65e-13 hbar GeV^-1) in seconds."""
    return g_per_GeV * HBAR / GEV


def f_a_GeV(m_eV):
    """Axion decay constant from the mass relation of Sec. 3.2: m_a = 6.3 eV 1e6 GeV / f_a."""
    return 6.3 * 1.0e6 / m_eV


def model_coupling_per_GeV(m_eV, c_gamma):
    """g = c_gamma 2 alpha / (pi f_a) in GeV^-1 (Sec. 3.2); c_gamma = 0.36 (DFSZ), -0.97 (KSVZ)."""
    return c_gamma * 2.0 * ALPHA / (math.pi * f_a_GeV(m_eV))


DFSZ_C_GAMMA = 0.36
KSVZ_C_GAMMA = -0.97


def conversion_probability_si(g_s, B_tesla, l_m, kappa_per_m=0.0):
    """Sec. 3.2 conversion probability in SI form: c / (4 mu0 hbar) (g B l)^2 sinc^2(kappa l / 2)."""
    x = kappa_per_m * l_m / 2.0
    s = 1.0 if x == 0.0 else math.sin(x) / x
    return C / (4.0 * MU0 * HBAR) * (g_s * B_tesla * l_m) ** 2 * s * s


def conversion_probability(g, B, l, kappa=0.0):
    """The same law in normalised units: (1/4) (g B l)^2 sinc^2(kappa l / 2)."""
    x = kappa * l / 2.0
    s = 1.0 if x == 0.0 else math.sin(x) / x
    return 0.25 * (g * B * l) ** 2 * s * s


def fps_estimate(a0=100.0, lambda0=8.0e-7, g_per_GeV=2.7e-13, E0=None):
    """The order-of-magnitude estimate of Sec. 2.2: laser field E0 for a0 (unless
    E0 in V/m is given), the axion field a laser generates within a wavelength in
    a field as strong as itself, phi ~ g E0 B0 / (2 mu0 hbar k0^2) with
    B0 = E0 / c, and the field it feeds back, E1 ~ g phi B0 c.  Returns (E0 in
    V/m, phi in 1/s, E1 in V/m)."""
    u = Units(lambda0)
    if E0 is None:
        E0 = a0 * u.E_u
    B0 = E0 / C
    g = g_seconds(g_per_GeV)
    k0 = 2.0 * math.pi / lambda0
    phi = g * E0 * B0 / (2.0 * MU0 * HBAR * k0 * k0)
    return E0, phi, g * phi * B0 * C


@dataclass(frozen=True)
class GenerationSetup:
    """The axion-generation benchmark of Sec. 3.2 in normalised units."""

    a0: float
    B: float          # background along y
    m: float          # Klein-Gordon mass
    g: float
    waist: float      # transverse width (lambda0)
    duration: float   # intensity FWHM (lambda0 / c)
    units: Units


def paper_generation_setup(lambda0=8.0e-7, a0=3.0, B_tesla=423.0, m_eV=1.0e-3, c_gamma=DFSZ_C_GAMMA,
                           width_lambda=5.0, fwhm_periods=5.0):
    """Sec. 3.2: 800 nm laser, a0 = 3, B = 423 T along y, m_a = 1 meV, DFSZ coupling,
    width 5 lambda0, FWHM duration 5 T0."""
    u = Units(lambda0)
    g = u.coupling(g_seconds(abs(model_coupling_per_GeV(m_eV, c_gamma))))
    return GenerationSetup(a0=a0, B=u.B(B_tesla), m=u.mass(m_eV), g=g, waist=width_lambda, duration=fwhm_periods,
                           units=u)

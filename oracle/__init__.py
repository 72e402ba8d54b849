"""Python access to the plain FP64 CPU oracle (oracle/axp_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; the product package never imports it.

The oracle follows arXiv 2406.16796 Sec. 2 step by step (see the header of
axp_oracle.c for the readings it takes where the paper is silent).  Arrays are
numpy float64 of shape (nz, ny, nx), x fastest, matching the C layout.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from paper_2406_16796_gb300.workloads import BC_CODE, FIELD_NAMES, AxionSpec, GridSpec, LaserSpec, SourceSpec

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "axp_oracle.c")
PSRC = os.path.join(HERE, "axp_oracle_particles.c")
LIB = os.path.join(HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force=False) -> str:
    """Compile liborc.so with gcc (-O2 -ffp-contract=off, OpenMP when available)."""
    with _lock:
        hdr = os.path.join(HERE, "axp_oracle.h")
        fresh = os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in (SRC, PSRC, hdr))
        if fresh and not force:
            return LIB
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", SRC, PSRC, "-o",
                LIB + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(LIB + ".tmp", LIB)
        return LIB


class _Params(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("d", C.c_double * 3), ("lo", C.c_double * 3), ("dt", C.c_double),
                ("m", C.c_double), ("g", C.c_double), ("B_ext", C.c_double * 3), ("E_ext", C.c_double * 3),
                ("axion_bc", (C.c_int32 * 2) * 3), ("em_bc", (C.c_int32 * 2) * 3), ("pml_cells", C.c_int32),
                ("pad_", C.c_int32), ("pml_sigma_max_dt", C.c_double)]


_DP = C.POINTER(C.c_double)


class _State(C.Structure):
    _fields_ = [("E0", _DP * 3), ("B0", _DP * 3), ("E1", _DP * 3), ("B1", _DP * 3), ("phi_cur", _DP),
                ("phi_old", _DP), ("ghost", ((_DP * 2) * 2) * 3), ("step", C.c_int64)]


class _Laser(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double * 3), ("pol", C.c_double * 3),
                ("centre", C.c_double * 3), ("waist", C.c_double), ("duration", C.c_double),
                ("phase", C.c_double)]


class _Axion(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double * 3), ("centre", C.c_double * 3),
                ("waist", C.c_double), ("length", C.c_double), ("speed", C.c_double), ("phase", C.c_double)]


class _Source(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double), ("pol", C.c_double * 3), ("centre", C.c_double * 3),
                ("waist", C.c_double), ("duration", C.c_double), ("t_centre", C.c_double), ("phase", C.c_double),
                ("plane", C.c_int64)]


class _Particles(C.Structure):
    _fields_ = [("count", C.c_int64), ("q", C.c_double), ("m", C.c_double), ("w", _DP), ("x0", _DP * 3),
                ("u0", _DP * 3), ("x1", _DP * 3), ("u1", _DP * 3), ("j0", _DP * 3), ("j1", _DP * 3)]


class _Diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("t", "H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "W", "sum_xB1z2",
                                          "sum_B1z2", "gauss_l2")]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.orc_validate.argtypes = [C.POINTER(_Params)]
        L.orc_step.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int64]
        L.orc_step_src.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Source), C.c_int64]
        L.orc_current.argtypes = [C.POINTER(_Params), C.POINTER(_State), _DP * 3]
        L.orc_source_now.argtypes = [C.POINTER(_Params), C.POINTER(_State), _DP]
        L.orc_gauss_residual.argtypes = [C.POINTER(_Params), C.POINTER(_State), _DP]
        L.orc_diagnostics.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Diag)]
        L.orc_inject_laser.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Laser)]
        L.orc_inject_axion.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Axion)]
        L.orc_sigma_cell.argtypes = [C.POINTER(_Params), C.c_int64, C.c_int64, C.c_int64, C.c_int]
        L.orc_sigma_cell.restype = C.c_double
        L.orc_outflow_solve.argtypes = [C.c_double] * 7 + [_DP, _DP]
        PP = C.POINTER(_Particles)
        L.orc_particles_validate.argtypes = [C.POINTER(_Params), PP]
        L.orc_particles_start.argtypes = [C.POINTER(_Params), PP]
        L.orc_particles_positions_now.argtypes = [C.POINTER(_Params), PP, _DP * 3, _DP * 3]
        L.orc_gather.argtypes = [C.POINTER(_Params), C.POINTER(_State), _DP, _DP, _DP, _DP, _DP, _DP]
        L.orc_kick.argtypes = [C.c_double, C.c_double] + [_DP] * 8
        L.orc_deposit.argtypes = [C.POINTER(_Params), C.c_double, _DP, _DP, _DP, _DP, _DP * 3, _DP * 3]
        L.orc_push.argtypes = [C.POINTER(_Params), C.POINTER(_State), PP]
        L.orc_step_plasma.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Source), PP, C.c_int64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def params_of(grid: GridSpec) -> _Params:
    p = _Params()
    for a in range(3):
        p.n[a] = int(grid.n[a])
        p.d[a] = float(grid.d[a])
        p.lo[a] = float(grid.lo[a])
        p.B_ext[a] = float(grid.B_ext[a])
        p.E_ext[a] = float(grid.E_ext[a])
        for s in range(2):
            p.axion_bc[a][s] = BC_CODE[grid.axion_bc[a][s]]
            p.em_bc[a][s] = BC_CODE[grid.em_bc[a][s]]
    p.dt, p.m, p.g = float(grid.dt), float(grid.m), float(grid.g)
    p.pml_cells = int(grid.pml_cells)
    p.pml_sigma_max_dt = float(grid.pml_sigma_max_dt)
    return p


def plane_shape(grid: GridSpec, a: int):
    """Shape of an outflow ghost plane for axis a, matching the C plane index."""
    nx, ny, nz = grid.n
    return {0: (nz, ny), 1: (nz, nx), 2: (ny, nx)}[a]


class OracleGrid:
    """A grid state advanced by the oracle.  Fields are numpy arrays (nz, ny, nx)."""

    def __init__(self, grid: GridSpec):
        self.grid = grid
        self.p = params_of(grid)
        rc = lib().orc_validate(C.byref(self.p))
        if rc:
            raise ValueError("invalid grid for the oracle (code %d)" % rc)
        shape = (grid.n[2], grid.n[1], grid.n[0])
        self.f = {name: np.zeros(shape) for name in FIELD_NAMES}
        self.phi_cur = np.zeros(shape)
        self.phi_old = np.zeros(shape)
        # ghost[a][side] = [cur plane, old plane] (outflow faces only)
        self.ghost = [[None, None] for _ in range(3)]
        for a in range(3):
            for s in range(2):
                if grid.axion_bc[a][s] == "outflow":
                    self.ghost[a][s] = [np.zeros(plane_shape(grid, a)), np.zeros(plane_shape(grid, a))]
        self.step_count = 0
        self.src = None  # soft source (_Source) or None
        self.parts = None  # macroparticles (dict of arrays) or None

    # -- state marshalling --
    def _state(self) -> _State:
        st = _State()
        for a, c in enumerate("xyz"):
            st.E0[a] = _ptr(self.f["E0" + c])
            st.B0[a] = _ptr(self.f["B0" + c])
            st.E1[a] = _ptr(self.f["E1" + c])
            st.B1[a] = _ptr(self.f["B1" + c])
        st.phi_cur = _ptr(self.phi_cur)
        st.phi_old = _ptr(self.phi_old)
        for a in range(3):
            for s in range(2):
                g = self.ghost[a][s]
                for lev in range(2):
                    st.ghost[a][s][lev] = _ptr(g[lev]) if g is not None else _DP()
        st.step = self.step_count
        return st

    def load(self, fields: dict):
        for name, arr in fields.items():
            if name in self.f:
                self.f[name][...] = arr
            elif name == "phi_cur":
                self.phi_cur[...] = arr
            elif name == "phi_old":
                self.phi_old[...] = arr
            else:
                raise KeyError(name)

    def set_ghost(self, a, side, cur, old):
        self.ghost[a][side][0][...] = cur
        self.ghost[a][side][1][...] = old

    # -- method --
    def step(self, n: int = 1):
        st = self._state()
        src = C.byref(self.src) if self.src is not None else None
        if self.parts is None:
            lib().orc_step_src(C.byref(self.p), C.byref(st), src, int(n))
        else:
            pc = self._parts_struct()
            lib().orc_step_plasma(C.byref(self.p), C.byref(st), src, C.byref(pc), int(n))
        self.step_count = st.step

    # -- perturbed-particle current (Sec. 2.2) --
    def attach_particles(self, q, m, w, x0, u0, x1=None, u1=None):
        """One species of macroparticles: weights w (count,), positions x0, x1 and
        momenta u0, u1 (3, count) at the present integer time.  Deposits j^n and
        moves the positions to the next half-integer time."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        n = w.shape[0]
        z = np.zeros((3, n))
        cells = self.phi_cur.shape
        self.parts = {"q": float(q), "m": float(m), "w": w.copy(),
                      "x0": np.array(x0, dtype=np.float64).reshape(3, n).copy(),
                      "u0": np.array(u0, dtype=np.float64).reshape(3, n).copy(),
                      "x1": (z.copy() if x1 is None else np.array(x1, dtype=np.float64).reshape(3, n).copy()),
                      "u1": (z.copy() if u1 is None else np.array(u1, dtype=np.float64).reshape(3, n).copy()),
                      "j0": np.zeros((3,) + cells), "j1": np.zeros((3,) + cells)}
        pc = self._parts_struct()
        if lib().orc_particles_validate(C.byref(self.p), C.byref(pc)):
            self.parts = None
            raise ValueError("particles need a positive mass and periodic E/B along every active axis")
        lib().orc_particles_start(C.byref(self.p), C.byref(pc))

    def _parts_struct(self) -> _Particles:
        P = self.parts
        for k in ("x0", "u0", "x1", "u1", "j0", "j1"):
            assert P[k].flags.c_contiguous
        return _Particles(P["w"].shape[0], P["q"], P["m"], _ptr(P["w"]),
                          *[(_DP * 3)(*[_ptr(P[k][a]) for a in range(3)]) for k in ("x0", "u0", "x1", "u1", "j0",
                                                                                    "j1")])

    def particles_now(self) -> dict:
        """Positions at the present integer time, momenta, and the currents j^n."""
        P = self.parts
        n = P["w"].shape[0]
        x0n, x1n = np.zeros((3, n)), np.zeros((3, n))
        pc = self._parts_struct()
        lib().orc_particles_positions_now(C.byref(self.p), C.byref(pc), (_DP * 3)(*[_ptr(x0n[a]) for a in range(3)]),
                                          (_DP * 3)(*[_ptr(x1n[a]) for a in range(3)]))
        return {"x0": x0n, "x1": x1n, "u0": P["u0"].copy(), "u1": P["u1"].copy(), "j0": P["j0"].copy(),
                "j1": P["j1"].copy(), "x0_half": P["x0"].copy(), "x1_half": P["x1"].copy()}

    def gather(self, x0, x1):
        """Fields felt at x0 (+ x1) from the present arrays: (E_nop, B_nop, E_p, B_p)."""
        out = [np.zeros(3) for _ in range(4)]
        st = self._state()
        lib().orc_gather(C.byref(self.p), C.byref(st), _ptr(np.array(x0, dtype=np.float64)),
                         _ptr(np.array(x1, dtype=np.float64)), *[_ptr(o) for o in out])
        return tuple(out)

    def deposit(self, qw, x0, x1, u0, u1):
        """Current of one particle alone: (j0, j1), each (3, nz, ny, nx)."""
        j0, j1 = np.zeros((3,) + self.phi_cur.shape), np.zeros((3,) + self.phi_cur.shape)
        lib().orc_deposit(C.byref(self.p), float(qw), *[_ptr(np.array(v, dtype=np.float64)) for v in (x0, x1, u0, u1)],
                          (_DP * 3)(*[_ptr(j0[a]) for a in range(3)]), (_DP * 3)(*[_ptr(j1[a]) for a in range(3)]))
        return j0, j1

    def set_soft_source(self, S: SourceSpec | None):
        """Laser entering through an x-plane for the following steps (None: off)."""
        if S is None:
            self.src = None
            return
        n0 = self.grid.n[0]
        if not (1 <= S.plane <= n0 - 1) or S.pol[0] != 0 or not S.k > 0:
            raise ValueError("invalid soft source")
        self.src = _Source(S.amplitude, S.k, (C.c_double * 3)(*S.pol), (C.c_double * 3)(*S.centre), S.waist,
                           S.duration, S.t_centre, S.phase, int(S.plane))

    def current(self):
        """J^n (without g) at the E locations, shape (3, nz, ny, nx)."""
        J = np.zeros((3,) + self.phi_cur.shape)
        arr = (_DP * 3)(*[_ptr(J[a]) for a in range(3)])
        st = self._state()
        lib().orc_current(C.byref(self.p), C.byref(st), arr)
        return J

    def source_now(self):
        S = np.zeros(self.phi_cur.shape)
        st = self._state()
        lib().orc_source_now(C.byref(self.p), C.byref(st), _ptr(S))
        return S

    def gauss_residual(self):
        R = np.zeros(self.phi_cur.shape)
        st = self._state()
        lib().orc_gauss_residual(C.byref(self.p), C.byref(st), _ptr(R))
        return R

    def diagnostics(self) -> dict:
        d = _Diag()
        st = self._state()
        lib().orc_diagnostics(C.byref(self.p), C.byref(st), C.byref(d))
        return {name: getattr(d, name) for name, _ in _Diag._fields_}

    def inject_laser(self, L: LaserSpec):
        c = _Laser(L.amplitude, (C.c_double * 3)(*L.k), (C.c_double * 3)(*L.pol), (C.c_double * 3)(*L.centre),
                   L.waist, L.duration, L.phase)
        st = self._state()
        lib().orc_inject_laser(C.byref(self.p), C.byref(st), C.byref(c))

    def inject_axion(self, A: AxionSpec):
        c = _Axion(A.amplitude, (C.c_double * 3)(*A.k), (C.c_double * 3)(*A.centre), A.waist, A.length, A.speed,
                   A.phase)
        st = self._state()
        lib().orc_inject_axion(C.byref(self.p), C.byref(st), C.byref(c))

    def sigma(self, i, j, k, axion=True):
        return lib().orc_sigma_cell(C.byref(self.p), i, j, k, 1 if axion else 0)

    def fields(self) -> dict:
        out = {k: v.copy() for k, v in self.f.items()}
        out["phi_cur"] = self.phi_cur.copy()
        out["phi_old"] = self.phi_old.copy()
        return out


def kick(q_over_m, dt, u0, u1, Enop, Bnop, Ep, Bp):
    """One Boris momentum update of order 0 and its first-order part: (u0', u1')."""
    o0, o1 = np.zeros(3), np.zeros(3)
    lib().orc_kick(float(q_over_m), float(dt), *[_ptr(np.array(v, dtype=np.float64)) for v in
                                                 (u0, u1, Enop, Bnop, Ep, Bp)], _ptr(o0), _ptr(o1))
    return o0, o1


def outflow_solve(dt, dxa, m, g_cur, g_old, p0_cur, S_g):
    V, U = C.c_double(), C.c_double()
    lib().orc_outflow_solve(dt, dxa, m, g_cur, g_old, p0_cur, S_g, C.byref(V), C.byref(U))
    return V.value, U.value


def run_workload(w, steps=None, grid=None):
    """Set up a workload's initial condition and advance it; returns the OracleGrid."""
    og = OracleGrid(grid or w.grid)
    for L in w.lasers:
        og.inject_laser(L)
    for A in w.axions:
        og.inject_axion(A)
    og.step(w.steps if steps is None else steps)
    return og

"""Python binding of the C ABI in include/axp.h (argument marshalling only).

Every function of the header is exposed under the same name; all compute
runs in libaxp.so's CUDA kernels.  PyTorch supplies device memory (the grid
workspace is a torch uint8 tensor) and the CUDA stream.  There is no CPU
fallback: importing this module on a machine where libaxp.so cannot be
loaded raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build
from .workloads import BC_CODE, AxionSpec, GridSpec, LaserSpec, SourceSpec

AXP_OK, AXP_E_INVAL, AXP_E_UNSTABLE, AXP_E_NOMEM, AXP_E_CUDA, AXP_E_TIMEOUT, AXP_E_NONFINITE, AXP_E_STATE = range(8)
AXP_FP64, AXP_FP32_SPLIT = 0, 1
AXP_KERNEL_AUTO, AXP_KERNEL_GENERAL, AXP_KERNEL_FUSED, AXP_KERNEL_TM2D, AXP_KERNEL_AX3D, AXP_KERNEL_BLOCK1D = 0, 1, 2, 3, 4, 5
AXP_KERNEL_TM2D_LIST = 6
FIELD_IDS = {n: i for i, n in enumerate(("E0x", "E0y", "E0z", "B0x", "B0y", "B0z",
                                          "E1x", "E1y", "E1z", "B1x", "B1y", "B1z"))}
FIELD_IDS["phi_cur"] = 12
FIELD_IDS["phi_old"] = 13


class AxpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, axp_status_str(status), status))


class axp_grid_desc(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("d", C.c_double * 3), ("lo", C.c_double * 3), ("dt", C.c_double),
                ("m", C.c_double), ("g", C.c_double), ("axion_bc", (C.c_int32 * 2) * 3),
                ("em_bc", (C.c_int32 * 2) * 3), ("pml_cells", C.c_int32), ("precision", C.c_int32),
                ("pml_sigma_max_dt", C.c_double), ("diag_every", C.c_int32), ("diag_capacity", C.c_int32)]


class axp_laser_desc(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double * 3), ("pol", C.c_double * 3),
                ("centre", C.c_double * 3), ("waist", C.c_double), ("duration", C.c_double),
                ("phase", C.c_double)]


class axp_axion_desc(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double * 3), ("centre", C.c_double * 3),
                ("waist", C.c_double), ("length", C.c_double), ("speed", C.c_double), ("phase", C.c_double)]


class axp_source_desc(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("k", C.c_double), ("pol", C.c_double * 3), ("centre", C.c_double * 3),
                ("waist", C.c_double), ("duration", C.c_double), ("t_centre", C.c_double), ("phase", C.c_double),
                ("plane", C.c_int64)]


class axp_diag(C.Structure):
    _fields_ = [("step", C.c_int64)] + [(n, C.c_double) for n in (
        "t", "H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "W", "sum_xB1z2", "sum_B1z2", "gauss_l2")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_P = C.c_void_p
_D3 = C.c_double * 3


def lib():
    """Load libaxp.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        L = C.CDLL(path)
        sig = {
            "axp_status_str": ([C.c_int], C.c_char_p),
            "axp_workspace_bytes": ([C.POINTER(axp_grid_desc), C.POINTER(C.c_size_t)], C.c_int),
            "axp_create_grid": ([C.POINTER(axp_grid_desc), _P, C.c_size_t, _P, C.POINTER(_P)], C.c_int),
            "axp_destroy_grid": ([_P], C.c_int),
            "axp_set_background_field": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
            "axp_inject_laser": ([_P, C.POINTER(axp_laser_desc)], C.c_int),
            "axp_inject_axion": ([_P, C.POINTER(axp_axion_desc)], C.c_int),
            "axp_set_soft_source": ([_P, C.POINTER(axp_source_desc)], C.c_int),
            "axp_step": ([_P, C.c_int64], C.c_int),
            "axp_read_diagnostics": ([_P, C.POINTER(axp_diag), C.c_int64, C.POINTER(C.c_int64)], C.c_int),
            "axp_compute_diagnostics": ([_P, C.POINTER(axp_diag)], C.c_int),
            "axp_diagnostics_noalloc": ([C.POINTER(axp_grid_desc), C.POINTER(C.c_void_p), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.c_int64, _P, C.POINTER(axp_diag)], C.c_int),
            "axp_read_field": ([_P, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_write_field": ([_P, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_read_ghost": ([_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_write_ghost": ([_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_state_bytes": ([_P, C.POINTER(C.c_size_t)], C.c_int),
            "axp_save_state": ([_P, _P, C.c_size_t], C.c_int),
            "axp_load_state": ([_P, _P, C.c_size_t], C.c_int),
            "axp_get_step": ([_P, C.POINTER(C.c_int64)], C.c_int),
            "axp_synchronize": ([_P], C.c_int),
            "axp_set_kernel": ([_P, C.c_int32], C.c_int),
            "axp_shift_window": ([_P, C.c_int32, C.c_int64], C.c_int),
            "axp_set_moving_window": ([_P, C.c_int32, C.c_double, C.c_int32, C.c_int64], C.c_int),
            "axp_get_window_offset": ([_P, C.POINTER(C.c_int64)], C.c_int),
            "axp_get_kernel_path": ([_P, C.POINTER(C.c_int32)], C.c_int),
            "axp_get_launch_count": ([_P, C.POINTER(C.c_int64)], C.c_int),
            "axp_test_block1d_absent": ([_P, C.c_int32], C.c_int),
            "axp_rows_bytes": ([_P, C.c_int64, C.POINTER(C.c_size_t)], C.c_int),
            "axp_pack_rows": ([_P, C.c_int64, C.c_int64, _P, C.c_size_t], C.c_int),
            "axp_unpack_rows": ([_P, C.c_int64, C.c_int64, _P, C.c_size_t], C.c_int),
            "axp_compute_diagnostics_rows": ([_P, C.c_int64, C.c_int64, C.POINTER(axp_diag)], C.c_int),
            "axp_particles_bytes": ([_P, C.c_int64, C.POINTER(C.c_size_t)], C.c_int),
            "axp_attach_particles": ([_P, C.c_int64, C.c_double, C.c_double, _P, C.c_size_t], C.c_int),
            "axp_write_particles": ([_P, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_read_particles": ([_P, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_read_particle_current": ([_P, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_detach_particles": ([_P], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    """Names of the functions declared in include/axp.h."""
    hdr = open(os.path.join(_build.INCLUDE, "axp.h")).read()
    import re

    return sorted(set(re.findall(r"\b(axp_[a-z_]+)\s*\(", hdr)))


def _check(st, where):
    if st != AXP_OK:
        raise AxpError(st, where)


# ---- same-name wrappers (marshalling only) ----

def axp_status_str(st):
    return lib().axp_status_str(int(st)).decode()


def axp_workspace_bytes(desc):
    n = C.c_size_t()
    _check(lib().axp_workspace_bytes(C.byref(desc), C.byref(n)), "axp_workspace_bytes")
    return n.value


def axp_create_grid(desc, dev_ptr, nbytes, stream_ptr):
    h = _P()
    _check(lib().axp_create_grid(C.byref(desc), _P(dev_ptr), nbytes, _P(stream_ptr), C.byref(h)), "axp_create_grid")
    return h


def axp_destroy_grid(h):
    _check(lib().axp_destroy_grid(h), "axp_destroy_grid")


def axp_set_background_field(h, B_ext=None, E_ext=None):
    b = _D3(*B_ext) if B_ext is not None else None
    e = _D3(*E_ext) if E_ext is not None else None
    _check(lib().axp_set_background_field(h, b, e), "axp_set_background_field")


def axp_inject_laser(h, laser: axp_laser_desc):
    _check(lib().axp_inject_laser(h, C.byref(laser)), "axp_inject_laser")


def axp_inject_axion(h, ax: axp_axion_desc):
    _check(lib().axp_inject_axion(h, C.byref(ax)), "axp_inject_axion")


def axp_set_soft_source(h, src):
    _check(lib().axp_set_soft_source(h, C.byref(src) if src is not None else None), "axp_set_soft_source")


def axp_step(h, nsteps):
    _check(lib().axp_step(h, int(nsteps)), "axp_step")


def axp_read_diagnostics(h, max_records=4096):
    buf = (axp_diag * max(1, max_records))()
    n = C.c_int64()
    _check(lib().axp_read_diagnostics(h, buf, int(max_records), C.byref(n)), "axp_read_diagnostics")
    return [buf[i].as_dict() for i in range(n.value)]


def axp_compute_diagnostics(h):
    d = axp_diag()
    _check(lib().axp_compute_diagnostics(h, C.byref(d)), "axp_compute_diagnostics")
    return d.as_dict()


def axp_diagnostics_noalloc(desc, dev_ptrs, B_ext, E_ext, step, stream_ptr):
    """Diagnostics of caller-held FP64 device fields without any device allocation.
    dev_ptrs: 14 device addresses (E0xyz, B0xyz, E1xyz, B1xyz, phi^{n+1/2}, phi^{n-1/2})."""
    ptrs = (C.c_void_p * 14)(*[int(p) for p in dev_ptrs])
    d = axp_diag()
    _check(lib().axp_diagnostics_noalloc(C.byref(desc), ptrs, _D3(*B_ext), _D3(*E_ext), int(step),
                                         _P(stream_ptr), C.byref(d)), "axp_diagnostics_noalloc")
    return d.as_dict()


def axp_read_field(h, which, ncells):
    out = np.empty(ncells, dtype=np.float64)
    _check(lib().axp_read_field(h, int(which), out.ctypes.data_as(C.POINTER(C.c_double)), out.nbytes),
           "axp_read_field")
    return out


def axp_write_field(h, which, values):
    a = np.ascontiguousarray(values, dtype=np.float64).ravel()
    _check(lib().axp_write_field(h, int(which), a.ctypes.data_as(C.POINTER(C.c_double)), a.nbytes),
           "axp_write_field")


def axp_read_ghost(h, axis, side, level, nplane):
    out = np.empty(nplane, dtype=np.float64)
    _check(lib().axp_read_ghost(h, axis, side, level, out.ctypes.data_as(C.POINTER(C.c_double)), out.nbytes),
           "axp_read_ghost")
    return out


def axp_write_ghost(h, axis, side, level, values):
    a = np.ascontiguousarray(values, dtype=np.float64).ravel()
    _check(lib().axp_write_ghost(h, axis, side, level, a.ctypes.data_as(C.POINTER(C.c_double)), a.nbytes),
           "axp_write_ghost")


def axp_state_bytes(h):
    n = C.c_size_t()
    _check(lib().axp_state_bytes(h, C.byref(n)), "axp_state_bytes")
    return n.value


def axp_save_state(h, host_ptr, nbytes):
    _check(lib().axp_save_state(h, _P(host_ptr), nbytes), "axp_save_state")


def axp_load_state(h, host_ptr, nbytes):
    _check(lib().axp_load_state(h, _P(host_ptr), nbytes), "axp_load_state")


def axp_get_step(h):
    n = C.c_int64()
    _check(lib().axp_get_step(h, C.byref(n)), "axp_get_step")
    return n.value


def axp_synchronize(h):
    _check(lib().axp_synchronize(h), "axp_synchronize")


def axp_set_kernel(h, k):
    _check(lib().axp_set_kernel(h, int(k)), "axp_set_kernel")


def axp_shift_window(h, axis, cells):
    _check(lib().axp_shift_window(h, int(axis), int(cells)), "axp_shift_window")


def axp_set_moving_window(h, axis, velocity, shift_cells=1, start_step=0):
    _check(lib().axp_set_moving_window(h, int(axis), float(velocity), int(shift_cells), int(start_step)),
           "axp_set_moving_window")


def axp_get_window_offset(h):
    n = C.c_int64()
    _check(lib().axp_get_window_offset(h, C.byref(n)), "axp_get_window_offset")
    return n.value


def axp_get_kernel_path(h):
    p = C.c_int32()
    _check(lib().axp_get_kernel_path(h, C.byref(p)), "axp_get_kernel_path")
    return p.value


def axp_get_launch_count(h):
    n = C.c_int64()
    _check(lib().axp_get_launch_count(h, C.byref(n)), "axp_get_launch_count")
    return n.value


def axp_rows_bytes(h, nrows):
    n = C.c_size_t()
    _check(lib().axp_rows_bytes(h, int(nrows), C.byref(n)), "axp_rows_bytes")
    return n.value


def axp_pack_rows(h, row0, nrows, dev_ptr, nbytes):
    _check(lib().axp_pack_rows(h, int(row0), int(nrows), _P(dev_ptr), nbytes), "axp_pack_rows")


def axp_unpack_rows(h, row0, nrows, dev_ptr, nbytes):
    _check(lib().axp_unpack_rows(h, int(row0), int(nrows), _P(dev_ptr), nbytes), "axp_unpack_rows")


def axp_compute_diagnostics_rows(h, row0, row1):
    d = axp_diag()
    _check(lib().axp_compute_diagnostics_rows(h, int(row0), int(row1), C.byref(d)), "axp_compute_diagnostics_rows")
    return d.as_dict()


def axp_test_block1d_absent(h, block):
    _check(lib().axp_test_block1d_absent(h, int(block)), "axp_test_block1d_absent")


# ---- descriptors from the workload specs ----

def axp_particles_bytes(h, count):
    n = C.c_size_t()
    _check(lib().axp_particles_bytes(h, int(count), C.byref(n)), "axp_particles_bytes")
    return n.value


def axp_attach_particles(h, count, q, m, dev_ptr, nbytes):
    _check(lib().axp_attach_particles(h, int(count), float(q), float(m), dev_ptr, nbytes), "axp_attach_particles")


def axp_write_particles(h, rows: np.ndarray):
    a = np.ascontiguousarray(rows, dtype=np.float64)
    _check(lib().axp_write_particles(h, a.ctypes.data_as(C.POINTER(C.c_double)), a.nbytes), "axp_write_particles")


def axp_read_particles(h, count):
    out = np.empty((13, int(count)), dtype=np.float64)
    _check(lib().axp_read_particles(h, out.ctypes.data_as(C.POINTER(C.c_double)), out.nbytes), "axp_read_particles")
    return out


def axp_read_particle_current(h, order, ncells):
    out = np.empty((3, int(ncells)), dtype=np.float64)
    _check(lib().axp_read_particle_current(h, int(order), out.ctypes.data_as(C.POINTER(C.c_double)), out.nbytes),
           "axp_read_particle_current")
    return out


def axp_detach_particles(h):
    _check(lib().axp_detach_particles(h), "axp_detach_particles")


def desc_of(grid: GridSpec, diag_every=0, diag_capacity=0) -> axp_grid_desc:
    d = axp_grid_desc()
    for a in range(3):
        d.n[a] = int(grid.n[a])
        d.d[a] = float(grid.d[a])
        d.lo[a] = float(grid.lo[a])
        for s in range(2):
            d.axion_bc[a][s] = BC_CODE[grid.axion_bc[a][s]]
            d.em_bc[a][s] = BC_CODE[grid.em_bc[a][s]]
    d.dt, d.m, d.g = float(grid.dt), float(grid.m), float(grid.g)
    d.pml_cells = int(grid.pml_cells)
    d.precision = AXP_FP32_SPLIT if grid.precision == "fp32" else AXP_FP64
    d.pml_sigma_max_dt = float(grid.pml_sigma_max_dt)
    d.diag_every = int(diag_every)
    d.diag_capacity = int(diag_capacity if diag_capacity else (1 if diag_every else 0))
    return d


def laser_of(L: LaserSpec) -> axp_laser_desc:
    return axp_laser_desc(L.amplitude, _D3(*L.k), _D3(*L.pol), _D3(*L.centre), L.waist, L.duration, L.phase)


def source_of(S: SourceSpec) -> axp_source_desc:
    return axp_source_desc(S.amplitude, S.k, _D3(*S.pol), _D3(*S.centre), S.waist, S.duration, S.t_centre, S.phase,
                           int(S.plane))


def axion_of(A: AxionSpec) -> axp_axion_desc:
    return axp_axion_desc(A.amplitude, _D3(*A.k), _D3(*A.centre), A.waist, A.length, A.speed, A.phase)


class Grid:
    """A grid whose workspace is a torch CUDA tensor; a thin owner of one handle."""

    def __init__(self, grid: GridSpec, diag_every=0, diag_capacity=0, stream=None, device=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("axp needs a CUDA device; there is no CPU fallback")
        self.spec = grid
        self.desc = desc_of(grid, diag_every, diag_capacity)
        self.nbytes = axp_workspace_bytes(self.desc)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.h = axp_create_grid(self.desc, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)
        axp_set_background_field(self.h, grid.B_ext, grid.E_ext)
        self.cells = grid.cells
        self.shape = (grid.n[2], grid.n[1], grid.n[0])

    def close(self):
        if getattr(self, "h", None):
            axp_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def inject_laser(self, L: LaserSpec):
        axp_inject_laser(self.h, laser_of(L))

    def inject_axion(self, A: AxionSpec):
        axp_inject_axion(self.h, axion_of(A))

    def set_soft_source(self, S: SourceSpec | None):
        """Laser entering through an x-plane for the following steps (None: off)."""
        axp_set_soft_source(self.h, source_of(S) if S is not None else None)

    def step(self, n=1):
        axp_step(self.h, n)

    def synchronize(self):
        axp_synchronize(self.h)

    def diagnostics(self):
        return axp_compute_diagnostics(self.h)

    def read_diagnostics(self, max_records=4096):
        return axp_read_diagnostics(self.h, max_records)

    def read(self, name):
        return axp_read_field(self.h, FIELD_IDS[name], self.cells).reshape(self.shape)

    def write(self, name, values):
        axp_write_field(self.h, FIELD_IDS[name], values)

    def load(self, state: dict):
        for k, v in state.items():
            self.write(k, v)

    def fields(self):
        return {k: self.read(k) for k in FIELD_IDS}

    def plane(self, a):
        nx, ny, nz = self.spec.n
        return {0: ny * nz, 1: nx * nz, 2: nx * ny}[a]

    def read_ghost(self, axis, side, level):
        return axp_read_ghost(self.h, axis, side, level, self.plane(axis))

    def write_ghost(self, axis, side, level, values):
        axp_write_ghost(self.h, axis, side, level, values)

    def shift_window(self, axis, cells):
        axp_shift_window(self.h, axis, cells)

    def set_moving_window(self, axis, velocity=1.0, shift_cells=1, start_step=0):
        axp_set_moving_window(self.h, axis, velocity, shift_cells, start_step)

    def window_offset(self):
        return axp_get_window_offset(self.h)

    def set_kernel(self, k):
        axp_set_kernel(self.h, k)

    def kernel_path(self):
        return axp_get_kernel_path(self.h)

    def launches(self):
        return axp_get_launch_count(self.h)

    @property
    def step_count(self):
        return axp_get_step(self.h)

    def save_state(self):
        n = axp_state_bytes(self.h)
        buf = np.empty(n, dtype=np.uint8)
        axp_save_state(self.h, buf.ctypes.data, n)
        return buf

    def load_state(self, buf: np.ndarray):
        axp_load_state(self.h, buf.ctypes.data, buf.nbytes)

    # -- macroparticles (perturbed-particle current) --
    def attach_particles(self, q, m, w, x0, u0, x1=None, u1=None):
        """One species: weights w (count,), positions x0, x1 and momenta u0, u1
        (3, count) at the present time step; the workspace is a torch tensor."""
        import torch

        w = np.asarray(w, dtype=np.float64)
        n = w.shape[0]
        z = np.zeros((3, n))
        rows = np.concatenate([w[None], np.asarray(x0, dtype=np.float64).reshape(3, n),
                               np.asarray(u0, dtype=np.float64).reshape(3, n),
                               z if x1 is None else np.asarray(x1, dtype=np.float64).reshape(3, n),
                               z if u1 is None else np.asarray(u1, dtype=np.float64).reshape(3, n)])
        nbytes = axp_particles_bytes(self.h, n)
        with torch.cuda.device(self.device):
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        # the workspace of particles already attached stays referenced when this is refused
        axp_attach_particles(self.h, n, q, m, ws.data_ptr(), nbytes)
        self.particle_ws = ws
        self.particle_count = n
        axp_write_particles(self.h, rows)

    def write_particles(self, rows: np.ndarray):
        axp_write_particles(self.h, rows)

    def read_particles(self) -> dict:
        """Positions and momenta at the present time step: w, x0, u0, x1, u1."""
        r = axp_read_particles(self.h, self.particle_count)
        return {"w": r[0], "x0": r[1:4], "u0": r[4:7], "x1": r[7:10], "u1": r[10:13]}

    def particle_current(self, order):
        """j^n of order 0 or 1, shape (3, nz, ny, nx)."""
        return axp_read_particle_current(self.h, order, self.cells).reshape((3,) + self.shape)

    def detach_particles(self):
        axp_detach_particles(self.h)
        self.particle_ws = None

"""Groups of 2D grids stepped together: binding of the axp_group_* C ABI.

All compute runs in libaxp.so; PyTorch provides the workspace and the stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import axp as _axp

_P = C.c_void_p
_sig_done = False


def lib():
    global _sig_done
    L = _axp.lib()
    if not _sig_done:
        sig = {
            "axp_group_workspace_bytes": ([C.c_int32, C.c_int32, C.POINTER(C.c_size_t)], C.c_int),
            "axp_group_create": ([C.c_int32, C.c_int32, _P, C.c_size_t, _P, C.POINTER(_P)], C.c_int),
            "axp_group_destroy": ([_P], C.c_int),
            "axp_group_add": ([_P, _P, C.c_int64, C.POINTER(C.c_int32)], C.c_int),
            "axp_group_remove": ([_P, C.c_int32], C.c_int),
            "axp_group_run": ([_P, C.c_int64], C.c_int),
            "axp_group_progress": ([_P, C.POINTER(C.c_int64), C.c_int32], C.c_int),
            "axp_group_set_chunk": ([_P, C.c_int32], C.c_int),
            "axp_group_use_graphs": ([_P, C.c_int32], C.c_int),
            "axp_group_launch_count": ([_P, C.POINTER(C.c_int64)], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _sig_done = True
    return L


def _check(st, where):
    if st != _axp.AXP_OK:
        raise _axp.AxpError(st, where)


def axp_group_workspace_bytes(max_grids, max_tiles):
    n = C.c_size_t()
    _check(lib().axp_group_workspace_bytes(int(max_grids), int(max_tiles), C.byref(n)), "axp_group_workspace_bytes")
    return n.value


# written columns per tile of the group kernel: 250 for a member of even width
# (two columns per thread), 123 for one of odd width; the library's own count
# decides admission (axp_group_add refuses a member beyond max_tiles)
VX_EVEN, VX_ODD = 250, 123


def tiles_of(nx, ny, chunk=64):
    vx = VX_EVEN if nx % 2 == 0 else VX_ODD
    return -(-nx // vx) * -(-ny // chunk)


class Group:
    """Up to max_grids FP32-split 2D grids (axp.Grid objects) advanced together."""

    def __init__(self, max_grids, max_tiles, stream=None, graphs=False, chunk=None):
        import torch

        self.nbytes = axp_group_workspace_bytes(max_grids, max_tiles)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        torch.cuda.current_stream().synchronize()
        h = _P()
        _check(lib().axp_group_create(int(max_grids), int(max_tiles), _P(self.workspace.data_ptr()), self.nbytes,
                                      _P(self.stream.cuda_stream), C.byref(h)), "axp_group_create")
        self.h = h
        self.max_grids = max_grids
        self.members = {}
        if chunk is not None:
            _check(lib().axp_group_set_chunk(self.h, int(chunk)), "axp_group_set_chunk")
        if graphs:
            _check(lib().axp_group_use_graphs(self.h, 1), "axp_group_use_graphs")

    def add(self, grid, steps):
        """Join an axp.Grid for `steps` more steps; returns its member index, or
        None when the group has no room (AXP_E_NOMEM)."""
        m = C.c_int32()
        st = lib().axp_group_add(self.h, grid.h, int(steps), C.byref(m))
        if st == _axp.AXP_E_NOMEM:
            return None
        _check(st, "axp_group_add")
        self.members[m.value] = grid
        return m.value

    def remove(self, member):
        _check(lib().axp_group_remove(self.h, int(member)), "axp_group_remove")
        return self.members.pop(member)

    def run(self, nsteps):
        _check(lib().axp_group_run(self.h, int(nsteps)), "axp_group_run")

    def progress(self):
        buf = (C.c_int64 * self.max_grids)()
        _check(lib().axp_group_progress(self.h, buf, self.max_grids), "axp_group_progress")
        return np.frombuffer(buf, dtype=np.int64).copy()

    def launches(self):
        n = C.c_int64()
        _check(lib().axp_group_launch_count(self.h, C.byref(n)), "axp_group_launch_count")
        return n.value

    def close(self):
        if getattr(self, "h", None):
            for m in list(self.members):
                self.remove(m)
            lib().axp_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Batches of 1D conversion runs: binding of the axp_batch_* C ABI, the tiling
autotuner, and the parameter-scan driver.

All compute runs in libaxp.so; PyTorch provides the workspace and the stream.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import axp as _axp
from .workloads import ScanInstance

_P = C.c_void_p


class axp_batch_instance(C.Structure):
    _fields_ = [("nx", C.c_int64), ("dx", C.c_double), ("dt", C.c_double), ("m", C.c_double), ("g", C.c_double),
                ("By", C.c_double), ("Bz", C.c_double), ("amplitude", C.c_double), ("k", C.c_double),
                ("steps", C.c_int64)]


_sig_done = False


def lib():
    global _sig_done
    L = _axp.lib()
    if not _sig_done:
        sig = {
            "axp_batch_workspace_bytes": ([C.c_int32, C.c_int64, C.POINTER(C.c_size_t)], C.c_int),
            "axp_batch_create": ([C.c_int32, C.c_int64, _P, C.c_size_t, _P, C.POINTER(_P)], C.c_int),
            "axp_batch_destroy": ([_P], C.c_int),
            "axp_batch_add": ([_P, C.POINTER(axp_batch_instance), C.POINTER(C.c_int32)], C.c_int),
            "axp_batch_remove": ([_P, C.c_int32], C.c_int),
            "axp_batch_run": ([_P, C.c_int64], C.c_int),
            "axp_batch_progress": ([_P, C.POINTER(C.c_int64), C.c_int32], C.c_int),
            "axp_batch_result": ([_P, C.c_int32, C.POINTER(_axp.axp_diag)], C.c_int),
            "axp_batch_results": ([_P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(_axp.axp_diag)], C.c_int),
            "axp_batch_read_state": ([_P, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "axp_batch_set_tiling": ([_P, C.c_int32, C.c_int32, C.c_int32], C.c_int),
            "axp_batch_get_tiling": ([_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
            "axp_batch_use_graphs": ([_P, C.c_int32], C.c_int),
            "axp_batch_launch_count": ([_P, C.POINTER(C.c_int64)], C.c_int),
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


def axp_batch_workspace_bytes(max_instances, max_cells):
    n = C.c_size_t()
    _check(lib().axp_batch_workspace_bytes(int(max_instances), int(max_cells), C.byref(n)), "axp_batch_workspace_bytes")
    return n.value


def instance_of(nx, dx, dt, m, g, By, Bz, amplitude, k, steps):
    return axp_batch_instance(int(nx), dx, dt, m, g, By, Bz, amplitude, k, int(steps))


def scan_instance(inst: ScanInstance, cfl=0.95, amplitude=1e-3):
    """The 1D conversion set-up for one scan draw: dx = lambda/32, a whole number of
    wavelengths in the box (the nearest to the box length), B_ext along y."""
    dx = 1.0 / 32.0
    waves = max(1, round(inst.nx * dx))
    k = 2.0 * math.pi * waves / (inst.nx * dx)
    return instance_of(inst.nx, dx, cfl * dx, inst.m, inst.g, inst.B0, 0.0, amplitude, k, inst.steps)


class Batch:
    """Slots for up to max_instances 1D runs totalling max_cells cells."""

    def __init__(self, max_instances, max_cells, stream=None, graphs=False):
        import torch

        self.nbytes = axp_batch_workspace_bytes(max_instances, max_cells)
        # a stream of its own (graph capture needs a non-default stream)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        # the allocation is ordered on the current stream; the batch works on its own
        torch.cuda.current_stream().synchronize()
        h = _P()
        _check(lib().axp_batch_create(int(max_instances), int(max_cells), _P(self.workspace.data_ptr()), self.nbytes,
                                      _P(self.stream.cuda_stream), C.byref(h)), "axp_batch_create")
        self.h = h
        self.max_instances = max_instances
        self.nx = {}
        if graphs:
            self.use_graphs(True)

    def use_graphs(self, enable=True):
        _check(lib().axp_batch_use_graphs(self.h, 1 if enable else 0), "axp_batch_use_graphs")

    def launches(self):
        n = C.c_int64()
        _check(lib().axp_batch_launch_count(self.h, C.byref(n)), "axp_batch_launch_count")
        return n.value

    def close(self):
        if getattr(self, "h", None):
            lib().axp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, inst: axp_batch_instance):
        s = C.c_int32()
        _check(lib().axp_batch_add(self.h, C.byref(inst), C.byref(s)), "axp_batch_add")
        self.nx[s.value] = inst.nx
        return s.value

    def try_add(self, inst):
        s = C.c_int32()
        st = lib().axp_batch_add(self.h, C.byref(inst), C.byref(s))
        if st == _axp.AXP_E_NOMEM:
            return None
        _check(st, "axp_batch_add")
        self.nx[s.value] = inst.nx
        return s.value

    def remove(self, slot):
        _check(lib().axp_batch_remove(self.h, int(slot)), "axp_batch_remove")
        self.nx.pop(slot, None)

    def run(self, nsteps):
        _check(lib().axp_batch_run(self.h, int(nsteps)), "axp_batch_run")

    def progress(self):
        buf = (C.c_int64 * self.max_instances)()
        _check(lib().axp_batch_progress(self.h, buf, self.max_instances), "axp_batch_progress")
        return np.frombuffer(buf, dtype=np.int64).copy()

    def result(self, slot):
        d = _axp.axp_diag()
        _check(lib().axp_batch_result(self.h, int(slot), C.byref(d)), "axp_batch_result")
        return d.as_dict()

    def results(self, slots):
        """result() of several slots in one launch and one synchronisation."""
        slots = [int(x) for x in slots]
        if not slots:
            return []
        arr = (C.c_int32 * len(slots))(*slots)
        out = (_axp.axp_diag * len(slots))()
        _check(lib().axp_batch_results(self.h, arr, len(slots), out), "axp_batch_results")
        return [d.as_dict() for d in out]

    def read_state(self, slot, which):
        n = self.nx[slot]
        out = np.empty(n, dtype=np.float64)
        _check(lib().axp_batch_read_state(self.h, int(slot), int(which), out.ctypes.data_as(C.POINTER(C.c_double)),
                                          out.nbytes), "axp_batch_read_state")
        return out

    def set_tiling(self, block_steps, segment_cells, threads):
        _check(lib().axp_batch_set_tiling(self.h, int(block_steps), int(segment_cells), int(threads)),
               "axp_batch_set_tiling")

    def tiling(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().axp_batch_get_tiling(self.h, C.byref(a), C.byref(b), C.byref(c)), "axp_batch_get_tiling")
        return a.value, b.value, c.value

    def autotune(self, probe_steps=64, candidates=None):
        """Time each candidate tiling on the batch as it stands (the probe steps are
        real steps: every tiling gives bit-identical results) and keep the fastest.
        Returns (best tiling, {tiling: seconds per probe})."""
        import torch

        if candidates is None:
            # segments that fill a block's 8 cells per thread with their halo
            candidates = [(bs, 8 * th - 6 * bs, th) for th in (256, 512) for bs in (16, 32, 48, 64)]
        times = {}
        for cand in candidates:
            self.set_tiling(*cand)
            self.run(min(probe_steps, cand[0]))  # rebuild the work table outside the timing
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(self.stream)
            self.run(probe_steps)
            ev1.record(self.stream)
            ev1.synchronize()
            times[cand] = ev0.elapsed_time(ev1) / 1e3
        best = min(times, key=times.get)
        self.set_tiling(*best)
        return best, times


def run_scan(instances, max_cells=None, tune=True, chunk_steps=1024, graphs=True, tiling=None, phases=None):
    """Admit every instance, run them all to completion, return (results per instance
    index, wall seconds from the first admission to the last result, tiling).  The
    autotuner's probe steps are real steps and are inside the timing.  A given
    `tiling` (block_steps, segment_cells, threads) is used as it is, untuned.  A dict
    passed as `phases` receives the wall seconds of admission, tuning, stepping and
    read-out, and the device seconds of the stepping (CUDA events on the batch's stream)."""
    import torch

    total = sum(i.nx for i in instances)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = Batch(len(instances), max_cells or total, graphs=graphs)
    slots = [b.add(i) for i in instances]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if tiling is not None:
        b.set_tiling(*tiling)
    elif tune:
        tiling, _ = b.autotune()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(b.stream)
    while True:
        done = b.progress()
        rem = max(int(inst.steps) - int(done[s]) for inst, s in zip(instances, slots))
        if rem <= 0:
            break
        b.run(min(rem, chunk_steps))
    ev1.record(b.stream)
    ev1.synchronize()
    t3 = time.perf_counter()
    res = b.results(slots)
    el = time.perf_counter() - t0
    if phases is not None:
        phases.update(admit_s=t1 - t0, tune_s=t2 - t1, steps_s=t3 - t2, readout_s=el - (t3 - t0),
                      steps_device_s=ev0.elapsed_time(ev1) / 1e3)
    b.close()
    return res, el, tiling or b.tiling()

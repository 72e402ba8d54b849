"""The C-ABI library builds, loads and exports every function include/axp.h
declares; descriptor validation is host logic and runs without a GPU."""
import ctypes as C
import math
import re
import subprocess

import pytest

from paper_2406_16796_gb300 import _build, axp
from paper_2406_16796_gb300 import workloads as W


def header_functions():
    src = open(_build.INCLUDE + "/axp.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(axp_[a-z0-9_]+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    L = axp.lib()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (axp_[a-z0-9_]+)\b", out))
    assert set(names) <= exported


def test_status_strings():
    for s in range(8):
        assert axp.axp_status_str(s)


def _desc(**kw):
    w = W.pulse_2d(nx=64, ny=32)
    return axp.desc_of(w.grid.replace(**kw))


def test_workspace_bytes_and_layout_grow_with_size():
    a = axp.axp_workspace_bytes(_desc())
    b = axp.axp_workspace_bytes(axp.desc_of(W.pulse_2d(nx=128, ny=32).grid))
    assert b > a > 12 * 64 * 32 * 8
    f = axp.axp_workspace_bytes(_desc(precision="fp32"))
    assert f < a


def test_stability_bounds_are_enforced():
    w = W.vacuum_1d(nx=64)
    ok = axp.desc_of(w.grid.replace(dt=w.grid.d[0] * 0.999))
    axp.axp_workspace_bytes(ok)
    with pytest.raises(axp.AxpError) as e:
        axp.axp_workspace_bytes(axp.desc_of(w.grid.replace(dt=w.grid.d[0] * 1.001)))
    assert e.value.status == axp.AXP_E_UNSTABLE
    # axion bound dt^2 (4/dx^2 + m^2) <= 4 with a heavy axion
    with pytest.raises(axp.AxpError) as e:
        axp.axp_workspace_bytes(axp.desc_of(w.grid.replace(dt=w.grid.d[0] * 0.99, m=20.0)))
    assert e.value.status == axp.AXP_E_UNSTABLE


@pytest.mark.parametrize("bad", ["periodic_mismatch", "size1_nonperiodic", "em_outflow", "n0", "pml_too_thick"])
def test_invalid_descriptors(bad):
    g = W.pulse_2d(nx=64, ny=32).grid
    if bad == "periodic_mismatch":
        g = g.replace(axion_bc=W._bcs("periodic", "pml"))
    elif bad == "size1_nonperiodic":
        g = g.replace(n=(64, 1, 1), axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"))
    elif bad == "em_outflow":
        g = g.replace(em_bc=W._bcs("outflow", "pml"), axion_bc=W._bcs("outflow", "pml"))
    elif bad == "n0":
        g = g.replace(n=(0, 32, 1))
    else:
        g = g.replace(pml_cells=100)
    with pytest.raises(axp.AxpError) as e:
        axp.axp_workspace_bytes(axp.desc_of(g))
    assert e.value.status == axp.AXP_E_INVAL


def test_create_rejects_small_or_null_workspace():
    d = _desc()
    h = C.c_void_p()
    assert axp.lib().axp_create_grid(C.byref(d), None, 0, None, C.byref(h)) == axp.AXP_E_INVAL


def test_batch_workspace_validation():
    from paper_2406_16796_gb300 import batch

    a = batch.axp_batch_workspace_bytes(4, 10000)
    b = batch.axp_batch_workspace_bytes(4, 20000)
    assert b > a > 2 * 8 * 10000 * 4
    with pytest.raises(axp.AxpError):
        batch.axp_batch_workspace_bytes(0, 10000)
    with pytest.raises(axp.AxpError):
        batch.axp_batch_workspace_bytes(4, 4)

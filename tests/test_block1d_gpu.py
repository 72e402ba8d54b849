"""The time-blocked 1D kernel (FP64, periodic along x) against the oracle.

The kernel advances windows held in shared memory for blocks of steps, with a
bounded grid-wide wait between blocks, in the single-pass kernels' arithmetic:
every field within 1e-12 of the oracle (normwise, after N steps), on sizes that
divide unevenly among the blocks, step counts that are not multiples of the
block length, every component and coupling term active, and diagnostics taken
between launches.  How the steps are split into launches changes no bit.  The
failure-detection case removes one participant of the grid-wide wait and
checks that the others give up and the host is told."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]


def line_grid(nx, **kw):
    d = (0.05, 0.05, 0.05)
    return W.GridSpec(n=(nx, 1, 1), d=d, dt=0.7 * d[0], m=1.1, g=0.7, B_ext=(0.4, 1.0, -0.3), **kw)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("nx", [256, 300, 1000, 4096, 5003])
def test_block1d_matches_the_oracle(nx):
    from paper_2406_16796_gb300 import axp

    grid = line_grid(nx)
    st = W.random_state(grid, seed=nx)
    og = oracle.OracleGrid(grid)
    og.load(st)
    g = axp.Grid(grid)
    g.load(st)
    assert g.kernel_path() == axp.AXP_KERNEL_BLOCK1D
    g.step(1)  # (the first step also takes the state to the staggered form)
    l0 = g.launches()
    g.step(28)  # two full blocks of 12 steps and a partial one, one launch
    og.step(29)
    assert g.launches() - l0 == 1
    got, ref = g.fields(), og.fields()
    for k in NAMES:
        assert rel(got[k], ref[k]) < 1e-12, (nx, k, rel(got[k], ref[k]))
    d, dr = g.diagnostics(), og.diagnostics()
    for key in ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "sum_xB1z2", "gauss_l2"):
        assert d[key] == pytest.approx(dr[key], rel=1e-11), key
    g.close()


def test_block1d_launch_splits_and_diagnostics_ring():
    """Runs split at any step count, and at diagnostic steps, give the same bits;
    the diagnostics ring records what the general path records (1e-11)."""
    from paper_2406_16796_gb300 import axp

    grid = line_grid(777)
    st = W.random_state(grid, seed=9)
    runs = {}
    for name, kernel, chunks in (("one", axp.AXP_KERNEL_BLOCK1D, [45]),
                                 ("split", axp.AXP_KERNEL_BLOCK1D, [1, 7, 8, 9, 3, 17]),
                                 ("general", axp.AXP_KERNEL_GENERAL, [45])):
        g = axp.Grid(grid, diag_every=10, diag_capacity=8)
        g.set_kernel(kernel)
        g.load(st)
        for c in chunks:
            g.step(c)
        assert g.kernel_path() == kernel
        runs[name] = (g.fields(), g.read_diagnostics())
        g.close()
    for k in NAMES:
        assert np.array_equal(runs["split"][0][k], runs["one"][0][k]), k
        assert rel(runs["general"][0][k], runs["one"][0][k]) < 1e-12, k
    for name in ("split", "general"):
        assert [r["step"] for r in runs[name][1]] == [10, 20, 30, 40]
        for ra, rb in zip(runs[name][1], runs["one"][1]):
            for key in ("H_phi", "H_g1", "gauss_l2"):
                if name == "split":
                    assert ra[key] == rb[key], (name, key)
                else:
                    assert ra[key] == pytest.approx(rb[key], rel=1e-11), (name, key)


def test_block1d_runs_the_1d_conversion_workload():
    """The 1D conversion set-up (Nx = 4096, dx = lambda/32, CFL 0.95, g = 1e-4,
    B0 = 1, CW laser) for 1000 steps from the oracle's initial state, every
    field within 1e-12, and the automatic kernel choice takes this kernel."""
    from paper_2406_16796_gb300 import axp

    w = W.vacuum_1d(nx=4096)
    og = oracle.OracleGrid(w.grid)
    og.inject_laser(w.lasers[0])
    g = axp.Grid(w.grid)
    g.load(og.fields())  # the same initial bits on both sides
    og.step(1000)
    assert g.kernel_path() == axp.AXP_KERNEL_BLOCK1D
    g.step(1000)
    got, ref = g.fields(), og.fields()
    for k in NAMES:
        if np.any(ref[k]):
            assert rel(got[k], ref[k]) < 1e-12, (k, rel(got[k], ref[k]))
        else:
            assert not np.any(got[k]), k
    g.close()


def test_block1d_wait_gives_up_when_a_block_never_arrives():
    """Failure detection without a fault: one block leaves before the first
    grid-wide wait; the others' bounded waits give up within about a second,
    the next synchronising call reports AXP_E_TIMEOUT once, and the grid and
    the context stay usable."""
    from paper_2406_16796_gb300 import axp

    grid = line_grid(4096)
    st = W.random_state(grid, seed=77)
    g = axp.Grid(grid)
    g.load(st)
    assert g.kernel_path() == axp.AXP_KERNEL_BLOCK1D
    axp.axp_test_block1d_absent(g.h, 5)
    t0 = time.perf_counter()
    g.step(40)
    with pytest.raises(axp.AxpError) as e:
        g.synchronize()
    assert e.value.status == axp.AXP_E_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    g.synchronize()  # reported once, then cleared
    # the handle still steps (from whatever state the aborted launch left)
    g.load(st)
    og = oracle.OracleGrid(grid)
    og.load(st)
    g.step(16)
    og.step(16)
    got, ref = g.fields(), og.fields()
    for k in NAMES:
        assert rel(got[k], ref[k]) < 1e-12, k
    g.close()

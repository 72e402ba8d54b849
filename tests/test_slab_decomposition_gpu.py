"""The slab decomposition of one grid, run through the product kernels on one GPU.

Two slab grids, each a half of a periodic grid along its march axis plus halo
rows on both sides, take turns with the same GPU: each advances k steps in its
own kernels, and between rounds the host swaps halo rows of every array (both
axion levels included) through the grid API.  No kernel waits on another; the
exchange happens between launches.  After several rounds the owned rows must
match the undivided grid run on the same GPU and the undivided oracle run, at
the kernel's tolerance: the slabs go through the staggered-state conversions at
every exchange, the undivided run does not.  The 2D case takes the 2D TM kernel
(the pulse's component set), the 3D case the axion-box kernel."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]


def axp_mod():
    from paper_2406_16796_gb300 import axp

    return axp


def rows(a, axis, lo, hi):
    idx = np.arange(lo, hi) % a.shape[axis]
    return np.take(a, idx, axis=axis)


def put_rows(a, axis, lo, hi, v):
    sl = [slice(None)] * 3
    sl[axis] = slice(lo, hi)
    a[tuple(sl)] = v


CASES = {
    # grid cells, split axis of the (nz, ny, nx) arrays, active arrays, precision, kernel, steps per round
    "2d_tm2d_fp64": dict(n=(192, 128, 1), axis=1, active=["E0z", "B0x", "B0y"] + [f for f in W.FIELD_NAMES if f[1] == "1"],
                         prec="fp64", kernel="AXP_KERNEL_TM2D", k=6, tol=1e-12),
    "2d_tm2d_fp32": dict(n=(192, 128, 1), axis=1, active=["E0z", "B0x", "B0y"] + [f for f in W.FIELD_NAMES if f[1] == "1"],
                         prec="fp32", kernel="AXP_KERNEL_TM2D", k=6, tol=1e-4),
    "3d_ax3d_fp32": dict(n=(40, 36, 64), axis=0, active=[f for f in W.FIELD_NAMES if f[1] == "1"], prec="fp32",
                         kernel="AXP_KERNEL_AX3D", k=4, tol=1e-4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_slabs_with_halo_swaps_match_the_undivided_grid(case):
    axp = axp_mod()
    c = CASES[case]
    n, axis, k, rounds = c["n"], c["axis"], c["k"], 3
    d = (0.05, 0.05, 0.05)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    glob = W.GridSpec(n=n, d=d, dt=dt, m=0.8, g=0.7, B_ext=(0.0, 0.6, 1.0) if n[2] == 1 else (0.0, 1.0, 0.0),
                      precision=c["prec"])
    start = W.random_state(glob, seed=515, active=c["active"])
    N = start["E0x"].shape[axis]
    own = N // 2
    w = k + 6  # the integer-time reach (k + 2) and the staggered-state conversions' reach, with margin
    ln = list(n)
    ln[2 - axis] = own + 2 * w
    slab_spec = glob.replace(n=tuple(ln))
    slabs = []
    for r in range(2):
        g = axp.Grid(slab_spec)
        g.set_kernel(getattr(axp, c["kernel"]))
        g.load({name: rows(start[name], axis, r * own - w, r * own + own + w) for name in NAMES})
        slabs.append(g)
    for _ in range(rounds):
        for g in slabs:
            g.step(k)
            assert g.kernel_path() == getattr(axp, c["kernel"])
        f = [g.fields() for g in slabs]
        for r in range(2):
            other = f[1 - r]
            new = {}
            for name in NAMES:
                a = f[r][name].copy()
                # lower halo from the other slab's top owned rows, upper halo from its bottom ones
                put_rows(a, axis, 0, w, rows(other[name], axis, own, own + w))
                put_rows(a, axis, own + w, own + 2 * w, rows(other[name], axis, w, 2 * w))
                new[name] = a
            slabs[r].load(new)
    got = {name: np.concatenate([rows(g.fields()[name], axis, w, w + own) for g in slabs], axis=axis) for name in NAMES}
    for g in slabs:
        g.close()

    whole = axp.Grid(glob)
    whole.set_kernel(getattr(axp, c["kernel"]))
    whole.load(start)
    whole.step(k * rounds)
    ref_gpu = whole.fields()
    whole.close()
    og = oracle.OracleGrid(glob.replace(precision="fp64"))
    og.load(start)
    og.step(k * rounds)
    ref = og.fields()
    for name in NAMES:
        nr = np.linalg.norm(ref[name])
        if name not in c["active"] and name not in ("phi_cur", "phi_old"):
            assert not np.any(got[name]) and nr == 0, name
            continue
        assert nr > 0, name
        assert np.linalg.norm(got[name] - ref[name]) <= c["tol"] * nr, (name, np.linalg.norm(got[name] - ref[name]) / nr)
        assert np.linalg.norm(got[name] - ref_gpu[name]) <= c["tol"] * nr, name

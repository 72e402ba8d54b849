"""The 2D pulse workload at its full size (4096 x 2048 cells), stepped by the
grid API in the launch configuration the bench times, checked against the
oracle on sampled sub-boxes.

After N steps a cell depends only on cells within a few cells per step of it,
so the oracle steps a 256 x 256 sub-box cut out of the same initial state.  Its
cut sides get an absorbing layer like the grid's edges.  Its cells farther than
layer + 3 N + 2 cells from every cut side (a generous margin: one step's reach is
one cell, and the axion current's stencil adds two once) must equal the full-size run's:
1e-12 normwise in FP64 (the fused path's tolerance), 1e-4 in FP32 split.  Sides
that lie on the grid's own edges keep their true layer.  The initial state is
random, so every sub-box carries non-trivial fields, layers included."""
import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]
N_STEPS = 20
S = 256  # sub-box edge, cells


def boxes(nx, ny):
    """(x0, y0) of the sampled sub-boxes: two corners, an x edge, the interior, the top edge."""
    return [(0, 0), (nx - S, 0), (0, ny // 2 - S // 2), (nx // 2 - S // 2, ny // 2 - S // 2), (nx // 3, ny - S)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_pulse_grid_matches_the_oracle_on_sub_boxes(prec):
    from paper_2406_16796_gb300 import axp

    w = W.pulse_2d(precision=prec)  # 4096 x 2048, PML of 20 cells on every side
    grid = w.grid
    nx, ny, L = grid.n[0], grid.n[1], grid.pml_cells
    g = axp.Grid(grid)
    # the workload's component set: laser (E0z; B0x, B0y), every order-1 array, phi
    active = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
    g.load(W.random_state(grid, seed=20240624 + 1, active=active))
    start = g.fields()
    g.step(N_STEPS)
    assert g.kernel_path() in (axp.AXP_KERNEL_TM2D, axp.AXP_KERNEL_TM2D_LIST)
    end = g.fields()
    g.close()
    margin = L + 3 * N_STEPS + 2
    tol = 1e-12 if prec == "fp64" else 1e-4
    for x0, y0 in boxes(nx, ny):
        sl = (0, slice(y0, y0 + S), slice(x0, x0 + S))
        sub = grid.replace(n=(S, S, 1), precision="fp64")
        og = oracle.OracleGrid(sub)
        og.load({k: start[k][sl][None] for k in NAMES})
        og.step(N_STEPS)
        ref = og.fields()
        # the exact region: away from the cut sides (a side on the grid's edge is not cut)
        xlo = 0 if x0 == 0 else margin
        xhi = S if x0 + S == nx else S - margin
        ylo = 0 if y0 == 0 else margin
        yhi = S if y0 + S == ny else S - margin
        assert xhi - xlo >= 64 and yhi - ylo >= 64
        for k in NAMES:
            a = end[k][sl][ylo:yhi, xlo:xhi]
            b = ref[k][0, ylo:yhi, xlo:xhi]
            nb = np.linalg.norm(b)
            if k in ("E0x", "E0y", "B0z"):  # outside the component set: stay zero
                assert not np.any(a) and nb == 0, (x0, y0, k)
                continue
            assert nb > 0, (x0, y0, k)
            assert np.linalg.norm(a - b) <= tol * nb, (prec, x0, y0, k, np.linalg.norm(a - b) / nb)


def test_full_size_axion_box_matches_the_oracle_on_sub_boxes():
    """The 3D axion box at its full size (512^3, FP32 split, periodic), stepped by
    the 3D kernel, against the oracle on two 128^3 sub-boxes (one across the
    periodic seam) cut from the same start.  Every side of a sub-box is cut, so
    the exact region lies layer + 3 N + 2 cells inside each side.  Arrays are read
    one at a time to keep the host's memory small."""
    from paper_2406_16796_gb300 import axp

    w = W.axion_3d(precision="fp32")  # 512^3, axion plane wave along x, B_ext along y
    grid = w.grid
    n = grid.n[0]
    steps, s3, lay = 10, 128, 4
    g = axp.Grid(grid)
    g.inject_axion(w.axions[0])
    origins = [(200, 150, 300), (n - 64, n - 64, n - 64)]  # the second box wraps around the seam

    def cut(a, o):
        idx = [(np.arange(s3) + o[d]) % n for d in range(3)]
        return a[np.ix_(idx[2], idx[1], idx[0])]

    start = {k: [cut(g.read(k), o) for o in origins] for k in NAMES}
    g.step(steps)
    assert g.kernel_path() == axp.AXP_KERNEL_AX3D
    end = {k: [cut(g.read(k), o) for o in origins] for k in NAMES}
    g.close()
    bc = W._bcs("pml", "pml", "pml")
    sub = grid.replace(n=(s3, s3, s3), precision="fp64", axion_bc=bc, em_bc=bc, pml_cells=lay)
    m = lay + 3 * steps + 2
    inner = (slice(m, s3 - m),) * 3
    for b in range(len(origins)):
        og = oracle.OracleGrid(sub)
        og.load({k: start[k][b] for k in NAMES})
        og.step(steps)
        ref = og.fields()
        for k in ("E1x", "E1y", "E1z", "B1x", "B1y", "B1z", "phi_cur", "phi_old"):
            a, r = end[k][b][inner], ref[k][inner]
            nr = np.linalg.norm(r)
            if nr == 0:
                assert not np.any(a), (b, k)
                continue
            assert np.linalg.norm(a - r) <= 1e-4 * nr, (b, k, np.linalg.norm(a - r) / nr)
        # the axion wave drives E1 along B_ext (y) through J = (D_t phi) B_ext
        assert np.linalg.norm(ref["phi_cur"][inner]) > 0 and np.linalg.norm(ref["E1y"][inner]) > 0


def test_full_size_pulse_work_lists_equal_the_uniform_grid():
    """At the full 4096 x 2048 size the FP64 2D kernel's two launch forms, the
    balanced work lists and the uniform grid of strips by chunks, give the same
    fields bit for bit after a few steps from the same random state."""
    from paper_2406_16796_gb300 import axp

    grid = W.pulse_2d(precision="fp64").grid
    active = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]
    st = W.random_state(grid, seed=20240624 + 7, active=active)
    out = {}
    for kernel in (axp.AXP_KERNEL_TM2D_LIST, axp.AXP_KERNEL_TM2D):
        g = axp.Grid(grid)
        g.set_kernel(kernel)
        g.load(st)
        assert g.kernel_path() == kernel
        g.step(3)
        out[kernel] = g.fields()
        g.close()
    for k in NAMES:
        assert np.array_equal(out[axp.AXP_KERNEL_TM2D_LIST][k], out[axp.AXP_KERNEL_TM2D][k]), k

"""The slab decomposition driver with its product engine (grids of the C ABI,
rows packed and unpacked in device buffers) on one GPU.

Several slabs of one grid run in one process on one device (run_local): each
advances k steps in its own launches, then the halo rows move through device
buffers between launches.  No kernel waits on another.  The owned rows must
match the undivided grid run on the same GPU (the same kernel, the same
arithmetic per cell) and the oracle, and the slabs' combined diagnostics the
undivided grid's record."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import slab
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]
TM_ACTIVE = ["E0z", "B0x", "B0y"] + [f for f in W.FIELD_NAMES if f[1] == "1"]

CASES = {
    # grid, active arrays, expected kernel, steps per round, rounds, ranks
    "2d_pml_tm2d": (W.pulse_2d(nx=200, ny=240, m=0.7, g=0.5).grid.replace(pml_cells=8), TM_ACTIVE, "TM2D", 6, 4, 3),
    "2d_periodic_y_tm2d": (W.beam_2d(160, 200, m=0.7, g=0.5, pml_cells=8).grid.replace(
        em_bc=W._bcs("pml", "periodic"), axion_bc=W._bcs("pml", "periodic")), TM_ACTIVE, "TM2D", 5, 4, 2),
    "3d_axion_box": (W.axion_3d(n=48, g=0.5).grid, [f for f in W.FIELD_NAMES if f[1] == "1"], "AX3D", 3, 3, 2),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_local_slabs_match_the_undivided_grid(case, prec):
    from paper_2406_16796_gb300 import axp

    glob, active, kern, k, rounds, world = CASES[case]
    glob = glob.replace(precision=prec)
    if case.startswith("3d") and prec == "fp64":
        pytest.skip("the 3D axion-box kernel's FP64 slabs are covered by the FP32 case")
    start = W.random_state(glob, seed=99, active=active)
    runs = [slab.SlabRun(glob, r, world, k, slab.LocalComm()) for r in range(world)]
    for r in runs:
        r.load_global(start)
        ok = {getattr(axp, "AXP_KERNEL_" + kern)}
        if kern == "TM2D" and prec == "fp64":
            ok.add(axp.AXP_KERNEL_TM2D_LIST)  # (the work-list form, where the planner prefers it)
        assert r.engine.grid.kernel_path() in ok
    slab.run_local(runs, rounds)
    ax = 2 - slab.split_axis(glob)
    got = {name: np.concatenate([r.owned(r.engine.fields())[name] for r in runs], axis=ax) for name in NAMES}
    rec = slab.combine([r.engine.owned_record() for r in runs])
    for r in runs:
        r.engine.close()

    whole = axp.Grid(glob)
    whole.load(start)
    whole.step(k * rounds)
    ref_gpu, rec_gpu = whole.fields(), whole.diagnostics()
    whole.close()
    og = oracle.OracleGrid(glob.replace(precision="fp64"))
    og.load(start)
    og.step(k * rounds)
    ref = og.fields()
    tol = 1e-12 if prec == "fp64" else 1e-4
    for name in NAMES:
        nr = np.linalg.norm(ref[name])
        if nr == 0:
            assert not np.any(got[name]), name
            continue
        assert np.linalg.norm(got[name] - ref_gpu[name]) <= tol * nr, (name, np.linalg.norm(got[name] - ref_gpu[name]) / nr)
        assert np.linalg.norm(got[name] - ref[name]) <= tol * nr, (name, np.linalg.norm(got[name] - ref[name]) / nr)
    for key in ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "sum_xB1z2", "sum_B1z2", "gauss_l2"):
        assert rec[key] == pytest.approx(rec_gpu[key], rel=1e-12 if prec == "fp64" else 1e-5), key

"""Groups of 2D grids stepped by one launch per step against the grids stepped
alone and against the oracle.

A member's states are compared bit for bit between the mix and a group of one
(the same kernel), and to FP32 rounding with axp_step on the grid alone (the
single-grid kernel); one case also goes to the FP64 oracle at the FP32 split
tolerance (fields 1e-4 after the run, conversion probability 1e-3)."""
import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = ("E0z", "B0x", "B0y", "E1x", "E1y", "E1z", "B1x", "B1y", "B1z", "phi_cur", "phi_old")
ACTIVE = ["E0z", "B0x", "B0y"] + [n for n in W.FIELD_NAMES if n[1] == "1"]


def mods():
    from paper_2406_16796_gb300 import axp, group

    return axp, group


def grid_of(n, m, g, Bz, bc, pml=6, d=(0.05, 0.07)):
    dt = 0.5 / np.sqrt(1 / d[0] ** 2 + 1 / d[1] ** 2)
    kw = {}
    if bc == "pml":
        kw = dict(axion_bc=W._bcs("pml", "pml"), em_bc=W._bcs("pml", "pml"), pml_cells=pml)
    elif bc == "periodic_x_pml_y":
        kw = dict(axion_bc=W._bcs("periodic", "pml"), em_bc=W._bcs("periodic", "pml"), pml_cells=pml)
    return W.GridSpec(n=(n[0], n[1], 1), d=(d[0], d[1], 0.06), dt=dt, m=m, g=g, B_ext=(0.1, -0.2, Bz),
                      precision="fp32", **kw)


MEMBERS = [
    dict(n=(300, 90), m=1.1, g=0.7, Bz=1.0, bc="periodic", steps=30),
    dict(n=(520, 130), m=0.0, g=0.3, Bz=0.5, bc="pml", steps=17),
    dict(n=(64, 200), m=2.0, g=1.3, Bz=-1.0, bc="periodic_x_pml_y", steps=25),
    dict(n=(700, 33), m=0.4, g=0.9, Bz=2.0, bc="periodic_x_pml_y", steps=8),
]


def loaded(axp, spec, seed):
    grid = grid_of(spec["n"], spec["m"], spec["g"], spec["Bz"], spec["bc"])
    st = W.random_state(grid, seed=seed, active=ACTIVE)
    g = axp.Grid(grid)
    g.load(st)
    return g, grid, st


def test_group_member_is_identical_alone_and_in_the_mix():
    """A grid's states do not depend on the other members, the tile height or the
    launch count: bit-identical alone (a group of one, another tiling) and in
    the mix.  Against the single-grid 2D kernel (a separately compiled kernel
    of the same body) they agree to FP32 rounding."""
    axp, group = mods()
    G = group.Group(8, 2000, chunk=24)
    grids = []
    for i, spec in enumerate(MEMBERS):
        g, grid, st = loaded(axp, spec, 500 + i)
        grids.append((g, G.add(g, spec["steps"])))
    G.run(max(s["steps"] for s in MEMBERS) + 5)  # extra launches leave finished members alone
    p = G.progress()
    assert [p[m] for _, m in grids] == [s["steps"] for s in MEMBERS]
    for (g, m), spec, i in zip(grids, MEMBERS, range(len(MEMBERS))):
        G.remove(m)
        assert g.step_count == spec["steps"]
        solo, _, _ = loaded(axp, spec, 500 + i)
        G1 = group.Group(1, 400, chunk=40)
        m1 = G1.add(solo, spec["steps"])
        for _ in range(spec["steps"]):
            G1.run(1)
        G1.remove(m1)
        G1.close()
        single, _, _ = loaded(axp, spec, 500 + i)
        single.set_kernel(axp.AXP_KERNEL_TM2D)
        single.step(spec["steps"])
        a, b, c = g.fields(), solo.fields(), single.fields()
        for k in NAMES:
            assert np.array_equal(a[k], b[k]), (spec, k)
            nc = np.linalg.norm(c[k])
            assert np.linalg.norm(a[k] - c[k]) <= 1e-5 * (nc if nc > 0 else 1.0), (spec, k)
        for x in (g, solo, single):
            x.close()
    G.close()


def test_group_member_matches_oracle():
    axp, group = mods()
    spec = MEMBERS[2]
    g, grid, st = loaded(axp, spec, 77)
    og = oracle.OracleGrid(grid.replace(precision="fp64"))
    og.load(st)
    G = group.Group(2, 400)
    m = G.add(g, spec["steps"])
    G.run(spec["steps"])
    G.remove(m)
    og.step(spec["steps"])
    ref, got = og.fields(), g.fields()
    for k in NAMES:
        nb = np.linalg.norm(ref[k])
        assert np.linalg.norm(got[k] - ref[k]) / (nb if nb > 0 else 1.0) < 1e-4, k
    assert g.diagnostics()["H_phi"] == pytest.approx(og.diagnostics()["H_phi"], rel=1e-3)
    G.close()
    g.close()


def test_group_admission_release_graphs_and_guard():
    """Members join and leave between runs (the pulse set-up with its laser), graph
    replay gives the states of direct launches, and a member's grid refuses
    direct calls until it is handed back."""
    axp, group = mods()
    specs = [W.pulse_2d(nx=nx, ny=ny, m=0.5 * W.K0, g=1e-4, precision="fp32") for nx, ny in ((256, 128), (512, 256),
                                                                                             (300, 150))]
    results = []
    for graphs in (False, True):
        G = group.Group(2, 200, graphs=graphs)
        gs = []
        for w in specs:
            g = axp.Grid(w.grid.replace(pml_cells=10))
            g.inject_laser(w.lasers[0])
            gs.append(g)
        m0 = G.add(gs[0], 60)
        m1 = G.add(gs[1], 90)
        with pytest.raises(axp.AxpError) as e:
            gs[0].step(1)
        assert e.value.status == axp.AXP_E_STATE
        assert G.add(gs[2], 10) is None  # both member indices are taken
        for _ in range(3):
            G.run(20)
        assert list(G.progress()[[m0, m1]]) == [60, 60]
        G.remove(m0)
        m2 = G.add(gs[2], 40)
        for _ in range(2):
            G.run(20)
        assert list(G.progress()[[m1, m2]]) == [90, 40]
        G.remove(m1)
        G.remove(m2)
        assert [g.step_count for g in gs] == [60, 90, 40]
        results.append([(g.fields(), g.diagnostics()) for g in gs])
        for g in gs:
            g.close()
        G.close()
    for (fa, da), (fb, db) in zip(*results):
        for k in NAMES:
            assert np.array_equal(fa[k], fb[k]), k
        assert da["P_g2a"] == db["P_g2a"]


def test_group_rejects_grids_it_cannot_step():
    axp, group = mods()
    G = group.Group(2, 100)
    g64 = axp.Grid(grid_of((64, 40), 0.1, 0.1, 1.0, "periodic").replace(precision="fp64"))
    with pytest.raises(axp.AxpError) as e:
        G.add(g64, 5)
    assert e.value.status == axp.AXP_E_INVAL
    g3 = axp.Grid(W.axion_3d(n=16, precision="fp32").grid)
    with pytest.raises(axp.AxpError):
        G.add(g3, 5)
    big = axp.Grid(grid_of((2000, 2000), 0.1, 0.1, 1.0, "periodic"))
    assert G.add(big, 5) is None  # more tiles than the group holds
    for g in (g64, g3, big):
        g.close()
    G.close()

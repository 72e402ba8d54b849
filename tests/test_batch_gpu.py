"""Batches of 1D conversion runs (parameter scans, serving) against the oracle.

Tolerances are those of the FP32 split path: fields normwise <= 1e-4 after the
run, conversion probability <= 1e-3 relative."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def batch_mod():
    from paper_2406_16796_gb300 import batch

    return batch


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def inst(nx, m, g, By, Bz, steps, amplitude=1e-3, waves=None):
    B = batch_mod()
    dx = 1.0 / 32.0
    w = waves or max(1, round(nx * dx))
    k = 2 * math.pi * w / (nx * dx)
    return B.instance_of(nx, dx, 0.95 * dx, m, g, By, Bz, amplitude, k, steps)


def oracle_run(i, steps):
    grid = W.GridSpec(n=(int(i.nx), 1, 1), d=(i.dx, i.dx, i.dx), dt=i.dt, m=i.m, g=i.g, B_ext=(0.0, i.By, i.Bz))
    og = oracle.OracleGrid(grid)
    og.inject_laser(W.LaserSpec(amplitude=i.amplitude, k=(i.k, 0, 0), pol=(0, 1, 0)))
    og.step(steps)
    return og


INSTANCES = [
    dict(nx=64, m=0.0, g=3e-2, By=1.0, Bz=0.0),
    dict(nx=700, m=2.0, g=1e-2, By=2.0, Bz=0.5),
    dict(nx=6400, m=0.5 * W.K0, g=5e-3, By=1.5, Bz=-0.3),
    dict(nx=9000, m=0.1, g=2e-2, By=0.7, Bz=0.2),
]


def test_batch_matches_oracle_with_segmented_instances():
    B = batch_mod()
    steps = 120
    insts = [inst(steps=steps, **d) for d in INSTANCES]
    b = B.Batch(8, sum(int(i.nx) for i in insts) + 100)
    b.set_tiling(32, 1536, 256)  # 6400 and 9000 run as segments with halos
    slots = [b.add(i) for i in insts]
    b.run(steps)
    assert list(b.progress()[slots]) == [steps] * len(slots)
    for i, s in zip(insts, slots):
        og = oracle_run(i, steps)
        ref = og.fields()
        got = {"B0z": b.read_state(s, 1), "B1y": b.read_state(s, 4), "B1z": b.read_state(s, 5),
               "phi_cur": b.read_state(s, 6)}
        got["phi_old"] = got["phi_cur"] - b.read_state(s, 7)
        for k, v in got.items():
            assert rel(v, ref[k].ravel()) < 1e-4, (int(i.nx), k, rel(v, ref[k].ravel()))
        d, dr = b.result(s), og.diagnostics()
        assert d["step"] == steps
        for key in ("P_g2a", "H_phi", "H_g0", "H_g1"):
            assert d[key] == pytest.approx(dr[key], rel=1e-3), (int(i.nx), key, d[key], dr[key])
    b.close()


def test_batch_instance_is_identical_alone_and_in_the_mix():
    """Each instance's arithmetic does not depend on the other instances, the block
    length or the segmentation: bit-identical states."""
    B = batch_mod()
    x = inst(nx=9000, m=0.3, g=1e-2, By=1.0, Bz=0.1, steps=200)
    alone = B.Batch(1, 9000)
    sa = alone.add(x)
    alone.set_tiling(16, 3584, 512)
    alone.run(200)
    mix = B.Batch(6, 40000)
    others = [inst(nx=n, m=0.1 * j, g=1e-3, By=2.0, Bz=0.0, steps=150 + 10 * j) for j, n in enumerate((100, 3000, 7000, 12000))]
    for o in others[:2]:
        mix.add(o)
    sm = mix.add(x)
    for o in others[2:]:
        mix.add(o)
    mix.set_tiling(64, 1536, 256)
    mix.run(200)
    for which in range(8):
        assert np.array_equal(alone.read_state(sa, which), mix.read_state(sm, which)), which
    alone.close()
    mix.close()


def test_batch_completion_admission_and_release():
    B = batch_mod()
    b = B.Batch(3, 3000)
    s1 = b.add(inst(nx=1000, m=0.0, g=1e-3, By=1.0, Bz=0.0, steps=50))
    s2 = b.add(inst(nx=1500, m=1.0, g=1e-3, By=1.0, Bz=0.0, steps=200))
    assert b.try_add(inst(nx=600, m=0.0, g=1e-3, By=1.0, Bz=0.0, steps=10)) is None  # not enough cells
    b.run(300)
    p = b.progress()
    assert p[s1] == 50 and p[s2] == 200
    b.remove(s1)  # frees cells [0, 1000); [2500, 3000) is free too, but not contiguous with it
    assert b.try_add(inst(nx=1400, m=0.0, g=1e-3, By=1.0, Bz=0.0, steps=10)) is None
    s3 = b.add(inst(nx=900, m=0.0, g=1e-3, By=1.0, Bz=0.0, steps=10))  # reuses the released cells
    b.run(20)
    p = b.progress()
    assert p[s3] == 10 and p[s2] == 200
    b.remove(s2)
    b.remove(s3)  # all released ranges coalesce into one
    s4 = b.add(inst(nx=2900, m=0.0, g=1e-3, By=1.0, Bz=0.0, steps=5))
    b.run(5)
    assert b.progress()[s4] == 5
    b.close()


def test_batch_matches_single_grid_fp32():
    """The batch and the single-grid FP32 path agree to the FP32 tolerance (their
    operation orders differ, so agreement is to rounding, not bit for bit)."""
    from paper_2406_16796_gb300 import axp

    B = batch_mod()
    x = inst(nx=4096, m=0.2 * W.K0, g=1e-4, By=1.0, Bz=0.0, steps=400)
    b = B.Batch(1, 4096)
    s = b.add(x)
    b.run(400)
    w = W.vacuum_1d(nx=4096, m=x.m, g=x.g, precision="fp32")
    g = axp.Grid(w.grid)
    g.inject_laser(w.lasers[0])
    g.step(400)
    assert rel(b.read_state(s, 6), g.read("phi_cur").ravel()) < 1e-4
    assert rel(b.read_state(s, 5), g.read("B1z").ravel()) < 1e-4
    assert b.result(s)["P_g2a"] == pytest.approx(g.diagnostics()["P_g2a"], rel=1e-4)
    b.close()
    g.close()


def test_batch_graph_replay_is_identical_to_direct_launches():
    """A run replayed from a captured CUDA graph gives the states of the same run
    launched directly, and admission between runs invalidates the graph."""
    B = batch_mod()
    xs = [inst(nx=n, m=0.2, g=1e-3, By=1.0, Bz=0.0, steps=300) for n in (500, 2500, 8000)]
    runs = []
    for graphs in (False, True):
        b = B.Batch(4, 20000, graphs=graphs)
        slots = [b.add(x) for x in xs[:2]]
        for _ in range(3):
            b.run(40)  # the second and third calls replay the graph
        slots.append(b.add(xs[2]))
        for _ in range(4):
            b.run(40)
        assert b.launches() > 0
        runs.append([[b.read_state(s, w) for w in range(8)] for s in slots])
        assert list(b.progress()[slots]) == [280, 280, 160]
        b.close()
    for a, c in zip(*runs):
        for w in range(8):
            assert np.array_equal(a[w], c[w]), w


def test_scan_draws_meet_the_conversion_probability_tolerance():
    """Scan draws (masses, couplings and fields from the scan distribution, shorter
    boxes and runs so the oracle finishes in seconds): the FP32 split batch and the
    FP32 split single grid give P(gamma->a) within 1e-3 of the FP64 oracle.  Small
    (m dt)^2 next to 2 dt^2/dx^2 is the case that needs the mass term kept apart."""
    from paper_2406_16796_gb300 import axp

    B = batch_mod()
    draws = W.scan_instances(count=5, nx_range=(1024, 2048), steps_range=(4000, 9000))
    draws.append(W.ScanInstance(1100, 0.2387, 1.4e-6, 8.9, 9000))
    b = B.Batch(len(draws), sum(d.nx for d in draws))
    xs = [B.scan_instance(d) for d in draws]
    slots = [b.add(x) for x in xs]
    b.run(max(d.steps for d in draws))
    for d, x, s in zip(draws, xs, slots):
        og = oracle_run(x, d.steps)
        want = og.diagnostics()["P_g2a"]
        got = b.result(s)["P_g2a"]
        assert got == pytest.approx(want, rel=1e-3), (d, got, want)
        w = W.scan_workload(d, precision="fp32")
        g = axp.Grid(w.grid)
        g.inject_laser(w.lasers[0])
        g.step(d.steps)
        assert g.diagnostics()["P_g2a"] == pytest.approx(want, rel=1e-3), d
        g.close()
    b.close()


def test_batched_results_equal_the_per_slot_results():
    """axp_batch_results: one launch for many slots, each record bit-identical to
    the slot's own axp_batch_result; a free slot in the list is refused."""
    from paper_2406_16796_gb300 import axp

    B = batch_mod()
    xs = [inst(nx=n, m=0.3, g=1e-3, By=1.0, Bz=0.2, steps=150) for n in (700, 3000, 9000, 1500)]
    b = B.Batch(6, 20000)
    slots = [b.add(x) for x in xs]
    b.run(150)
    many = b.results(slots[::-1])
    for s, d in zip(slots[::-1], many):
        assert d == b.result(s)
    b.remove(slots[1])
    with pytest.raises(axp.AxpError) as e:
        b.results([slots[0], slots[1]])
    assert e.value.status == axp.AXP_E_INVAL
    b.close()


@pytest.mark.parametrize("tiling", [(32, 1856, 256), (8, 4000, 512)])
def test_smallest_instances_match_the_oracle(tiling):
    """Instances of 8 to 33 cells: one to five threads hold cells (the last with a
    partial run of fewer than 8), the periodic neighbours wrap within those threads,
    and the rest of the block is idle."""
    B = batch_mod()
    steps = 90
    insts = [inst(nx=n, m=0.4 * j, g=2e-2, By=1.0, Bz=0.3 * j, steps=steps, waves=1)
             for j, n in enumerate((8, 9, 13, 16, 17, 33))]
    b = B.Batch(8, 200)
    b.set_tiling(*tiling)
    slots = [b.add(i) for i in insts]
    b.run(steps)
    for i, s, d in zip(insts, slots, b.results(slots)):
        og = oracle_run(i, steps)
        ref = og.fields()
        got = {"B0z": b.read_state(s, 1), "B1y": b.read_state(s, 4), "B1z": b.read_state(s, 5),
               "phi_cur": b.read_state(s, 6)}
        for k, v in got.items():
            assert rel(v, ref[k].ravel()) < 1e-4, (int(i.nx), k, rel(v, ref[k].ravel()))
        assert d["P_g2a"] == pytest.approx(og.diagnostics()["P_g2a"], rel=1e-3), int(i.nx)
    b.close()

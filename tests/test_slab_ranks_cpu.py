"""The slab decomposition driver (paper_2406_16796_gb300/slab.py) over gloo
ranks on CPU.

The driver's own plan, exchange schedule and torch.distributed messages run
here as they do between GPUs; only the engine that steps a slab is the oracle
(test infrastructure) instead of a grid of the C ABI.  After several rounds of
k steps and halo exchanges, the owned rows of every rank must equal the
undivided oracle run bit for bit: split axis periodic (2D and 3D) or absorbing
(PML on the grid's edges, and a layer inside the halo at every cut), two and
three ranks.  The fixed-order combination of the ranks' diagnostic records is
checked through the same messages."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2406_16796_gb300 import slab
from paper_2406_16796_gb300 import workloads as W

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def grid_of(n, bc):
    d = (0.05, 0.07, 0.06)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / math.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    b = W._bcs(*[bc if n[a] > 1 else "periodic" for a in range(3)])
    return W.GridSpec(n=n, d=d, dt=dt, lo=(0.2, -0.3, 0.1), m=1.1, g=0.7, B_ext=(0.3, -0.2, 1.0), axion_bc=b,
                      em_bc=b, pml_cells=3)


CASES = {
    # global cells, boundary kind, steps between exchanges, rounds
    "2d_periodic": ((20, 60, 1), "periodic", 3, 4),
    "2d_pml": ((18, 80, 1), "pml", 2, 4),
    "3d_periodic": ((6, 5, 40), "periodic", 2, 3),
}


class OracleEngine:
    """A slab stepped by the CPU oracle; rows move as float64 CPU tensors."""

    def __init__(self, p):
        import oracle

        self.plan = p
        self.og = oracle.OracleGrid(p.spec)
        self.ax = 2 - p.axis

    def _arrays(self):
        f = self.og.f
        return [f[k] for k in W.FIELD_NAMES] + [self.og.phi_cur, self.og.phi_old]

    def step(self, k):
        self.og.step(k)

    def pack(self, start, count):
        idx = np.arange(start, start + count)
        return torch.from_numpy(np.stack([np.take(a, idx, axis=self.ax) for a in self._arrays()]).copy())

    def empty(self, count):
        shape = list(self.og.phi_cur.shape)
        shape[self.ax] = count
        return torch.empty([len(NAMES)] + shape, dtype=torch.float64)

    def unpack(self, start, count, buf):
        v = buf.numpy()
        for q, a in enumerate(self._arrays()):
            sl = [slice(None)] * 3
            sl[self.ax] = slice(start, start + count)
            a[tuple(sl)] = v[q]

    def load(self, state):
        self.og.load(state)

    def fields(self):
        return self.og.fields()


def _rank_main(rank, world, port, case, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, bc, k, rounds = CASES[case]
        glob = grid_of(n, bc)
        start = W.random_state(glob, seed=2718)
        run = slab.SlabRun(glob, rank, world, k, slab.TorchComm(), engine_factory=OracleEngine)
        run.load_global(start)
        run.run(rounds)
        out[rank] = run.owned(run.engine.fields())
        # the records' fixed-order combination through the same messages
        rec = {key: float(rank + 1) * (i + 1) for i, key in enumerate(slab.SUMS)}
        rec.update(step=k * rounds, t=0.5)
        tot = slab.combine(run.comm.gather_records(rec))
        if rank == 0:
            out["combined"] = tot
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_slab_ranks_equal_the_undivided_oracle(case, world):
    import oracle

    n, bc, k, rounds = CASES[case]
    glob = grid_of(n, bc)
    start = W.random_state(glob, seed=2718)
    og = oracle.OracleGrid(glob)
    og.load(start)
    og.step(k * rounds)
    ref = og.fields()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, free_port(), case, out), nprocs=world, start_method="spawn")
    ax = 2 - slab.split_axis(glob)
    got = {name: np.concatenate([out[r][name] for r in range(world)], axis=ax) for name in NAMES}
    for name in NAMES:
        assert got[name].shape == ref[name].shape
        assert np.array_equal(got[name], ref[name]), (case, world, name, np.abs(got[name] - ref[name]).max())
    tot = out["combined"]
    for i, key in enumerate(slab.SUMS):
        assert tot[key] == sum(float(r + 1) * (i + 1) for r in range(world))
    assert tot["P_g2a"] == tot["H_phi"] / tot["H_g0"] and tot["step"] == k * rounds


def test_plan_rows_halo_and_boundaries():
    g = W.pulse_2d(nx=64, ny=300).grid  # PML along y, 20 cells
    for world in (1, 2, 3, 4):
        plans = [slab.plan(g, r, world, 5) for r in range(world)]
        assert plans[0].own_lo == 0 and plans[-1].own_hi == 300
        for a, b in zip(plans, plans[1:]):
            assert a.own_hi == b.own_lo
        for p in plans:
            assert p.spec.n[1] == p.hi - p.lo and p.spec.n[0] == 64
            assert p.spec.lo[1] == pytest.approx(g.lo[1] + p.lo * g.d[1])
            if world > 1:
                assert p.width == 5 + 2 + slab.MARGIN + g.pml_cells
            assert 0 <= p.lo and p.hi <= 300  # an absorbing axis does not wrap
            assert p.spec.em_bc[1] == ("pml", "pml") and p.spec.axion_bc[1] == ("pml", "pml")
    per = g.replace(em_bc=W._bcs("pml", "periodic"), axion_bc=W._bcs("pml", "periodic"))
    p = slab.plan(per, 0, 2, 5)
    assert p.lo == -(5 + 2 + slab.MARGIN) and p.spec.em_bc[1] == ("periodic", "periodic")
    with pytest.raises(ValueError):
        slab.plan(g, 0, 40, 5)  # slabs thinner than their halo
    with pytest.raises(ValueError):
        slab.plan(g.replace(axion_bc=W._bcs("pml", "outflow")), 0, 2, 5)

"""Slab decomposition of one grid across ranks (one device per rank).

The update of Sec. 2.3 is explicit: one step at a cell reads its neighbours
one cell away, and the axion current's two-cell stencil widens that once.  So
a rank that holds its owned rows of the grid plus `halo` rows on each side,
along the grid's slowest axis with more than one cell (y in 2D, z in 3D), can
take k steps alone while halo >= k + 2, and then refreshes its halo rows from
its neighbours' owned rows.  The kernels never wait on another rank: the
exchange runs between launches, each rank packing rows of its own state into
a local buffer that a point-to-point message carries into the neighbour's
local buffer, from which the neighbour unpacks them (no peer memory is handed
to any kernel).

Boundaries along the split axis:
  * periodic: every slab grid is itself periodic along the axis; what wraps in
    at its seams is wrong data that stays inside the halo.
  * absorbing (PML): the slabs at the grid's edges keep the real layer; every
    cut side carries a layer of the same thickness inside the halo, so the halo
    is widened by the layer (its damping stays inside the halo too).
The margin of 4 rows beyond k + 2 covers the staggered-state conversion of the
single-pass kernels at the first step and the diagnostics' reconstruction.

Diagnostics: each slab sums its owned rows (axp_compute_diagnostics_rows); the
energies and sums add up across slabs, gathered and added in rank order (a
fixed order, so the result does not depend on timing); the ratios are formed
from the totals.

The host logic here (plan, exchange schedule, combination) does not touch a
device; the engine that steps a slab and packs its rows is a grid of the C ABI
(`GridEngine`), and the messages go through `TorchComm` (torch.distributed:
NCCL between devices, gloo on CPU) or, for several slabs on one device in one
process, `LocalComm`.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass
from typing import List, Sequence

from .workloads import GridSpec

# the additive quantities of a diagnostics record
SUMS = ("H_phi", "H_g0", "H_g1", "W", "sum_xB1z2", "sum_B1z2", "gauss_l2")
MARGIN = 4


def split_axis(spec: GridSpec) -> int:
    """Axis (0 = x, 1 = y, 2 = z) whose rows the slabs own: the slowest with n > 1."""
    return 2 if spec.n[2] > 1 else (1 if spec.n[1] > 1 else 0)


@dataclass
class SlabPlan:
    """Rows of one rank's slab, in global row indices along the split axis.

    own_lo, own_hi: the owned rows [own_lo, own_hi);
    lo, hi: the slab's rows [lo, hi) (periodic: may run past either end);
    halo_lo, halo_hi: halo rows below and above the owned ones;
    spec: the slab's own grid (its sizes, origin and boundaries)."""

    rank: int
    world: int
    k: int
    axis: int
    rows: int
    periodic: bool
    own_lo: int
    own_hi: int
    halo_lo: int
    halo_hi: int
    width: int  # the halo width of every cut or periodic seam
    spec: GridSpec

    @property
    def lo(self) -> int:
        return self.own_lo - self.halo_lo

    @property
    def hi(self) -> int:
        return self.own_hi + self.halo_hi

    @property
    def up(self) -> int:
        return (self.rank + 1) % self.world

    @property
    def down(self) -> int:
        return (self.rank - 1) % self.world

    def halo_lo_of(self, r: int) -> int:
        """Halo rows below rank r's owned rows."""
        return self.width if (self.periodic or r > 0) else 0

    def halo_hi_of(self, r: int) -> int:
        """Halo rows above rank r's owned rows."""
        return self.width if (self.periodic or r < self.world - 1) else 0


def owned_range(rows: int, rank: int, world: int):
    """Balanced split of `rows` rows: rank r owns [r rows / world, (r+1) rows / world)."""
    return rows * rank // world, rows * (rank + 1) // world


def halo_width(spec: GridSpec, k: int) -> int:
    a = split_axis(spec)
    periodic = spec.em_bc[a][0] == "periodic"
    return k + 2 + MARGIN + (0 if periodic else spec.pml_cells)


def plan(spec: GridSpec, rank: int, world: int, k: int) -> SlabPlan:
    """The slab of rank `rank` of `world` for k steps between exchanges."""
    if world < 1 or not 0 <= rank < world or k < 1:
        raise ValueError("rank %d of %d, k = %d" % (rank, world, k))
    a = split_axis(spec)
    rows = spec.n[a]
    periodic = spec.em_bc[a][0] == "periodic"
    for side in range(2):
        for bc in (spec.em_bc[a][side], spec.axion_bc[a][side]):
            if bc not in ("periodic", "pml"):
                raise ValueError("slabs need a periodic or absorbing (PML) split axis, not %r" % bc)
    if any(bc == "outflow" for ax in spec.axion_bc for bc in ax):
        raise ValueError("outflow ghost planes are not split across slabs")
    own_lo, own_hi = owned_range(rows, rank, world)
    h = halo_width(spec, k) if world > 1 else 0
    if world > 1 and min(owned_range(rows, r, world)[1] - owned_range(rows, r, world)[0] for r in range(world)) < h:
        raise ValueError("%d rows over %d ranks leave slabs thinner than their %d-row halo" % (rows, world, h))
    halo_lo = h if (world > 1 and (periodic or rank > 0)) else 0
    halo_hi = h if (world > 1 and (periodic or rank < world - 1)) else 0
    n = list(spec.n)
    n[a] = own_hi - own_lo + halo_lo + halo_hi
    lo = list(spec.lo)
    lo[a] = spec.lo[a] + (own_lo - halo_lo) * spec.d[a]
    em, ax = [list(x) for x in spec.em_bc], [list(x) for x in spec.axion_bc]
    if not periodic:  # cut sides carry a layer (inside the halo); grid edges keep theirs
        if rank > 0:
            em[a][0] = ax[a][0] = "pml"
        if rank < world - 1:
            em[a][1] = ax[a][1] = "pml"
    sub = dataclasses.replace(spec, n=tuple(n), lo=tuple(lo), em_bc=tuple(tuple(x) for x in em),
                              axion_bc=tuple(tuple(x) for x in ax))
    return SlabPlan(rank, world, k, a, rows, periodic, own_lo, own_hi, halo_lo, halo_hi, h, sub)


def schedule(p: SlabPlan):
    """The two exchange phases of a round, as (send_to, send_rows, recv_from,
    recv_rows), rows in this slab's own indices [start, start + count):
    phase 0 moves rows upwards (the top owned rows fill the upper neighbour's low
    halo), phase 1 downwards.  A phase with nothing to move is None."""
    if p.world == 1:
        return [(None, None), (None, None)]
    own = p.own_hi - p.own_lo
    base = p.halo_lo  # slab index of the first owned row
    out = []
    # phase 0: upwards.  Rank r sends its top rows to r+1's low halo (which exists
    # unless r+1 wraps past a non-periodic edge) and fills its own low halo from r-1.
    send = (p.up, (base + own - p.halo_lo_of(p.up), p.halo_lo_of(p.up))) if p.halo_lo_of(p.up) else None
    recv = (p.down, (0, p.halo_lo)) if p.halo_lo else None
    out.append((send, recv))
    # phase 1: downwards
    send = (p.down, (base, p.halo_hi_of(p.down))) if p.halo_hi_of(p.down) else None
    recv = (p.up, (base + own, p.halo_hi)) if p.halo_hi else None
    out.append((send, recv))
    return out


def combine(records: Sequence[dict]) -> dict:
    """One record from the slabs' records (owned rows each), summed in rank order."""
    tot = {k: 0.0 for k in SUMS}
    for r in records:
        for k in SUMS:
            tot[k] += r[k]
    out = dict(tot)
    out["step"] = records[0]["step"]
    out["t"] = records[0]["t"]
    out["P_g2a"] = tot["H_phi"] / tot["H_g0"] if tot["H_g0"] > 0 else 0.0
    out["P_a2g"] = tot["H_g1"] / tot["H_phi"] if tot["H_phi"] > 0 else 0.0
    return out


# ---------------------------------------------------------------------------
# engines and communicators
# ---------------------------------------------------------------------------

class GridEngine:
    """A slab stepped by a grid of the C ABI on this process's device; rows move
    through device buffers (axp_pack_rows / axp_unpack_rows)."""

    def __init__(self, p: SlabPlan, stream=None, device=None):
        from . import axp

        self.axp = axp
        self.plan = p
        self.grid = axp.Grid(p.spec, stream=stream, device=device)

    def step(self, k: int):
        self.grid.step(k)

    def pack(self, start: int, count: int):
        import torch

        n = self.axp.axp_rows_bytes(self.grid.h, count)
        buf = torch.empty(n, dtype=torch.uint8, device=self.grid.device)
        self.axp.axp_pack_rows(self.grid.h, start, count, buf.data_ptr(), n)
        return buf

    def empty(self, count: int):
        import torch

        n = self.axp.axp_rows_bytes(self.grid.h, count)
        return torch.empty(n, dtype=torch.uint8, device=self.grid.device)

    def unpack(self, start: int, count: int, buf):
        self.axp.axp_unpack_rows(self.grid.h, start, count, buf.data_ptr(), buf.numel())

    def load(self, state: dict):
        self.grid.load(state)

    def inject_laser(self, L):
        self.grid.inject_laser(L)

    def inject_axion(self, A):
        self.grid.inject_axion(A)

    def fields(self) -> dict:
        return self.grid.fields()

    def owned_record(self) -> dict:
        p = self.plan
        return self.axp.axp_compute_diagnostics_rows(self.grid.h, p.halo_lo, p.halo_lo + p.own_hi - p.own_lo)

    def close(self):
        self.grid.close()


class TorchComm:
    """Point-to-point messages between ranks with torch.distributed (one slab per
    rank).  Sends and receives of a phase are posted together, so no ordering of
    the ranks can deadlock."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group

    def phase(self, send, send_buf, recv, recv_buf):
        ops = []
        if send is not None:
            ops.append(self.dist.P2POp(self.dist.isend, send_buf, send[0], group=self.group))
        if recv is not None:
            ops.append(self.dist.P2POp(self.dist.irecv, recv_buf, recv[0], group=self.group))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()

    def gather_records(self, rec: dict) -> List[dict]:
        import torch

        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        mine = torch.tensor([rec[k] for k in SUMS] + [float(rec["step"]), rec["t"]], dtype=torch.float64, device=dev)
        allr = [torch.empty_like(mine) for _ in range(self.dist.get_world_size(self.group))]
        self.dist.all_gather(allr, mine, group=self.group)
        out = []
        for t in allr:
            v = t.cpu().tolist()
            r = dict(zip(SUMS, v[:len(SUMS)]))
            r["step"], r["t"] = int(v[len(SUMS)]), v[len(SUMS) + 1]
            out.append(r)
        return out


class SlabRun:
    """One rank's part of a decomposed grid: plan, engine and communicator."""

    def __init__(self, spec: GridSpec, rank: int, world: int, k: int, comm, engine_factory=GridEngine):
        self.plan = plan(spec, rank, world, k)
        self.engine = engine_factory(self.plan)
        self.comm = comm

    def load_global(self, state: dict):
        """Set this slab from a whole-grid host state (numpy arrays of shape
        (nz, ny, nx)): its rows [lo, hi), wrapped along a periodic axis."""
        import numpy as np

        p = self.plan
        ax = 2 - p.axis  # array axis of the split axis
        idx = np.arange(p.lo, p.hi) % p.rows
        self.engine.load({k: np.take(v, idx, axis=ax) for k, v in state.items()})

    def owned(self, fields: dict) -> dict:
        """The owned rows of this slab's host fields."""
        import numpy as np

        p = self.plan
        ax = 2 - p.axis
        return {k: np.take(v, np.arange(p.halo_lo, p.halo_lo + p.own_hi - p.own_lo), axis=ax)
                for k, v in fields.items()}

    def exchange(self):
        for send, recv in schedule(self.plan):
            sbuf = self.engine.pack(*send[1]) if send is not None else None
            rbuf = self.engine.empty(recv[1][1]) if recv is not None else None
            self.comm.phase(send, sbuf, recv, rbuf)
            if recv is not None:
                self.engine.unpack(recv[1][0], recv[1][1], rbuf)

    def run(self, rounds: int):
        """rounds x (k steps, then a halo exchange)."""
        for _ in range(rounds):
            self.engine.step(self.plan.k)
            self.exchange()

    def diagnostics(self) -> dict:
        """The whole grid's record (right after an exchange: every halo row exact)."""
        return combine(self.comm.gather_records(self.engine.owned_record()))


def run_local(runs: Sequence["SlabRun"], rounds: int):
    """Several slabs of one grid in one process (one device): k steps each, then
    the two exchange phases with every send packed before any receive is
    unpacked (sends read owned rows, receives write halo rows)."""
    for _ in range(rounds):
        for r in runs:
            r.engine.step(r.plan.k)
        for ph in range(2):
            bufs = {}
            for r in runs:
                send, _ = schedule(r.plan)[ph]
                if send is not None:
                    bufs[(r.plan.rank, send[0])] = r.engine.pack(*send[1])
            for r in runs:
                _, recv = schedule(r.plan)[ph]
                if recv is not None:
                    r.engine.unpack(recv[1][0], recv[1][1], bufs[(recv[0], r.plan.rank)])


class LocalComm:
    """Placeholder communicator of slabs run together by run_local: records are
    combined by the caller."""

    def phase(self, *a):
        raise RuntimeError("slabs in one process exchange through run_local")

"""Serving loop for conversion-probability requests: continuous batching.

Requests (1D and 2D conversion runs, each with its own size, mass, coupling,
field and step count) arrive over time.  The server admits an arrived request
as soon as device memory and a slot are free for it, keeps its state resident
on the device until it finishes, and advances all live requests together:

* 1D requests live in one axp_batch (one cell pool, first-fit admission; one
  persistent time-blocked launch advances them all);
* 2D requests each own an FP32-split grid (admitted while the 2D memory budget
  holds its workspace) and are members of one axp_group (one launch per step
  advances all of them).

Each round issues work on both streams (sized so that a round takes about
`round_s` of device time), then polls progress; finished requests are read
out (FP64 diagnostics), removed, and their memory goes back to the pool at
once.  Nothing is recomputed on the host: every step runs in libaxp.so.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import axp as _axp
from . import batch as _batch
from . import group as _group
from . import workloads as W


@dataclass
class Record:
    index: int
    ndim: int
    arrival: float
    admitted: float = -1.0
    finished: float = -1.0
    P_g2a: float = float("nan")
    H_phi: float = float("nan")

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class ServeStats:
    records: list
    wall_s: float
    rounds: int
    launches: int
    max_live: int
    extra: dict = field(default_factory=dict)

    def summary(self):
        lat = np.array([r.latency for r in self.records])
        done = len(self.records)
        first = min(r.arrival for r in self.records)
        last = max(r.finished for r in self.records)
        out = {"requests": done, "sims_per_s": done / max(last - first, 1e-9), "wall_s": self.wall_s,
               "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
               "mean_latency_s": float(lat.mean()), "p99_tail_samples": int((lat >= np.percentile(lat, 99)).sum()),
               "rounds": self.rounds, "gpu_launches": self.launches, "max_live": self.max_live}
        # per class (1D and 2D requests)
        for nd in (1, 2):
            cl = np.array([r.latency for r in self.records if r.ndim == nd])
            if len(cl):
                out["class_%dd" % nd] = {"requests": int(len(cl)), "p50_latency_s": float(np.percentile(cl, 50)),
                                         "p99_latency_s": float(np.percentile(cl, 99)),
                                         "mean_latency_s": float(cl.mean()),
                                         "p99_tail_samples": int((cl >= np.percentile(cl, 99)).sum())}
        return out


def batch_instance(r: W.Request):
    return _batch.scan_instance(W.ScanInstance(r.n[0], r.m, r.g, r.B0, r.steps))


class Server:
    """Continuous-batching server on one GPU.

    mem_1d_cells: cells of the 1D pool (64 bytes per cell: two copies of eight
    FP32 arrays); mem_2d_bytes: budget for the 2D grids' workspaces."""

    def __init__(self, mem_1d_cells=16 << 20, max_1d=4096, mem_2d_bytes=8 << 30, max_2d=256, max_tiles=65536,
                 round_s=0.02, graphs=True):
        self.batch = _batch.Batch(max_1d, mem_1d_cells, graphs=graphs)
        self.group = _group.Group(max_2d, max_tiles, graphs=graphs)
        self.mem_2d = mem_2d_bytes
        self.max_tiles = max_tiles
        self.used_2d = 0
        self.round_s = round_s
        # device rates (cell-updates/s) used to size a round; refined as it runs
        self.rate_1d = 1.0e11
        self.rate_2d = 1.0e10

    def close(self):
        self.group.close()
        self.batch.close()

    # -- admission ---------------------------------------------------------
    def _admit_1d(self, r):
        return self.batch.try_add(batch_instance(r))

    def _admit_2d(self, r):
        w = W.request_workload(r, precision="fp32")
        desc = _axp.desc_of(w.grid)
        need = _axp.axp_workspace_bytes(desc)
        if self.used_2d + need > self.mem_2d:
            return None
        if _group.tiles_of(r.n[0], r.n[1]) > self.group_free_tiles():
            return None
        g = _axp.Grid(w.grid)
        g.inject_laser(w.lasers[0])
        m = self.group.add(g, r.steps)
        if m is None:
            g.close()
            return None
        self.used_2d += need
        return m, g, need

    def group_free_tiles(self):
        used = sum(_group.tiles_of(g.spec.n[0], g.spec.n[1]) for g in self.group.members.values())
        return self.max_tiles - used

    # -- the loop ------------------------------------------------------------
    def serve(self, requests, clock_scale=1.0):
        """Run the request stream to completion.  Arrival times are seconds from
        the start (scaled by clock_scale); returns ServeStats."""
        import torch

        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = collections.deque(order)
        queue = []
        live1, live2 = {}, {}  # slot -> index; member -> (index, grid, bytes)
        recs = {i: Record(i, requests[i].ndim, requests[i].arrival * clock_scale) for i in order}
        done = []
        rounds = 0
        launches0 = self.batch.launches() + self.group.launches()
        max_live = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        while len(done) < len(requests):
            t = now()
            while pending and recs[pending[0]].arrival <= t:
                queue.append(pending.popleft())
            # admit in arrival order; a request that does not fit yet lets later ones by
            keep = []
            for i in queue:
                r = requests[i]
                if r.ndim == 1:
                    s = self._admit_1d(r)
                    if s is None:
                        keep.append(i)
                        continue
                    live1[s] = i
                else:
                    a = self._admit_2d(r)
                    if a is None:
                        keep.append(i)
                        continue
                    live2[a[0]] = (i, a[1], a[2])
                recs[i].admitted = now()
            queue = keep
            max_live = max(max_live, len(live1) + len(live2))
            if not live1 and not live2:
                if pending:
                    time.sleep(max(0.0, recs[pending[0]].arrival - now()))
                    continue
                raise RuntimeError("requests that can never be admitted: %s" % queue)
            # one round of device work on both streams
            cells1 = sum(self.batch.nx[s] for s in live1)
            cells2 = sum(live2[m][1].cells for m in live2)
            k1 = int(min(4096, max(64, self.round_s * self.rate_1d / max(cells1, 1)))) if live1 else 0
            k2 = int(min(1024, max(8, self.round_s * self.rate_2d / max(cells2, 1)))) if live2 else 0
            k1 = 1 << (k1.bit_length() - 1) if k1 else 0  # powers of two keep the captured graphs few
            k2 = 1 << (k2.bit_length() - 1) if k2 else 0
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            if k1:
                e1[0].record(self.batch.stream)
                self.batch.run(k1)
                e1[1].record(self.batch.stream)
            if k2:
                e2[0].record(self.group.stream)
                self.group.run(k2)
                e2[1].record(self.group.stream)
            rounds += 1
            if k1:
                prog = self.batch.progress()
                d1 = e1[0].elapsed_time(e1[1]) / 1e3
                if d1 > 0:
                    self.rate_1d = 0.5 * self.rate_1d + 0.5 * cells1 * k1 / d1
                t = now()
                fin = [s for s in live1 if prog[s] >= requests[live1[s]].steps]
                for s, d in zip(fin, self.batch.results(fin)):
                    i = live1.pop(s)
                    self.batch.remove(s)
                    recs[i].P_g2a, recs[i].H_phi, recs[i].finished = d["P_g2a"], d["H_phi"], now()
                    done.append(i)
            if k2:
                prog = self.group.progress()
                d2 = e2[0].elapsed_time(e2[1]) / 1e3
                if d2 > 0:
                    self.rate_2d = 0.5 * self.rate_2d + 0.5 * cells2 * k2 / d2
                for m in [m for m in live2 if prog[m] >= requests[live2[m][0]].steps]:
                    i, g, need = live2.pop(m)
                    self.group.remove(m)
                    d = g.diagnostics()
                    g.close()
                    self.used_2d -= need
                    recs[i].P_g2a, recs[i].H_phi, recs[i].finished = d["P_g2a"], d["H_phi"], now()
                    done.append(i)
        wall = now()
        launches = self.batch.launches() + self.group.launches() - launches0
        return ServeStats([recs[i] for i in sorted(done)], wall, rounds, launches, max_live)

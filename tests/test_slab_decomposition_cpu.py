"""The slab decomposition a grid larger than one GPU would take, checked on CPU.

One step's dependency cone is one cell wide on each side: E and B each read one
neighbour per half-step, and the axion reads one per step.  The axion current
widens it once more, by its two-cell stencil (the central gradient of phi and
the face average).  So a rank that owns a slab of rows along the march axis (y
in 2D, z in 3D) can advance it k steps on its own. It needs k + 2 halo rows on
each side, refreshed from its neighbours' owned rows every k steps.

Here gloo ranks on CPU each step their slab with the oracle and swap halo rows
of every array, both axion levels included, by send/recv.  After several rounds
the owned rows must equal the undivided oracle run from the same start, bit for
bit.  The slabs' own grids are periodic along the split axis: what wraps in at
their seams is wrong data, and the halo absorbs it.  A halo one row short fails
the same comparison."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2406_16796_gb300 import workloads as W

NAMES = list(W.FIELD_NAMES) + ["phi_cur", "phi_old"]
CASES = {
    # global cells, split axis of the (nz, ny, nx) arrays, steps between exchanges, rounds
    "2d_split_y": dict(n=(24, 48, 1), axis=1, k=3, rounds=4),
    "3d_split_z": dict(n=(8, 6, 36), axis=0, k=2, rounds=3),
}


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def grid_of(n):
    d = (0.05, 0.07, 0.06)
    nd = [a for a in range(3) if n[a] > 1]
    dt = 0.5 / np.sqrt(sum(1.0 / d[a] ** 2 for a in nd))
    return W.GridSpec(n=n, d=d, dt=dt, m=1.1, g=0.7, B_ext=(0.3, -0.2, 1.0), E_ext=(0.0, 0.0, 0.0))


def rows(a, axis, lo, hi):
    """Rows lo..hi-1 of `a` along `axis`, wrapping periodically."""
    idx = np.arange(lo, hi) % a.shape[axis]
    return np.take(a, idx, axis=axis)


def _rank_main(rank, world, port, case, out):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASES[case]
        n, axis, k, rounds = c["n"], c["axis"], c["k"], c["rounds"]
        glob = grid_of(n)
        start = W.random_state(glob, seed=4242)
        N = start["E0x"].shape[axis]
        own = N // world
        w = k + 2
        r0 = rank * own
        # this rank's slab grid: owned rows plus w halo rows on each side
        ln = list(n)
        ln[2 - axis] = own + 2 * w  # (nx, ny, nz) order of GridSpec.n
        og = oracle.OracleGrid(glob.replace(n=tuple(ln)))
        og.load({name: rows(start[name], axis, r0 - w, r0 + own + w) for name in NAMES})
        up, down = (rank + 1) % world, (rank - 1) % world

        def pack(f, lo, hi):
            return torch.from_numpy(np.stack([rows(f[name], axis, lo, hi) for name in NAMES]))

        for _ in range(rounds):
            og.step(k)
            f = og.fields()
            # my top owned rows become the upper neighbour's lower halo, my bottom
            # owned rows the lower neighbour's upper halo
            top, bottom = pack(f, own, own + w), pack(f, w, 2 * w)
            from_down, from_up = torch.empty_like(top), torch.empty_like(bottom)
            reqs = [dist.isend(top, up, tag=0), dist.isend(bottom, down, tag=1),
                    dist.irecv(from_down, down, tag=0), dist.irecv(from_up, up, tag=1)]
            for q in reqs:
                q.wait()
            for i, name in enumerate(NAMES):
                a = f[name]
                sl_lo = [slice(None)] * 3
                sl_hi = [slice(None)] * 3
                sl_lo[axis] = slice(0, w)
                sl_hi[axis] = slice(own + w, own + 2 * w)
                a[tuple(sl_lo)] = from_down[i].numpy()
                a[tuple(sl_hi)] = from_up[i].numpy()
            og.load(f)
        f = og.fields()
        mine = torch.from_numpy(np.stack([rows(f[name], axis, w, w + own) for name in NAMES]))
        if rank == 0:
            parts = [mine]
            for src in range(1, world):
                t = torch.empty_like(mine)
                dist.recv(t, src)
                parts.append(t)
            whole = torch.cat(parts, dim=1 + axis).numpy()
            ref = oracle.OracleGrid(glob)
            ref.load(start)
            ref.step(k * rounds)
            rf = ref.fields()
            bad = [name for i, name in enumerate(NAMES) if not np.array_equal(whole[i], rf[name])]
            moved = all(not np.array_equal(rf[name], start[name]) for name in NAMES)
            out.put((bad, moved))
        else:
            dist.send(mine, 0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_slabs_with_halo_exchange_equal_the_undivided_run(case):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    bad, moved = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert moved, "every array must change over the run"
    assert bad == [], bad


@pytest.mark.parametrize("case", sorted(CASES))
def test_a_halo_one_row_short_is_caught(case):
    """k + 2 halo rows reproduce the undivided run after k steps and k + 1 do not:
    the bound is tight, and the comparison can fail."""
    import oracle

    c = CASES[case]
    n, axis = c["n"], c["axis"]
    glob = grid_of(n)
    start = W.random_state(glob, seed=4243)
    own = start["E0x"].shape[axis] // 2
    for k in (1, 3):
        ref = oracle.OracleGrid(glob)
        ref.load(start)
        ref.step(k)
        rf = ref.fields()

        def slab_matches(w):
            ln = list(n)
            ln[2 - axis] = own + 2 * w
            og = oracle.OracleGrid(glob.replace(n=tuple(ln)))
            og.load({name: rows(start[name], axis, -w, own + w) for name in NAMES})
            og.step(k)
            f = og.fields()
            return all(np.array_equal(rows(f[name], axis, w, w + own), rows(rf[name], axis, 0, own)) for name in NAMES)

        assert slab_matches(k + 2), k
        assert not slab_matches(k + 1), k

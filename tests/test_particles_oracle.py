"""Pins of the oracle's perturbed-particle current (arXiv 2406.16796 Sec. 2.2, FPS
particle method) against what the mathematics fixes, independent of how the
oracle writes its formulas:

- the quadratic B-spline shape: partition of unity, exact first moment, exact
  interpolation of a linear field and of its derivative, total deposited current;
- the Boris rotation: angle 2 atan(|q B dt / 2m| / gamma) and its sense;
- every first-order quantity (fields felt, momentum update, current, and a
  whole coupled run of fields and particles) is the derivative of the
  corresponding order-0 quantity, checked by central differences of order-0
  runs alone;
- the k = 0 response of a cold plasma: the leapfrog plasma oscillation
  sin(w dt/2) = w_p dt/2 exactly, and the R/L cutoffs of a magnetised plasma.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_16796_gb300.workloads import GridSpec

pytestmark = pytest.mark.filterwarnings("ignore")


def grid1d(n=16, d=0.25, dt=0.1, B_ext=(0.0, 0.0, 0.0), g=0.0):
    return GridSpec(n=(n, 1, 1), d=(d, d, d), dt=dt, B_ext=B_ext, g=g)


def grid2d(nx=12, ny=10, d=0.25, dt=0.1):
    return GridSpec(n=(nx, ny, 1), d=(d, d, d), dt=dt)


def node_pos(grid, kind, a, idx):
    """Position of node idx (i, j, k) of component a; kind 1 = E_a, 2 = B_a."""
    out = []
    for b in range(3):
        off = 0.5
        if kind == 1 and b == a:
            off = 1.0
        if kind == 2 and b != a:
            off = 1.0
        out.append(grid.lo[b] + (idx[b] + off) * grid.d[b])
    return np.array(out)


def interior_point(grid, rng, margin=3.0):
    """A position at least `margin` cells from the seam, and not within 0.05
    cells of any knot of either staggering (so central differences do not
    straddle a change of the spline's second derivative)."""
    while True:
        x = np.zeros(3)
        for b in range(3):
            if grid.n[b] > 1:
                x[b] = grid.lo[b] + grid.d[b] * rng.uniform(margin, grid.n[b] - margin)
        ok = True
        for b in range(3):
            if grid.n[b] > 1:
                f = ((x[b] - grid.lo[b]) / grid.d[b]) % 0.5
                ok = ok and 0.05 < f < 0.45
        if ok:
            return x


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("a", [0, 1, 2])
def test_gather_is_exact_on_linear_fields(kind, a):
    """A field linear in position (away from the periodic seam) is interpolated
    exactly by the quadratic B-spline, and its first-order part is exactly the
    field's gradient along x1: pins the staggered node positions, the weights
    and the derivative's sign and scale."""
    rng = np.random.default_rng(3 + kind * 10 + a)
    grid = grid2d()
    og = O.OracleGrid(grid)
    alpha, beta = 0.7, np.array([1.3, -0.4, 0.0])
    name = ("E0" if kind == 1 else "B0") + "xyz"[a]
    F = og.f[name]
    for k in range(grid.n[2]):
        for j in range(grid.n[1]):
            for i in range(grid.n[0]):
                F[k, j, i] = alpha + beta @ node_pos(grid, kind, a, (i, j, k))
    for _ in range(5):
        x0 = interior_point(grid, rng)
        x1 = rng.normal(size=3) * 0.1
        Enop, Bnop, Ep, Bp = og.gather(x0, x1)
        nop, p = (Enop, Ep) if kind == 1 else (Bnop, Bp)
        assert abs(nop[a] - (alpha + beta @ x0)) < 1e-13
        assert abs(p[a] - beta @ x1) < 1e-13
        others = [c for c in range(3) if c != a]
        assert np.all(np.abs(nop[others]) == 0) and np.all(np.abs(p[others]) == 0)


def test_deposit_moments():
    """One particle deposits a total current q w v over all nodes (partition of
    unity), centred on the particle (first moment), and its first-order part
    totals q w v1 (the derivative terms sum to zero)."""
    rng = np.random.default_rng(11)
    grid = grid2d()
    og = O.OracleGrid(grid)
    dV = grid.d[0] * grid.d[1] * grid.d[2]
    for _ in range(4):
        x0 = interior_point(grid, rng)
        x1 = rng.normal(size=3) * 0.05
        u0 = rng.normal(size=3) * 0.5
        u1 = rng.normal(size=3) * 0.1
        qw = -0.37
        j0, j1 = og.deposit(qw, x0, x1, u0, u1)
        g0 = math.sqrt(1 + u0 @ u0)
        v0 = u0 / g0
        v1 = (g0 * g0 * u1 - u0 * (u0 @ u1)) / g0 ** 3
        for a in range(3):
            assert abs(j0[a].sum() * dV - qw * v0[a]) < 1e-14
            assert abs(j1[a].sum() * dV - qw * v1[a]) < 1e-14
            # first moment along x of the order-0 current: the particle's position
            idx = np.argwhere(j0[a] != 0)
            mom = sum(j0[a][tuple(t)] * node_pos(grid, 1, a, (t[2], t[1], t[0]))[0] for t in idx)
            assert abs(mom * dV - qw * v0[a] * x0[0]) < 1e-13


def test_boris_rotation_angle_and_sense():
    """Pure magnetic field: |u| is kept and u turns by 2 atan(|q B dt/(2m)|/gamma)
    per step; an electron (q < 0) in B along +z turns counter-clockwise in (x, y)."""
    q, m, dt, B = -1.0, 1.0, 0.3, 2.0
    u = np.array([1.5, 0.0, 0.2])
    gam = math.sqrt(1 + u @ u)
    u_new, _ = O.kick(q / m, dt, u, np.zeros(3), np.zeros(3), np.array([0.0, 0.0, B]), np.zeros(3), np.zeros(3))
    assert abs(np.linalg.norm(u_new) - np.linalg.norm(u)) < 1e-14
    ang = math.atan2(u_new[1], u_new[0]) - math.atan2(u[1], u[0])
    assert ang > 0
    assert abs(ang - 2.0 * math.atan(abs(q * B * dt / (2 * m)) / gam)) < 1e-14
    assert u_new[2] == u[2]


def test_kick_first_order_is_its_derivative():
    """The first-order momentum update equals the central difference of the
    order-0 update along (u1, E_p, B_p)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        u0, u1 = rng.normal(size=3), rng.normal(size=3)
        E, B, Ep, Bp = rng.normal(size=3), rng.normal(size=3) * 2, rng.normal(size=3), rng.normal(size=3)
        qm, dt, eps = -1.7, 0.21, 1e-6
        _, d = O.kick(qm, dt, u0, u1, E, B, Ep, Bp)
        z = np.zeros(3)
        up, _ = O.kick(qm, dt, u0 + eps * u1, z, E + eps * Ep, B + eps * Bp, z, z)
        um, _ = O.kick(qm, dt, u0 - eps * u1, z, E - eps * Ep, B - eps * Bp, z, z)
        fd = (up - um) / (2 * eps)
        assert np.max(np.abs(fd - d)) < 1e-8 * (1 + np.max(np.abs(d)))


def test_gather_first_order_is_its_derivative():
    """F_p equals the central difference of F_nop along (x1, F1): the fields
    F0 + eps F1 felt at x0 + eps x1 (Sec. 2.2 expansion), on random fields."""
    rng = np.random.default_rng(9)
    grid = grid2d()
    og = O.OracleGrid(grid)
    F0 = {k: rng.normal(size=og.f[k].shape) for k in og.f}
    F1 = {k: rng.normal(size=og.f[k].shape) for k in og.f}
    for name in og.f:
        if name[1] == "0":
            og.f[name][...] = F0[name]
        else:
            og.f[name][...] = F1[name.replace("1", "0", 1)]
    for _ in range(6):
        x0 = interior_point(grid, rng)
        x1 = rng.normal(size=3) * 0.3
        x1[2] = 0.0
        Enop, Bnop, Ep, Bp = og.gather(x0, x1)
        eps = 1e-6
        outs = []
        for sgn in (1, -1):
            o2 = O.OracleGrid(grid)
            for name in o2.f:
                if name[1] == "0":
                    o2.f[name][...] = F0[name] + sgn * eps * F1[name]
            outs.append(o2.gather(x0 + sgn * eps * x1, np.zeros(3)))
        fdE = (outs[0][0] - outs[1][0]) / (2 * eps)
        fdB = (outs[0][1] - outs[1][1]) / (2 * eps)
        assert np.max(np.abs(fdE - Ep)) < 1e-7
        assert np.max(np.abs(fdB - Bp)) < 1e-7


def test_deposit_first_order_is_its_derivative():
    rng = np.random.default_rng(13)
    grid = grid2d()
    og = O.OracleGrid(grid)
    for _ in range(4):
        x0 = interior_point(grid, rng)
        x1 = rng.normal(size=3) * 0.3
        u0, u1 = rng.normal(size=3), rng.normal(size=3)
        _, j1 = og.deposit(-0.8, x0, x1, u0, u1)
        eps = 1e-6
        z = np.zeros(3)
        jp, _ = og.deposit(-0.8, x0 + eps * x1, z, u0 + eps * u1, z)
        jm, _ = og.deposit(-0.8, x0 - eps * x1, z, u0 - eps * u1, z)
        fd = (jp - jm) / (2 * eps)
        assert np.max(np.abs(fd - j1)) < 1e-7 * (1 + np.max(np.abs(j1)))


def uniform_plasma(grid, ppc, density, q=-1.0, m=1.0):
    """ppc particles per cell at equal spacing along x (1D grid), at rest."""
    n = grid.n[0] * ppc
    x = grid.lo[0] + (np.arange(n) + 0.5) * grid.d[0] / ppc
    X = np.zeros((3, n))
    X[0] = x
    dV = grid.d[0] * grid.d[1] * grid.d[2]
    w = np.full(n, density * dV / ppc)
    return q, m, w, X


def k0_map(grid, ppc, density, comps):
    """One-step linear map of a uniform first-order state (u1 components and
    E1 components listed in comps) of a cold plasma at rest, columns from unit
    initial states."""
    q, m, w, X = uniform_plasma(grid, ppc, density)
    n = w.shape[0]
    M = np.zeros((len(comps), len(comps)))
    for c, (kind0, a0) in enumerate(comps):
        og = O.OracleGrid(grid)
        u1 = np.zeros((3, n))
        if kind0 == "u":
            u1[a0] = 1.0
        else:
            og.f["E1" + "xyz"[a0]][...] = 1.0
        og.attach_particles(q, m, w, X, np.zeros((3, n)), None, u1)
        og.step(1)
        st = og.particles_now()
        for r, (kind, a) in enumerate(comps):
            if kind == "u":
                vals = st["u1"][a]
            else:
                vals = og.f["E1" + "xyz"[a]].ravel()
            assert np.ptp(vals) < 1e-13  # the state stays uniform
            M[r, c] = vals.mean()
    return M


def test_cold_plasma_oscillation_is_the_leapfrog_oscillator():
    """k = 0 first-order response of a cold plasma at rest: u1x and E1x form a
    leapfrog oscillator, so the one-step map has determinant 1 and trace
    2 - (w_p dt)^2, i.e. sin(w dt/2) = w_p dt/2 with w_p^2 = n q^2/m."""
    grid = grid1d(n=8, d=0.5, dt=0.2)
    density = 3.0
    M = k0_map(grid, 4, density, [("u", 0), ("E", 0)])
    wp2 = density * 1.0 / 1.0
    assert abs(np.linalg.det(M) - 1.0) < 1e-13
    assert abs(np.trace(M) - (2.0 - wp2 * grid.dt ** 2)) < 1e-13


def test_magnetised_plasma_cutoffs():
    """k = 0 response of a cold electron plasma in B along z: the two frequencies
    of the (u1x, u1y, E1x, E1y) map are the R and L cutoffs
    sqrt(w_c^2/4 + w_p^2) +- w_c/2, to the scheme's second order in w dt."""
    dt = 0.005
    B = 1.5
    grid = grid1d(n=8, d=0.5, dt=dt, B_ext=(0.0, 0.0, B))
    density = 1.0
    M = k0_map(grid, 2, density, [("u", 0), ("u", 1), ("E", 0), ("E", 1)])
    ev = np.linalg.eigvals(M)
    assert np.max(np.abs(np.abs(ev) - 1.0)) < 1e-12
    w = np.sort(np.abs(np.angle(ev)) / dt)
    wc, wp = B, 1.0
    wR = math.sqrt(wc * wc / 4 + wp * wp) + wc / 2
    wL = math.sqrt(wc * wc / 4 + wp * wp) - wc / 2
    assert np.allclose(w, [wL, wL, wR, wR], rtol=2e-5, atol=0)


def test_positions_round_trip():
    """Positions handed in at t_n come back at t_n after the half-step shift."""
    rng = np.random.default_rng(21)
    grid = grid2d()
    og = O.OracleGrid(grid)
    n = 40
    X = np.zeros((3, n))
    X[0] = rng.uniform(0, grid.n[0] * grid.d[0], n)
    X[1] = rng.uniform(0, grid.n[1] * grid.d[1], n)
    U = rng.normal(size=(3, n)) * 0.3
    X1, U1 = rng.normal(size=(3, n)) * 0.01, rng.normal(size=(3, n)) * 0.01
    og.attach_particles(-1.0, 1.0, np.ones(n), X, U, X1, U1)
    st = og.particles_now()
    L = np.array([grid.n[0] * grid.d[0], grid.n[1] * grid.d[1], 1.0])
    dx = (st["x0"] - X + L[:, None] / 2) % L[:, None] - L[:, None] / 2
    assert np.max(np.abs(dx[:2])) < 1e-13
    assert np.max(np.abs(st["x1"] - X1)) < 1e-15


def test_invalid_particles_are_refused():
    absorbing = (("pml", "pml"), ("periodic", "periodic"), ("periodic", "periodic"))
    grid = GridSpec(n=(64, 1, 1), d=(0.25, 0.25, 0.25), dt=0.1, pml_cells=8, em_bc=absorbing, axion_bc=absorbing)
    og = O.OracleGrid(grid)
    with pytest.raises(ValueError):
        og.attach_particles(-1.0, 1.0, np.ones(2), np.zeros((3, 2)), np.zeros((3, 2)))
    og = O.OracleGrid(grid1d())
    with pytest.raises(ValueError):
        og.attach_particles(-1.0, 0.0, np.ones(2), np.zeros((3, 2)), np.zeros((3, 2)))


def test_coupled_run_first_order_is_the_derivative_of_order_zero():
    """A whole coupled run (fields and particles, several steps) of the FPS
    system equals, in its first-order part, the central difference of two
    order-0 runs started from (order 0) +- eps (order 1).  Order 0 here is a
    laser in a warm magnetised plasma, so every term of Sec. 2.2 is exercised
    (v0 != 0, F0 with gradients, B_nop != 0).  g = 0: with an axion coupling the
    FPS system is not a linearisation of order 0 alone."""
    rng = np.random.default_rng(17)
    grid = GridSpec(n=(24, 1, 1), d=(0.25, 0.25, 0.25), dt=0.2, B_ext=(0.0, 0.3, 0.8))
    L = grid.n[0] * grid.d[0]
    kx = 2 * math.pi * 2 / L
    npart = 96
    X = np.zeros((3, npart))
    X[0] = rng.uniform(0, L, npart)
    U0 = rng.normal(size=(3, npart)) * 0.2
    X1 = np.zeros((3, npart))
    X1[0] = rng.normal(size=npart) * 0.02
    U1 = rng.normal(size=(3, npart)) * 0.05
    w = np.full(npart, 0.5 * grid.d[0] ** 3 * grid.n[0] / npart)

    def fields0(og):
        xs = grid.lo[0] + (np.arange(grid.n[0]) + 0.5) * grid.d[0]
        xf = xs + grid.d[0] / 2
        og.f["E0y"][...] = 0.3 * np.cos(kx * xs)
        og.f["B0z"][...] = 0.3 * np.cos(kx * xf)
        og.f["E0x"][...] = 0.1 * np.sin(kx * xf)

    F1 = {k: rng.normal(size=(1, 1, grid.n[0])) * 0.1 for k in ("E1x", "E1y", "E1z", "B1x", "B1y", "B1z")}
    steps = 6

    fps = O.OracleGrid(grid)
    fields0(fps)
    for k, v in F1.items():
        fps.f[k][...] = v
    fps.attach_particles(-1.0, 1.0, w, X, U0, X1, U1)
    fps.step(steps)
    st = fps.particles_now()

    eps = 1e-6
    runs = []
    for sgn in (1, -1):
        og = O.OracleGrid(grid)
        fields0(og)
        for k, v in F1.items():
            og.f[k.replace("1", "0", 1)][...] += sgn * eps * v
        og.attach_particles(-1.0, 1.0, w, X + sgn * eps * X1, U0 + sgn * eps * U1)
        og.step(steps)
        runs.append((og.fields(), og.particles_now()))
    for k in ("x", "y", "z"):
        for f in ("E", "B"):
            fd = (runs[0][0][f + "0" + k] - runs[1][0][f + "0" + k]) / (2 * eps)
            got = fps.f[f + "1" + k]
            assert np.max(np.abs(fd - got)) < 2e-6 * (1 + np.max(np.abs(got))), (f, k)
    fdu = (runs[0][1]["u0"] - runs[1][1]["u0"]) / (2 * eps)
    assert np.max(np.abs(fdu - st["u1"])) < 2e-6 * (1 + np.max(np.abs(st["u1"])))
    dx = runs[0][1]["x0"] - runs[1][1]["x0"]
    dx = (dx + L / 2) % L - L / 2
    assert np.max(np.abs(dx[0] / (2 * eps) - st["x1"][0])) < 2e-6
    fdj = (runs[0][1]["j0"] - runs[1][1]["j0"]) / (2 * eps)
    assert np.max(np.abs(fdj - st["j1"])) < 2e-6 * (1 + np.max(np.abs(st["j1"])))
    # the run is not trivial: first-order fields and currents grew from the particles
    assert np.max(np.abs(st["j1"])) > 1e-3 and np.max(np.abs(st["u1"] - U1)) > 1e-3


def test_magnetised_plasma_x_and_o_mode_dispersion():
    """Sec. 3.4's set-up in miniature: the first-order fields and particles of a
    cold electron plasma at rest in B along z (k along x) carry the cold-plasma
    modes.  The exact one-step map of a periodic 64-cell box (fields and particle
    momenta, built column by column from oracle steps) is diagonalised; at each
    of the box's lowest wave numbers the field-carrying frequencies are the
    O mode w^2 = w_p^2 + k^2 (E along B) and the two X-mode branches,
    k^2 = w^2 - w_p^2 (w^2 - w_p^2)/(w^2 - w_UH^2), w_UH^2 = w_p^2 + w_c^2
    (E across B).  k enters through its Yee form (2/dx) sin(k dx/2); what
    remains is the time discretisation's O((w dt)^2) (w dt <= 0.12 here) and
    the spline's O((k dx)^2) filtering of the plasma response, so the bound
    widens with k."""
    n, d, ppc = 64, 0.02, 2
    wp, wc = 5.0, 4.0
    dt = 0.5 * d
    grid = grid1d(n=n, d=d, dt=dt, B_ext=(0.0, 0.0, wc))
    npart = n * ppc
    X = np.zeros((3, npart))
    X[0] = (np.arange(npart) + 0.5) * d / ppc
    w = np.full(npart, wp ** 2 * d ** 3 / ppc)  # density w_p^2 (q = -1, m = 1)
    names = ["E1x", "E1y", "E1z", "B1x", "B1y", "B1z"]
    D = 6 * n + 3 * npart
    M = np.zeros((D, D))
    for i in range(D):
        vec = np.zeros(D)
        vec[i] = 1.0
        og = O.OracleGrid(grid)
        for c, k in enumerate(names):
            og.f[k][0, 0, :] = vec[c * n:(c + 1) * n]
        og.attach_particles(-1.0, 1.0, w, X, np.zeros((3, npart)), None, vec[6 * n:].reshape(3, npart))
        og.step(1)
        M[:, i] = np.concatenate([og.f[k][0, 0, :] for k in names] + [og.particles_now()["u1"].ravel()])
    ev, V = np.linalg.eig(M)
    assert np.max(np.abs(np.abs(ev) - 1.0)) < 1e-12  # no growth, no damping
    found = {}
    for j in range(D):
        om = abs(np.angle(ev[j])) / dt
        v = V[:, j]
        fld = v[:6 * n].reshape(6, n)
        if om < 1e-6 or np.linalg.norm(fld) < 1e-2 * np.linalg.norm(v):
            continue
        F = np.abs(np.fft.fft(fld, axis=1)) ** 2
        Fm = F.sum(axis=0)
        folded = Fm[: n // 2 + 1] + np.r_[Fm[0], Fm[:0:-1]][: n // 2 + 1]
        m = int(np.argmax(folded))
        found.setdefault(m, []).append((om, names[int(F[:, m].argmax())]))
    L = n * d
    for m, tol in ((0, 3e-4), (1, 1e-3), (2, 4e-3)):
        ke = 2.0 / d * math.sin(math.pi * m / L * d)
        U = wp ** 2 + wc ** 2
        b, c = U + wp ** 2 + ke ** 2, wp ** 4 + ke ** 2 * U
        x_lo, x_hi = math.sqrt((b - math.sqrt(b * b - 4 * c)) / 2), math.sqrt((b + math.sqrt(b * b - 4 * c)) / 2)
        o_mode = math.sqrt(wp ** 2 + ke ** 2)
        got = found[m]
        for target, across in ((x_lo, True), (o_mode, False), (x_hi, True)):
            best = min(got, key=lambda t: abs(t[0] - target))
            assert abs(best[0] - target) <= tol * target, (m, target, best)
            # the O mode's field lies along B, the X modes' across it
            assert (best[1] != "E1z") == across, (m, target, best)
        # nothing else carries fields at this wave number
        for wv, _ in got:
            assert min(abs(wv - t) for t in (x_lo, o_mode, x_hi)) <= tol * wv, (m, wv)


def test_boris_e_cross_b_drift():
    """Crossed uniform fields (E along y, B along z, |E| << |B|): a particle
    starting at rest gyrates about a guide centre drifting at E x B / B^2; over
    whole gyration periods its mean velocity is the drift, to the scheme's
    O((w_c dt)^2) and the relativistic O((E/B)^2)."""
    q, m, dt, B, E = -1.0, 1.0, 0.05, 2.0, 0.01
    h_rot = 2.0 * math.atan(abs(q) * B * dt / (2.0 * m))  # Boris turn per step
    steps = int(round(200 * 2.0 * math.pi / h_rot))  # about 200 gyrations
    u = np.zeros(3)
    z = np.zeros(3)
    vsum = np.zeros(3)
    for _ in range(steps):
        u, _ = O.kick(q / m, dt, u, z, np.array([0.0, E, 0.0]), np.array([0.0, 0.0, B]), z, z)
        vsum += u / math.sqrt(1.0 + u @ u)
    v = vsum / steps
    drift = E / B  # (E x B)_x / B^2 for E = E y-hat, B = B z-hat
    assert abs(v[0] - drift) < 5e-3 * drift
    assert abs(v[1]) < 5e-3 * drift and v[2] == 0.0

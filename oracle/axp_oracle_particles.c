/*
 * axp_oracle_particles.c -- plain FP64 CPU oracle of the perturbed-particle
 * current of arXiv 2406.16796, Sec. 2.2 (FPS method: the particle motion and
 * the current split into an order-0 part and its first-order perturbation).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU baseline leg of bench.py.  Shares no code with the CUDA path.
 *
 * What the paper fixes (Sec. 2.2):
 *  - fields felt by a particle at x0 + x1: F = F_nop + F_p with
 *    F_nop = sum_ijk S(r_ijk - x0) F0_ijk and
 *    F_p   = sum_ijk [dS(r_ijk - x)/dx at x0 . x1] F0_ijk + sum_ijk S(r_ijk - x0) F1_ijk;
 *  - dx1/dt = v1,  dp1/dt = q (E_p + v0 x B_p + v1 x B_nop),
 *    v1 = (dv/dp) p1 = (gamma0^2 u1 - u0 (u0 . u1)) / gamma0^3   (c = 1);
 *  - j0 + j1 at node ijk = (q/dV) [S(r - x0) v0 + (dS/dx at x0 . x1) v0 + S(r - x0) v1].
 *  - Sec. 2.3: the particles are pushed by the fields of both orders between
 *    the axion update and the second field half-steps.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *  - S is the quadratic B-spline (three nodes per active axis), the smooth
 *    shape whose derivative the first-order terms need; every component is
 *    gathered from (and every current deposited on) its own staggered nodes,
 *    j_a on the E_a nodes.
 *  - The order-0 push is the relativistic Boris scheme (half kick, rotation,
 *    half kick) with the fields at t_{n+1/2} at the position x^{n+1/2};
 *    momenta live at integer times, positions at half-integer times, and
 *    the current j^{n+1} is deposited at x^{n+1} = x^{n+1/2} + (dt/2) v^{n+1}
 *    with v^{n+1}: it is centred on the E interval [n+1/2, n+3/2] it enters.
 *  - The order-1 push is the first-order part of the order-0 push taken
 *    along (x1, u1, F_p): each Boris operation differentiated once.  Its
 *    continuum limit is the paper's equation for dp1/dt.
 *  - The uniform background (B_ext, E_ext) is part of F_nop; having no
 *    gradient, it adds nothing to F_p.
 *  - The macroparticle volume dV of the current is the cell volume d0 d1 d2;
 *    a particle of weight w stands for w physical particles.
 *  - Positions wrap into [lo, lo + n d) along every active (periodic) axis.
 */
#include "axp_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static int64_t cells_of(const orc_params *p) { return p->n[0] * p->n[1] * p->n[2]; }
static int64_t wrap_index(int64_t c, int64_t n) { return ((c % n) + n) % n; }

int orc_particles_validate(const orc_params *p, const orc_particles *P)
{
    if (orc_validate(p)) return 1;
    if (P->count < 0 || !(P->m > 0.0)) return 1;
    for (int a = 0; a < 3; a++)
        if (p->n[a] > 1 && (p->em_bc[a][0] != ORC_PERIODIC || p->em_bc[a][1] != ORC_PERIODIC)) return 1;
    return 0;
}

/* Node offset (in cells) of a staggered component along axis b:
 * kind 1 = E_a (face along a), kind 2 = B_a (faces along the other two). */
static double node_offset(int kind, int a, int b)
{
    if (kind == 1) return b == a ? 1.0 : 0.5;
    return b == a ? 0.5 : 1.0;
}

/* One axis of the shape: the nodes ic-1, ic, ic+1 nearest to the particle,
 * their quadratic B-spline weights W and dW/dx.  Along an invariant axis the
 * one node 0 has weight 1 and no derivative. */
typedef struct {
    int64_t node[3];
    double W[3], dW[3];
    int nn;
} axis_shape;

static void shape_axis(const orc_params *p, int kind, int a, int b, double x, axis_shape *s)
{
    if (p->n[b] == 1) {
        s->nn = 1;
        s->node[0] = 0;
        s->W[0] = 1.0;
        s->dW[0] = 0.0;
        return;
    }
    const double xi = (x - p->lo[b]) / p->d[b] - node_offset(kind, a, b);
    const double c = floor(xi + 0.5);
    const double del = xi - c;
    s->nn = 3;
    for (int t = 0; t < 3; t++) s->node[t] = wrap_index((int64_t)c + t - 1, p->n[b]);
    s->W[0] = 0.5 * (0.5 - del) * (0.5 - del);
    s->W[1] = 0.75 - del * del;
    s->W[2] = 0.5 * (0.5 + del) * (0.5 + del);
    /* d/dx = (1/d) d/d(del) */
    s->dW[0] = -(0.5 - del) / p->d[b];
    s->dW[1] = -2.0 * del / p->d[b];
    s->dW[2] = (0.5 + del) / p->d[b];
}

/* Visit every node of a component's stencil: weight S and the directional
 * derivative (dS/dx . x1). */
typedef struct {
    int64_t idx;
    double S, dS;
} node_weight;

static int stencil(const orc_params *p, int kind, int a, const double x0[3], const double x1[3], node_weight out[27])
{
    axis_shape sh[3];
    for (int b = 0; b < 3; b++) shape_axis(p, kind, a, b, x0[b], &sh[b]);
    int m = 0;
    for (int tk = 0; tk < sh[2].nn; tk++)
        for (int tj = 0; tj < sh[1].nn; tj++)
            for (int ti = 0; ti < sh[0].nn; ti++) {
                const double Wx = sh[0].W[ti], Wy = sh[1].W[tj], Wz = sh[2].W[tk];
                out[m].idx = sh[0].node[ti] + p->n[0] * (sh[1].node[tj] + p->n[1] * sh[2].node[tk]);
                out[m].S = Wx * Wy * Wz;
                out[m].dS = sh[0].dW[ti] * Wy * Wz * x1[0] + Wx * sh[1].dW[tj] * Wz * x1[1] +
                            Wx * Wy * sh[2].dW[tk] * x1[2];
                m++;
            }
    return m;
}

void orc_gather(const orc_params *p, const orc_state *s, const double x0[3], const double x1[3], double Enop[3],
                double Bnop[3], double Ep[3], double Bp[3])
{
    node_weight nw[27];
    for (int a = 0; a < 3; a++) {
        int m = stencil(p, 1, a, x0, x1, nw);
        double f0 = 0.0, fp = 0.0;
        for (int t = 0; t < m; t++) {
            f0 = f0 + nw[t].S * s->E0[a][nw[t].idx];
            fp = fp + nw[t].dS * s->E0[a][nw[t].idx] + nw[t].S * s->E1[a][nw[t].idx];
        }
        Enop[a] = f0 + p->E_ext[a];
        Ep[a] = fp;
        m = stencil(p, 2, a, x0, x1, nw);
        f0 = 0.0;
        fp = 0.0;
        for (int t = 0; t < m; t++) {
            f0 = f0 + nw[t].S * s->B0[a][nw[t].idx];
            fp = fp + nw[t].dS * s->B0[a][nw[t].idx] + nw[t].S * s->B1[a][nw[t].idx];
        }
        Bnop[a] = f0 + p->B_ext[a];
        Bp[a] = fp;
    }
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* velocity of both orders from the momenta: v0 = u0/gamma0 and
 * v1 = (gamma0^2 u1 - u0 (u0 . u1)) / gamma0^3 */
static void velocities(const double u0[3], const double u1[3], double v0[3], double v1[3])
{
    const double g0 = sqrt(1.0 + dot3(u0, u0));
    const double uu = dot3(u0, u1);
    for (int a = 0; a < 3; a++) {
        v0[a] = u0[a] / g0;
        v1[a] = (g0 * g0 * u1[a] - u0[a] * uu) / (g0 * g0 * g0);
    }
}

void orc_kick(double q_over_m, double dt, const double u0[3], const double u1[3], const double Enop[3],
              const double Bnop[3], const double Ep[3], const double Bp[3], double u0_out[3], double u1_out[3])
{
    const double h = q_over_m * dt / 2.0;
    double um[3], dum[3], t[3], dtv[3], up[3], dup[3], sv[3], dsv[3], c1[3], c2[3], c3[3];
    /* half kick */
    for (int a = 0; a < 3; a++) {
        um[a] = u0[a] + h * Enop[a];
        dum[a] = u1[a] + h * Ep[a];
    }
    /* rotation vector t = h B / gamma(u-) and its first-order part */
    const double gm = sqrt(1.0 + dot3(um, um));
    const double dgm = dot3(um, dum) / gm;
    for (int a = 0; a < 3; a++) {
        t[a] = h * Bnop[a] / gm;
        dtv[a] = h * Bp[a] / gm - t[a] * dgm / gm;
    }
    /* u' = u- + u- x t */
    cross3(um, t, c1);
    cross3(dum, t, c2);
    cross3(um, dtv, c3);
    for (int a = 0; a < 3; a++) {
        up[a] = um[a] + c1[a];
        dup[a] = dum[a] + c2[a] + c3[a];
    }
    /* s = 2 t / (1 + t.t) */
    const double tt = dot3(t, t), dtt = 2.0 * dot3(t, dtv);
    for (int a = 0; a < 3; a++) {
        sv[a] = 2.0 * t[a] / (1.0 + tt);
        dsv[a] = 2.0 * dtv[a] / (1.0 + tt) - 2.0 * t[a] * dtt / ((1.0 + tt) * (1.0 + tt));
    }
    /* u+ = u- + u' x s, then the second half kick */
    cross3(up, sv, c1);
    cross3(dup, sv, c2);
    cross3(up, dsv, c3);
    for (int a = 0; a < 3; a++) {
        u0_out[a] = (um[a] + c1[a]) + h * Enop[a];
        u1_out[a] = ((dum[a] + c2[a]) + c3[a]) + h * Ep[a];
    }
}

void orc_deposit(const orc_params *p, double qw, const double x0[3], const double x1[3], const double u0[3],
                 const double u1[3], double *j0[3], double *j1[3])
{
    const double dV = p->d[0] * p->d[1] * p->d[2];
    double v0[3], v1[3];
    velocities(u0, u1, v0, v1);
    node_weight nw[27];
    for (int a = 0; a < 3; a++) {
        const int m = stencil(p, 1, a, x0, x1, nw);
        for (int t = 0; t < m; t++) {
            j0[a][nw[t].idx] = j0[a][nw[t].idx] + qw / dV * (nw[t].S * v0[a]);
            j1[a][nw[t].idx] = j1[a][nw[t].idx] + qw / dV * (nw[t].dS * v0[a] + nw[t].S * v1[a]);
        }
    }
}

static double wrap_position(const orc_params *p, int b, double x)
{
    if (p->n[b] == 1) return x;
    const double L = (double)p->n[b] * p->d[b];
    if (x >= p->lo[b] + L) return x - L;
    if (x < p->lo[b]) return x + L;
    return x;
}

static void zero_currents(const orc_params *p, orc_particles *P)
{
    for (int a = 0; a < 3; a++) {
        memset(P->j0[a], 0, sizeof(double) * (size_t)cells_of(p));
        memset(P->j1[a], 0, sizeof(double) * (size_t)cells_of(p));
    }
}

static void load(const orc_particles *P, int64_t q, double x0[3], double x1[3], double u0[3], double u1[3])
{
    for (int a = 0; a < 3; a++) {
        x0[a] = P->x0[a][q];
        x1[a] = P->x1[a][q];
        u0[a] = P->u0[a][q];
        u1[a] = P->u1[a][q];
    }
}

void orc_particles_start(const orc_params *p, orc_particles *P)
{
    if (orc_particles_validate(p, P)) {
        fprintf(stderr, "orc_particles_start: invalid particles\n");
        abort();
    }
    zero_currents(p, P);
    for (int64_t q = 0; q < P->count; q++) {
        double x0[3], x1[3], u0[3], u1[3], v0[3], v1[3];
        load(P, q, x0, x1, u0, u1);
        orc_deposit(p, P->q * P->w[q], x0, x1, u0, u1, P->j0, P->j1);
        velocities(u0, u1, v0, v1);
        for (int a = 0; a < 3; a++) {
            P->x0[a][q] = wrap_position(p, a, x0[a] + (p->dt / 2.0) * v0[a]);
            P->x1[a][q] = x1[a] + (p->dt / 2.0) * v1[a];
        }
    }
}

void orc_particles_positions_now(const orc_params *p, const orc_particles *P, double *x0n[3], double *x1n[3])
{
    for (int64_t q = 0; q < P->count; q++) {
        double x0[3], x1[3], u0[3], u1[3], v0[3], v1[3];
        load(P, q, x0, x1, u0, u1);
        velocities(u0, u1, v0, v1);
        for (int a = 0; a < 3; a++) {
            x0n[a][q] = wrap_position(p, a, x0[a] - (p->dt / 2.0) * v0[a]);
            x1n[a][q] = x1[a] - (p->dt / 2.0) * v1[a];
        }
    }
}

void orc_push(const orc_params *p, const orc_state *s, orc_particles *P)
{
    zero_currents(p, P);
    const double dt = p->dt;
    for (int64_t q = 0; q < P->count; q++) {
        double x0[3], x1[3], u0[3], u1[3];
        double Enop[3], Bnop[3], Ep[3], Bp[3], u0n[3], u1n[3], v0[3], v1[3], xc0[3], xc1[3];
        load(P, q, x0, x1, u0, u1);
        /* fields at t_{n+1/2} felt at x^{n+1/2} */
        orc_gather(p, s, x0, x1, Enop, Bnop, Ep, Bp);
        /* u^n -> u^{n+1} */
        orc_kick(P->q / P->m, dt, u0, u1, Enop, Bnop, Ep, Bp, u0n, u1n);
        velocities(u0n, u1n, v0, v1);
        for (int a = 0; a < 3; a++) {
            /* x^{n+1} (where j^{n+1} is deposited) and x^{n+3/2} */
            xc0[a] = x0[a] + (dt / 2.0) * v0[a];
            xc1[a] = x1[a] + (dt / 2.0) * v1[a];
            P->x0[a][q] = wrap_position(p, a, x0[a] + dt * v0[a]);
            P->x1[a][q] = x1[a] + dt * v1[a];
            P->u0[a][q] = u0n[a];
            P->u1[a][q] = u1n[a];
        }
        orc_deposit(p, P->q * P->w[q], xc0, xc1, u0n, u1n, P->j0, P->j1);
    }
}

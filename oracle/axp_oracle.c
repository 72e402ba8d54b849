/*
 * axp_oracle.c -- plain FP64 CPU oracle of the axion-coupled Yee field update
 * (arXiv 2406.16796, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU baseline leg of bench.py.  Shares no code with the CUDA path.
 *
 * Written to be read against the paper, not to be fast: every array access
 * goes through the boundary-aware accessors below, every step of the time
 * scheme is its own loop, and nothing is fused or reordered beyond what the
 * equations state.  Build with -ffp-contract=off so that no multiply-add is
 * contracted and results are identical on every host.
 *
 * Readings of the paper that this file implements (each is also listed in
 * the design notes):
 *  - D_t phi in the second E half-step is (phi^{n+3/2} - phi^{n+1/2})/dt, the
 *    difference centred on n+1 (Sec. 2.3 prints D_t phi^{n+1/2}).
 *  - (D_t phi) B0 is formed at cell centres with the 4-point Bbar of Sec. 2.3
 *    and averaged to E locations over the two adjacent cells, the same rule
 *    the paper prints for the cross term E0 x grad phi.
 *  - E0^{n+1}, B0^{n+1} in the second E1 half-step are the order-0 fields of
 *    the same step, advanced first.
 *  - The uniform background B_ext, E_ext is held as constants and added to the
 *    averaged order-0 fields; arrays hold the laser part only.
 *  - Along a non-periodic axis E and B are zero outside the grid.  An optional
 *    absorbing layer of the same cubic profile as the axion PML damps E and B
 *    of both orders: F <- ((1 - s h/2) F + h X)/(1 + s h/2) per half-step h.
 *  - Axion ghosts are one cell deep; cells outside along two or more
 *    non-periodic axes (corners) hold 0.
 *  - Outflow (Sec. 2.4 item 3) is applied per face along the face normal, with
 *    the source S at the ghost computed by the same averaging rule (which sees
 *    the zero closure of the laser fields plus the uniform background).
 *  - PML (Sec. 2.4 item 4): sigma = (1 - i/N)^3 sigma_max with i = 0 at the
 *    outermost cell; at corners the largest sigma of the axes; outside the
 *    layer the ghost is 0.
 *  - A laser "injected" into the box (Sec. 3.2) may enter through an x-plane
 *    as an electric and a magnetic current sheet on the plane, which launch
 *    the incident wave towards +x only (orc_step_src).
 */
#include "axp_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static int64_t ncells(const orc_params *p) { return p->n[0] * p->n[1] * p->n[2]; }

static int64_t cidx(const orc_params *p, int64_t i, int64_t j, int64_t k)
{
    return i + p->n[0] * (j + p->n[1] * k);
}

/* Declares the (i, j, k) of flat cell index c_ (x fastest). */
#define CELL_IJK(c_)                                                   \
    const int64_t i = (c_) % p->n[0], j = ((c_) / p->n[0]) % p->n[1], \
                  k = (c_) / (p->n[0] * p->n[1])

static int64_t wrapi(int64_t c, int64_t n) { return ((c % n) + n) % n; }

static int em_periodic(const orc_params *p, int a) { return p->em_bc[a][0] == ORC_PERIODIC; }
static int ax_periodic(const orc_params *p, int a) { return p->axion_bc[a][0] == ORC_PERIODIC; }

static void die(const char *msg)
{
    fprintf(stderr, "axp oracle: %s\n", msg);
    abort();
}

int orc_validate(const orc_params *p)
{
    for (int a = 0; a < 3; a++) {
        if (p->n[a] < 1 || !(p->d[a] > 0)) return 1;
        for (int s = 0; s < 2; s++) {
            if ((p->em_bc[a][s] == ORC_PERIODIC) != (p->axion_bc[a][s] == ORC_PERIODIC)) return 2;
            if (p->em_bc[a][s] == ORC_OUTFLOW) return 3;
        }
        if ((p->em_bc[a][0] == ORC_PERIODIC) != (p->em_bc[a][1] == ORC_PERIODIC)) return 4;
        if (p->n[a] == 1 && p->em_bc[a][0] != ORC_PERIODIC) return 5;
    }
    if (!(p->dt > 0)) return 6;
    return 0;
}

/* Field component value at an integer index that may lie outside the grid:
 * periodic axes wrap, non-periodic axes close with zero. */
static double fld(const orc_params *p, const double *F, int64_t i, int64_t j, int64_t k)
{
    int64_t c[3] = {i, j, k};
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= p->n[a]) {
            if (em_periodic(p, a)) c[a] = wrapi(c[a], p->n[a]);
            else return 0.0;
        }
    }
    return F[cidx(p, c[0], c[1], c[2])];
}

static int64_t plane_index(const orc_params *p, int a, const int64_t c[3])
{
    if (a == 0) return c[1] + p->n[1] * c[2];
    if (a == 1) return c[0] + p->n[0] * c[2];
    return c[0] + p->n[0] * c[1];
}

static int64_t plane_size(const orc_params *p, int a)
{
    if (a == 0) return p->n[1] * p->n[2];
    if (a == 1) return p->n[0] * p->n[2];
    return p->n[0] * p->n[1];
}

/* Axion field of one time level at a cell index that may be a ghost cell.
 * Sec. 2.4: reflect  phi_{-1/2} = phi_{1/2};  periodic  phi_{-1/2} = phi_{N-1/2};
 * outflow: the solved ghost value (stored plane G); PML: 0 beyond the layer. */
static double phi_at(const orc_params *p, const double *phi, double *const G[3][2],
                     int64_t i, int64_t j, int64_t k)
{
    int64_t c[3] = {i, j, k};
    int nout = 0, out_axis = -1;
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= p->n[a]) {
            if (ax_periodic(p, a)) c[a] = wrapi(c[a], p->n[a]);
            else { nout++; out_axis = a; }
        }
    }
    if (nout == 0) return phi[cidx(p, c[0], c[1], c[2])];
    if (nout > 1) return 0.0;
    int a = out_axis;
    int side = c[a] < 0 ? 0 : 1;
    if (c[a] < -1 || c[a] > p->n[a]) die("ghost deeper than one cell");
    switch (p->axion_bc[a][side]) {
    case ORC_REFLECT:
        c[a] = side ? p->n[a] - 1 : 0;
        return phi[cidx(p, c[0], c[1], c[2])];
    case ORC_PML:
        return 0.0;
    case ORC_OUTFLOW:
        if (!G[a][side]) die("missing outflow ghost plane");
        return G[a][side][plane_index(p, a, c)];
    default:
        die("bad axion boundary");
    }
    return 0.0;
}

/* ---- absorbing-layer profile (Sec. 2.4 item 4, Sec. 3.1) ---- */
static double sigma_axis(const orc_params *p, int a, int64_t c, int axion)
{
    const int32_t *bc = axion ? p->axion_bc[a] : p->em_bc[a];
    int64_t N = p->pml_cells;
    double smax = p->pml_sigma_max_dt / p->dt;
    double s = 0.0;
    if (N <= 0) return 0.0;
    if (bc[0] == ORC_PML && c < N) {
        double r = 1.0 - (double)c / (double)N;
        s = r * r * r * smax;
    }
    if (bc[1] == ORC_PML && c >= p->n[a] - N) {
        double r = 1.0 - (double)(p->n[a] - 1 - c) / (double)N;
        double v = r * r * r * smax;
        if (v > s) s = v;
    }
    return s;
}

double orc_sigma_cell(const orc_params *p, int64_t i, int64_t j, int64_t k, int axion)
{
    double s0 = sigma_axis(p, 0, i, axion), s1 = sigma_axis(p, 1, j, axion), s2 = sigma_axis(p, 2, k, axion);
    double s = s0;
    if (s1 > s) s = s1;
    if (s2 > s) s = s2;
    return s;
}

/* ---- discrete curls (Yee staggering of Sec. 2.3, Fig. 1) ---- */

/* (curl B)_a at the E_a location of cell (i,j,k): backward differences. */
static double curlB(const orc_params *p, double *const B[3], int a, int64_t i, int64_t j, int64_t k)
{
    const double dx = p->d[0], dy = p->d[1], dz = p->d[2];
    if (a == 0)
        return (fld(p, B[2], i, j, k) - fld(p, B[2], i, j - 1, k)) / dy
             - (fld(p, B[1], i, j, k) - fld(p, B[1], i, j, k - 1)) / dz;
    if (a == 1)
        return (fld(p, B[0], i, j, k) - fld(p, B[0], i, j, k - 1)) / dz
             - (fld(p, B[2], i, j, k) - fld(p, B[2], i - 1, j, k)) / dx;
    return (fld(p, B[1], i, j, k) - fld(p, B[1], i - 1, j, k)) / dx
         - (fld(p, B[0], i, j, k) - fld(p, B[0], i, j - 1, k)) / dy;
}

/* (curl E)_a at the B_a location of cell (i,j,k): forward differences. */
static double curlE(const orc_params *p, double *const E[3], int a, int64_t i, int64_t j, int64_t k)
{
    const double dx = p->d[0], dy = p->d[1], dz = p->d[2];
    if (a == 0)
        return (fld(p, E[2], i, j + 1, k) - fld(p, E[2], i, j, k)) / dy
             - (fld(p, E[1], i, j, k + 1) - fld(p, E[1], i, j, k)) / dz;
    if (a == 1)
        return (fld(p, E[0], i, j, k + 1) - fld(p, E[0], i, j, k)) / dz
             - (fld(p, E[2], i + 1, j, k) - fld(p, E[2], i, j, k)) / dx;
    return (fld(p, E[1], i + 1, j, k) - fld(p, E[1], i, j, k)) / dx
         - (fld(p, E[0], i, j + 1, k) - fld(p, E[0], i, j, k)) / dy;
}

static const int64_t UNIT[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* 2-point average of E0_a to the cell centre (Sec. 2.3), plus the background. */
static double Ebar(const orc_params *p, double *const E[3], int a, int64_t i, int64_t j, int64_t k)
{
    const int64_t *u = UNIT[a];
    return 0.5 * (fld(p, E[a], i, j, k) + fld(p, E[a], i - u[0], j - u[1], k - u[2])) + p->E_ext[a];
}

/* 4-point average of B0_a to the cell centre (Sec. 2.3), plus the background.
 * For a = x the terms are (j+1/2,k+1/2), (j+1/2,k-1/2), (j-1/2,k+1/2), (j-1/2,k-1/2);
 * y and z follow by the cyclic permutation x -> y -> z. */
static double Bbar(const orc_params *p, double *const B[3], int a, int64_t i, int64_t j, int64_t k)
{
    const int64_t *ub = UNIT[(a + 1) % 3], *uc = UNIT[(a + 2) % 3];
    double s = fld(p, B[a], i, j, k);
    s = s + fld(p, B[a], i - uc[0], j - uc[1], k - uc[2]);
    s = s + fld(p, B[a], i - ub[0], j - ub[1], k - ub[2]);
    s = s + fld(p, B[a], i - ub[0] - uc[0], j - ub[1] - uc[1], k - ub[2] - uc[2]);
    return 0.25 * s + p->B_ext[a];
}

/* Source S = g Ebar0 . Bbar0 at a cell centre (Sec. 2.3). */
static double source_at(const orc_params *p, double *const E0[3], double *const B0[3],
                        int64_t i, int64_t j, int64_t k)
{
    double s = Ebar(p, E0, 0, i, j, k) * Bbar(p, B0, 0, i, j, k);
    s = s + Ebar(p, E0, 1, i, j, k) * Bbar(p, B0, 1, i, j, k);
    s = s + Ebar(p, E0, 2, i, j, k) * Bbar(p, B0, 2, i, j, k);
    return p->g * s;
}

/* Two phi time levels (hi = later, lo = earlier) around an integer time. */
typedef struct {
    const double *hi, *lo;
    double *Ghi[3][2], *Glo[3][2]; /* ghost planes of the two levels */
} phi_pair;

static phi_pair make_pair(const double *hi, const double *lo, double *const Ghi[3][2], double *const Glo[3][2])
{
    phi_pair q;
    q.hi = hi;
    q.lo = lo;
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            q.Ghi[a][sd] = Ghi[a][sd];
            q.Glo[a][sd] = Glo[a][sd];
        }
    return q;
}

static double phi_hi(const orc_params *p, const phi_pair *q, int64_t i, int64_t j, int64_t k)
{
    return phi_at(p, q->hi, q->Ghi, i, j, k);
}
static double phi_lo(const orc_params *p, const phi_pair *q, int64_t i, int64_t j, int64_t k)
{
    return phi_at(p, q->lo, q->Glo, i, j, k);
}

/* phi at the integer time between the two levels: phi^n = (phi^{n+1/2} + phi^{n-1/2})/2 */
static double phi_mid(const orc_params *p, const phi_pair *q, int64_t i, int64_t j, int64_t k)
{
    return 0.5 * (phi_hi(p, q, i, j, k) + phi_lo(p, q, i, j, k));
}

/* Central difference of phi^n along axis b at a cell centre: (phi_{c+1} - phi_{c-1})/(2 d_b). */
static double dphi(const orc_params *p, const phi_pair *q, int b, int64_t i, int64_t j, int64_t k)
{
    const int64_t *u = UNIT[b];
    return (phi_mid(p, q, i + u[0], j + u[1], k + u[2]) - phi_mid(p, q, i - u[0], j - u[1], k - u[2]))
         / (2.0 * p->d[b]);
}

/* Component a of the cell-centred axion current density without the factor g:
 * P_a = (D_t phi) Bbar0_a - (Ebar0 x grad phi)_a, with (a,b,c) cyclic. */
static double P_comp(const orc_params *p, const phi_pair *q, double *const E0[3], double *const B0[3],
                     int a, int64_t i, int64_t j, int64_t k)
{
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double Dt = (phi_hi(p, q, i, j, k) - phi_lo(p, q, i, j, k)) / p->dt;
    double cross = Ebar(p, E0, b, i, j, k) * dphi(p, q, c, i, j, k)
                 - Ebar(p, E0, c, i, j, k) * dphi(p, q, b, i, j, k);
    return Dt * Bbar(p, B0, a, i, j, k) - cross;
}

/* Axion current at the E locations: J_a(c + a/2) = (P_a(c) + P_a(c + a))/2. */
static void current_into(const orc_params *p, const phi_pair *q, double *const E0[3], double *const B0[3],
                         double *J[3])
{
    for (int a = 0; a < 3; a++) {
        const int64_t *u = UNIT[a];
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < ncells(p); c++) {
            CELL_IJK(c);
            J[a][c] = 0.5 * (P_comp(p, q, E0, B0, a, i, j, k) + P_comp(p, q, E0, B0, a, i + u[0], j + u[1], k + u[2]));
        }
    }
}

/* One half-step of length h for a field with optional absorbing-layer damping:
 * dF/dt = X - sigma F, trapezoidal in time. */
static double half_update(double F, double X, double sig, double h)
{
    if (sig == 0.0) return F + h * X;
    return ((1.0 - sig * h / 2.0) * F + h * X) / (1.0 + sig * h / 2.0);
}

/* ---- soft source (laser entering through an x-plane) ---- */

static void position(const orc_params *p, int kind, int a, int64_t i, int64_t j, int64_t k, double x[3]);

/* Time-dependent factor of the incident wave at lab position x, time t:
 * env(t - t_c - (x - x_c)) cos(k (x - x_c) - w (t - t_c) + phase). */
static double src_wave(const orc_params *p, const orc_source *q, double x, double t)
{
    double w = (2.0 / p->dt) * asin((p->dt / p->d[0]) * sin(q->k * p->d[0] / 2.0));
    double e = 1.0;
    if (q->duration > 0) {
        double L = q->duration / sqrt(2.0 * log(2.0));
        double u = (t - q->t_centre) - (x - q->centre[0]);
        e = exp(-(u * u) / (L * L));
    }
    return e * cos(q->k * (x - q->centre[0]) - w * (t - q->t_centre) + q->phase);
}

/* Sheet weight of polarisation component a (1 = y, 2 = z) at transverse cell
 * (j, k): A pol_a f / dx at the E_a location of cell (plane, j, k); its B
 * partner on the sheet (B_z for E_y, B_y for E_z) has the same y and z.  Zero
 * where either cell next to the sheet lies in an absorbing layer. */
static double src_weight(const orc_params *p, const orc_source *q, int a, int64_t j, int64_t k)
{
    if (orc_sigma_cell(p, q->plane, j, k, 0) != 0.0 || orc_sigma_cell(p, q->plane - 1, j, k, 0) != 0.0) return 0.0;
    double f = 1.0;
    if (q->waist > 0) {
        double x[3];
        position(p, 1, a, q->plane, j, k, x);
        double r2 = 0.0;
        if (p->n[1] > 1) r2 = r2 + (x[1] - q->centre[1]) * (x[1] - q->centre[1]);
        if (p->n[2] > 1) r2 = r2 + (x[2] - q->centre[2]) * (x[2] - q->centre[2]);
        f = exp(-r2 / (q->waist * q->waist));
    }
    return ((q->amplitude * q->pol[a]) * f) / p->d[0];
}

/* Electric sheet, in the E update of cell (plane, j, k) at time t: the update
 * of E_y uses B_z of the face on the plane, which lies on the incident-free
 * side, so the incident B_z/dx is added to its curl; likewise E_z takes
 * -B_y,inc/dx.  With B_inc = xhat x E_inc both terms are +A pol f tau/dx, tau
 * the wave factor at the face (x = x_p). */
static double src_e_term(const orc_params *p, const orc_source *q, int a, int64_t i, int64_t j, int64_t k, double t)
{
    if (!q || i != q->plane || a == 0) return 0.0;
    double xp = p->lo[0] + (double)q->plane * p->d[0];
    return src_weight(p, q, a, j, k) * src_wave(p, q, xp, t);
}

/* Magnetic sheet, in the B update of the face (plane-1, j, k) at time t: the
 * curl there reads E of cell `plane`, on the incident side, so the incident
 * part is taken out: B_y gets -E_z,inc/dx, B_z gets +E_y,inc/dx, with the
 * wave factor at the E cells (x = x_p + dx/2). */
static double src_b_term(const orc_params *p, const orc_source *q, int a, int64_t i, int64_t j, int64_t k, double t)
{
    if (!q || i != q->plane - 1 || a == 0) return 0.0;
    double xe = p->lo[0] + ((double)q->plane + 0.5) * p->d[0];
    double tau = src_wave(p, q, xe, t);
    if (a == 1) return -(src_weight(p, q, 2, j, k) * tau);
    return src_weight(p, q, 1, j, k) * tau;
}

/* jp: the particle current of this order (NULL without particles), Ampere's law
 * curl B = dE/dt + j (natural units) */
static void e_half(const orc_params *p, double *E[3], double *const B[3], double *const J[3], double coef_g,
                   const orc_source *src, double t, double *const jp[3])
{
    const double h = p->dt / 2.0;
    for (int a = 0; a < 3; a++) {
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < ncells(p); c++) {
            CELL_IJK(c);
            double X = curlB(p, B, a, i, j, k);
            if (J) X = X - coef_g * J[a][c];
            if (jp) X = X - jp[a][c];
            if (src && i == src->plane) X = X + src_e_term(p, src, a, i, j, k, t);
            E[a][c] = half_update(E[a][c], X, orc_sigma_cell(p, i, j, k, 0), h);
        }
    }
}

static void b_half(const orc_params *p, double *B[3], double *const E[3], const orc_source *src, double t)
{
    const double h = p->dt / 2.0;
    for (int a = 0; a < 3; a++) {
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < ncells(p); c++) {
            CELL_IJK(c);
            double X = -curlE(p, E, a, i, j, k);
            if (src && i == src->plane - 1) X = X + src_b_term(p, src, a, i, j, k, t);
            B[a][c] = half_update(B[a][c], X, orc_sigma_cell(p, i, j, k, 0), h);
        }
    }
}

/* Sec. 2.4 item 3: the two-equation outflow solve at the x_min face, written
 * for one ghost cell.  Inputs: phi^{n-1}_{-1/2} (g_cur), phi^{n-2}_{-1/2}
 * (g_old), phi^{n-1}_{1/2} (p0_cur) and S^{n-1}_{-1/2}.  Outputs
 * V = phi^{n-1}_{-3/2} and U = phi^{n}_{-1/2}. */
void orc_outflow_solve(double dt, double dxa, double m, double g_cur, double g_old,
                       double p0_cur, double S_g, double *V_out, double *U_out)
{
    double r = dt / dxa;
    double r2 = (dt * dt) / (dxa * dxa);
    double rhs = -2.0 * g_cur + 2.0 * g_old - (dt * dt) * (S_g - m * m * g_cur) + r * p0_cur
               - r2 * (p0_cur - 2.0 * g_cur);
    double V = rhs / (r + r2);
    double U = g_old + r * (p0_cur - V);
    *V_out = V;
    *U_out = U;
}

static void step_impl(const orc_params *p, orc_state *s, const orc_source *src, orc_particles *P, int64_t nsteps);

void orc_step(const orc_params *p, orc_state *s, int64_t nsteps) { step_impl(p, s, NULL, NULL, nsteps); }

void orc_step_src(const orc_params *p, orc_state *s, const orc_source *src, int64_t nsteps)
{
    step_impl(p, s, src, NULL, nsteps);
}

void orc_step_plasma(const orc_params *p, orc_state *s, const orc_source *src, orc_particles *P, int64_t nsteps)
{
    if (P && orc_particles_validate(p, P)) die("invalid particles");
    step_impl(p, s, src, P, nsteps);
}

/* Sec. 2.3 time scheme; with particles, Sec. 2.3's step order puts the particle
 * push between the axion update and the second field half-steps, and the
 * current j^n (j^{n+1}) enters the first (second) E half-steps of its order. */
static void step_impl(const orc_params *p, orc_state *s, const orc_source *src, orc_particles *P, int64_t nsteps)
{
    if (orc_validate(p)) die("invalid parameters");
    if (src && (src->plane < 1 || src->plane > p->n[0] - 1 || src->pol[0] != 0.0)) die("invalid soft source");
    const int64_t N = ncells(p);
    double *J[3], *S = malloc(sizeof(double) * N), *phi_new = malloc(sizeof(double) * N);
    for (int a = 0; a < 3; a++) J[a] = malloc(sizeof(double) * N);
    double *Gnew[3][2] = {{0}};
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++)
            if (p->axion_bc[a][sd] == ORC_OUTFLOW) {
                if (!s->ghost[a][sd][0] || !s->ghost[a][sd][1]) die("outflow face without ghost planes");
                Gnew[a][sd] = malloc(sizeof(double) * plane_size(p, a));
            }
    const double dt = p->dt, m2 = p->m * p->m;

    for (int64_t it = 0; it < nsteps; it++) {
        double *Gcur[3][2], *Gold[3][2];
        for (int a = 0; a < 3; a++)
            for (int sd = 0; sd < 2; sd++) {
                Gcur[a][sd] = s->ghost[a][sd][0];
                Gold[a][sd] = s->ghost[a][sd][1];
            }

        /* 1. axion current J^n from phi^{n+1/2}, phi^{n-1/2}, E0^n, B0^n */
        phi_pair qn = make_pair(s->phi_cur, s->phi_old, Gcur, Gold);
        current_into(p, &qn, s->E0, s->B0, J);

        /* source times: the E half-steps read B at t_n and t_{n+1}, the B half-steps E at t_{n+1/2} */
        const double t_n = (double)s->step * dt, t_h = ((double)s->step + 0.5) * dt;
        const double t_n1 = (double)(s->step + 1) * dt;

        /* 2.-5. first half-steps, order 0 before order 1 (Eq. update_E and the B1 half-step) */
        e_half(p, s->E0, s->B0, NULL, 0.0, src, t_n, P ? P->j0 : NULL);
        e_half(p, s->E1, s->B1, J, p->g, NULL, 0.0, P ? P->j1 : NULL);
        b_half(p, s->B0, s->E0, src, t_h);
        b_half(p, s->B1, s->E1, NULL, 0.0);

        /* 8.-9. source S^{n+1/2} and the axion leapfrog (Eq. update_axion), PML form in the layer */
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < N; c++) {
            CELL_IJK(c);
            S[c] = source_at(p, s->E0, s->B0, i, j, k);
            double ph = s->phi_cur[c];
            double lap = 0.0;
            for (int a = 0; a < 3; a++) {
                const int64_t *u = UNIT[a];
                double up = phi_at(p, s->phi_cur, Gcur, i + u[0], j + u[1], k + u[2]);
                double dn = phi_at(p, s->phi_cur, Gcur, i - u[0], j - u[1], k - u[2]);
                lap = lap + ((up + dn) - 2.0 * ph) / (p->d[a] * p->d[a]);
            }
            double sig = orc_sigma_cell(p, i, j, k, 1);
            if (sig == 0.0) {
                phi_new[c] = 2.0 * ph - s->phi_old[c] + (dt * dt) * ((lap - m2 * ph) + S[c]);
            } else {
                double Y = ((S[c] - m2 * ph) + lap) - sig * sig * ph;
                phi_new[c] = ((dt * dt) * Y + sig * dt * s->phi_old[c] + 2.0 * ph - s->phi_old[c]) / (1.0 + sig * dt);
            }
        }

        /* 9b. outflow ghosts at the new level (needed by J^{n+1} and the next step) */
        for (int a = 0; a < 3; a++)
            for (int sd = 0; sd < 2; sd++) {
                if (!Gnew[a][sd]) continue;
                int b = (a + 1) % 3, c2 = (a + 2) % 3;
                int64_t ca[3];
                for (int64_t tb = 0; tb < p->n[b]; tb++)
                    for (int64_t tc = 0; tc < p->n[c2]; tc++) {
                        ca[b] = tb;
                        ca[c2] = tc;
                        ca[a] = sd ? p->n[a] : -1;
                        int64_t pi = plane_index(p, a, ca);
                        double Sg = source_at(p, s->E0, s->B0, ca[0], ca[1], ca[2]);
                        int64_t ci[3] = {ca[0], ca[1], ca[2]};
                        ci[a] = sd ? p->n[a] - 1 : 0;
                        double p0 = s->phi_cur[cidx(p, ci[0], ci[1], ci[2])];
                        double V, U;
                        orc_outflow_solve(dt, p->d[a], p->m, Gcur[a][sd][pi], Gold[a][sd][pi], p0, Sg, &V, &U);
                        Gnew[a][sd][pi] = U;
                    }
            }

        /* particles pushed by the fields of both orders at t_{n+1/2}; j^{n+1} */
        if (P) orc_push(p, s, P);

        /* 10.-12. second half-steps of B (both orders) and of E0 */
        b_half(p, s->B0, s->E0, src, t_h);
        b_half(p, s->B1, s->E1, NULL, 0.0);
        e_half(p, s->E0, s->B0, NULL, 0.0, src, t_n1, P ? P->j0 : NULL);

        /* 13.-14. J^{n+1} from phi^{n+3/2}, phi^{n+1/2}, E0^{n+1}, B0^{n+1}; second E1 half-step */
        phi_pair qn1 = make_pair(phi_new, s->phi_cur, Gnew, Gcur);
        current_into(p, &qn1, s->E0, s->B0, J);
        e_half(p, s->E1, s->B1, J, p->g, NULL, 0.0, P ? P->j1 : NULL);

        /* 17. rotate the axion levels: old <- cur, cur <- new (copies keep the caller's buffers) */
        memcpy(s->phi_old, s->phi_cur, sizeof(double) * N);
        memcpy(s->phi_cur, phi_new, sizeof(double) * N);
        for (int a = 0; a < 3; a++)
            for (int sd = 0; sd < 2; sd++) {
                if (!Gnew[a][sd]) continue;
                size_t bytes = sizeof(double) * plane_size(p, a);
                memcpy(s->ghost[a][sd][1], s->ghost[a][sd][0], bytes);
                memcpy(s->ghost[a][sd][0], Gnew[a][sd], bytes);
            }
        s->step += 1;
    }
    free(phi_new);
    free(S);
    for (int a = 0; a < 3; a++) {
        free(J[a]);
        for (int sd = 0; sd < 2; sd++) free(Gnew[a][sd]);
    }
}

/* J^n of the present state (phi_cur, phi_old, E0, B0), without the factor g. */
void orc_current(const orc_params *p, const orc_state *s, double *J[3])
{
    double *Gcur[3][2], *Gold[3][2];
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            Gcur[a][sd] = s->ghost[a][sd][0];
            Gold[a][sd] = s->ghost[a][sd][1];
        }
    phi_pair q = make_pair(s->phi_cur, s->phi_old, Gcur, Gold);
    current_into(p, &q, s->E0, s->B0, J);
}

/* S = g Ebar0 . Bbar0 of the present E0, B0 at every cell centre. */
void orc_source_now(const orc_params *p, const orc_state *s, double *S)
{
    for (int64_t k = 0; k < p->n[2]; k++)
        for (int64_t j = 0; j < p->n[1]; j++)
            for (int64_t i = 0; i < p->n[0]; i++) S[cidx(p, i, j, k)] = source_at(p, s->E0, s->B0, i, j, k);
}

static void ghosts_now(const orc_state *s, double *Gcur[3][2], double *Gold[3][2])
{
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            Gcur[a][sd] = s->ghost[a][sd][0];
            Gold[a][sd] = s->ghost[a][sd][1];
        }
}

/* Gauss residual R = div E1 + g Bbar0 . grad_c phi^n at every cell centre
 * (modified Gauss law for the order-1 field, Sec. 2.2). */
void orc_gauss_residual(const orc_params *p, const orc_state *s, double *R)
{
    double *Gcur[3][2], *Gold[3][2];
    ghosts_now(s, Gcur, Gold);
    phi_pair q = make_pair(s->phi_cur, s->phi_old, Gcur, Gold);
    for (int64_t k = 0; k < p->n[2]; k++)
        for (int64_t j = 0; j < p->n[1]; j++)
            for (int64_t i = 0; i < p->n[0]; i++) {
                double div = 0.0, bg = 0.0;
                for (int a = 0; a < 3; a++) {
                    const int64_t *u = UNIT[a];
                    div = div + (fld(p, s->E1[a], i, j, k) - fld(p, s->E1[a], i - u[0], j - u[1], k - u[2])) / p->d[a];
                    bg = bg + Bbar(p, s->B0, a, i, j, k) * dphi(p, &q, a, i, j, k);
                }
                R[cidx(p, i, j, k)] = div + p->g * bg;
            }
}

static int in_region(const orc_params *p, const int64_t c[3])
{
    for (int a = 0; a < 3; a++) {
        if (p->n[a] == 1 || em_periodic(p, a)) continue;
        int64_t N = p->pml_cells;
        int lo_abs = p->em_bc[a][0] == ORC_PML || p->axion_bc[a][0] == ORC_PML;
        int hi_abs = p->em_bc[a][1] == ORC_PML || p->axion_bc[a][1] == ORC_PML;
        if (lo_abs && c[a] < N) return 0;
        if (hi_abs && c[a] >= p->n[a] - N) return 0;
    }
    return 1;
}

/* Energy diagnostics at the present integer time (Sec. 3.2 and 3.3 energy
 * densities; the centroid of Sec. 3.4).  H_phi uses D_t phi^n, the forward
 * difference of phi^n to the next cell per axis, and phi^n itself.  Sums run
 * over the cells outside the absorbing layers, in index order. */
void orc_diagnostics(const orc_params *p, const orc_state *s, orc_diag *out)
{
    double *Gcur[3][2], *Gold[3][2];
    ghosts_now(s, Gcur, Gold);
    phi_pair q = make_pair(s->phi_cur, s->phi_old, Gcur, Gold);
    const double dV = p->d[0] * p->d[1] * p->d[2];
    double Hphi = 0, Hg0 = 0, Hg1 = 0, X = 0, sxb = 0, sb = 0, gl2 = 0;
    double *R = malloc(sizeof(double) * ncells(p));
    orc_gauss_residual(p, s, R);
    for (int64_t k = 0; k < p->n[2]; k++)
        for (int64_t j = 0; j < p->n[1]; j++)
            for (int64_t i = 0; i < p->n[0]; i++) {
                int64_t cc[3] = {i, j, k};
                if (!in_region(p, cc)) continue;
                int64_t c = cidx(p, i, j, k);
                double Dt = (s->phi_cur[c] - s->phi_old[c]) / p->dt;
                double ph = 0.5 * (s->phi_cur[c] + s->phi_old[c]);
                double g2 = 0.0;
                for (int a = 0; a < 3; a++) {
                    const int64_t *u = UNIT[a];
                    double dfw = (phi_mid(p, &q, i + u[0], j + u[1], k + u[2]) - ph) / p->d[a];
                    g2 = g2 + dfw * dfw;
                }
                Hphi = Hphi + 0.5 * ((Dt * Dt + g2) + p->m * p->m * ph * ph) * dV;
                double e0 = 0, e1 = 0, x = 0;
                for (int a = 0; a < 3; a++) {
                    e0 = e0 + s->E0[a][c] * s->E0[a][c] + s->B0[a][c] * s->B0[a][c];
                    e1 = e1 + s->E1[a][c] * s->E1[a][c] + s->B1[a][c] * s->B1[a][c];
                    x = x + (s->E0[a][c] + p->E_ext[a]) * s->E1[a][c] + (s->B0[a][c] + p->B_ext[a]) * s->B1[a][c];
                }
                Hg0 = Hg0 + 0.5 * e0 * dV;
                Hg1 = Hg1 + 0.5 * e1 * dV;
                X = X + x * dV;
                double xb = p->lo[0] + (double)(i + 1) * p->d[0];
                double bz2 = s->B1[2][c] * s->B1[2][c] * dV;
                sxb = sxb + xb * bz2;
                sb = sb + bz2;
                gl2 = gl2 + R[c] * R[c] * dV;
            }
    free(R);
    out->t = (double)s->step * p->dt;
    out->H_phi = Hphi;
    out->H_g0 = Hg0;
    out->H_g1 = Hg1;
    out->P_g2a = Hg0 > 0 ? Hphi / Hg0 : 0.0;
    out->P_a2g = Hphi > 0 ? Hg1 / Hphi : 0.0;
    out->W = Hphi + X;
    out->sum_xB1z2 = sxb;
    out->sum_B1z2 = sb;
    out->gauss_l2 = gl2;
}

/* ---- initial conditions ---- */

/* Position of a staggered component: 'kind' 0 = cell centre, 1 = E_a, 2 = B_a. */
static void position(const orc_params *p, int kind, int a, int64_t i, int64_t j, int64_t k, double x[3])
{
    int64_t c[3] = {i, j, k};
    for (int b = 0; b < 3; b++) {
        double off = 0.5;
        if (kind == 1 && b == a) off = 1.0;
        if (kind == 2 && b != a) off = 1.0;
        x[b] = p->lo[b] + ((double)c[b] + off) * p->d[b];
    }
}

static double envelope(const double x[3], const double centre[3], const double khat[3],
                       double waist, double len, double shift)
{
    double dx[3] = {x[0] - centre[0], x[1] - centre[1], x[2] - centre[2]};
    double xi = khat[0] * dx[0] + khat[1] * dx[1] + khat[2] * dx[2];
    double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2] - xi * xi;
    double e = 1.0;
    if (waist > 0) e = e * exp(-r2 / (waist * waist));
    if (len > 0) e = e * exp(-((xi - shift) * (xi - shift)) / (len * len));
    return e;
}

/* Laser: E = A pol env cos(k.(x - x_c) + phase) at integer time 0, and
 * B = curl_h(pol F) with F = (A / cos(theta/2)) env sin(...) / |K|, where
 * K_d = (2/d_d) sin(k_d d_d / 2) and sin(theta/2) = dt |K| / 2 (Yee
 * dispersion).  For a CW wave commensurate with a periodic box this is the
 * exact discrete eigenmode of the half-step scheme; B is divergence-free by
 * construction.  Fields are added to the present E0, B0. */
void orc_inject_laser(const orc_params *p, orc_state *s, const orc_laser *L)
{
    const int64_t N = ncells(p);
    double K2 = 0.0, kk = 0.0;
    for (int a = 0; a < 3; a++) {
        double Ka = (2.0 / p->d[a]) * sin(L->k[a] * p->d[a] / 2.0);
        K2 = K2 + Ka * Ka;
        kk = kk + L->k[a] * L->k[a];
    }
    double Kmag = sqrt(K2), kmag = sqrt(kk);
    double sh = p->dt * Kmag / 2.0;
    double ch = sqrt(1.0 - sh * sh);
    double khat[3] = {0, 0, 0};
    if (kmag > 0)
        for (int a = 0; a < 3; a++) khat[a] = L->k[a] / kmag;
    double len = L->duration > 0 ? L->duration / sqrt(2.0 * log(2.0)) : 0.0;
    double *F[3];
    for (int a = 0; a < 3; a++) F[a] = calloc(N, sizeof(double));
    for (int a = 0; a < 3; a++)
        for (int64_t k = 0; k < p->n[2]; k++)
            for (int64_t j = 0; j < p->n[1]; j++)
                for (int64_t i = 0; i < p->n[0]; i++) {
                    double x[3];
                    position(p, 1, a, i, j, k, x);
                    double env = envelope(x, L->centre, khat, L->waist, len, 0.0);
                    double ph = L->k[0] * (x[0] - L->centre[0]) + L->k[1] * (x[1] - L->centre[1])
                              + L->k[2] * (x[2] - L->centre[2]) + L->phase;
                    int64_t c = cidx(p, i, j, k);
                    s->E0[a][c] = s->E0[a][c] + L->amplitude * L->pol[a] * env * cos(ph);
                    F[a][c] = (L->amplitude / ch) * L->pol[a] * env * sin(ph) / Kmag;
                }
    for (int a = 0; a < 3; a++)
        for (int64_t k = 0; k < p->n[2]; k++)
            for (int64_t j = 0; j < p->n[1]; j++)
                for (int64_t i = 0; i < p->n[0]; i++) {
                    int64_t c = cidx(p, i, j, k);
                    s->B0[a][c] = s->B0[a][c] + curlE(p, F, a, i, j, k);
                }
    for (int a = 0; a < 3; a++) free(F[a]);
}

/* Axion wave phi(x, t) = A env(xi - v t, r) sin(k.(x - x_c) - w t + phase),
 * evaluated at t = +dt/2 (phi_cur) and t = -dt/2 (phi_old), as Sec. 3.1 sets
 * its test pulse at two time levels.  w solves the discrete Klein-Gordon
 * dispersion cos(w dt) = 1 - dt^2 (K^2 + m^2)/2, K_d = (2/d_d) sin(k_d d_d/2).
 * Outflow ghost planes receive the same profile at the ghost centres. */
void orc_inject_axion(const orc_params *p, orc_state *s, const orc_axion *A)
{
    double K2 = 0.0, kk = 0.0;
    for (int a = 0; a < 3; a++) {
        double Ka = (2.0 / p->d[a]) * sin(A->k[a] * p->d[a] / 2.0);
        K2 = K2 + Ka * Ka;
        kk = kk + A->k[a] * A->k[a];
    }
    double cw = 1.0 - p->dt * p->dt * (K2 + p->m * p->m) / 2.0;
    double w = acos(cw) / p->dt;
    double kmag = sqrt(kk);
    double khat[3] = {0, 0, 0};
    if (kmag > 0)
        for (int a = 0; a < 3; a++) khat[a] = A->k[a] / kmag;
    for (int lev = 0; lev < 2; lev++) {
        double t = lev == 0 ? 0.5 * p->dt : -0.5 * p->dt;
        double *phi = lev == 0 ? s->phi_cur : s->phi_old;
        for (int64_t k = 0; k < p->n[2]; k++)
            for (int64_t j = 0; j < p->n[1]; j++)
                for (int64_t i = 0; i < p->n[0]; i++) {
                    double x[3];
                    position(p, 0, 0, i, j, k, x);
                    double env = envelope(x, A->centre, khat, A->waist, A->length, A->speed * t);
                    double ph = A->k[0] * (x[0] - A->centre[0]) + A->k[1] * (x[1] - A->centre[1])
                              + A->k[2] * (x[2] - A->centre[2]) - w * t + A->phase;
                    int64_t c = cidx(p, i, j, k);
                    phi[c] = phi[c] + A->amplitude * env * sin(ph);
                }
        for (int a = 0; a < 3; a++)
            for (int sd = 0; sd < 2; sd++) {
                double *G = s->ghost[a][sd][lev];
                if (p->axion_bc[a][sd] != ORC_OUTFLOW || !G) continue;
                int b = (a + 1) % 3, c2 = (a + 2) % 3;
                for (int64_t tb = 0; tb < p->n[b]; tb++)
                    for (int64_t tc = 0; tc < p->n[c2]; tc++) {
                        int64_t ca[3];
                        ca[a] = sd ? p->n[a] : -1;
                        ca[b] = tb;
                        ca[c2] = tc;
                        double x[3];
                        position(p, 0, 0, ca[0], ca[1], ca[2], x);
                        double env = envelope(x, A->centre, khat, A->waist, A->length, A->speed * t);
                        double ph = A->k[0] * (x[0] - A->centre[0]) + A->k[1] * (x[1] - A->centre[1])
                                  + A->k[2] * (x[2] - A->centre[2]) - w * t + A->phase;
                        int64_t pi = plane_index(p, a, ca);
                        G[pi] = G[pi] + A->amplitude * env * sin(ph);
                    }
            }
    }
}

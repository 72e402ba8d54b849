/*
 * axp_oracle.h -- plain FP64 CPU oracle of the axion-coupled Yee field update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load or call this library.  It shares no code,
 * header, table or helper with the CUDA path under paper_2406_16796_gb300/.
 *
 * Method: arXiv 2406.16796, Sec. 2 (field equations Eq. wave_axion and the
 * modified Maxwell equations; FPS split of Sec. 2.2; time discretisation of
 * Sec. 2.3, Eqs. update_E / update_axion and the phi^n average; spatial
 * averaging operators of Sec. 2.3; axion boundary conditions of Sec. 2.4).
 * Natural units hbar = c = eps0 = 1, Heaviside-Lorentz.
 *
 * Layout: every field component is an array of n[0]*n[1]*n[2] doubles, x
 * fastest: element (i,j,k) sits at index i + n0*(j + n1*k).  With cell
 * centres at ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz) from the domain origin:
 *   phi    at the cell centre;
 *   E_x    at the centre + dx/2 (E_y, E_z cyclic);
 *   B_x    at the centre + dy/2 + dz/2 (B_y, B_z cyclic).
 * Time levels: E, B at integer n; phi at n+1/2 (phi_cur) and n-1/2 (phi_old).
 */
#ifndef AXP_ORACLE_H
#define AXP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_REFLECT = 1, ORC_OUTFLOW = 2, ORC_PML = 3 };

typedef struct {
    int64_t n[3];          /* cells per axis; invariant axes have n = 1 and must be periodic */
    double d[3];           /* cell size per axis */
    double lo[3];          /* domain origin (position of the low cell faces) */
    double dt;
    double m, g;           /* axion mass and coupling, natural units */
    double B_ext[3];       /* uniform static background fields (not stored in arrays) */
    double E_ext[3];
    int32_t axion_bc[3][2];/* per axis, per side (0 = low, 1 = high) */
    int32_t em_bc[3][2];   /* ORC_PERIODIC, ORC_PML (absorbing layer) or ORC_REFLECT (zero closure) */
    int32_t pml_cells;     /* absorbing layer thickness N */
    int32_t pad_;
    double pml_sigma_max_dt; /* sigma_max * dt */
} orc_params;

typedef struct {
    double *E0[3], *B0[3], *E1[3], *B1[3];  /* laser (order 0) and perturbation (order 1) */
    double *phi_cur, *phi_old;              /* phi^{n+1/2}, phi^{n-1/2} */
    /* outflow ghost planes [axis][side][0 = level of phi_cur, 1 = level of phi_old];
     * plane index: axis 0 -> j + n1*k, axis 1 -> i + n0*k, axis 2 -> i + n0*j.
     * NULL where the face is not an outflow face. */
    double *ghost[3][2][2];
    int64_t step;
} orc_state;

typedef struct {
    double amplitude;    /* E amplitude at integer time levels */
    double k[3];         /* carrier wave vector */
    double pol[3];       /* unit E polarisation, perpendicular to k */
    double centre[3];    /* pulse centre at t = 0 */
    double waist;        /* transverse 1/e field radius; 0 = plane wave */
    double duration;     /* intensity FWHM in time (c = 1); 0 = CW */
    double phase;
} orc_laser;

typedef struct {
    double amplitude;
    double k[3];         /* carrier wave vector; the wave moves along +k */
    double centre[3];    /* envelope centre at t = 0 */
    double waist;        /* transverse 1/e radius; 0 = plane */
    double length;       /* longitudinal 1/e half-length; 0 = CW */
    double speed;        /* envelope speed along k-hat */
    double phase;
} orc_axion;

typedef struct {
    double t;
    double H_phi, H_g0, H_g1;        /* axion, laser, perturbation energies */
    double P_g2a, P_a2g;             /* H_phi/H_g0 and H_g1/H_phi */
    double W;                        /* H_phi + sum(E0.E1 + B0.B1) dV (B0, E0 incl. background) */
    double sum_xB1z2, sum_B1z2;      /* centroid numerator / denominator */
    double gauss_l2;                 /* sum over cells of R^2 dV, R = div E1 + g Bbar0 . grad_c phi */
} orc_diag;

/* Laser entering through a fixed x-plane (Sec. 3.2 injects the laser into the
 * box), as a pair of current sheets on the plane x_p = lo[0] + plane d[0]: an
 * electric sheet on the E cells at index `plane` and a magnetic sheet on the B
 * faces at index plane-1 (the faces on x_p).  Together they launch the incident
 * wave towards +x only (a Huygens source: cells below the plane see the
 * incident wave removed, cells from `plane` on see it added).  Incident wave,
 * lab coordinates, t = step dt:
 *   E_inc = A pol f(y, z) env(t - t_c - (x - x_c)) cos(k (x - x_c) - w (t - t_c) + phase),
 *   B_inc = xhat x E_inc,
 * w from the Yee dispersion along x, sin(w dt/2)/dt = sin(k dx/2)/dx, so that a
 * CW wave is an exact discrete plane wave; f = exp(-r^2/waist^2) over the
 * active transverse axes (1 for waist = 0); env = exp(-u^2/L^2) with
 * L = duration/sqrt(2 ln 2) (1 for duration = 0).  The sheets stop where a
 * transverse absorbing layer begins. */
typedef struct {
    double amplitude;
    double k;            /* carrier wave number along +x, > 0 */
    double pol[3];       /* unit E polarisation, pol[0] = 0 */
    double centre[3];    /* x_c (envelope centre at t_c); y_c, z_c (beam axis) */
    double waist;
    double duration;     /* intensity FWHM in time (c = 1) */
    double t_centre;
    double phase;
    int64_t plane;       /* first cell on the +x side of the sheet, 1 <= plane <= n[0]-1 */
} orc_source;

/* Macroparticles of one species for the perturbed-particle current of Sec. 2.2
 * (FPS: p = p0 + p1, v = v0 + v1, j = j0 + j1).  Natural units (c = 1):
 * u = gamma v is the normalised momentum, du/dt = (q/m)(E + v x B).
 * Time levels inside a run: positions x0, x1 at t_{n+1/2}, momenta u0, u1 at
 * t_n, currents j0, j1 at t_n on the E_a positions (arrays of the grid's
 * layout).  orc_particles_start takes positions at t_n and moves them to
 * t_{n+1/2}; orc_particles_positions_now gives them back at t_n.
 * Every active axis (n > 1) must be periodic for E and B; positions wrap into
 * [lo, lo + n d) along active axes, x1 (a displacement) does not wrap. */
typedef struct {
    int64_t count;
    double q, m;            /* charge and mass of the species */
    double *w;              /* physical particles per macroparticle */
    double *x0[3], *u0[3];  /* order 0 */
    double *x1[3], *u1[3];  /* order 1 */
    double *j0[3], *j1[3];  /* current densities, ncells each */
} orc_particles;

int orc_validate(const orc_params *p);
void orc_step(const orc_params *p, orc_state *s, int64_t nsteps);
/* orc_step with a soft source (src may be NULL) */
void orc_step_src(const orc_params *p, orc_state *s, const orc_source *src, int64_t nsteps);
void orc_current(const orc_params *p, const orc_state *s, double *J[3]);
void orc_source_now(const orc_params *p, const orc_state *s, double *S);
void orc_gauss_residual(const orc_params *p, const orc_state *s, double *R);
void orc_diagnostics(const orc_params *p, const orc_state *s, orc_diag *out);
void orc_inject_laser(const orc_params *p, orc_state *s, const orc_laser *L);
void orc_inject_axion(const orc_params *p, orc_state *s, const orc_axion *A);
double orc_sigma_cell(const orc_params *p, int64_t i, int64_t j, int64_t k, int axion);
void orc_outflow_solve(double dt, double dxa, double m, double g_cur, double g_old,
                       double p0_cur, double S_g, double *V_out, double *U_out);

/* ---- perturbed-particle current (axp_oracle_particles.c) ---- */
int orc_particles_validate(const orc_params *p, const orc_particles *P);
/* positions given at t_n: deposit j0^n, j1^n, then move the positions to t_{n+1/2} */
void orc_particles_start(const orc_params *p, orc_particles *P);
/* positions at t_n of the present state (x0n, x1n: count doubles per axis) */
void orc_particles_positions_now(const orc_params *p, const orc_particles *P, double *x0n[3], double *x1n[3]);
/* fields felt by a particle at x0 (+ x1), from the state's present arrays:
 * F_nop = sum S F0 (+ background), F_p = sum (dS/dx . x1) F0 + sum S F1 */
void orc_gather(const orc_params *p, const orc_state *s, const double x0[3], const double x1[3], double Enop[3],
                double Bnop[3], double Ep[3], double Bp[3]);
/* one momentum update of both orders (Boris rotation and its first-order part) */
void orc_kick(double q_over_m, double dt, const double u0[3], const double u1[3], const double Enop[3],
              const double Bnop[3], const double Ep[3], const double Bp[3], double u0_out[3], double u1_out[3]);
/* adds one particle's current at positions x0 (+ x1) with momenta u0, u1 */
void orc_deposit(const orc_params *p, double qw, const double x0[3], const double x1[3], const double u0[3],
                 const double u1[3], double *j0[3], double *j1[3]);
/* the particle step between the field half-steps: kick with the present fields
 * (t_{n+1/2}), drift, deposit j^{n+1} */
void orc_push(const orc_params *p, const orc_state *s, orc_particles *P);
/* orc_step_src with particles (src may be NULL) */
void orc_step_plasma(const orc_params *p, orc_state *s, const orc_source *src, orc_particles *P, int64_t nsteps);

#ifdef __cplusplus
}
#endif
#endif

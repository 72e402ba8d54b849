/*
 * axp.h -- C ABI of the GB300 axion-coupled Yee field solver.
 *
 * Method: arXiv 2406.16796, "Modeling of axion and electromagnetic fields
 * coupling in a particle-in-cell code", Sec. 2 (Simulation Methods).  One
 * call of axp_step advances, per time step n -> n+1:
 *   - the zeroth-order (laser) fields E0, B0 and the first-order perturbation
 *     fields E1, B1 by the half-step Yee leapfrog of Sec. 2.3 (Eq. update_E,
 *     the B half-steps and the second E half-step);
 *   - the axion field phi by the leapfrog of Eq. update_axion, driven by
 *     S = g E0 . B0 averaged to cell centres (Sec. 2.3);
 *   - the axion current g[(D_t phi) B0 - E0 x grad phi] of Eq. update_E, which
 *     drives E1 (field perturbation separation, Sec. 2.2);
 *   - the axion boundary conditions of Sec. 2.4: periodic, reflect, outflow
 *     and PML; E and B use periodic wrap, a zero-field closure, or an
 *     absorbing layer with the PML's cubic profile.
 * Units: natural units hbar = c = eps0 = 1 (Sec. 2.1), any length unit.
 *
 * Memory: the caller owns all device memory.  axp_workspace_bytes() says how
 * much one grid needs; the caller allocates it (e.g. a torch uint8 tensor)
 * and passes the pointer to axp_create_grid().  The library allocates no
 * device memory of its own.  Host-side handles are small and freed by
 * axp_destroy_grid().
 *
 * Layout in the workspace (each array 256-byte aligned, x fastest, element
 * (i,j,k) at i + n0*(j + n1*k)): E0x E0y E0z B0x B0y B0z E1x E1y E1z B1x
 * B1y B1z, then the axion arrays, the axion current J, outflow ghost planes,
 * diagnostic scratch and the diagnostic ring.  With cell centres at
 * lo + (i+1/2, j+1/2, k+1/2) d:  phi at the centre, E_a at centre + d_a/2,
 * B_a at centre + (d - d_a)/2 (Yee staggering, Sec. 2.3 and Fig. 1).
 * Time levels: E, B at integer n; phi at n+1/2 and n-1/2 (Sec. 2.3).
 *
 * Precision: AXP_FP64 stores and computes everything in double.
 * AXP_FP32_SPLIT stores all arrays in float, keeps E0/B0 and E1/B1 apart as
 * the paper's FPS method does (Sec. 2.2), holds phi as phi^{n+1/2} plus the
 * increment phi^{n+1/2} - phi^{n-1/2}, takes the uniform background fields as
 * double constants, and accumulates every diagnostic in double.
 *
 * Errors: every call returns an axp_status; nothing is thrown across the
 * ABI.  Kernel launch errors are returned by the call that launched;
 * asynchronous device errors are returned by the next synchronising call on
 * the handle (axp_read_diagnostics, axp_read_field, axp_synchronize, ...).
 * A handle is not thread-safe; distinct handles are independent.  All work of
 * a handle runs on the stream given at creation, in call order.
 */
#ifndef AXP_H
#define AXP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AXP_OK = 0,
    AXP_E_INVAL = 1,     /* bad argument, size or combination of options */
    AXP_E_UNSTABLE = 2,  /* dt violates the Yee CFL or the axion leapfrog bound */
    AXP_E_NOMEM = 3,     /* workspace too small / admission refused for lack of memory */
    AXP_E_CUDA = 4,      /* a CUDA call failed; the handle should be destroyed */
    AXP_E_TIMEOUT = 5,   /* a bounded device wait expired */
    AXP_E_NONFINITE = 6, /* a diagnostic came out NaN or Inf */
    AXP_E_STATE = 7      /* call not valid in the handle's present state */
} axp_status;

typedef enum { AXP_FP64 = 0, AXP_FP32_SPLIT = 1 } axp_precision;

/* Boundary kinds.  Axion: all four (Sec. 2.4).  E/B: AXP_BC_PERIODIC,
 * AXP_BC_PML (absorbing layer) or AXP_BC_REFLECT (fields are zero outside the
 * grid).  Periodic must be set on both sides of an axis for both E/B and the
 * axion; an axis with n = 1 must be periodic. */
typedef enum { AXP_BC_PERIODIC = 0, AXP_BC_REFLECT = 1, AXP_BC_OUTFLOW = 2, AXP_BC_PML = 3 } axp_bc;

typedef struct {
    int64_t n[3];             /* cells per axis, >= 1 */
    double d[3];              /* cell sizes, > 0 */
    double lo[3];             /* position of the grid's low faces */
    double dt;                /* time step */
    double m;                 /* axion mass (natural units) */
    double g;                 /* axion-photon coupling g_agg */
    int32_t axion_bc[3][2];   /* [axis][0 = low side, 1 = high side] */
    int32_t em_bc[3][2];
    int32_t pml_cells;        /* absorbing layer thickness N (Sec. 3.1 uses 20) */
    int32_t precision;        /* axp_precision */
    double pml_sigma_max_dt;  /* sigma_max * dt (Sec. 3.1 uses 0.2) */
    int32_t diag_every;       /* axp_step records diagnostics every K steps (0 = never) */
    int32_t diag_capacity;    /* diagnostic ring entries (>= 1 when diag_every > 0) */
} axp_grid_desc;

/* Laser (order-0 field) initial placement at integer time 0.  E = A pol env
 * cos(k.(x - centre) + phase) at the E locations; B is the discrete curl of
 * pol F, F = (A/cos(theta/2)) env sin(...)/|K|, K_d = (2/d_d) sin(k_d d_d/2),
 * sin(theta/2) = dt |K|/2, so a CW wave commensurate with a periodic box is an
 * exact eigenmode of the scheme and B is divergence-free.  env is
 * exp(-r_perp^2/waist^2) exp(-xi^2/L^2) with xi = khat.(x - centre) and
 * L = duration/sqrt(2 ln 2) (duration = intensity FWHM); waist = 0 or
 * duration = 0 drops that factor.  Fields are added to E0, B0. */
typedef struct {
    double amplitude;
    double k[3];
    double pol[3];
    double centre[3];
    double waist;
    double duration;
    double phase;
} axp_laser_desc;

/* Axion field at t = +dt/2 and t = -dt/2 (Sec. 3.1 sets its test pulse at two
 * time levels): phi = A env(xi - speed t) sin(k.(x - centre) - w t + phase),
 * with w from the discrete Klein-Gordon dispersion cos(w dt) =
 * 1 - dt^2 (K^2 + m^2)/2.  env as for the laser with the longitudinal 1/e
 * half-length `length`.  Added to phi; outflow ghosts receive the same
 * profile at the ghost centres. */
typedef struct {
    double amplitude;
    double k[3];
    double centre[3];
    double waist;
    double length;
    double speed;
    double phase;
} axp_axion_desc;

/* Diagnostics at an integer time (Sec. 3.2-3.4), accumulated in double over
 * the cells outside absorbing layers:
 *   H_phi = sum (1/2)[(D_t phi)^2 + |grad phi|^2 + m^2 phi^2] dV  (forward
 *           differences of phi^n, D_t phi^n = (phi^{n+1/2} - phi^{n-1/2})/dt)
 *   H_g0  = sum (1/2)(E0^2 + B0^2) dV (laser part, background excluded)
 *   H_g1  = sum (1/2)(E1^2 + B1^2) dV
 *   P_g2a = H_phi / H_g0,  P_a2g = H_g1 / H_phi   (0 when the divisor is 0)
 *   W     = H_phi + sum (E0.E1 + B0.B1) dV with the background included
 *   sum_xB1z2 / sum_B1z2 = laser centroid along x of Sec. 3.4
 *   gauss_l2 = sum R^2 dV, R = div E1 + g Bbar0 . grad_c phi^n (Sec. 2.2). */
typedef struct {
    int64_t step;
    double t;
    double H_phi, H_g0, H_g1;
    double P_g2a, P_a2g;
    double W;
    double sum_xB1z2, sum_B1z2;
    double gauss_l2;
} axp_diag;

/* Field identifiers for read/write.  Values are transferred as double. */
typedef enum {
    AXP_E0X = 0, AXP_E0Y, AXP_E0Z, AXP_B0X, AXP_B0Y, AXP_B0Z,
    AXP_E1X, AXP_E1Y, AXP_E1Z, AXP_B1X, AXP_B1Y, AXP_B1Z,
    AXP_PHI_CUR = 12, /* phi^{n+1/2} */
    AXP_PHI_OLD = 13  /* phi^{n-1/2} */
} axp_field;

typedef struct axp_grid axp_grid;

/* Human-readable name of a status code.  Never NULL. */
const char *axp_status_str(axp_status s);

/* Bytes of device workspace a grid with this descriptor needs.  Validates the
 * descriptor: AXP_E_INVAL for bad sizes/boundaries, AXP_E_UNSTABLE when dt
 * exceeds the Yee bound dt <= 1/sqrt(sum_a 1/d_a^2) (over axes with n > 1) or
 * the axion bound dt^2 (sum_a 4/d_a^2 + m^2) <= 4. */
axp_status axp_workspace_bytes(const axp_grid_desc *desc, size_t *bytes);

/* Create a grid in caller-owned device memory `dev_workspace` (at least
 * axp_workspace_bytes, 256-byte aligned) on the current CUDA device.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Fields
 * start at zero.  *out receives the handle (host memory owned by the
 * library, released by axp_destroy_grid; the workspace stays the caller's). */
axp_status axp_create_grid(const axp_grid_desc *desc, void *dev_workspace, size_t bytes, void *cuda_stream,
                           axp_grid **out);
axp_status axp_destroy_grid(axp_grid *grid);

/* Uniform static background fields (Sec. 2.2 FPS: part of the order-0
 * field, stored as constants, never in the arrays).  Either pointer may be
 * NULL to leave that field unchanged. */
axp_status axp_set_background_field(axp_grid *grid, const double B_ext[3], const double E_ext[3]);

axp_status axp_inject_laser(axp_grid *grid, const axp_laser_desc *laser);
axp_status axp_inject_axion(axp_grid *grid, const axp_axion_desc *axion);

/* Laser entering through a fixed x-plane (Sec. 3.2: the laser is injected
 * into the box), as a soft source: an electric current sheet on the E cells
 * at x index `plane` and a magnetic one on the B faces at index plane-1 (the
 * faces on the plane x_p = lo + plane d[0]).  Together they launch the
 * incident wave towards +x only:
 *   E_inc = A pol f(y, z) env(t - t_centre - (x - centre[0]))
 *           cos(k (x - centre[0]) - w (t - t_centre) + phase),   B_inc = xhat x E_inc,
 * with t = step dt, x the lab position (a moving window moves the grid, not
 * the wave), w from the Yee dispersion along x, sin(w dt/2)/dt =
 * sin(k dx/2)/dx (a CW wave is then an exact discrete plane wave: nothing
 * appears behind the plane), f = exp(-r^2/waist^2) over the active
 * transverse axes around (centre[1], centre[2]) (1 for waist = 0) and env =
 * exp(-u^2/L^2), L = duration/sqrt(2 ln 2) (1 for duration = 0).  Added to the
 * order-0 half-steps: E_y, E_z of cell `plane` get +A pol f tau/dx in their
 * curl (tau the wave factor at x_p, at the time of the B they read); B_y, B_z
 * on the faces get -A pol_z f tau/dx and +A pol_y f tau/dx (tau at x_p + dx/2,
 * t_{n+1/2}).  The sheets stop where a transverse absorbing layer begins;
 * their transverse profile is taken when the source is set.
 * Requirements: a grid with n[0] >= 2; 1 <= plane <= n[0]-1 with the cells
 * plane-1 and plane outside the x absorbing layers; pol[0] = 0; k > 0;
 * finite values; waist, duration >= 0.  Otherwise AXP_E_INVAL, and
 * AXP_E_STATE for a grid that a group is stepping.  `src` = NULL switches the
 * source off.  The source is a setting of the handle (like the kernel choice),
 * not part of the saved state.  Steps with a source run on the general path,
 * or on the 2D TM kernel when the polarisation is along z. */
typedef struct {
    double amplitude;
    double k;
    double pol[3];
    double centre[3];
    double waist;
    double duration;
    double t_centre;
    double phase;
    int64_t plane;
} axp_source_desc;
axp_status axp_set_soft_source(axp_grid *grid, const axp_source_desc *src);

/* Advance nsteps >= 0 time steps, asynchronously on the grid's stream.  When
 * diag_every > 0, a diagnostic record is appended to the device ring after
 * every step whose new index is a multiple of diag_every (the oldest record
 * is overwritten when the ring is full). */
axp_status axp_step(axp_grid *grid, int64_t nsteps);

/* Copy up to `max` unread ring records (oldest first) to host `out`; *n gets
 * the count.  Synchronises the stream.  AXP_E_NONFINITE if any copied record
 * holds NaN/Inf. */
axp_status axp_read_diagnostics(axp_grid *grid, axp_diag *out, int64_t max, int64_t *n);

/* Diagnostics of the present state, computed now.  Synchronises. */
axp_status axp_compute_diagnostics(axp_grid *grid, axp_diag *out);

/* Diagnostics of FP64 fields the caller already holds, with no device
 * allocation at all.  The paper has no counterpart: this entry point serves
 * callers that cannot call cudaMalloc -- code whose fields live in memory
 * another allocator owns and that may not create an axp workspace, for
 * instance inside a latency-critical loop where cudaMalloc/cudaFree would
 * implicitly synchronise the device, or in a process whose device memory is
 * entirely handed to another framework's pool.
 *   desc        grid description (precision must be AXP_FP64; no outflow faces).
 *               desc->lo must be the grid's present lower corner: after moving
 *               window shifts, the shifted corner (the regular entry point adds
 *               the window's offset itself), since the B1z-weighted centroid
 *               sum uses absolute positions lo + (i+1) dx
 *   dev_fields  14 device pointers, each n0*n1*n2 doubles in the layout above:
 *               E0x E0y E0z B0x B0y B0z E1x E1y E1z B1x B1y B1z,
 *               phi^{n+1/2}, phi^{n-1/2}; E and B at the integer time `step`
 *   B_ext, E_ext  uniform background fields
 *   host_out    receives the record (same definitions as axp_compute_diagnostics)
 * The reduction's scratch is a fixed array inside the library, so grids are
 * limited to 8,388,608 cells (AXP_E_INVAL beyond, with a message on stderr).
 * The array lives on every GPU that loads the library until the process exits.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process.  Every call
 * synchronises its stream, so the entry point cannot be used inside a stream
 * capture.  A cudaDeviceReset of the device discards
 * the array and so the kept address: do not call this entry point on that
 * device again in the same process after a reset.  Every call shares the array and
 * rewrites what it uses, so results never depend on earlier calls, but calls
 * that overlap on the GPU (from other threads or streams) race.  The call
 * synchronises `cuda_stream` before returning. */
axp_status axp_diagnostics_noalloc(const axp_grid_desc *desc, const double *const dev_fields[14],
                                   const double B_ext[3], const double E_ext[3], int64_t step, void *cuda_stream,
                                   axp_diag *host_out);

/* Copy one field to/from host memory as n0*n1*n2 doubles (bytes must equal
 * 8 * cells).  Synchronises.  Writing marks the cached axion current stale. */
axp_status axp_read_field(axp_grid *grid, int32_t which, double *host_dst, size_t bytes);
axp_status axp_write_field(axp_grid *grid, int32_t which, const double *host_src, size_t bytes);

/* Macroparticles and the perturbed-particle current of Sec. 2.2 (FPS: the
 * particle momentum, velocity and current split into an order-0 part and its
 * first-order perturbation, j = j0 + j1).  One species per grid, FP64 grids
 * only, every active axis (n > 1) periodic for E and B.  Natural units
 * (c = 1): u = gamma v is the normalised momentum, du/dt = (q/m)(E + v x B);
 * a macroparticle of weight w stands for w physical particles in the cell
 * volume dV = d0 d1 d2.
 *
 * Each step (Sec. 2.3 step order) pushes the particles between the axion
 * update and the second field half-steps, with the fields of both orders at
 * t_{n+1/2} felt at x0 + x1 (Sec. 2.2: F_nop = sum S(r - x0) F0 plus the
 * uniform background, F_p = sum (dS/dx . x1) F0 + sum S F1), the order-0
 * momentum by the relativistic Boris scheme and u1 by the first-order part of
 * the same operations (continuum limit dp1/dt = q (E_p + v0 x B_p + v1 x
 * B_nop)).  The current j^{n+1} = (q w/dV)[S v0] and (q w/dV)[(dS/dx . x1) v0 +
 * S v1], deposited at x^{n+1} with v^{n+1}, enters the second E half-steps of
 * its order and the next step's first ones (curl B = dE/dt + j).  S is the
 * quadratic B-spline on each component's own staggered nodes.  A grid with
 * particles always takes the general (multi-pass) kernels: AXP_KERNEL_AUTO
 * chooses them, and forcing a single-pass kernel makes axp_step return
 * AXP_E_STATE.  Checkpoint images (axp_save_state) hold the fields only.
 *
 * axp_particles_bytes: device workspace for `count` particles on this grid.
 * axp_attach_particles: attach `count` particles of charge q and mass m > 0,
 *   kept in the caller's device workspace (256-byte aligned, at least
 *   axp_particles_bytes; owned by the caller, used until detach or destroy).
 *   They start at rest at the origin with weight 0 until written.
 *   AXP_E_INVAL: bad arguments, an FP32 grid or a non-periodic active axis;
 *   AXP_E_NOMEM: workspace too small; AXP_E_STATE: particles already attached
 *   or the grid is in a group.
 * axp_write_particles / axp_read_particles: host arrays of 13 rows of `count`
 *   doubles: w, x0 (x, y, z), u0 (x, y, z), x1 (x, y, z), u1 (x, y, z), positions
 *   and momenta at the grid's present time step.  Writing deposits j^n (so the
 *   next step's first E half-steps see it); non-finite values give
 *   AXP_E_NONFINITE.  Both synchronise.
 * axp_read_particle_current: j^n of order `order` (0 or 1) as 3 rows of cells
 *   doubles (x, y, z components on the E_x, E_y, E_z locations).
 * axp_detach_particles: the grid continues without particles. */
axp_status axp_particles_bytes(const axp_grid *grid, int64_t count, size_t *bytes);
axp_status axp_attach_particles(axp_grid *grid, int64_t count, double q, double m, void *dev_workspace,
                                size_t bytes);
axp_status axp_write_particles(axp_grid *grid, const double *host_src, size_t bytes);
axp_status axp_read_particles(axp_grid *grid, double *host_dst, size_t bytes);
axp_status axp_read_particle_current(axp_grid *grid, int32_t order, double *host_dst, size_t bytes);
axp_status axp_detach_particles(axp_grid *grid);

/* Outflow ghost planes of axis `axis`, side `side` (level 0 = phi^{n+1/2},
 * 1 = phi^{n-1/2}) as doubles; plane index: axis 0 -> j + n1 k,
 * axis 1 -> i + n0 k, axis 2 -> i + n0 j.  AXP_E_INVAL unless that face is
 * an outflow face. */
axp_status axp_read_ghost(axp_grid *grid, int32_t axis, int32_t side, int32_t level, double *host_dst,
                          size_t bytes);
axp_status axp_write_ghost(axp_grid *grid, int32_t axis, int32_t side, int32_t level, const double *host_src,
                           size_t bytes);

/* Complete checkpoint: the state, ghosts, step count, background and window,
 * as an opaque byte image of axp_state_bytes() bytes.  The image holds only
 * the arrays that can be non-zero: the order-0 components the injected laser
 * couples to, all order-1 components and both axion levels; the cached axion
 * current is recomputed after a load.  Its size therefore follows the grid's
 * injected components at the time of the save.  A grid that the single-pass
 * kernels are stepping keeps E half a step ahead of B (leapfrog staggering);
 * its image is taken in that form, without a conversion, unless the grid has
 * a soft source (then E is converted to integer time first).  Loading into a
 * grid of the same descriptor resumes bit for bit, a staggered image as the
 * uninterrupted run would have continued (arrays outside the image are set to
 * zero); a staggered image cannot be loaded into a grid with a soft source
 * (AXP_E_STATE).  Both synchronise. */
axp_status axp_state_bytes(const axp_grid *grid, size_t *bytes);
axp_status axp_save_state(axp_grid *grid, void *host_dst, size_t bytes);
axp_status axp_load_state(axp_grid *grid, const void *host_src, size_t bytes);

/* Slab decomposition of one grid across devices (the rows exchange that a
 * domain decomposition of the explicit scheme of Sec. 2.3 needs; the paper
 * itself runs inside EPOCH's own decomposition).  Rows are the cells with one
 * index along the grid's slowest axis with more than one cell (z in 3D, y in
 * 2D, x in 1D); row r is the contiguous range of n0*n1 (3D), n0 (2D) or 1
 * (1D) elements at offset r times that.  A slab grid holds its owned rows
 * plus halo rows on each side; k steps on their own leave the owned rows
 * exact while the halo is at least k + 2 rows wide (one step's dependency
 * cone is one cell wide, the axion current's stencil widens it once), wider
 * by the absorbing layer where a slab's cut side carries one.
 *
 * axp_pack_rows copies rows [row0, row0 + nrows) of the 14 arrays of the
 * present state (the 12 fields, phi^{n+1/2}, then the second axion level, in
 * the grid's storage precision and present representation) into the device
 * buffer dev_dst, array after array; axp_unpack_rows writes such a buffer
 * into rows of this grid.  Both are asynchronous on the grid's stream and
 * allocate nothing; bytes must equal axp_rows_bytes(nrows).  The state's
 * representation (integer time, or the staggered state of the single-pass
 * kernels) must be the same on both sides: slabs that exchange rows take the
 * same kernel path and the same steps.  AXP_E_INVAL for rows outside the
 * grid; AXP_E_STATE for a grid with macroparticles (they do not move between
 * slabs).
 *
 * axp_compute_diagnostics_rows: the record of axp_compute_diagnostics
 * restricted to the cells whose row lies in [row0, row1) (and in the physical
 * region).  Its energies and sums (H_phi, H_g0, H_g1, W, sum_xB1z2, sum_B1z2,
 * gauss_l2) add up across slabs; the ratios are formed from the sums.
 * Synchronises. */
axp_status axp_rows_bytes(const axp_grid *grid, int64_t nrows, size_t *bytes);
axp_status axp_pack_rows(axp_grid *grid, int64_t row0, int64_t nrows, void *dev_dst, size_t bytes);
axp_status axp_unpack_rows(axp_grid *grid, int64_t row0, int64_t nrows, const void *dev_src, size_t bytes);
axp_status axp_compute_diagnostics_rows(axp_grid *grid, int64_t row0, int64_t row1, axp_diag *out);

/* Current step index n, and a wait for all queued work of the handle. */
axp_status axp_get_step(const axp_grid *grid, int64_t *step);
axp_status axp_synchronize(axp_grid *grid);

/* Moving window (Sec. 3.2: the simulation window moves at the speed of light
 * after the laser has entered it).  A shift by `cells` along `axis` moves the
 * integer-time state -- every field array of both orders and both axion
 * levels -- towards lower index along that axis; the `cells` entering at the
 * high end are vacuum (zero), the ones leaving at the low end are dropped, and
 * the grid origin moves by cells x d[axis] (later injections and the laser
 * centroid use the moved origin).  The axis must not be periodic and the grid
 * must have no outflow axion side (outflow ghost planes do not move); one
 * window axis per grid.
 *
 * axp_shift_window shifts once, now.  axp_set_moving_window makes axp_step
 * move the window at `velocity` (units of c, in (0, 1]) from step
 * `start_step` on: the window's travel accumulates velocity x dt / d[axis]
 * cells per step and each time it reaches `shift_cells` the state is shifted
 * by shift_cells between two steps.  velocity = 0 stops the window.  The
 * window state is part of checkpoints. */
axp_status axp_shift_window(axp_grid *grid, int32_t axis, int64_t cells);
axp_status axp_set_moving_window(axp_grid *grid, int32_t axis, double velocity, int32_t shift_cells,
                                 int64_t start_step);
/* Cells shifted so far. */
axp_status axp_get_window_offset(const axp_grid *grid, int64_t *cells);

/* Kernel selection for axp_step.  AXP_KERNEL_AUTO (default) uses the fastest
 * single-pass kernel that supports the grid's shape, boundaries and active
 * field components, else the general multi-pass kernels.
 * AXP_KERNEL_GENERAL forces the general kernels (one pass per stage of the
 * time scheme, in the oracle's operation order); AXP_KERNEL_FUSED forces the
 * generic single-pass kernel (1D/2D/3D, periodic, reflect and PML edges);
 * AXP_KERNEL_TM2D forces the single-pass kernel specialised for 2D grids with
 * an (E0z; B0x, B0y) laser and periodic or PML edges (at most 2^32 cells), on
 * its uniform launch grid of x strips by march chunks;
 * AXP_KERNEL_TM2D_LIST forces the same kernel on per-block work lists (FP64
 * grids without a soft source): the host cuts each x strip into tiles of about
 * equal cost and lets two short tiles share a block, so that every block, all
 * resident at once, finishes at about the same time (the work list sits in the
 * workspace and is copied there, host to device on the grid's stream, by the
 * first axp_step after a change of kernel, soft source or background field;
 * a grid too wide for the list's 2048 items makes axp_step return AXP_E_CUDA);
 * AUTO takes whichever of the two forms the planner's cost model prefers;
 * AXP_KERNEL_AX3D forces the single-pass kernel specialised for periodic 3D
 * grids with no laser fields and no uniform E (an axion wave in a uniform B);
 * AXP_KERNEL_BLOCK1D forces the time-blocked kernel for FP64 1D grids that
 * are periodic along x (at least 256 cells, no soft source): the single-pass
 * kernels' staggered scheme reduced to 1D, its curl updates folded into one
 * multiply-add per difference (within 1e-12 of the general path after 20000
 * steps), over windows held in shared memory for blocks of steps, in one
 * cooperative launch per run of steps; any split of a run into launches gives
 * the same bits.  Should one of its
 * bounded grid-wide waits give up, the next synchronising call on the handle
 * (axp_synchronize, diagnostics, reads, axp_save_state) returns
 * AXP_E_TIMEOUT.  Forcing a kernel that does not support the grid makes
 * axp_step return AXP_E_STATE. */
typedef enum {
    AXP_KERNEL_AUTO = 0,
    AXP_KERNEL_GENERAL = 1,
    AXP_KERNEL_FUSED = 2,
    AXP_KERNEL_TM2D = 3,
    AXP_KERNEL_AX3D = 4,
    AXP_KERNEL_BLOCK1D = 5,
    AXP_KERNEL_TM2D_LIST = 6
} axp_kernel;
axp_status axp_set_kernel(axp_grid *grid, int32_t kernel);
/* Which path the next axp_step will take (an axp_kernel value other than AUTO). */
axp_status axp_get_kernel_path(axp_grid *grid, int32_t *path);

/* Failure detection test for the time-blocked 1D kernel (no counterpart in
 * the paper): in the next launch of that kernel on this grid, block `block`
 * leaves before its first grid-wide wait, as a participant that never
 * arrives.  The other blocks' bounded waits give up after about a second, the
 * launch ends, the state is left partly advanced, and the next synchronising
 * call returns AXP_E_TIMEOUT.  -1 cancels.  Nothing faults or hangs. */
axp_status axp_test_block1d_absent(axp_grid *grid, int32_t block);

/* Number of kernel launches issued by this handle since creation (for
 * launch accounting in benchmarks). */
axp_status axp_get_launch_count(const axp_grid *grid, int64_t *count);

/* ------------------------------------------------------------------------
 * Batches of 1D conversion runs (parameter scans and serving).
 *
 * Each instance is the 1D photon -> axion set-up of Sec. 3.2 in a periodic
 * box: a CW laser E0y along x (placed as the exact discrete eigenmode, as
 * axp_inject_laser does), a uniform background B_ext = (0, By, Bz), and the
 * axion field initially zero.  Every instance has its own size, mass,
 * coupling, background, laser and step count.  All instances are stored in
 * FP32 split form (as AXP_FP32_SPLIT) and advanced together: one launch
 * advances every unfinished instance by up to `block_steps` steps, each
 * (instance, segment) work item keeping its cells in registers (8 per
 * thread) for the whole block (time blocking; segments of large instances
 * carry a halo of 3 cells per step).  Diagnostics are accumulated in FP64.
 *
 * Memory: the caller provides one device workspace sized for a maximum number
 * of instances and a total number of cells; instances are admitted into it
 * first-fit and their cells released on removal (admission by device memory).
 * The batch's per-launch bookkeeping lives on the device, so a sequence of
 * axp_batch_run calls can be captured in a CUDA graph.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t nx;           /* cells (periodic box), >= 8 */
    double dx, dt;        /* dt <= dx (Yee bound) and the axion bound */
    double m, g;          /* axion mass and coupling */
    double By, Bz;        /* uniform background field (B_ext,x = 0) */
    double amplitude;     /* laser E amplitude */
    double k;             /* laser wave number (2 pi x whole wavelengths / box) */
    int64_t steps;        /* total steps to run */
} axp_batch_instance;

typedef struct axp_batch axp_batch;

/* Workspace bytes for up to max_instances instances totalling max_cells cells. */
axp_status axp_batch_workspace_bytes(int32_t max_instances, int64_t max_cells, size_t *bytes);
axp_status axp_batch_create(int32_t max_instances, int64_t max_cells, void *dev_workspace, size_t bytes,
                            void *cuda_stream, axp_batch **out);
axp_status axp_batch_destroy(axp_batch *batch);

/* Admit an instance (initial fields written on the batch's stream).  *slot
 * receives its slot; AXP_E_NOMEM when no slot or no contiguous cell range is
 * free, AXP_E_UNSTABLE / AXP_E_INVAL for bad parameters. */
axp_status axp_batch_add(axp_batch *batch, const axp_batch_instance *inst, int32_t *slot);
/* Release a slot and its cells (the instance need not be finished). */
axp_status axp_batch_remove(axp_batch *batch, int32_t slot);

/* Advance every admitted, unfinished instance by up to nsteps steps,
 * asynchronously on the batch's stream (ceil(nsteps / block_steps) launches of
 * the persistent kernel plus one bookkeeping launch each). */
axp_status axp_batch_run(axp_batch *batch, int64_t nsteps);

/* Replay each axp_batch_run as one CUDA graph (captured on first use and kept
 * while the step count, the tiling and the set of admitted instances are
 * unchanged).  Needs a batch created on a non-default stream. */
axp_status axp_batch_use_graphs(axp_batch *batch, int32_t enable);
/* Kernel launches issued (graph replays count their nodes). */
axp_status axp_batch_launch_count(const axp_batch *batch, int64_t *count);

/* Steps done so far per slot (-1 for free slots), copied to host; synchronises. */
axp_status axp_batch_progress(axp_batch *batch, int64_t *steps_done, int32_t max_slots);

/* FP64 diagnostics of one slot's present state (same definitions as axp_diag);
 * synchronises. */
axp_status axp_batch_result(axp_batch *batch, int32_t slot, axp_diag *out);
/* The same for n slots at once (host array `slots`, n <= max_instances; out[q]
 * receives slot slots[q]'s record): one launch, one copy, one synchronisation.
 * Each record is bit-identical to axp_batch_result's.  AXP_E_INVAL if a listed
 * slot is free, AXP_E_NONFINITE if a record holds NaN/Inf. */
axp_status axp_batch_results(axp_batch *batch, const int32_t *slots, int32_t n, axp_diag *out);

/* Stored state of one slot as nx doubles: which = 0 E0y, 1 B0z, 2 E1y, 3 E1z,
 * 4 B1y, 5 B1z, 6 phi^{n+1/2}, 7 phi^{n+1/2} - phi^{n-1/2}.  B and phi are at
 * the present step n; the E arrays hold E^{n+1/2} (the leapfrog-staggered
 * state the batch advances).  Synchronises. */
axp_status axp_batch_read_state(axp_batch *batch, int32_t slot, int32_t which, double *host_dst, size_t bytes);

/* Time blocking: steps per launch, core cells per segment, threads per CTA
 * (default 32, 1856, 256: a segment and its halo fill the block).
 * block_steps in [1, 256]; threads a multiple of 32 in [64, 512]; a work item
 * holds 8 cells per thread, so segment_cells + 6 block_steps <= 8 threads
 * (instances of up to 8 threads cells run whole). */
axp_status axp_batch_set_tiling(axp_batch *batch, int32_t block_steps, int32_t segment_cells, int32_t threads);
axp_status axp_batch_get_tiling(const axp_batch *batch, int32_t *block_steps, int32_t *segment_cells,
                                int32_t *threads);

/* ------------------------------------------------------------------------
 * Groups of 2D grids stepped together (continuous batching of 2D runs).
 *
 * A group advances many independent 2D grids -- each created with
 * axp_create_grid in FP32 split precision, with the (E0z; B0x, B0y) laser
 * polarisation of the 2D pulse set-up (Sec. 3.2) or none, periodic or
 * absorbing (PML on E/B and phi together) sides, no uniform background E,
 * and diag_every = 0 -- by one persistent launch per time step.  Each launch
 * moves every unfinished member on by exactly one step of the same scheme
 * axp_step runs; members differ in size, mass, coupling, fields and step
 * count.  Results equal those of axp_step on the grid alone (the same
 * arithmetic per cell).
 *
 * While a grid is a member, every axp_* call on the grid itself returns
 * AXP_E_STATE; axp_group_remove hands it back with its step count advanced
 * by the steps the group ran on it, after which diagnostics, reads and
 * further axp_step calls work as usual.  Memory: the group's workspace holds
 * only per-member parameters and the tile table (the grids keep their own
 * workspaces); admission is bounded by max_grids and max_tiles, where a grid
 * of nx x ny cells takes ceil(nx / 251) x ceil(ny / chunk) tiles.
 * ------------------------------------------------------------------------ */
typedef struct axp_group axp_group;

axp_status axp_group_workspace_bytes(int32_t max_grids, int32_t max_tiles, size_t *bytes);
axp_status axp_group_create(int32_t max_grids, int32_t max_tiles, void *dev_workspace, size_t bytes,
                            void *cuda_stream, axp_group **out);
/* AXP_E_STATE while members remain. */
axp_status axp_group_destroy(axp_group *group);
/* Join a grid that will run `steps` more steps; *member receives its index.
 * Synchronises the grid's stream.  AXP_E_INVAL for grids the group cannot
 * step (among them grids with a soft source), AXP_E_NOMEM when no member
 * index or too few tiles are free. */
axp_status axp_group_add(axp_group *group, axp_grid *grid, int64_t steps, int32_t *member);
/* Hand a member's grid back (finished or not); synchronises the group's stream. */
axp_status axp_group_remove(axp_group *group, int32_t member);
/* nsteps launches on the group's stream, asynchronous. */
axp_status axp_group_run(axp_group *group, int64_t nsteps);
/* Steps done per member index (-1 for free indices); synchronises. */
axp_status axp_group_progress(axp_group *group, int64_t *steps_done, int32_t max_members);
/* y planes per tile (default 64, >= 8); only while the group is empty. */
axp_status axp_group_set_chunk(axp_group *group, int32_t rows);
/* Replay each axp_group_run as one CUDA graph, kept while the step count and
 * the membership are unchanged.  Needs a non-default stream. */
axp_status axp_group_use_graphs(axp_group *group, int32_t enable);
axp_status axp_group_launch_count(const axp_group *group, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif /* AXP_H */

// axp_internal.h -- definitions shared by the CUDA translation units of libaxp.
//
// Method: arXiv 2406.16796 Sec. 2.3-2.4.  This header holds the grid handle,
// the by-value kernel view of a grid, and the boundary-aware index helpers
// used by the general (multi-pass) kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "axp.h"

namespace axp {

constexpr int kFields = 12;  // E0xyz B0xyz E1xyz B1xyz
constexpr int kE0 = 0, kB0 = 3, kE1 = 6, kB1 = 9;
constexpr int kDiagSlots = 10;  // per-cell accumulators of the diagnostics kernel

// Per-grid parameters in the arithmetic type T, passed to kernels by value.
template <typename T>
struct View {
    T *f[kFields];
    T *phi_cur;   // phi^{n+1/2}
    T *phi_b;     // FP64: phi^{n-1/2};  FP32 split: increment pi^n = phi^{n+1/2} - phi^{n-1/2}
    T *phi_next;  // FP32 split: buffer that receives phi^{n+3/2}; unused for FP64
    T *J[3];      // axion current (without g) at the E locations
    T *gh[3][2][3];  // outflow ghost planes [axis][side][level: 0 = n+1/2, 1 = n-1/2, 2 = n+3/2]
    const T *sig_em[3];  // absorbing-layer profile per axis (E/B), length n[a]
    const T *sig_ax[3];  // PML profile per axis (axion)
    int64_t n[3];
    int64_t N;
    T d[3];
    // 1/d, 1/(2d) and 1/d^2 per axis where d is a power of two, else 0.  Then
    // x / d and x * (1/d) are the same correctly rounded value, and the general
    // kernels multiply; otherwise they divide (set by set_reciprocals).
    T rd[3], rd2[3], rdd[3];
    T lo[3];
    T dt, h;     // h = dt / 2
    T g, m2;
    T Bext[3], Eext[3];
    int periodic[3];
    int axbc[3][2];
    int region_lo[3], region_hi[3];  // diagnostics region [lo, hi) per axis
    // cells a general kernel visits: all (vaxis < 0), or those whose index along
    // vaxis lies in [vlo, vhi); Nv of them
    int vaxis;
    int64_t vlo, vhi, Nv;
    // current density j^n of the attached macroparticles, order 0 and order 1, at
    // the E locations (null without particles)
    T *jp[2][3];
};

// Macroparticles of one species attached to a FP64 grid (perturbed-particle
// current, Sec. 2.2).  All arrays sit in the caller's particle workspace.
// Positions x0, x1 are at t_{n+1/2}, momenta u0, u1 (u = gamma v) at t_n, and
// j[order] holds the current density j^n deposited by the last push.
struct Particles {
    int64_t count;
    double q, m;
    char *ws;
    size_t bytes;
    double *w, *x0[3], *u0[3], *x1[3], *u1[3];
    double *j[2][3];
    double *scratch[6];  // read-back of the positions at t_n (x0, x1)
};

// A named NVTX range over one entry point of the C ABI: a span on a profiler's
// timeline (nsys, ncu's range filters); without a tool attached it costs a
// check of an unset function pointer.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// The exact reciprocals of View::rd, rd2 and rdd, from v.d: kept only where
// both the divisor and its reciprocal are normal numbers and their product is
// exactly 1 (d a power of two), so that multiplying gives the division's bits.
template <typename T>
inline void set_reciprocals(View<T> &v)
{
    auto exact = [](T den) -> T {
        int e = 0;
        if (!(den > T(0)) || !std::isnormal(den) || std::frexp(den, &e) != T(0.5)) return T(0);
        const T r = T(1) / den;
        return std::isnormal(r) && r * den == T(1) ? r : T(0);
    };
    for (int a = 0; a < 3; a++) {
        v.rd[a] = exact(v.d[a]);
        v.rd2[a] = exact(T(2) * v.d[a]);
        v.rdd[a] = exact(v.d[a] * v.d[a]);
    }
}

constexpr int kSchedItems = 2048;

struct Workspace {
    size_t off_fields[2][kFields];  // two field sets: the fused step reads one and writes the other
    size_t off_phi[4];              // axion buffers; roles are tracked by the handle
    size_t off_J[3];
    size_t off_P[3];  // scratch of the general path's current: P at cell centres
    size_t off_ghost[3][2][3];
    size_t off_sig_em[3], off_sig_ax[3];
    // per axis, 6 x n[a] coefficients of the layer updates as products (fused 2D kernel):
    // E/B: a = (1 - s h/2)/(1 + s h/2), b = h/(1 + s h/2), and for two half-steps a^2,
    // b (1 + a); axion: c1 = dt^2/(1 + s dt), c2 = (1 - s dt)/(1 + s dt).  All decrease
    // with s, so the corner value (largest s of the axes) is the smallest of the axes'.
    size_t off_pml_tab[3];
    // soft source: per (j, k) of the x-plane, A pol_a f / dx for a = y, z (zero in layers)
    size_t off_src[2];
    size_t off_sched;  // 2D grids: kSchedItems work-list items (int4) of the 2D kernel
    size_t off_partials;
    size_t off_ring;
    size_t off_flag;
    size_t total;
    int diag_blocks;
    size_t elem;
};

}  // namespace axp

struct axp_grid {
    axp_grid_desc desc;
    double B_ext[3], E_ext[3];
    cudaStream_t stream;
    int device;
    char *ws;
    size_t ws_bytes;
    axp::Workspace layout;
    // current roles of the axion buffers (indices into off_phi): phi^{n+1/2}, the
    // second level (phi^{n-1/2} or the increment), and two spares
    int phi_cur_slot, phi_b_slot, phi_next_slot, phi_next_b_slot;
    int fset;         // field set holding the present state
    bool staggered;   // E arrays hold E^{n+1/2} (fused-path state) instead of E^n
    int ghost_level_slot[3];  // which stored plane currently holds level 0/1/2
    int64_t step;
    bool J_valid;       // J holds J^n of the present state
    int32_t kernel_choice;
    int64_t ring_written;  // records appended since creation
    int64_t ring_read;     // records returned to the caller
    int64_t launches;
    uint32_t active;       // bit per field array that may be non-zero
    bool phi_active;
    void *group;           // the axp_group stepping this grid, or null
    // CUDA graphs of consecutive fused 1D steps, one per buffer-role configuration;
    // cfg_version changes whenever fields, background or kernel choice change
    int64_t cfg_version;
    // moving window: axis (-1: none), speed in units of c, cells per shift, first
    // step at which it moves, distance travelled since the last shift (cells)
    int32_t win_axis;
    double win_velocity;
    int32_t win_cells;
    int64_t win_start;
    double win_travel;
    int64_t win_offset;  // cells shifted so far
    cudaStream_t capture_stream;
    int n_step_graphs;
    int64_t step_graph_key[8];
    cudaGraphExec_t step_graph[8];
    // soft source (axp_set_soft_source); its sheet weights sit in off_src
    bool src_on;
    axp_source_desc src;
    // the time-blocked 1D kernel has run: its barrier-timeout word (off_flag + 4)
    // is checked by the next synchronising call
    bool coop_used;
    int32_t coop_absent;  // failure-detection test: block that skips the next launch's barriers (-1: none)
    // launch plan of the 2D single-pass kernel, made for configuration tm_plan_key
    // (-1: none): tile width, and either the uniform grid (chunk sizes, chunk rows)
    // or tm_list_blocks blocks of tm_list_per_block work-list items in off_sched
    int64_t tm_plan_key;
    int32_t tm_tx, tm_chunk, tm_chunk_first, tm_chunk_edge, tm_nchunks;
    int32_t tm_list_blocks, tm_list_per_block;
    std::vector<int4> tm_items;  // the work lists (host copy)
    bool tm_items_uploaded;      // tm_items are in off_sched
    // the other field set holds E^{n-1/2} of the present staggered state E^{n+1/2}:
    // the last change of state was a single-pass step (made at configuration
    // half_prev_cfg), so E^n follows cell by cell from the two levels
    bool half_prev;
    int64_t half_prev_cfg;
    // attached macroparticles (Sec. 2.2), or null; a grid with particles takes the
    // general path
    axp::Particles *parts;
};

namespace axp {

size_t elem_size(const axp_grid_desc &d);
bool compute_layout(const axp_grid_desc &d, Workspace *w);

template <typename T>
View<T> make_view(axp_grid *g);
// view whose E0/E1 arrays are taken from field set `eset` (B and the rest from the present set)
template <typename T>
View<T> make_view_eset(axp_grid *g, int eset);

// launchers implemented in the .cu files (return cudaGetLastError())
template <typename T>
cudaError_t general_step(axp_grid *g, int64_t nsteps);
template <typename T>
cudaError_t general_current(axp_grid *g);  // J^n of the present state
template <typename T>
cudaError_t diag_compute(axp_grid *g, axp_diag *dev_dst);
template <typename T>
cudaError_t diag_compute_rows(axp_grid *g, axp_diag *dev_dst, int axis, int64_t lo, int64_t hi);
template <typename T>
cudaError_t inject_laser(axp_grid *g, const axp_laser_desc &L);
template <typename T>
cudaError_t inject_axion(axp_grid *g, const axp_axion_desc &A);
template <typename T>
cudaError_t fused_step(axp_grid *g, int64_t nsteps, bool *handled);
// macroparticles: workspace size and layout, the deposit of j^n with the move of
// the positions to t_{n+1/2}, the push between the field half-steps (fields of the
// view at t_{n+1/2}), and the positions at t_n into the read-back scratch
size_t particles_bytes(const axp_grid_desc &d, int64_t count);
void particles_layout(const axp_grid_desc &d, Particles *P);
cudaError_t particles_start(axp_grid *g);
cudaError_t particles_push(axp_grid *g, const View<double> &v);
cudaError_t particles_now(axp_grid *g);
// time-blocked 1D kernel (FP64, periodic): eligibility and steps on the integer-time state
bool block1d_supported(const axp_grid *g);
cudaError_t block1d_step(axp_grid *g, int64_t nsteps);
template <typename T>
bool fused_supported(const axp_grid *g);
// the path axp_step will take under the handle's kernel choice (an axp_kernel value)
template <typename T>
int32_t fused_path(axp_grid *g);
// staggered <-> integer-time conversion of E (E^{n+1/2} = E^n + h (curl B^n - g J^n))
template <typename T>
cudaError_t enter_staggered(axp_grid *g);
template <typename T>
cudaError_t exit_staggered(axp_grid *g, bool in_place);
// mask of E0/B0 components that can become non-zero (bits 0-2 E0xyz, 3-5 B0xyz)
uint32_t order0_closure(const axp_grid *g);
cudaError_t ensure_integer(axp_grid *g);
// buffer roles after one more fused step (field sets and axion slots alternate)
void rotate_roles(axp_grid *g);
// grid origin along axis a, moved by the window's shifts
inline double lo_of(const axp_grid *g, int a)
{
    return g->desc.lo[a] + (a == g->win_axis ? (double)g->win_offset * g->desc.d[a] : 0.0);
}
// Soft source: the incident wave's time factor env(t - t_c - (x - x_c)) cos(k (x - x_c)
// - w (t - t_c) + phase) at lab position x and time t (host, FP64).
double source_wave(const axp_grid *g, double x, double t);
// lab x of the sheet's B faces (the plane itself) and of its E cells
inline double source_x_b(const axp_grid *g) { return lo_of(g, 0) + (double)g->src.plane * g->desc.d[0]; }
inline double source_x_e(const axp_grid *g) { return lo_of(g, 0) + ((double)g->src.plane + 0.5) * g->desc.d[0]; }
// step times: t_n, t_{n+1/2}, t_{n+1} of step n
inline double time_n(const axp_grid *g, int64_t n) { return (double)n * g->desc.dt; }
inline double time_half(const axp_grid *g, int64_t n) { return ((double)n + 0.5) * g->desc.dt; }
// shift the integer-time state by s cells along axis (moving window)
template <typename T>
cudaError_t shift_window(axp_grid *g, int axis, int64_t s);
// the same shift applied to the staggered state with only the bands at the ends
// of the axis taken through integer time; *done = false where it does not apply
template <typename T>
cudaError_t shift_staggered(axp_grid *g, int axis, int64_t s, bool *done);
// destroy the cached step graphs (and the capture stream when `all`)
void release_step_graphs(axp_grid *g, bool all);

axp_diag *ring_slot(axp_grid *g, int64_t index);

}  // namespace axp

// api.cu -- host side of the C ABI declared in include/axp.h.
//
// Validation, workspace layout in caller-owned device memory, handle state,
// host<->device transfers and checkpointing.  No device memory is allocated
// here: every array lives in the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "axp_internal.h"

using namespace axp;

namespace {

constexpr size_t kAlign = 256;
constexpr uint64_t kStateMagic = 0x32505841u;  // "AXP2"

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t cells(const axp_grid_desc &d) { return d.n[0] * d.n[1] * d.n[2]; }

int64_t plane_size(const axp_grid_desc &d, int a)
{
    return a == 0 ? d.n[1] * d.n[2] : (a == 1 ? d.n[0] * d.n[2] : d.n[0] * d.n[1]);
}

axp_status validate(const axp_grid_desc *d)
{
    if (!d) return AXP_E_INVAL;
    if (d->precision != AXP_FP64 && d->precision != AXP_FP32_SPLIT) return AXP_E_INVAL;
    if (!(d->dt > 0) || !std::isfinite(d->dt) || !std::isfinite(d->m) || !std::isfinite(d->g)) return AXP_E_INVAL;
    if (d->pml_cells < 0 || !(d->pml_sigma_max_dt >= 0)) return AXP_E_INVAL;
    if (d->diag_every < 0 || (d->diag_every > 0 && d->diag_capacity < 1) || d->diag_capacity < 0) return AXP_E_INVAL;
    double inv2 = 0.0;
    for (int a = 0; a < 3; a++) {
        if (d->n[a] < 1 || !(d->d[a] > 0) || !std::isfinite(d->lo[a])) return AXP_E_INVAL;
        for (int s = 0; s < 2; s++) {
            const int ab = d->axion_bc[a][s], eb = d->em_bc[a][s];
            if (ab < AXP_BC_PERIODIC || ab > AXP_BC_PML) return AXP_E_INVAL;
            if (eb != AXP_BC_PERIODIC && eb != AXP_BC_REFLECT && eb != AXP_BC_PML) return AXP_E_INVAL;
            if ((ab == AXP_BC_PERIODIC) != (eb == AXP_BC_PERIODIC)) return AXP_E_INVAL;
            if ((ab == AXP_BC_PML || eb == AXP_BC_PML) && d->pml_cells > d->n[a]) return AXP_E_INVAL;
        }
        if ((d->em_bc[a][0] == AXP_BC_PERIODIC) != (d->em_bc[a][1] == AXP_BC_PERIODIC)) return AXP_E_INVAL;
        if (d->n[a] == 1 && d->em_bc[a][0] != AXP_BC_PERIODIC) return AXP_E_INVAL;
        if (d->n[a] > 1) inv2 += 1.0 / (d->d[a] * d->d[a]);
    }
    if (cells(*d) > ((int64_t)1 << 40)) return AXP_E_INVAL;
    if (inv2 > 0) {
        // Yee: dt <= 1/sqrt(sum 1/d^2); axion leapfrog: dt^2 (sum 4/d^2 + m^2) <= 4
        if (d->dt * std::sqrt(inv2) > 1.0) return AXP_E_UNSTABLE;
        if (d->dt * d->dt * (4.0 * inv2 + d->m * d->m) > 4.0) return AXP_E_UNSTABLE;
    } else if (d->dt * d->dt * d->m * d->m > 4.0) {
        return AXP_E_UNSTABLE;
    }
    return AXP_OK;
}

template <typename T>
void sigma_tables(const axp_grid_desc &d, bool axion, std::vector<T> out[3])
{
    const double smax = d.pml_sigma_max_dt / d.dt;
    const int64_t N = d.pml_cells;
    for (int a = 0; a < 3; a++) {
        out[a].assign(d.n[a], T(0));
        const int32_t *bc = axion ? d.axion_bc[a] : d.em_bc[a];
        if (N <= 0) continue;
        for (int64_t c = 0; c < d.n[a]; c++) {
            double s = 0.0;
            if (bc[0] == AXP_BC_PML && c < N) {
                const double r = 1.0 - (double)c / (double)N;
                s = r * r * r * smax;
            }
            if (bc[1] == AXP_BC_PML && c >= d.n[a] - N) {
                const double r = 1.0 - (double)(d.n[a] - 1 - c) / (double)N;
                const double v = r * r * r * smax;
                if (v > s) s = v;
            }
            out[a][c] = (T)s;
        }
    }
}

// The layer coefficients of off_pml_tab from the FP64 profiles (em: E/B, ax: axion).
template <typename T>
void layer_coefficients(const axp_grid_desc &d, const std::vector<double> em[3], const std::vector<double> ax[3],
                        std::vector<T> out[3])
{
    const double h = d.dt / 2.0, dt = d.dt;
    for (int a = 0; a < 3; a++) {
        const int64_t n = d.n[a];
        out[a].assign(6 * n, T(0));
        for (int64_t c = 0; c < n; c++) {
            const double se = em[a][c], sa = ax[a][c];
            const double A = (1.0 - se * h / 2.0) / (1.0 + se * h / 2.0), B = h / (1.0 + se * h / 2.0);
            out[a][c] = (T)A;                      // one damped half-step: a F + b X
            out[a][n + c] = (T)B;
            out[a][2 * n + c] = (T)(A * A);        // two: a^2 F + b (1 + a) X
            out[a][3 * n + c] = (T)(B * (1.0 + A));
            out[a][4 * n + c] = (T)(dt * dt / (1.0 + sa * dt));
            out[a][5 * n + c] = (T)((1.0 - sa * dt) / (1.0 + sa * dt));
        }
    }
}

template <typename T>
cudaError_t upload_layer_tables(const axp_grid_desc &d, char *ws, const Workspace &w, cudaStream_t stream)
{
    std::vector<double> em64[3], ax64[3];
    sigma_tables<double>(d, false, em64);
    sigma_tables<double>(d, true, ax64);
    std::vector<T> em[3], ax[3], tab[3];
    sigma_tables<T>(d, false, em);
    sigma_tables<T>(d, true, ax);
    layer_coefficients<T>(d, em64, ax64, tab);
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; a++) {
        e = cudaMemcpyAsync(ws + w.off_sig_em[a], em[a].data(), em[a].size() * sizeof(T), cudaMemcpyHostToDevice,
                            stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws + w.off_sig_ax[a], ax[a].data(), ax[a].size() * sizeof(T), cudaMemcpyHostToDevice,
                                stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws + w.off_pml_tab[a], tab[a].data(), tab[a].size() * sizeof(T),
                                cudaMemcpyHostToDevice, stream);
    }
    // the host vectors must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
}

axp_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return AXP_OK;
    fprintf(stderr, "axp: CUDA error %s\n", cudaGetErrorString(e));
    return AXP_E_CUDA;
}

bool finite_diag(const axp_diag &d)
{
    const double v[] = {d.t, d.H_phi, d.H_g0, d.H_g1, d.P_g2a, d.P_a2g, d.W, d.sum_xB1z2, d.sum_B1z2, d.gauss_l2};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

bool is_fp32(const axp_grid *g) { return g->desc.precision == AXP_FP32_SPLIT; }

// A grid-wide wait of the time-blocked 1D kernel that gave up leaves a word in
// the workspace; synchronising calls report it once (AXP_E_TIMEOUT) and clear it.
axp_status latched_status(axp_grid *g)
{
    if (!g->coop_used) return AXP_OK;
    int *flag = (int *)(g->ws + g->layout.off_flag) + 1;
    int v = 0;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (!v) return AXP_OK;
    e = cudaMemset(flag, 0, sizeof(int));
    return e == cudaSuccess ? AXP_E_TIMEOUT : cuda_status(e);
}

struct StateHeader {
    uint64_t magic;
    uint64_t bytes;
    axp_grid_desc desc;
    double B_ext[3], E_ext[3];
    int64_t step;
    int32_t J_valid;
    uint32_t active;
    int32_t phi_active;
    int32_t win_axis;    // moving window (-1: none) and its state
    int32_t win_cells;
    int32_t staggered;   // 1: E arrays hold E^{n+1/2} (the single-pass kernels' state)
    double win_velocity, win_travel;
    int64_t win_start, win_offset;
};

}  // namespace

namespace axp {

size_t elem_size(const axp_grid_desc &d) { return d.precision == AXP_FP32_SPLIT ? 4 : 8; }

bool compute_layout(const axp_grid_desc &d, Workspace *w)
{
    std::memset(w, 0, sizeof(*w));
    const size_t e = elem_size(d);
    const size_t arr = align_up((size_t)cells(d) * e);
    size_t off = 0;
    w->off_flag = off;
    off += kAlign;
    for (int set = 0; set < 2; set++)
        for (int f = 0; f < kFields; f++) {
            w->off_fields[set][f] = off;
            off += arr;
        }
    // FP64 keeps two levels and one spare; 1D grids get a second spare, which the
    // time-blocked 1D kernel uses to double-buffer both levels
    const bool line = d.n[1] == 1 && d.n[2] == 1;
    const int nphi = d.precision == AXP_FP32_SPLIT || line ? 4 : 3;
    for (int p = 0; p < 4; p++) {
        if (p < nphi) {
            w->off_phi[p] = off;
            off += arr;
        }
    }
    for (int a = 0; a < 3; a++) {
        w->off_J[a] = off;
        off += arr;
    }
    for (int a = 0; a < 3; a++) {  // P at cell centres (general path scratch)
        w->off_P[a] = off;
        off += arr;
    }
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++)
            for (int l = 0; l < 3; l++) {
                if (d.axion_bc[a][s] != AXP_BC_OUTFLOW) continue;
                w->off_ghost[a][s][l] = off;
                off += align_up((size_t)plane_size(d, a) * e);
            }
    for (int a = 0; a < 3; a++) {
        w->off_sig_em[a] = off;
        off += align_up((size_t)d.n[a] * e);
        w->off_sig_ax[a] = off;
        off += align_up((size_t)d.n[a] * e);
        w->off_pml_tab[a] = off;
        off += align_up((size_t)6 * d.n[a] * e);
    }
    for (int c = 0; c < 2; c++) {  // soft-source sheet weights of E_y and E_z over the plane
        w->off_src[c] = off;
        off += align_up((size_t)plane_size(d, 0) * e);
    }
    if (d.n[1] > 1 && d.n[2] == 1) {  // work lists of the 2D kernel
        w->off_sched = off;
        off += align_up((size_t)kSchedItems * 16);
    }
    int64_t nb = (cells(d) + 255) / 256;
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    w->diag_blocks = (int)nb;
    w->off_partials = off;
    off += align_up((size_t)nb * 7 * sizeof(double));
    w->off_ring = off;
    off += align_up((size_t)(d.diag_capacity + 1) * sizeof(axp_diag));
    w->total = off;
    w->elem = e;
    return true;
}

axp_diag *ring_slot(axp_grid *g, int64_t index)
{
    const int64_t cap = g->desc.diag_capacity > 0 ? g->desc.diag_capacity : 1;
    return (axp_diag *)(g->ws + g->layout.off_ring) + (index % cap);
}

static axp_diag *scratch_slot(axp_grid *g)
{
    return (axp_diag *)(g->ws + g->layout.off_ring) + g->desc.diag_capacity;
}

template <typename T>
View<T> make_view_eset(axp_grid *g, int eset)
{
    View<T> v;
    std::memset(&v, 0, sizeof(v));
    const axp_grid_desc &d = g->desc;
    const Workspace &w = g->layout;
    for (int f = 0; f < kFields; f++) {
        const bool is_e = (f >= kE0 && f < kE0 + 3) || (f >= kE1 && f < kE1 + 3);
        v.f[f] = (T *)(g->ws + w.off_fields[is_e ? eset : g->fset][f]);
    }
    v.phi_cur = (T *)(g->ws + w.off_phi[g->phi_cur_slot]);
    v.phi_b = (T *)(g->ws + w.off_phi[g->phi_b_slot]);
    v.phi_next = (T *)(g->ws + w.off_phi[g->phi_next_slot]);
    for (int a = 0; a < 3; a++) {
        v.J[a] = (T *)(g->ws + w.off_J[a]);
        for (int s = 0; s < 2; s++)
            for (int l = 0; l < 3; l++) {
                const size_t off = w.off_ghost[a][s][g->ghost_level_slot[l]];
                v.gh[a][s][l] = off ? (T *)(g->ws + off) : nullptr;
            }
        v.sig_em[a] = (const T *)(g->ws + w.off_sig_em[a]);
        v.sig_ax[a] = (const T *)(g->ws + w.off_sig_ax[a]);
        v.n[a] = d.n[a];
        v.d[a] = (T)d.d[a];
        v.lo[a] = (T)lo_of(g, a);
        v.Bext[a] = (T)g->B_ext[a];
        v.Eext[a] = (T)g->E_ext[a];
        v.periodic[a] = d.em_bc[a][0] == AXP_BC_PERIODIC;
        for (int s = 0; s < 2; s++) v.axbc[a][s] = d.axion_bc[a][s];
        int rlo = 0, rhi = (int)d.n[a];
        if (d.n[a] > 1 && !v.periodic[a]) {
            if (d.em_bc[a][0] == AXP_BC_PML || d.axion_bc[a][0] == AXP_BC_PML) rlo = d.pml_cells;
            if (d.em_bc[a][1] == AXP_BC_PML || d.axion_bc[a][1] == AXP_BC_PML) rhi = (int)d.n[a] - d.pml_cells;
        }
        v.region_lo[a] = rlo;
        v.region_hi[a] = rhi;
    }
    v.N = cells(d);
    v.vaxis = -1;
    v.Nv = v.N;
    v.dt = (T)d.dt;
    v.h = (T)(d.dt / 2.0);
    v.g = (T)d.g;
    v.m2 = (T)(d.m * d.m);
    set_reciprocals(v);
    if (g->parts && sizeof(T) == sizeof(double))
        for (int o = 0; o < 2; o++)
            for (int a = 0; a < 3; a++) v.jp[o][a] = (T *)g->parts->j[o][a];
    return v;
}

template <typename T>
View<T> make_view(axp_grid *g)
{
    return make_view_eset<T>(g, g->fset);
}

template View<double> make_view<double>(axp_grid *);
template View<float> make_view<float>(axp_grid *);
template View<double> make_view_eset<double>(axp_grid *, int);
template View<float> make_view_eset<float>(axp_grid *, int);

cudaError_t ensure_integer(axp_grid *g)
{
    if (!g->staggered) return cudaSuccess;
    return g->desc.precision == AXP_FP32_SPLIT ? exit_staggered<float>(g, true) : exit_staggered<double>(g, true);
}

// Which order-0 components can become non-zero: the injected/written ones and
// everything the discrete curls couple them to along the grid's active axes.
uint32_t order0_closure(const axp_grid *g)
{
    uint32_t m = (g->active & 7u) | (((g->active >> kB0) & 7u) << 3);
    bool ax[3];
    for (int a = 0; a < 3; a++) ax[a] = g->desc.n[a] > 1;
    for (int it = 0; it < 6; it++) {
        uint32_t nm = m;
        for (int a = 0; a < 3; a++) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            // (curl E)_a = D_b E_c - D_c E_b feeds B_a; (curl B)_a likewise feeds E_a
            if ((ax[b] && (m >> c & 1)) || (ax[c] && (m >> b & 1))) nm |= 1u << (3 + a);
            if ((ax[b] && (m >> (3 + c) & 1)) || (ax[c] && (m >> (3 + b) & 1))) nm |= 1u << a;
        }
        m = nm;
    }
    return m;
}

}  // namespace axp

namespace axp {

double source_wave(const axp_grid *g, double x, double t)
{
    const axp_source_desc &q = g->src;
    const double dt = g->desc.dt, dx = g->desc.d[0];
    const double w = (2.0 / dt) * std::asin((dt / dx) * std::sin(q.k * dx / 2.0));
    double e = 1.0;
    if (q.duration > 0) {
        const double L = q.duration / std::sqrt(2.0 * std::log(2.0));
        const double u = (t - q.t_centre) - (x - q.centre[0]);
        e = std::exp(-(u * u) / (L * L));
    }
    return e * std::cos(q.k * (x - q.centre[0]) - w * (t - q.t_centre) + q.phase);
}

}  // namespace axp

namespace {

// Sheet weights A pol_a f / dx of E_y (c = 0) and E_z (c = 1) over the (j, k) of
// the plane, f the transverse Gaussian at each component's own position; zero
// where the cells next to the sheet lie in a transverse absorbing layer.
template <typename T>
cudaError_t upload_source_weights(axp_grid *g)
{
    const axp_grid_desc &d = g->desc;
    const axp_source_desc &q = g->src;
    std::vector<double> em[3];
    sigma_tables<double>(d, false, em);
    const int64_t ny = d.n[1], nz = d.n[2];
    std::vector<T> w[2];
    for (int c = 0; c < 2; c++) {
        const int a = c + 1;
        w[c].assign(ny * nz, T(0));
        for (int64_t k = 0; k < nz; k++)
            for (int64_t j = 0; j < ny; j++) {
                if (em[1][j] != 0.0 || em[2][k] != 0.0) continue;
                double f = 1.0;
                if (q.waist > 0) {
                    // position of E_a: + d/2 along the other axes, + d along its own
                    const double y = lo_of(g, 1) + ((double)j + (a == 1 ? 1.0 : 0.5)) * d.d[1];
                    const double z = lo_of(g, 2) + ((double)k + (a == 2 ? 1.0 : 0.5)) * d.d[2];
                    double r2 = 0.0;
                    if (ny > 1) r2 = r2 + (y - q.centre[1]) * (y - q.centre[1]);
                    if (nz > 1) r2 = r2 + (z - q.centre[2]) * (z - q.centre[2]);
                    f = std::exp(-r2 / (q.waist * q.waist));
                }
                w[c][j + ny * k] = (T)(((q.amplitude * q.pol[a]) * f) / d.d[0]);
            }
    }
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 2 && e == cudaSuccess; c++)
        e = cudaMemcpyAsync(g->ws + g->layout.off_src[c], w[c].data(), w[c].size() * sizeof(T),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);  // the host vectors must outlive the copies
    return e;
}

}  // namespace

extern "C" {

const char *axp_status_str(axp_status s)
{
    switch (s) {
    case AXP_OK: return "ok";
    case AXP_E_INVAL: return "invalid argument";
    case AXP_E_UNSTABLE: return "time step violates the stability bound";
    case AXP_E_NOMEM: return "not enough memory";
    case AXP_E_CUDA: return "CUDA error";
    case AXP_E_TIMEOUT: return "bounded device wait expired";
    case AXP_E_NONFINITE: return "non-finite diagnostic";
    case AXP_E_STATE: return "call not valid in this state";
    }
    return "unknown status";
}

axp_status axp_workspace_bytes(const axp_grid_desc *desc, size_t *bytes)
{
    if (!bytes) return AXP_E_INVAL;
    const axp_status st = validate(desc);
    if (st != AXP_OK) return st;
    Workspace w;
    compute_layout(*desc, &w);
    *bytes = w.total;
    return AXP_OK;
}

axp_status axp_create_grid(const axp_grid_desc *desc, void *dev_workspace, size_t bytes, void *cuda_stream,
                           axp_grid **out)
{
    axp::TraceRange trace_("axp_create_grid");
    if (!out || !dev_workspace) return AXP_E_INVAL;
    *out = nullptr;
    axp_status st = validate(desc);
    if (st != AXP_OK) return st;
    if ((uintptr_t)dev_workspace % kAlign) return AXP_E_INVAL;
    Workspace w;
    compute_layout(*desc, &w);
    if (bytes < w.total) return AXP_E_NOMEM;
    axp_grid *g = new (std::nothrow) axp_grid();
    if (!g) return AXP_E_NOMEM;
    g->desc = *desc;
    g->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return AXP_E_CUDA;
    }
    g->ws = (char *)dev_workspace;
    g->ws_bytes = bytes;
    g->layout = w;
    g->phi_cur_slot = 0;
    g->phi_b_slot = 1;
    g->phi_next_slot = 2;
    g->phi_next_b_slot = 3;
    g->fset = 0;
    g->staggered = false;
    for (int l = 0; l < 3; l++) g->ghost_level_slot[l] = l;
    g->J_valid = false;
    g->kernel_choice = AXP_KERNEL_AUTO;
    g->win_axis = -1;
    g->coop_absent = -1;
    g->tm_plan_key = -1;
    cudaError_t e = cudaMemsetAsync(g->ws, 0, w.total, g->stream);
    if (e == cudaSuccess) {
        // absorbing-layer profiles and coefficients, computed once on the host
        e = desc->precision == AXP_FP32_SPLIT ? upload_layer_tables<float>(*desc, g->ws, w, g->stream)
                                              : upload_layer_tables<double>(*desc, g->ws, w, g->stream);
    }
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e);
    }
    *out = g;
    return AXP_OK;
}

axp_status axp_destroy_grid(axp_grid *grid)
{
    if (!grid) return AXP_E_INVAL;
    if (grid->group) return AXP_E_STATE;
    release_step_graphs(grid, true);
    delete grid->parts;
    delete grid;
    return AXP_OK;
}

axp_status axp_set_background_field(axp_grid *g, const double B_ext[3], const double E_ext[3])
{
    if (!g) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    g->cfg_version++;
    for (int a = 0; a < 3; a++) {
        if (B_ext && !std::isfinite(B_ext[a])) return AXP_E_INVAL;
        if (E_ext && !std::isfinite(E_ext[a])) return AXP_E_INVAL;
    }
    const cudaError_t e = ensure_integer(g);
    if (e != cudaSuccess) return cuda_status(e);
    for (int a = 0; a < 3; a++) {
        if (B_ext) g->B_ext[a] = B_ext[a];
        if (E_ext) g->E_ext[a] = E_ext[a];
    }
    g->J_valid = false;
    return AXP_OK;
}

axp_status axp_inject_laser(axp_grid *g, const axp_laser_desc *L)
{
    axp::TraceRange trace_("axp_inject_laser");
    if (!g || !L) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    g->cfg_version++;
    double kk = 0;
    for (int a = 0; a < 3; a++) {
        if (!std::isfinite(L->k[a]) || !std::isfinite(L->pol[a]) || !std::isfinite(L->centre[a])) return AXP_E_INVAL;
        kk += L->k[a] * L->k[a];
    }
    if (!(kk > 0) || !std::isfinite(L->amplitude) || L->waist < 0 || L->duration < 0) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = is_fp32(g) ? inject_laser<float>(g, *L) : inject_laser<double>(g, *L);
    g->J_valid = false;
    for (int a = 0; a < 3; a++) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        if (L->pol[a] != 0) g->active |= 1u << (kE0 + a);
        // B = curl(pol F): B_a = D_b F_c - D_c F_b along the grid's active axes
        if ((g->desc.n[b] > 1 && L->pol[c] != 0) || (g->desc.n[c] > 1 && L->pol[b] != 0)) g->active |= 1u << (kB0 + a);
    }
    return cuda_status(e);
}


axp_status axp_set_soft_source(axp_grid *g, const axp_source_desc *q)
{
    if (!g) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (q) {
        const axp_grid_desc &d = g->desc;
        bool ok = std::isfinite(q->amplitude) && std::isfinite(q->k) && q->k > 0 && std::isfinite(q->t_centre) &&
                  std::isfinite(q->phase) && std::isfinite(q->waist) && q->waist >= 0 &&
                  std::isfinite(q->duration) && q->duration >= 0 && q->pol[0] == 0.0;
        for (int a = 0; a < 3; a++) ok = ok && std::isfinite(q->pol[a]) && std::isfinite(q->centre[a]);
        ok = ok && d.n[0] >= 2 && q->plane >= 1 && q->plane <= d.n[0] - 1;
        if (ok) {
            // both cells next to the sheet outside the x absorbing layers
            const int64_t N = d.pml_cells;
            const bool lo_abs = d.em_bc[0][0] == AXP_BC_PML || d.axion_bc[0][0] == AXP_BC_PML;
            const bool hi_abs = d.em_bc[0][1] == AXP_BC_PML || d.axion_bc[0][1] == AXP_BC_PML;
            if (lo_abs && q->plane - 1 < N) ok = false;
            if (hi_abs && q->plane > d.n[0] - 1 - N) ok = false;
        }
        if (!ok) return AXP_E_INVAL;
    }
    g->cfg_version++;
    // the staggered state was formed with the old source: return to integer time first
    cudaError_t e = ensure_integer(g);
    if (e != cudaSuccess) return cuda_status(e);
    if (!q) {
        g->src_on = false;
        return AXP_OK;
    }
    g->src = *q;
    g->src_on = true;
    e = is_fp32(g) ? upload_source_weights<float>(g) : upload_source_weights<double>(g);
    if (e != cudaSuccess) {
        g->src_on = false;
        return cuda_status(e);
    }
    // the sheets drive E_y/B_z (pol_y) and E_z/B_y (pol_z)
    if (q->pol[1] != 0) g->active |= (1u << (kE0 + 1)) | (1u << (kB0 + 2));
    if (q->pol[2] != 0) g->active |= (1u << (kE0 + 2)) | (1u << (kB0 + 1));
    g->J_valid = false;
    return AXP_OK;
}

axp_status axp_inject_axion(axp_grid *g, const axp_axion_desc *A)
{
    axp::TraceRange trace_("axp_inject_axion");
    if (!g || !A) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    g->cfg_version++;
    for (int a = 0; a < 3; a++)
        if (!std::isfinite(A->k[a]) || !std::isfinite(A->centre[a])) return AXP_E_INVAL;
    if (!std::isfinite(A->amplitude) || A->waist < 0 || A->length < 0) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = is_fp32(g) ? inject_axion<float>(g, *A) : inject_axion<double>(g, *A);
    g->J_valid = false;
    g->phi_active = true;
    return cuda_status(e);
}

static axp_status run_steps(axp_grid *g, int64_t nsteps)
{
    cudaError_t e;
    bool handled = false;
    if (g->kernel_choice != AXP_KERNEL_GENERAL) {
        e = is_fp32(g) ? fused_step<float>(g, nsteps, &handled) : fused_step<double>(g, nsteps, &handled);
        if (e != cudaSuccess) return cuda_status(e);
        if (!handled && g->kernel_choice != AXP_KERNEL_AUTO) return AXP_E_STATE;
    }
    if (!handled) {
        e = ensure_integer(g);
        if (e == cudaSuccess) e = is_fp32(g) ? general_step<float>(g, nsteps) : general_step<double>(g, nsteps);
    } else {
        e = cudaSuccess;
    }
    return cuda_status(e);
}

// Shift the window by `cells` along `axis`: the integer-time state moves towards
// lower index and vacuum enters at the high end.
static axp_status shift_now(axp_grid *g, int axis, int64_t cells)
{
    bool done = false;
    cudaError_t e = is_fp32(g) ? shift_staggered<float>(g, axis, cells, &done)
                               : shift_staggered<double>(g, axis, cells, &done);
    if (e == cudaSuccess && !done) {
        e = ensure_integer(g);
        if (e == cudaSuccess) e = is_fp32(g) ? shift_window<float>(g, axis, cells) : shift_window<double>(g, axis, cells);
    }
    if (e != cudaSuccess) return cuda_status(e);
    if (g->win_axis < 0) g->win_axis = axis;
    g->win_offset += cells;
    g->cfg_version++;
    return AXP_OK;
}

static bool window_axis_ok(const axp_grid *g, int32_t axis)
{
    if (axis < 0 || axis > 2 || g->desc.n[axis] < 2) return false;
    if (g->desc.em_bc[axis][0] == AXP_BC_PERIODIC) return false;
    if (g->win_axis >= 0 && g->win_axis != axis) return false;  // one window axis per grid
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++)
            if (g->desc.axion_bc[a][s] == AXP_BC_OUTFLOW) return false;  // ghost planes do not move
    return true;
}

axp_status axp_step(axp_grid *g, int64_t nsteps)
{
    axp::TraceRange trace_("axp_step");
    if (!g || nsteps < 0) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (nsteps == 0) return AXP_OK;
    if (g->win_velocity <= 0.0) return run_steps(g, nsteps);
    // moving window: run up to each shift, then shift by win_cells
    const int a = g->win_axis;
    const double u = g->win_velocity * g->desc.dt / g->desc.d[a];  // cells per step
    int64_t left = nsteps;
    while (left > 0) {
        int64_t k = left;
        if (g->step < g->win_start) {
            k = std::min<int64_t>(left, g->win_start - g->step);
        } else {
            const double need = (double)g->win_cells - g->win_travel;
            k = std::min<int64_t>(left, std::max<int64_t>(1, (int64_t)std::ceil(need / u - 1e-9)));
        }
        const int64_t s0 = g->step;
        axp_status st = run_steps(g, k);
        if (st != AXP_OK) return st;
        left -= k;
        const int64_t moving = g->step - std::max(s0, g->win_start);
        if (moving > 0) g->win_travel += (double)moving * u;
        if (g->win_travel >= (double)g->win_cells - 1e-9) {
            if ((st = shift_now(g, a, g->win_cells)) != AXP_OK) return st;
            g->win_travel -= (double)g->win_cells;
        }
    }
    return AXP_OK;
}

axp_status axp_shift_window(axp_grid *g, int32_t axis, int64_t cells)
{
    if (!g || cells < 0) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (!window_axis_ok(g, axis) || cells >= g->desc.n[axis]) return AXP_E_INVAL;
    if (cells == 0) return AXP_OK;
    return shift_now(g, axis, cells);
}

axp_status axp_set_moving_window(axp_grid *g, int32_t axis, double velocity, int32_t shift_cells, int64_t start_step)
{
    if (!g) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (velocity == 0.0) {
        g->win_velocity = 0.0;
        return AXP_OK;
    }
    if (!window_axis_ok(g, axis) || !(velocity > 0.0) || velocity > 1.0 || shift_cells < 1 ||
        shift_cells >= g->desc.n[axis] || start_step < 0)
        return AXP_E_INVAL;
    g->win_axis = axis;
    g->win_velocity = velocity;
    g->win_cells = shift_cells;
    g->win_start = start_step;
    g->win_travel = 0.0;
    return AXP_OK;
}

axp_status axp_get_window_offset(const axp_grid *g, int64_t *cells)
{
    if (!g || !cells) return AXP_E_INVAL;
    *cells = g->win_offset;
    return AXP_OK;
}

axp_status axp_synchronize(axp_grid *g)
{
    if (!g) return AXP_E_INVAL;
    const axp_status st = cuda_status(cudaStreamSynchronize(g->stream));
    return st != AXP_OK ? st : latched_status(g);
}

axp_status axp_read_diagnostics(axp_grid *g, axp_diag *out, int64_t max, int64_t *n)
{
    axp::TraceRange trace_("axp_read_diagnostics");
    if (!g || !n || max < 0 || (max > 0 && !out)) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    *n = 0;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const axp_status lat = latched_status(g);
    if (lat != AXP_OK) return lat;
    const int64_t cap = g->desc.diag_capacity;
    if (cap <= 0) return AXP_OK;
    if (g->ring_written - g->ring_read > cap) g->ring_read = g->ring_written - cap;
    int64_t cnt = g->ring_written - g->ring_read;
    if (cnt > max) cnt = max;
    bool finite = true;
    for (int64_t r = 0; r < cnt; r++) {
        e = cudaMemcpy(out + r, ring_slot(g, g->ring_read + r), sizeof(axp_diag), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
        finite = finite && finite_diag(out[r]);
    }
    g->ring_read += cnt;
    *n = cnt;
    return finite ? AXP_OK : AXP_E_NONFINITE;
}

axp_status axp_compute_diagnostics(axp_grid *g, axp_diag *out)
{
    axp::TraceRange trace_("axp_compute_diagnostics");
    if (!g || !out) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    axp_diag *dst = scratch_slot(g);
    cudaError_t e = is_fp32(g) ? diag_compute<float>(g, dst) : diag_compute<double>(g, dst);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dst, sizeof(axp_diag), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const axp_status lat = latched_status(g);
    if (lat != AXP_OK) return lat;
    return finite_diag(*out) ? AXP_OK : AXP_E_NONFINITE;
}

static void *field_ptr(axp_grid *g, int which)
{
    if (which >= 0 && which < kFields) return g->ws + g->layout.off_fields[g->fset][which];
    if (which == AXP_PHI_CUR) return g->ws + g->layout.off_phi[g->phi_cur_slot];
    return g->ws + g->layout.off_phi[g->phi_b_slot];
}

axp_status axp_read_field(axp_grid *g, int32_t which, double *dst, size_t bytes)
{
    if (!g || !dst || which < 0 || which > AXP_PHI_OLD) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    const int64_t N = cells(g->desc);
    if (bytes != (size_t)N * 8) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const axp_status lat = latched_status(g);
    if (lat != AXP_OK) return lat;
    if (!is_fp32(g)) return cuda_status(cudaMemcpy(dst, field_ptr(g, which), bytes, cudaMemcpyDeviceToHost));
    std::vector<float> tmp(N), inc;
    e = cudaMemcpy(tmp.data(), field_ptr(g, which == AXP_PHI_OLD ? AXP_PHI_CUR : which), N * 4,
                   cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && which == AXP_PHI_OLD) {
        inc.resize(N);
        e = cudaMemcpy(inc.data(), g->ws + g->layout.off_phi[g->phi_b_slot], N * 4, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_status(e);
    for (int64_t c = 0; c < N; c++) dst[c] = which == AXP_PHI_OLD ? (double)tmp[c] - (double)inc[c] : (double)tmp[c];
    return AXP_OK;
}

axp_status axp_write_field(axp_grid *g, int32_t which, const double *src, size_t bytes)
{
    if (!g || !src || which < 0 || which > AXP_PHI_OLD) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    g->cfg_version++;
    const int64_t N = cells(g->desc);
    if (bytes != (size_t)N * 8) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    g->J_valid = false;
    bool nonzero = false;
    for (int64_t c = 0; c < N && !nonzero; c++) nonzero = src[c] != 0.0;
    if (nonzero) {
        if (which < kFields) g->active |= 1u << which;
        else g->phi_active = true;
    }
    if (!is_fp32(g)) return cuda_status(cudaMemcpy(field_ptr(g, which), src, bytes, cudaMemcpyHostToDevice));
    std::vector<float> tmp(N);
    if (which < kFields) {
        for (int64_t c = 0; c < N; c++) tmp[c] = (float)src[c];
        return cuda_status(cudaMemcpy(field_ptr(g, which), tmp.data(), N * 4, cudaMemcpyHostToDevice));
    }
    // increment storage: keep the other level, recompute pi = phi_cur - phi_old
    std::vector<double> cur(N), old(N);
    axp_status st = axp_read_field(g, AXP_PHI_CUR, cur.data(), N * 8);
    if (st == AXP_OK) st = axp_read_field(g, AXP_PHI_OLD, old.data(), N * 8);
    if (st != AXP_OK) return st;
    if (which == AXP_PHI_CUR) cur.assign(src, src + N);
    else old.assign(src, src + N);
    std::vector<float> inc(N);
    for (int64_t c = 0; c < N; c++) {
        tmp[c] = (float)cur[c];
        inc[c] = (float)(cur[c] - old[c]);
    }
    e = cudaMemcpy(g->ws + g->layout.off_phi[g->phi_cur_slot], tmp.data(), N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->ws + g->layout.off_phi[g->phi_b_slot], inc.data(), N * 4, cudaMemcpyHostToDevice);
    return cuda_status(e);
}

static axp_status ghost_io(axp_grid *g, int32_t axis, int32_t side, int32_t level, double *dst, const double *src,
                           size_t bytes)
{
    if (!g || axis < 0 || axis > 2 || side < 0 || side > 1 || level < 0 || level > 1) return AXP_E_INVAL;
    if (g->desc.axion_bc[axis][side] != AXP_BC_OUTFLOW) return AXP_E_INVAL;
    const int64_t P = plane_size(g->desc, axis);
    if (bytes != (size_t)P * 8) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    char *dev = g->ws + g->layout.off_ghost[axis][side][g->ghost_level_slot[level]];
    if (!is_fp32(g)) {
        if (dst) return cuda_status(cudaMemcpy(dst, dev, bytes, cudaMemcpyDeviceToHost));
        g->J_valid = false;
        return cuda_status(cudaMemcpy(dev, src, bytes, cudaMemcpyHostToDevice));
    }
    std::vector<float> tmp(P);
    if (dst) {
        e = cudaMemcpy(tmp.data(), dev, P * 4, cudaMemcpyDeviceToHost);
        for (int64_t c = 0; c < P; c++) dst[c] = tmp[c];
        return cuda_status(e);
    }
    for (int64_t c = 0; c < P; c++) tmp[c] = (float)src[c];
    g->J_valid = false;
    return cuda_status(cudaMemcpy(dev, tmp.data(), P * 4, cudaMemcpyHostToDevice));
}

// ---- macroparticles (Sec. 2.2) ----

axp_status axp_particles_bytes(const axp_grid *g, int64_t count, size_t *bytes)
{
    if (!g || !bytes || count < 0) return AXP_E_INVAL;
    *bytes = particles_bytes(g->desc, count);
    return AXP_OK;
}

axp_status axp_attach_particles(axp_grid *g, int64_t count, double q, double m, void *ws, size_t bytes)
{
    axp::TraceRange trace_("axp_attach_particles");
    if (!g || !ws || count < 0 || !std::isfinite(q) || !std::isfinite(m) || !(m > 0.0)) return AXP_E_INVAL;
    if (g->group || g->parts) return AXP_E_STATE;
    if (is_fp32(g) || (uintptr_t)ws % kAlign) return AXP_E_INVAL;
    for (int a = 0; a < 3; a++)
        if (g->desc.n[a] > 1 && (g->desc.em_bc[a][0] != AXP_BC_PERIODIC || g->desc.em_bc[a][1] != AXP_BC_PERIODIC))
            return AXP_E_INVAL;
    const size_t need = particles_bytes(g->desc, count);
    if (bytes < need) return AXP_E_NOMEM;
    cudaError_t e = ensure_integer(g);
    if (e != cudaSuccess) return cuda_status(e);
    Particles *P = new (std::nothrow) Particles();
    if (!P) return AXP_E_NOMEM;
    P->count = count;
    P->q = q;
    P->m = m;
    P->ws = (char *)ws;
    P->bytes = bytes;
    particles_layout(g->desc, P);
    e = cudaMemsetAsync(ws, 0, need, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        delete P;
        return cuda_status(e);
    }
    g->parts = P;
    g->active = (1u << kFields) - 1;  // the currents can drive every component
    g->cfg_version++;
    return AXP_OK;
}

axp_status axp_detach_particles(axp_grid *g)
{
    if (!g) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (!g->parts) return AXP_OK;
    const cudaError_t e = cudaStreamSynchronize(g->stream);
    delete g->parts;
    g->parts = nullptr;
    g->cfg_version++;
    return cuda_status(e);
}

// rows of the host image: w, x0 xyz, u0 xyz, x1 xyz, u1 xyz
static double *particle_row(Particles *P, int r)
{
    if (r == 0) return P->w;
    if (r < 4) return P->x0[r - 1];
    if (r < 7) return P->u0[r - 4];
    if (r < 10) return P->x1[r - 7];
    return P->u1[r - 10];
}

axp_status axp_write_particles(axp_grid *g, const double *src, size_t bytes)
{
    axp::TraceRange trace_("axp_write_particles");
    if (!g || !src) return AXP_E_INVAL;
    if (g->group || !g->parts) return AXP_E_STATE;
    Particles *P = g->parts;
    if (bytes != (size_t)P->count * 13 * sizeof(double)) return AXP_E_INVAL;
    for (int64_t i = 0; i < P->count * 13; i++)
        if (!std::isfinite(src[i])) return AXP_E_NONFINITE;
    cudaError_t e = ensure_integer(g);
    for (int r = 0; r < 13 && e == cudaSuccess && P->count > 0; r++)
        e = cudaMemcpyAsync(particle_row(P, r), src + (size_t)r * P->count, (size_t)P->count * sizeof(double),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = particles_start(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    g->cfg_version++;
    return cuda_status(e);
}

axp_status axp_read_particles(axp_grid *g, double *dst, size_t bytes)
{
    if (!g || !dst) return AXP_E_INVAL;
    if (g->group || !g->parts) return AXP_E_STATE;
    Particles *P = g->parts;
    if (bytes != (size_t)P->count * 13 * sizeof(double)) return AXP_E_INVAL;
    cudaError_t e = ensure_integer(g);
    if (e == cudaSuccess) e = particles_now(g);
    for (int r = 0; r < 13 && e == cudaSuccess && P->count > 0; r++) {
        const double *from = particle_row(P, r);
        if (r >= 1 && r < 4) from = P->scratch[r - 1];
        if (r >= 7 && r < 10) from = P->scratch[3 + r - 7];
        e = cudaMemcpyAsync(dst + (size_t)r * P->count, from, (size_t)P->count * sizeof(double), cudaMemcpyDeviceToHost,
                            g->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    return cuda_status(e);
}

axp_status axp_read_particle_current(axp_grid *g, int32_t order, double *dst, size_t bytes)
{
    if (!g || !dst || order < 0 || order > 1) return AXP_E_INVAL;
    if (!g->parts) return AXP_E_STATE;
    const int64_t N = cells(g->desc);
    if (bytes != (size_t)N * 3 * sizeof(double)) return AXP_E_INVAL;
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; a++)
        e = cudaMemcpyAsync(dst + (size_t)a * N, g->parts->j[order][a], (size_t)N * sizeof(double),
                            cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    return cuda_status(e);
}

axp_status axp_read_ghost(axp_grid *g, int32_t axis, int32_t side, int32_t level, double *dst, size_t bytes)
{
    if (!dst) return AXP_E_INVAL;
    if (g && g->group) return AXP_E_STATE;
    return ghost_io(g, axis, side, level, dst, nullptr, bytes);
}

axp_status axp_write_ghost(axp_grid *g, int32_t axis, int32_t side, int32_t level, const double *src, size_t bytes)
{
    if (!src) return AXP_E_INVAL;
    if (g && g->group) return AXP_E_STATE;
    if (g) g->cfg_version++;
    return ghost_io(g, axis, side, level, nullptr, src, bytes);
}

// Checkpoint image: header, then the state packed by role -- the field arrays
// that can be non-zero (the order-0 components in the closure of the injected
// ones, every order-1 component), phi^{n+1/2}, the second axion level and the
// outflow ghost planes of levels n+1/2 and n-1/2.  The other order-0 arrays are
// zero by construction and the cached current J is a function of the stored
// state, so neither is stored: a load zeroes the first and marks J for
// recomputation.  A grid that the single-pass kernels are stepping holds E at
// n+1/2 (the leapfrog-staggered state); its image keeps that form (flagged in
// the header), so a save and a load convert nothing and a resumed run is bit
// for bit the uninterrupted one.  With a soft source the staggered E carries the
// source's sheet terms, so such a grid saves its integer-time state instead.
static uint32_t stored_fields(const axp_grid *g)
{
    const uint32_t c0 = order0_closure(g);
    return (c0 & 7u) | (((c0 >> 3) & 7u) << kB0) | (0x3Fu << kE1);
}

static void state_regions(axp_grid *g, uint32_t fields, std::vector<std::pair<char *, size_t>> *out)
{
    const size_t arr = (size_t)cells(g->desc) * g->layout.elem;
    for (int f = 0; f < kFields; f++)
        if (fields >> f & 1u) out->push_back({g->ws + g->layout.off_fields[g->fset][f], arr});
    out->push_back({g->ws + g->layout.off_phi[g->phi_cur_slot], arr});
    out->push_back({g->ws + g->layout.off_phi[g->phi_b_slot], arr});
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++)
            for (int l = 0; l < 2; l++) {
                const size_t off = g->layout.off_ghost[a][sd][g->ghost_level_slot[l]];
                if (off) out->push_back({g->ws + off, (size_t)plane_size(g->desc, a) * g->layout.elem});
            }
}

static size_t image_bytes(axp_grid *g, uint32_t fields)
{
    std::vector<std::pair<char *, size_t>> r;
    state_regions(g, fields, &r);
    size_t total = sizeof(StateHeader);
    for (auto &x : r) total += x.second;
    return total;
}

axp_status axp_state_bytes(const axp_grid *g, size_t *bytes)
{
    if (!g || !bytes) return AXP_E_INVAL;
    axp_grid *gm = const_cast<axp_grid *>(g);
    *bytes = image_bytes(gm, stored_fields(gm));
    return AXP_OK;
}

axp_status axp_save_state(axp_grid *g, void *dst, size_t bytes)
{
    axp::TraceRange trace_("axp_save_state");
    size_t need;
    if (!g || !dst || axp_state_bytes(g, &need) != AXP_OK || bytes != need) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    cudaError_t e = g->src_on ? ensure_integer(g) : cudaSuccess;
    if (e != cudaSuccess) return cuda_status(e);
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kStateMagic;
    h.staggered = g->staggered ? 1 : 0;
    h.bytes = need;
    h.desc = g->desc;
    for (int a = 0; a < 3; a++) {
        h.B_ext[a] = g->B_ext[a];
        h.E_ext[a] = g->E_ext[a];
    }
    h.step = g->step;
    h.J_valid = 0;
    h.active = g->active;
    h.phi_active = g->phi_active;
    h.win_axis = g->win_axis;
    h.win_cells = g->win_cells;
    h.win_velocity = g->win_velocity;
    h.win_travel = g->win_travel;
    h.win_start = g->win_start;
    h.win_offset = g->win_offset;
    std::memcpy(dst, &h, sizeof(h));
    std::vector<std::pair<char *, size_t>> r;
    state_regions(g, stored_fields(g), &r);
    char *p = (char *)dst + sizeof(h);
    for (auto &x : r) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, x.first, x.second, cudaMemcpyDeviceToHost, g->stream);
        p += x.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return latched_status(g);
}

axp_status axp_load_state(axp_grid *g, const void *src, size_t bytes)
{
    axp::TraceRange trace_("axp_load_state");
    if (!g || !src || bytes < sizeof(StateHeader)) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    StateHeader h;
    std::memcpy(&h, src, sizeof(h));
    if (h.magic != kStateMagic || h.bytes != bytes || std::memcmp(&h.desc, &g->desc, sizeof(axp_grid_desc)) != 0)
        return AXP_E_INVAL;
    if (h.staggered && g->src_on) return AXP_E_STATE;  // (its staggered E carries no sheet terms)
    // the image's array set follows from its own record of the injected components
    const uint32_t active_before = g->active;
    g->active = h.active;
    const uint32_t fields = stored_fields(g);
    if (image_bytes(g, fields) != bytes) {
        g->active = active_before;
        return AXP_E_INVAL;
    }
    g->cfg_version++;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    g->staggered = h.staggered != 0;
    g->half_prev = false;
    // arrays outside the image are zero in both field sets (kernels never touch them)
    const size_t arr = (size_t)cells(g->desc) * g->layout.elem;
    for (int set = 0; set < 2 && e == cudaSuccess; set++)
        for (int f = 0; f < kFields && e == cudaSuccess; f++)
            if (!(fields >> f & 1u)) e = cudaMemsetAsync(g->ws + g->layout.off_fields[set][f], 0, arr, g->stream);
    std::vector<std::pair<char *, size_t>> r;
    state_regions(g, fields, &r);
    const char *p = (const char *)src + sizeof(h);
    for (auto &x : r) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(x.first, p, x.second, cudaMemcpyHostToDevice, g->stream);
        p += x.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int a = 0; a < 3; a++) {
        g->B_ext[a] = h.B_ext[a];
        g->E_ext[a] = h.E_ext[a];
    }
    g->step = h.step;
    g->J_valid = false;  // recomputed from the loaded state when a step needs it
    g->phi_active = h.phi_active != 0;
    g->win_axis = h.win_axis;
    g->win_cells = h.win_cells;
    g->win_velocity = h.win_velocity;
    g->win_travel = h.win_travel;
    g->win_start = h.win_start;
    g->win_offset = h.win_offset;
    g->ring_read = g->ring_written;
    return AXP_OK;
}

axp_status axp_get_step(const axp_grid *g, int64_t *step)
{
    if (!g || !step) return AXP_E_INVAL;
    *step = g->step;
    return AXP_OK;
}

axp_status axp_set_kernel(axp_grid *g, int32_t kernel)
{
    if (!g || kernel < AXP_KERNEL_AUTO || kernel > AXP_KERNEL_TM2D_LIST) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    g->cfg_version++;
    g->kernel_choice = kernel;
    return AXP_OK;
}

axp_status axp_get_kernel_path(axp_grid *g, int32_t *path)
{
    if (!g || !path) return AXP_E_INVAL;
    *path = is_fp32(g) ? fused_path<float>(g) : fused_path<double>(g);
    return AXP_OK;
}

// ---- slab decomposition: rows of the present state along the slowest axis ----

static int rows_axis(const axp_grid_desc &d) { return d.n[2] > 1 ? 2 : (d.n[1] > 1 ? 1 : 0); }

static int64_t row_cells(const axp_grid_desc &d)
{
    const int a = rows_axis(d);
    int64_t r = 1;
    for (int b = 0; b < a; b++) r *= d.n[b];
    return r;
}

// the 14 arrays of the present state in a fixed order: fields, phi^{n+1/2}, second level
static void state_arrays(axp_grid *g, char *out[kFields + 2])
{
    for (int f = 0; f < kFields; f++) out[f] = g->ws + g->layout.off_fields[g->fset][f];
    out[kFields] = g->ws + g->layout.off_phi[g->phi_cur_slot];
    out[kFields + 1] = g->ws + g->layout.off_phi[g->phi_b_slot];
}

axp_status axp_rows_bytes(const axp_grid *g, int64_t nrows, size_t *bytes)
{
    if (!g || !bytes || nrows < 0) return AXP_E_INVAL;
    *bytes = (size_t)(kFields + 2) * (size_t)nrows * (size_t)row_cells(g->desc) * g->layout.elem;
    return AXP_OK;
}

static axp_status rows_copy(axp_grid *g, int64_t row0, int64_t nrows, char *dev, size_t bytes, bool pack)
{
    size_t need;
    if (!g || !dev || axp_rows_bytes(g, nrows, &need) != AXP_OK || bytes != need) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    const int a = rows_axis(g->desc);
    if (row0 < 0 || row0 + nrows > g->desc.n[a]) return AXP_E_INVAL;
    const size_t chunk = (size_t)nrows * (size_t)row_cells(g->desc) * g->layout.elem;
    const size_t off = (size_t)row0 * (size_t)row_cells(g->desc) * g->layout.elem;
    char *arr[kFields + 2];
    state_arrays(g, arr);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < kFields + 2 && e == cudaSuccess; q++)
        e = pack ? cudaMemcpyAsync(dev + q * chunk, arr[q] + off, chunk, cudaMemcpyDeviceToDevice, g->stream)
                 : cudaMemcpyAsync(arr[q] + off, dev + q * chunk, chunk, cudaMemcpyDeviceToDevice, g->stream);
    if (!pack) {
        g->J_valid = false;
        g->cfg_version++;
    }
    return cuda_status(e);
}

axp_status axp_pack_rows(axp_grid *g, int64_t row0, int64_t nrows, void *dev_dst, size_t bytes)
{
    if (g && g->parts) return AXP_E_STATE;  // particles do not move between slabs
    return rows_copy(g, row0, nrows, (char *)dev_dst, bytes, true);
}

axp_status axp_unpack_rows(axp_grid *g, int64_t row0, int64_t nrows, const void *dev_src, size_t bytes)
{
    if (g && g->parts) return AXP_E_STATE;
    return rows_copy(g, row0, nrows, (char *)const_cast<void *>(dev_src), bytes, false);
}

axp_status axp_compute_diagnostics_rows(axp_grid *g, int64_t row0, int64_t row1, axp_diag *out)
{
    axp::TraceRange trace_("axp_compute_diagnostics_rows");
    if (!g || !out || row0 < 0 || row1 < row0) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    const int a = rows_axis(g->desc);
    if (row1 > g->desc.n[a]) return AXP_E_INVAL;
    axp_diag *dst = scratch_slot(g);
    cudaError_t e = is_fp32(g) ? diag_compute_rows<float>(g, dst, a, row0, row1)
                               : diag_compute_rows<double>(g, dst, a, row0, row1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dst, sizeof(axp_diag), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const axp_status lat = latched_status(g);
    if (lat != AXP_OK) return lat;
    return finite_diag(*out) ? AXP_OK : AXP_E_NONFINITE;
}

axp_status axp_test_block1d_absent(axp_grid *g, int32_t block)
{
    if (!g || block < -1) return AXP_E_INVAL;
    g->coop_absent = block;
    return AXP_OK;
}

axp_status axp_get_launch_count(const axp_grid *g, int64_t *count)
{
    if (!g || !count) return AXP_E_INVAL;
    *count = g->launches;
    return AXP_OK;
}

}  // extern "C"

// kernels_fused.cu -- host side of the fused single-pass step: eligibility,
// parameter setup, launch geometry and the per-step buffer rotation.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <utility>

#include "kernels_fused.cuh"
#include "kernels_ax3d.cuh"
#include "kernels_line1d.cuh"
#include "kernels_tm2d.cuh"
#include "kernels_tm2d_x2.cuh"

namespace axp {

cudaError_t fused_dispatch_f64(int mode, int set, const fused::Params<double> &P, int nchunks, cudaStream_t s,
                               int *occ);
cudaError_t fused_dispatch_f32(int mode, int set, const fused::Params<float> &P, int nchunks, cudaStream_t s,
                               int *occ);
cudaError_t tm2d_dispatch_f64(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ, int tx);
cudaError_t tm2d_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ, int tx);
cudaError_t tm2d_x2_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ, int cols);
cudaError_t tm2d_list_dispatch_f64(const fused::Params<double> &P, const int4 *items, int nblocks, int per_block,
                                   cudaStream_t s, int *occ, int tx);
cudaError_t ax3d_dispatch_f64(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ);
cudaError_t ax3d_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ);

namespace {

constexpr uint32_t kSets[4] = {0u, (4u) | (3u << 3), (3u) | (4u << 3), 63u};

int grid_mode(const axp_grid *g)
{
    const int64_t *n = g->desc.n;
    if (n[0] < 2) return 0;
    if (n[1] == 1 && n[2] == 1) return 1;
    if (n[2] == 1) return 2;
    if (n[1] > 1 && n[2] > 1) return 3;
    return 0;
}

int pick_set(const axp_grid *g)
{
    const uint32_t m = order0_closure(g);
    for (int s = 0; s < 4; s++)
        if ((m & ~kSets[s]) == 0) return s;
    return 3;
}

template <typename T>
cudaError_t dispatch(int mode, int set, const fused::Params<T> &P, int nchunks, cudaStream_t s, int *occ);
template <>
cudaError_t dispatch<double>(int mode, int set, const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ)
{
    return fused_dispatch_f64(mode, set, P, nchunks, s, occ);
}
template <>
cudaError_t dispatch<float>(int mode, int set, const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ)
{
    return fused_dispatch_f32(mode, set, P, nchunks, s, occ);
}

template <typename T>
cudaError_t dispatch_tm2d(const fused::Params<T> &P, int nchunks, cudaStream_t s, int *occ, int tx);
template <>
cudaError_t dispatch_tm2d<double>(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ, int tx)
{
    return tm2d_dispatch_f64(P, nchunks, s, occ, tx);
}
template <>
cudaError_t dispatch_tm2d<float>(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ, int tx)
{
    return tm2d_dispatch_f32(P, nchunks, s, occ, tx);
}

template <typename T>
cudaError_t dispatch_ax3d(const fused::Params<T> &P, int nchunks, cudaStream_t s, int *occ);
template <>
cudaError_t dispatch_ax3d<double>(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ)
{
    return ax3d_dispatch_f64(P, nchunks, s, occ);
}
template <>
cudaError_t dispatch_ax3d<float>(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ)
{
    return ax3d_dispatch_f32(P, nchunks, s, occ);
}

// The 3D kernel specialised for an axion box: 3D grid periodic on every axis
// (E/B and axion), no order-0 field active, no uniform background E.
bool ax3d_supported(const axp_grid *g)
{
    if (grid_mode(g) != 3 || g->src_on) return false;
    if (order0_closure(g) != 0) return false;
    for (int a = 0; a < 3; a++) {
        if (g->E_ext[a] != 0.0) return false;
        if (g->desc.n[a] > (1 << 30)) return false;
        if (g->desc.em_bc[a][0] != AXP_BC_PERIODIC) return false;
        for (int s = 0; s < 2; s++)
            if (g->desc.axion_bc[a][s] != AXP_BC_PERIODIC) return false;
    }
    return (int64_t)g->desc.n[0] * g->desc.n[1] * g->desc.n[2] < ((int64_t)1 << 40);
}

// The 2D kernel specialised for the (E0z; B0x, B0y) laser: 2D grid, order-0
// closure inside that set, every non-periodic side absorbing for both E/B and
// the axion, no uniform background E, at most 2^32 cells.  A soft source is
// taken when it drives E0z only (its polarisation along z keeps the closure
// inside the set).
bool tm2d_supported(const axp_grid *g);

// The two-column form of the 2D kernel: FP32 split, an even number of columns (a
// pair never straddles the grid's edge and stays 8-byte aligned), no soft source.
template <typename T>
bool tm2d_x2_eligible(const axp_grid *g)
{
#ifdef AXP_TM2D_ONE_COLUMN
    return false;
#else
    return sizeof(T) == 4 && !g->src_on && g->desc.n[0] % 2 == 0 && tm2d_supported(g);
#endif
}

bool tm2d_supported(const axp_grid *g)
{
    if (grid_mode(g) != 2) return false;
    if (order0_closure(g) & ~kSets[1]) return false;
    for (int a = 0; a < 3; a++) {
        if (g->E_ext[a] != 0.0) return false;
        if (g->desc.n[a] > (1 << 30)) return false;
        if (g->desc.em_bc[a][0] == AXP_BC_PERIODIC) continue;
        for (int s = 0; s < 2; s++)
            if (g->desc.axion_bc[a][s] != AXP_BC_PML || g->desc.em_bc[a][s] != AXP_BC_PML) return false;
    }
    return (int64_t)g->desc.n[0] * g->desc.n[1] <= ((int64_t)1 << 32);  // 32-bit element offsets
}

template <typename T>
fused::Params<T> make_params(axp_grid *g)
{
    fused::Params<T> P;
    const axp_grid_desc &d = g->desc;
    const Workspace &w = g->layout;
    const int in = g->fset, out = 1 - g->fset;
    for (int q = 0; q < 6; q++) {
        const int fe = q < 3 ? kE0 + q : kE1 + (q - 3);
        const int fb = q < 3 ? kB0 + q : kB1 + (q - 3);
        P.Ein[q] = (const T *)(g->ws + w.off_fields[in][fe]);
        P.Bin[q] = (const T *)(g->ws + w.off_fields[in][fb]);
        P.Eout[q] = (T *)(g->ws + w.off_fields[out][fe]);
        P.Bout[q] = (T *)(g->ws + w.off_fields[out][fb]);
    }
    P.phi = (const T *)(g->ws + w.off_phi[g->phi_cur_slot]);
    P.phib = (const T *)(g->ws + w.off_phi[g->phi_b_slot]);
    P.phi_out = (T *)(g->ws + w.off_phi[g->phi_next_slot]);
    P.phib_out = d.precision == AXP_FP32_SPLIT ? (T *)(g->ws + w.off_phi[g->phi_next_b_slot]) : nullptr;
    double s_idx2 = 0.0;
    bool pml = false;
    for (int a = 0; a < 3; a++) {
        P.sig_em[a] = (const T *)(g->ws + w.off_sig_em[a]);
        P.sig_ax[a] = (const T *)(g->ws + w.off_sig_ax[a]);
        P.pml_tab[a] = (const T *)(g->ws + w.off_pml_tab[a]);
        P.n[a] = (int)d.n[a];
        P.per[a] = d.em_bc[a][0] == AXP_BC_PERIODIC;
        for (int s = 0; s < 2; s++) {
            P.axbc[a][s] = d.axion_bc[a][s];
            const bool abs = d.axion_bc[a][s] == AXP_BC_PML || d.em_bc[a][s] == AXP_BC_PML;
            if (abs) pml = true;
            P.lay[a][s] = abs ? d.pml_cells : 0;
        }
        const double inv = 1.0 / d.d[a];
        P.idx[a] = (T)inv;
        P.hidx[a] = (T)(0.5 * inv);
        P.idx2[a] = (T)(inv * inv);
        P.lap_c[a] = (T)(d.dt * d.dt * inv * inv);
        if (d.n[a] > 1) s_idx2 += inv * inv;
        P.Bext[a] = (T)g->B_ext[a];
    }
    P.has_pml = pml && d.pml_cells > 0 && d.pml_sigma_max_dt > 0;
    // FP64: phi^{n+3/2} = lap_0 phi + sum_a lap_c[a] (phi_a+ + phi_a-) - phi^{n-1/2} + ...
    // FP32 split: pi^{n+1} = pi^n + lap_0 phi + sum_a lap_c[a] (second difference) + ...,
    // the mass term alone in lap_0 so that a small (m dt)^2 keeps its FP32 precision
    P.lap_0 = (T)(d.precision == AXP_FP32_SPLIT ? -d.dt * d.dt * d.m * d.m
                                                : 2.0 - d.dt * d.dt * (d.m * d.m + 2.0 * s_idx2));
    P.dt2g = (T)(d.dt * d.dt * d.g);
    P.h = (T)(d.dt / 2.0);
    P.dt = (T)d.dt;
    P.dt2 = (T)(d.dt * d.dt);
    P.inv_dt = (T)(1.0 / d.dt);
    P.g = (T)d.g;
    P.m2 = (T)(d.m * d.m);
    P.chunk = 1;
    P.chunk_edge = 1;
    P.chunk_first = 1;
    P.src_x = -1;
    P.src_w = (const T *)(g->ws + w.off_src[1]);
    P.src_b = P.src_e = T(0);
    if (g->src_on) {
        // the step from n: B^{n+1} from E^{n+1/2}, then E from B^{n+1}
        P.src_x = (int)g->src.plane;
        P.src_b = (T)(d.dt * source_wave(g, source_x_e(g), time_half(g, g->step)));
        P.src_e = (T)(d.dt / 2.0 * source_wave(g, source_x_b(g), time_n(g, g->step + 1)));
    }
    return P;
}

template <typename T, int MODE>
size_t ring_bytes(int set)
{
    static const int planes[4] = {fused::Lay<MODE, 0, 0>::PLANES, fused::Lay<MODE, 4, 3>::PLANES,
                                  fused::Lay<MODE, 3, 4>::PLANES, fused::Lay<MODE, 7, 7>::PLANES};
    return ((size_t)planes[set] * fused::Tile<T, MODE>::NT + 4 * fused::Tile<T, MODE>::TX) * sizeof(T);
}

template <typename T>
size_t smem_need(int mode, int set)
{
    if (mode == 1) return ring_bytes<T, 1>(set);
    if (mode == 2) return ring_bytes<T, 2>(set);
    return ring_bytes<T, 3>(set);
}

}  // namespace

template <typename T>
bool fused_supported(const axp_grid *g)
{
    const int mode = grid_mode(g);
    if (mode == 0 || g->src_on) return false;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device) != cudaSuccess) return false;
    if (smem_need<T>(mode, pick_set(g)) > (size_t)optin) return false;
    for (int a = 0; a < 3; a++) {
        if (g->E_ext[a] != 0.0) return false;
        if (g->desc.n[a] > (1 << 30)) return false;
        for (int s = 0; s < 2; s++)
            if (g->desc.axion_bc[a][s] == AXP_BC_OUTFLOW) return false;
    }
    if (mode >= 2 && g->desc.n[mode == 3 ? 2 : 1] < 1) return false;
    return true;
}

// steps per block of the time-blocked 1D kernel (halo tblock + 3 on each side):
// with 4096 cells over 152 SMs a window of 27 + 2 x 18 cells fits one pass of
// the kernel's 64 cells (T = 12, 14, 15 measured 1.80, 1.77, 1.76 us/step; from
// 16 the window takes two passes)
#ifndef AXP_LINE_BLOCK
#define AXP_LINE_BLOCK 15
#endif
constexpr int kLineBlock = AXP_LINE_BLOCK;
// blocks per SM of the time-blocked 1D kernel (each owns n / (SMs x this) cells)
#ifndef AXP_LINE_BLOCKS_PER_SM
#define AXP_LINE_BLOCKS_PER_SM 1
#endif
constexpr int kLineBlocksPerSM = AXP_LINE_BLOCKS_PER_SM;

// Which grids take the time-blocked 1D kernel: FP64, 1D and periodic along x,
// no soft source and no uniform E (as the other single-pass kernels), a window
// that fits shared memory, a spare pair of axion buffers and a device that
// supports cooperative launches.
bool block1d_supported(const axp_grid *g)
{
    const axp_grid_desc &d = g->desc;
    if (d.precision != AXP_FP64 || d.n[1] != 1 || d.n[2] != 1 || d.n[0] < 256 || g->src_on) return false;
    if (d.em_bc[0][0] != AXP_BC_PERIODIC || d.axion_bc[0][0] != AXP_BC_PERIODIC) return false;
    for (int a = 0; a < 3; a++)
        if (g->E_ext[a] != 0.0) return false;
    if (g->layout.off_phi[3] == 0) return false;
    int coop = 0, sms = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device) != cudaSuccess || !coop) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess || sms < 1) return false;
    const int64_t slots = (int64_t)sms * kLineBlocksPerSM, seg = (d.n[0] + slots - 1) / slots;
    return seg + 2 * (kLineBlock + 3) <= line1d::kMaxWindow;
}

// Runs of steps of the time-blocked 1D kernel on the staggered state: one
// cooperative launch per run, split at diagnostic steps.
cudaError_t block1d_step(axp_grid *g, int64_t nsteps)
{
    const axp_grid_desc &d = g->desc;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) return e;
    g->coop_used = true;
    g->half_prev = false;  // (its windows double-buffer both field sets)
    line1d::Args A;
    std::memset(&A, 0, sizeof(A));
    A.n = d.n[0];
    A.tblock = kLineBlock;
    A.halo = kLineBlock + 3;
    A.seg = (int)((d.n[0] + (int64_t)sms * kLineBlocksPerSM - 1) / ((int64_t)sms * kLineBlocksPerSM));
    const int blocks = (int)((d.n[0] + A.seg - 1) / A.seg);
    const size_t smem = (size_t)line1d::kArrays * (A.seg + 2 * A.halo) * sizeof(double);
    e = cudaFuncSetAttribute(line1d::k_line1d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(line1d::kArrays * line1d::kMaxWindow * sizeof(double)));
    if (e != cudaSuccess) return e;
    const double dx = d.d[0], dt = d.dt;
    A.cB = dt / 2.0 / dx;
    A.c2B = dt / dx;
    A.h2g = dt * d.g;
    A.lap_0 = 2.0 - dt * dt * (d.m * d.m + 2.0 / (dx * dx));
    A.lap_c = dt * dt / (dx * dx);
    A.dt2g = dt * dt * d.g;
    A.inv_dt = 1.0 / dt;
    A.q4dx = 1.0 / (4.0 * dx);
    for (int a = 0; a < 3; a++) A.Bext[a] = g->B_ext[a];
    const Workspace &w = g->layout;
    A.ctr = (unsigned *)(g->ws + w.off_flag);
    A.err = (int *)(g->ws + w.off_flag) + 1;  // read (and cleared) by the next synchronising call
    A.absent = g->coop_absent;
    g->coop_absent = -1;
    int64_t left = nsteps;
    while (left > 0) {
        int64_t k = left;
        if (d.diag_every > 0) k = std::min<int64_t>(k, d.diag_every - g->step % d.diag_every);
        const int sets[2] = {g->fset, 1 - g->fset};
        const int ph[2][2] = {{g->phi_cur_slot, g->phi_b_slot}, {g->phi_next_slot, g->phi_next_b_slot}};
        for (int p = 0; p < 2; p++) {
            for (int q = 0; q < 6; q++) {
                const int fe = q < 3 ? kE0 + q : kE1 + (q - 3), fb = q < 3 ? kB0 + q : kB1 + (q - 3);
                A.Ew[p][q] = (double *)(g->ws + w.off_fields[sets[p]][fe]);
                A.Bw[p][q] = (double *)(g->ws + w.off_fields[sets[p]][fb]);
                A.E[p][q] = A.Ew[p][q];
                A.B[p][q] = A.Bw[p][q];
            }
            A.phi[p][0] = (double *)(g->ws + w.off_phi[ph[p][0]]);
            A.phi[p][1] = (double *)(g->ws + w.off_phi[ph[p][1]]);
        }
        A.nsteps = k;
        if ((e = cudaMemsetAsync(A.ctr, 0, sizeof(unsigned), g->stream)) != cudaSuccess) return e;
        void *args[] = {&A};
        e = cudaLaunchCooperativeKernel((const void *)line1d::k_line1d, dim3(blocks), dim3(line1d::kThreads), args,
                                        smem, g->stream);
        if (e != cudaSuccess) return e;
        g->launches++;
        A.absent = -1;
        if (((k + A.tblock - 1) / A.tblock) & 1) {  // the state ended in the other buffer set
            g->fset = 1 - g->fset;
            std::swap(g->phi_cur_slot, g->phi_next_slot);
            std::swap(g->phi_b_slot, g->phi_next_b_slot);
        }
        g->step += k;
        left -= k;
        if (d.diag_every > 0 && g->step % d.diag_every == 0) {
            axp_diag *dst = ring_slot(g, g->ring_written);
            if ((e = diag_compute<double>(g, dst)) != cudaSuccess) return e;
            g->ring_written++;
        }
    }
    return cudaGetLastError();
}

// Cost, in plane-times of one tile, of a tile over planes [m0, m1) of a strip
// whose plain iteration costs r: the march runs m1 - m0 + 6 iterations (the
// pipeline's planes), and each iteration that runs the edge body over a y layer
// (or next to a non-periodic y side: t < ylo + 6 or t >= yhi) adds `layer`.
struct SpanCost {
    bool pery;
    int64_t ylo, yhi;
    double layer;
    double operator()(double r, int64_t m0, int64_t m1) const
    {
        const int64_t t0 = m0 - 2, t1 = m1 + 3;
        double c = r * (double)(t1 - t0 + 1);
        if (!pery) {
            auto len = [](int64_t a, int64_t b) { return b >= a ? b - a + 1 : (int64_t)0; };
            const int64_t lo_end = std::min(t1, ylo + 5), hi_beg = std::max(t0, yhi);
            c += layer * (double)(len(t0, lo_end) + len(hi_beg, t1) - len(hi_beg, lo_end));
        }
        return c;
    }
};

// A block's work list: at most kListTiles tiles (x: strip, y and z: planes
// [y, z); an empty tile has z <= y), and the sum of their costs.
constexpr int kListTiles = 3;
struct ListBlock {
    int4 t[kListTiles];
    int n;
    double cost;
};

// Cuts the strips `ids` (a plain iteration of each costs r) into blocks whose
// costs are at most T, for the smallest T found by bisection: every strip is cut
// from y = 0 into the longest tiles of cost <= T, and the strips' last tiles (the
// remainders) share blocks, up to kListTiles to a block, first fit in order of
// decreasing cost, where their costs add up to <= T.  T is
// feasible when that takes at most `limit` blocks and cuts no tile shorter than
// kMinTile planes (where the strip has them: shorter ones would spend more on the
// march's set-up than the balance gains).  Returns T, or -1 when no T is
// feasible.
double list_cut(const std::vector<int> &ids, double r, int64_t ny, const SpanCost &C, int64_t limit,
                std::vector<ListBlock> *blocks)
{
    constexpr int64_t kMinTile = 8;
    auto cut = [&](double T, std::vector<ListBlock> *outp) -> bool {
        std::vector<ListBlock> rem, out;
        for (const int s : ids) {
            int64_t m0 = 0;
            while (m0 < ny) {
                if (C(r, m0, m0 + 1) > T) return false;
                int64_t lo = m0 + 1, hi = ny;  // the largest m1 with cost <= T
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) / 2;
                    if (C(r, m0, mid) <= T) lo = mid;
                    else hi = mid - 1;
                }
                ListBlock b{};
                b.t[0] = make_int4(s, (int)m0, (int)lo, 0);
                b.n = 1;
                b.cost = C(r, m0, lo);
                (lo == ny ? rem : out).push_back(b);
                if ((int64_t)out.size() > limit) return false;
                m0 = lo;
            }
        }
        std::stable_sort(rem.begin(), rem.end(), [](const ListBlock &a, const ListBlock &b) { return a.cost > b.cost; });
        const size_t first_bin = out.size();
        for (const ListBlock &x : rem) {
            size_t k = first_bin;
            while (k < out.size() && (out[k].n == kListTiles || out[k].cost + x.cost > T)) k++;
            if (k == out.size()) {
                out.push_back(x);
            } else {
                out[k].t[out[k].n++] = x.t[0];
                out[k].cost += x.cost;
            }
        }
        if ((int64_t)out.size() > limit) return false;
        if (outp) *outp = std::move(out);
        return true;
    };
    if (ids.empty()) {
        blocks->clear();
        return 0.0;
    }
    double hi = C(r, 0, ny), lo = C(r, 0, std::min(ny, kMinTile));
    if (!cut(hi, nullptr)) return -1.0;
    if (cut(lo, nullptr)) hi = lo;
    for (int it = 0; it < 48 && hi - lo > 0.25; it++) {
        const double mid = 0.5 * (lo + hi);
        if (cut(mid, nullptr)) hi = mid;
        else lo = mid;
    }
    cut(hi, blocks);
    return hi;
}

// Work lists of the 2D kernel for a launch of `per_sm` blocks per SM, laid out
// for the order in which the block scheduler fills a GPU: with sms * per_sm
// blocks, blocks j and j + sms share an SM (j < sms).  A strip at a non-periodic
// x edge runs the edge body over its layer, and its block waits at each plane's
// barrier for the layer's warp: next to a block of another strip it takes
// kEdgeNextToInner plane-times per plane, next to another such block
// kEdgePair (block timestamps gave about 1.6; as the model's weight, 1.7 to 1.9
// ran the 4096 x 2048 pulse in 0.903-0.906 ms/step, 1.6 in 0.958, 1.4 in 1.11
// and 2.0 in 0.919: a weight at or below the measured ratio leaves the x-edge
// SMs the last to finish).  So with two blocks per SM the x-edge strips get SMs of their own
// (both blocks), as many as balance their cost against the other strips'; the
// number of such SMs is found by bisection (the other strips' cost grows with
// it, theirs falls).  Returns the costliest SM's cost in plane-times and fills
// `items` (kListTiles per block, every block of the launch listed), or -1 when no
// list fits one wave (`forced`: then one wave is not required).
double list_schedule(int64_t strips, bool xedge, int64_t ny, const SpanCost &C, int sms, int per_sm, bool forced,
                     std::vector<int4> *items)
{
#ifndef AXP_LIST_EDGE_PAIR
#define AXP_LIST_EDGE_PAIR 1.8
#endif
    constexpr double kEdgePair = AXP_LIST_EDGE_PAIR, kEdgeNextToInner = 1.82;
    const int64_t slots = (int64_t)sms * per_sm;
    std::vector<int> inner, edge, all;
    for (int s = 0; s < (int)strips; s++) {
        (xedge && (s == 0 || s == strips - 1) ? edge : inner).push_back(s);
        all.push_back(s);
    }
    std::vector<ListBlock> bi, be;
    double T = -1.0;
    int E = 0;  // SMs that take the x-edge strips
    if (!edge.empty() && per_sm == 2 && sms >= 2) {
        auto costs = [&](int e, std::vector<ListBlock> *oi, std::vector<ListBlock> *oe, double *ti, double *te) {
            *ti = list_cut(inner, 1.0, ny, C, 2 * (int64_t)(sms - e), oi);
            *te = list_cut(edge, kEdgePair, ny, C, 2 * (int64_t)e, oe);
        };
        // the smallest e whose edge cost no longer exceeds the inner cost
        int lo = 1, hi = sms - 1;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            double ti, te;
            std::vector<ListBlock> a, b;
            costs(mid, &a, &b, &ti, &te);
            if (te >= 0 && (ti < 0 || te <= ti)) hi = mid;
            else lo = mid + 1;
        }
        for (int e = std::max(1, lo - 1); e <= std::min(sms - 1, lo); e++) {
            double ti, te;
            std::vector<ListBlock> a, b;
            costs(e, &a, &b, &ti, &te);
            if (ti < 0 || te < 0) continue;
            if (T < 0 || std::max(ti, te) < T) {
                T = std::max(ti, te);
                E = e;
                bi = std::move(a);
                be = std::move(b);
            }
        }
    } else if (edge.empty()) {
        T = list_cut(inner, 1.0, ny, C, slots, &bi);
    } else {  // one block per SM: an x-edge strip's block is next to nothing, or next to inner blocks
        std::vector<ListBlock> a, b;
        const double ti = list_cut(inner, 1.0, ny, C, slots, &a);
        const double te = list_cut(edge, per_sm > 1 ? kEdgeNextToInner : kEdgePair, ny, C, slots, &b);
        if (ti >= 0 && te >= 0 && (int64_t)(a.size() + b.size()) <= slots) {
            T = std::max(ti, te);
            bi = std::move(a);
            be = std::move(b);
            for (ListBlock &x : be) bi.push_back(x);
            be.clear();
        }
    }
    if (T < 0) {
        if (!forced) return -1.0;
        // a grid of more strips than one wave holds: every strip at the edge rate
        T = list_cut(all, kEdgeNextToInner, ny, C, std::max(slots, strips), &bi);
        be.clear();
        E = 0;
        if (T < 0) return -1.0;
    }
    // lay the blocks out: x-edge blocks at j and j + sms for j < E, the others in
    // the remaining places, costliest first in the first wave and cheapest first in
    // the second (so that an SM's two blocks roughly even out); empty blocks pad
    // the launch to whole waves
    auto by_cost = [](const ListBlock &a, const ListBlock &b) { return a.cost > b.cost; };
    std::stable_sort(bi.begin(), bi.end(), by_cost);
    const int64_t nb = std::max<int64_t>(slots, (int64_t)(bi.size() + be.size()));
    const ListBlock none{};
    std::vector<ListBlock> lay((size_t)nb, none);
    std::vector<char> taken((size_t)nb, 0);
    for (size_t k = 0; k < be.size(); k++) {
        const int64_t pos = (int64_t)(k / 2) + (k % 2 ? sms : 0);
        lay[(size_t)pos] = be[k];
        taken[(size_t)pos] = 1;
    }
    for (int j = 0; j < E && per_sm == 2; j++) taken[(size_t)j] = taken[(size_t)(j + sms)] = 1;
    std::vector<int64_t> first, second;
    for (int64_t p = 0; p < nb; p++) {
        if (taken[(size_t)p]) continue;
        (p < sms ? first : second).push_back(p);
    }
#ifndef AXP_LIST_SAME_ORDER
    std::reverse(second.begin(), second.end());
#endif
    size_t k = 0;
    for (const int64_t p : first)
        if (k < bi.size()) lay[(size_t)p] = bi[k++];
    for (const int64_t p : second)
        if (k < bi.size()) lay[(size_t)p] = bi[k++];
    for (; k < bi.size(); k++) lay.push_back(bi[k]);  // (forced lists beyond one wave)
    items->clear();
    for (const ListBlock &b : lay)
        for (int k = 0; k < kListTiles; k++) items->push_back(b.t[k]);
    return T;
}

// The work-list form takes FP64 grids without a soft source.
template <typename T>
bool tm2d_list_eligible(const axp_grid *g)
{
    return sizeof(T) == 8 && !g->src_on && g->layout.off_sched != 0 && tm2d_supported(g);
}

// Launch plan of the 2D kernel, made once per configuration (kernel choice, soft
// source, and whether the folded-current form applies) and kept in the handle.
template <typename T>
cudaError_t tm2d_plan(axp_grid *g)
{
    fused::Params<T> P = make_params<T>(g);
    const bool foldp = P.Bext[0] == T(0) && P.Bext[1] == T(0) && P.idx[0] == P.idx[1];
    const int64_t key = ((int64_t)g->kernel_choice * 2 + (g->src_on ? 1 : 0)) * 2 + (foldp ? 1 : 0);
    if (g->tm_plan_key == key) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const bool x2 = tm2d_x2_eligible<T>(g);
    auto occ_of = [&](int width, int *o) -> cudaError_t {
        if constexpr (sizeof(T) == 4) {
            if (x2) return tm2d_x2_dispatch_f32(P, 0, g->stream, o, width);
        }
        return dispatch_tm2d<T>(P, 0, g->stream, o, width);
    };
    const bool want_list = g->kernel_choice == AXP_KERNEL_TM2D_LIST;
    const bool list_ok = tm2d_list_eligible<T>(g) && (want_list || g->kernel_choice == AXP_KERNEL_AUTO);
    double best_list = -1.0;
    int list_tx = 0;
    std::vector<int4> list_items;
    int tm_tx = tm2d::TX;
    // Tile width and march chunks: the fewest resident-block waves for the work
    // a wave does, (planes + pipeline) x columns x blocks per SM, divided by the
    // share of its issue rate an SM reaches with that many warps resident.  FP64:
    // below 8 warps the FP64 pipe's and the loads' latencies are no longer
    // hidden, sqrt(warps / 8); FP32: warps / 16, and kManyBlocks beyond two blocks
    // per SM; kOneBlock for one block per SM (all from measured tile widths).
    // Measured per-CTA times give the other two costs: a strip at a non-periodic x edge runs the edge body
    // over the x layer and takes kEdgeCost times as long per plane (its warps
    // wait at each plane's barrier for the layer's warp), and a chunk that
    // crosses a y layer runs the edge body over the layer and the pipeline's
    // planes next to it, kLayerCost plane-times each.  With one wave the x-edge
    // strips may get more, shorter chunks from the blocks the other strips
    // leave free, and the other strips' first and last chunks are shortened by
    // the y layer's extra cost.
    const double kEdgeCost = sizeof(T) == 8 ? 1.55 : 1.35;
    // A lone block per SM has nothing else to issue while its warps wait at a
    // plane's barrier: two blocks of half the width ran the 2D pulse 7% faster.
    const double kOneBlock = 0.92;
    const double kManyBlocks = 0.7;  // FP32 with more than two blocks per SM (the FP32 rule below)
    const double kLayerCost = sizeof(T) == 8 ? 0.93 : 0.32;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int64_t nx = g->desc.n[0], ny = g->desc.n[1];
    const bool xedge = g->desc.em_bc[0][0] != AXP_BC_PERIODIC;
    const bool ylay = g->desc.em_bc[1][0] != AXP_BC_PERIODIC && P.has_pml;
    const int64_t D = ylay ? (int64_t)std::lround(kLayerCost * (P.lay[1][0] + 7)) : 0;
    // the same costs tile by tile, for the work-list form
    const SpanCost span{g->desc.em_bc[1][0] == AXP_BC_PERIODIC, (int64_t)P.lay[1][0], ny - 1 - (int64_t)P.lay[1][1],
                        kLayerCost};
    // `rows` chunks over y: returns the costliest chunk in plane-times, with the
    // first and the middle chunk sizes (the last chunk is what remains, <= cf)
    auto split = [&](int64_t rows, int64_t *cf, int64_t *cm) -> double {
        const int64_t u0 = (ny + rows - 1) / rows;
        *cf = *cm = u0;
        if (D == 0 || rows < 3) return (double)(u0 + 6 + D);
        const int64_t c = (ny + 2 * D + rows - 1) / rows, f = c - D;
        const int64_t last = ny - f - (rows - 2) * c;
        if (f < 16 || last < 1 || last > f) return (double)(u0 + 6 + D);
        *cf = f;
        *cm = c;
        return (double)(c + 6);
    };
    double best = -1.0;
    int best_ce = 0, best_rows = 0, best_cf = 0;
    // tile widths in columns; the two-column form takes multiples of 64 (tx / 2 threads)
    const int halo = x2 ? tm2d_x2::HL + tm2d_x2::HR : tm2d::HL + tm2d::HR;
    for (int tx = tm2d::TX; tx >= 128; tx -= x2 ? 64 : 32) {
        int o = 0;
        if ((e = occ_of(tx, &o)) != cudaSuccess) return e;
        o = o > 0 ? o : 1;
        // warps of one-column threads holding as many columns (the two-column form
        // runs half as many threads with twice the work each)
        const double warps = (double)o * tx / 32.0;
        double u = warps >= 8.0 ? 1.0 : std::sqrt(warps / 8.0);
        if (sizeof(T) == 4) {
            // FP32 waits on memory, and more warps hide more of it: two 256-wide blocks
            // per SM (16 warps) beat 224 and 192 by 1-8% on 2048^2 to 8192 x 4096 grids,
            // while three or four narrower blocks per SM ran 15-30% slower
            u = std::min(warps, 16.0) / 16.0;
            if (o > 2) u *= kManyBlocks;
        }
        if (o < 2) u *= kOneBlock;
        const int64_t strips = (nx + (tx - halo) - 1) / (tx - halo);
        const int64_t slots = (int64_t)sms * o;
        const double r = xedge ? kEdgeCost : 1.0;
        if constexpr (sizeof(T) == 8) {
            int ol = 0;  // the work-list form at this tile width
            if (list_ok && (e = tm2d_list_dispatch_f64(P, nullptr, 0, kListTiles, g->stream, &ol, tx)) != cudaSuccess)
                return e;
            ol = ol > 0 ? ol : 1;
            // (grids too small for chunks of 16 planes on half the resident blocks are
            // latency-bound: there the uniform grid's shorter chunks did better)
            if (list_ok && (want_list || 2 * strips * (ny / 16) >= (int64_t)sms * ol)) {
                std::vector<int4> it;
                const double tl = list_schedule(strips, xedge, ny, span, sms, ol, want_list, &it);
                const double wl = (double)ol * tx / 32.0;
                const double ul = (wl >= 8.0 ? 1.0 : std::sqrt(wl / 8.0)) * (ol < 2 ? kOneBlock : 1.0);
                const double cost = tl * tx * ol / ul;
                if (tl > 0 && it.size() <= (size_t)kSchedItems && (best_list < 0 || cost < best_list)) {
                    best_list = cost;
                    list_tx = tx;
                    list_items = std::move(it);
                }
            }
        }
        // a grid too small to give every resident block a chunk of 16 planes takes
        // chunks down to 4 planes: the pipeline's extra planes then cost less than
        // the SMs they would leave idle (small grids are latency-bound)
        const int64_t min_chunk = strips * (ny / 16) < slots ? 4 : 16;
        for (int64_t nc = 1; nc <= 512 && ny / nc >= min_chunk; nc++) {  // the same chunks everywhere
            const int64_t chunk = (ny + nc - 1) / nc, rows = (ny + chunk - 1) / chunk;
            const int64_t waves = (strips * rows + slots - 1) / slots;
            const double cost = (double)waves * (double)(chunk + 6 + D) * r * tx * o / u;
            if (best < 0 || cost < best) {
                best = cost;
                tm_tx = tx;
                P.chunk = (int)chunk;
                best_cf = (int)chunk;
                best_ce = (int)chunk;
                best_rows = (int)rows;
            }
        }
        if (!xedge || strips < 3) continue;
        for (int64_t ni = 1; ni <= 64 && ny / ni >= 16; ni++) {  // shorter chunks at the x edges
            const int64_t ri = ni;
            int64_t cf = 0, cm = 0;
            const double ci_cost = split(ri, &cf, &cm);
            const int64_t left = slots - (strips - 2) * ri;
            if (left < 2) break;
            int64_t ne = std::min<int64_t>(left / 2, std::max<int64_t>(1, ny / 16));
            const int64_t ce = (ny + ne - 1) / ne, re = (ny + ce - 1) / ce;
            const double cost = std::max(ci_cost, (double)(ce + 6) * r + D) * tx * o / u;
            if (cost < best) {
                best = cost;
                tm_tx = tx;
                P.chunk = (int)cm;
                best_cf = (int)cf;
                best_ce = (int)ce;
                best_rows = (int)std::max(ri, re);
            }
        }
    }
    if (best < 0) {  // grids shorter than 16 planes: one chunk
        tm_tx = tm2d::TX;
        P.chunk = (int)ny;
        best_cf = (int)ny;
        best_ce = (int)ny;
        best_rows = 1;
    }
    // the work-list form of the SpanCost model, beside the uniform grid's
    g->tm_tx = tm_tx;
    g->tm_chunk = P.chunk;
    g->tm_chunk_first = best_cf;
    g->tm_chunk_edge = best_ce;
    g->tm_nchunks = best_rows;
    g->tm_list_blocks = 0;
    g->tm_list_per_block = kListTiles;
    if (want_list && best_list < 0) return cudaErrorInvalidValue;  // (more than kSchedItems items)
    // AUTO takes the lists where the model expects them 5% faster: measured on
    // 512^2 to 8192 x 4096 pulses, a smaller expected gain did not hold
    if (best_list >= 0 && (want_list || best_list < 0.95 * best)) {
        g->tm_tx = list_tx;
        g->tm_list_blocks = (int32_t)(list_items.size() / kListTiles);
        g->tm_items = std::move(list_items);
        g->tm_items_uploaded = false;
    }
    g->tm_plan_key = key;
    return cudaSuccess;
}

// Copies the work lists into the workspace once per plan (on the grid's stream,
// ordered before the launches that read them).
cudaError_t tm2d_upload_list(axp_grid *g)
{
    if (g->tm_items_uploaded) return cudaSuccess;
    const size_t bytes = g->tm_items.size() * sizeof(int4);
    if (g->tm_items.size() > (size_t)kSchedItems) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaMemcpyAsync(g->ws + g->layout.off_sched, g->tm_items.data(), bytes, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) g->tm_items_uploaded = true;
    return e;
}

template <typename T>
int32_t fused_path(axp_grid *g)
{
    const int32_t k = g->kernel_choice;
    if (k == AXP_KERNEL_GENERAL || g->parts) return AXP_KERNEL_GENERAL;
    const bool b1 = block1d_supported(g);
    if (k == AXP_KERNEL_BLOCK1D) return b1 ? AXP_KERNEL_BLOCK1D : AXP_KERNEL_GENERAL;
    if (k == AXP_KERNEL_AUTO && b1) return AXP_KERNEL_BLOCK1D;
    const bool tm = tm2d_supported(g), ax = ax3d_supported(g), fu = fused_supported<T>(g);
    if (k == AXP_KERNEL_TM2D) return tm ? AXP_KERNEL_TM2D : AXP_KERNEL_GENERAL;
    if (k == AXP_KERNEL_TM2D_LIST) return tm && tm2d_list_eligible<T>(g) ? AXP_KERNEL_TM2D_LIST : AXP_KERNEL_GENERAL;
    if (k == AXP_KERNEL_AX3D) return ax ? AXP_KERNEL_AX3D : AXP_KERNEL_GENERAL;
    if (k == AXP_KERNEL_FUSED) return fu ? AXP_KERNEL_FUSED : AXP_KERNEL_GENERAL;
    if (tm) return tm2d_plan<T>(g) == cudaSuccess && g->tm_list_blocks > 0 ? AXP_KERNEL_TM2D_LIST : AXP_KERNEL_TM2D;
    return ax ? AXP_KERNEL_AX3D : (fu ? AXP_KERNEL_FUSED : AXP_KERNEL_GENERAL);
}

// Fused 1D steps are short (microseconds), so runs of them replay from CUDA
// graphs of kGraphSteps launches.  kGraphSteps is a multiple of the periods of
// the buffer-role rotation (2 for the field sets and the FP32 axion slots, 3 for
// the FP64 axion slots), so a graph leaves the roles as it found them and one
// graph serves every replay from the same role configuration.
constexpr int kGraphSteps = 48;

int64_t roles_key(const axp_grid *g)
{
    return ((((g->cfg_version * 2 + g->fset) * 4 + g->phi_cur_slot) * 4 + g->phi_b_slot) * 4 + g->phi_next_slot) * 4 +
           g->phi_next_b_slot;
}

template <typename T, typename Launch>
cudaError_t step_graph(axp_grid *g, Launch &&launch_one, cudaGraphExec_t *out)
{
    const int64_t key = roles_key(g);
    for (int i = 0; i < g->n_step_graphs; i++)
        if (g->step_graph_key[i] == key) {
            *out = g->step_graph[i];
            return cudaSuccess;
        }
    if (g->n_step_graphs == 8) release_step_graphs(g, false);
    cudaError_t e = cudaSuccess;
    if (!g->capture_stream) e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    const int fset = g->fset, s0 = g->phi_cur_slot, s1 = g->phi_b_slot, s2 = g->phi_next_slot, s3 = g->phi_next_b_slot;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; k++) {
        le = launch_one(make_params<T>(g), g->capture_stream);
        rotate_roles(g);
    }
    e = cudaStreamEndCapture(g->capture_stream, &graph);
    g->fset = fset;  // (kGraphSteps rotations are the identity; restored regardless)
    g->phi_cur_slot = s0;
    g->phi_b_slot = s1;
    g->phi_next_slot = s2;
    g->phi_next_b_slot = s3;
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le != cudaSuccess ? le : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    g->step_graph_key[g->n_step_graphs] = key;
    g->step_graph[g->n_step_graphs++] = exec;
    *out = exec;
    return cudaSuccess;
}

template <typename T>
cudaError_t fused_step(axp_grid *g, int64_t nsteps, bool *handled)
{
    *handled = false;
    const int32_t path = fused_path<T>(g);
    if (path == AXP_KERNEL_GENERAL) return cudaSuccess;
    *handled = true;
    if (path == AXP_KERNEL_BLOCK1D) {
        cudaError_t e = enter_staggered<T>(g);
        return e != cudaSuccess ? e : block1d_step(g, nsteps);
    }
    const bool tm = path == AXP_KERNEL_TM2D || path == AXP_KERNEL_TM2D_LIST, ax = path == AXP_KERNEL_AX3D;
    const int mode = grid_mode(g);
    const int set = pick_set(g);
    cudaError_t e = enter_staggered<T>(g);
    if (e != cudaSuccess) return e;
    int tm_tx = tm2d::TX;  // tile width of the 2D kernel (chosen below)
    // FP32 split on an even-width grid without a soft source: the two-column form
    const bool x2 = tm && tm2d_x2_eligible<T>(g);
    auto dispatch_2d = [&](const fused::Params<T> &Pl, int nch, int *occp, int width) -> cudaError_t {
        if constexpr (sizeof(T) == 4) {
            if (x2) return tm2d_x2_dispatch_f32(Pl, nch, g->stream, occp, width);
        }
        return dispatch_tm2d<T>(Pl, nch, g->stream, occp, width);
    };
    auto launch = [&](const fused::Params<T> &Pl, int nch, int *occp) {
        if constexpr (sizeof(T) == 8) {
            if (tm && g->tm_plan_key >= 0 && g->tm_list_blocks > 0)
                return tm2d_list_dispatch_f64(Pl, (const int4 *)(g->ws + g->layout.off_sched),
                                              nch > 0 ? g->tm_list_blocks : 0, g->tm_list_per_block, g->stream, occp,
                                              tm_tx);
        }
        if (tm) return dispatch_2d(Pl, nch, occp, tm_tx);
        if (ax) return dispatch_ax3d<T>(Pl, nch, g->stream, occp);
        return dispatch<T>(mode, set, Pl, nch, g->stream, occp);
    };
    // launch geometry: as many march chunks as keep every resident CTA slot busy
    int occ = 0;
    fused::Params<T> P = make_params<T>(g);
    e = launch(P, 0, &occ);
    if (e != cudaSuccess) return e;
    int nchunks = 1;
    if (ax) {
        // z chunks: fewest waves of resident blocks for the (tile + pipeline) work
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const bool pairs = sizeof(T) == 4 && g->desc.n[0] % 2 == 0;  // the two-cell form's tiles
        const int64_t vx = pairs ? ax3d::x2::VXC : ax3d::VX, vy = pairs ? ax3d::x2::VYR : ax3d::Geo<T>::VY;
        const int64_t tiles = ((g->desc.n[0] + vx - 1) / vx) * ((g->desc.n[1] + vy - 1) / vy);
        const int64_t nz = g->desc.n[2], slots = (int64_t)sms * (occ > 0 ? occ : 1);
        double best = 0;
        for (int64_t nc = 1; nc <= 32 && nc <= nz; nc++) {
            const int64_t chunk = (nz + nc - 1) / nc, waves = (tiles * nc + slots - 1) / slots;
            const double cost = (double)waves * (double)(chunk + 3);
            if (nc == 1 || cost < best) {
                best = cost;
                P.chunk = (int)chunk;
                nchunks = (int)((nz + chunk - 1) / chunk);
            }
        }
    } else if (tm) {
        if ((e = tm2d_plan<T>(g)) != cudaSuccess) return e;
        tm_tx = g->tm_tx;
        P.chunk = g->tm_chunk;
        P.chunk_first = g->tm_chunk_first;
        P.chunk_edge = g->tm_chunk_edge;
        nchunks = g->tm_nchunks;
        if (g->tm_list_blocks > 0 && (e = tm2d_upload_list(g)) != cudaSuccess) return e;
    } else if (mode >= 2) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const int VX = mode == 3 ? fused::Tile<T, 3>::VX : fused::Tile<T, 2>::VX;
        const int VY = mode == 3 ? fused::Tile<T, 3>::VY : 1;
        const int64_t strips = ((g->desc.n[0] + VX - 1) / VX) * (mode == 3 ? (g->desc.n[1] + VY - 1) / VY : 1);
        const int64_t nm = g->desc.n[mode == 3 ? 2 : 1];
        const int64_t slots = (int64_t)sms * (occ > 0 ? occ : 1);
        int64_t nc = slots / strips;
        if (nc < 1) nc = 1;
        const int64_t min_chunk = 16;
        if (nm / nc < min_chunk) nc = nm / min_chunk > 0 ? nm / min_chunk : 1;
        int64_t chunk = (nm + nc - 1) / nc;
        nchunks = (int)((nm + chunk - 1) / chunk);
        P.chunk = (int)chunk;
    }
    int64_t it = 0;
    if (mode == 1 && !tm && !ax && g->desc.diag_every == 0 && nsteps >= kGraphSteps) {
        auto one = [&](const fused::Params<T> &Pl, cudaStream_t st) {
            return dispatch<T>(mode, set, Pl, nchunks, st, nullptr);
        };
        for (; it + kGraphSteps <= nsteps; it += kGraphSteps) {
            cudaGraphExec_t exec = nullptr;
            if ((e = step_graph<T>(g, one, &exec)) != cudaSuccess) return e;
            if ((e = cudaGraphLaunch(exec, g->stream)) != cudaSuccess) return e;
            g->launches += kGraphSteps;
            g->step += kGraphSteps;
            g->half_prev = true;  // the other set holds the last step's E^{n-1/2}
            g->half_prev_cfg = g->cfg_version;
        }
    }
    for (; it < nsteps; it++) {
        if (it > 0) {
            const int ch = P.chunk, che = P.chunk_edge, chf = P.chunk_first;
            P = make_params<T>(g);
            P.chunk = ch;
            P.chunk_edge = che;
            P.chunk_first = chf;
        }
        e = launch(P, nchunks, nullptr);
        if (e != cudaSuccess) return e;
        g->launches++;
        rotate_roles(g);
        g->step++;
        g->half_prev = true;  // the other set holds the last step's E^{n-1/2}
        g->half_prev_cfg = g->cfg_version;
        if (g->desc.diag_every > 0 && g->step % g->desc.diag_every == 0) {
            axp_diag *dst = ring_slot(g, g->ring_written);
            if ((e = diag_compute<T>(g, dst)) != cudaSuccess) return e;
            g->ring_written++;
        }
    }
    g->J_valid = false;
    return cudaGetLastError();
}

void release_step_graphs(axp_grid *g, bool all)
{
    if (g->n_step_graphs > 0) cudaStreamSynchronize(g->stream);  // no replay may still be running
    for (int i = 0; i < g->n_step_graphs; i++) cudaGraphExecDestroy(g->step_graph[i]);
    g->n_step_graphs = 0;
    if (all && g->capture_stream) {
        cudaStreamDestroy(g->capture_stream);
        g->capture_stream = nullptr;
    }
}

void rotate_roles(axp_grid *g)
{
    // the output field set becomes current; the axion buffers shift roles
    g->fset = 1 - g->fset;
    if (g->desc.precision == AXP_FP32_SPLIT) {
        std::swap(g->phi_cur_slot, g->phi_next_slot);
        std::swap(g->phi_b_slot, g->phi_next_b_slot);
    } else {
        const int old = g->phi_b_slot;
        g->phi_b_slot = g->phi_cur_slot;
        g->phi_cur_slot = g->phi_next_slot;
        g->phi_next_slot = old;
    }
}

bool tm2d_eligible(const axp_grid *g) { return tm2d_supported(g); }

template <typename T>
fused::Params<T> tm2d_params(axp_grid *g, int chunk)
{
    fused::Params<T> P = make_params<T>(g);
    P.chunk = chunk;
    P.chunk_edge = chunk;
    P.chunk_first = chunk;
    return P;
}

template fused::Params<float> tm2d_params<float>(axp_grid *, int);
template int32_t fused_path<double>(axp_grid *);
template int32_t fused_path<float>(axp_grid *);
template bool fused_supported<double>(const axp_grid *);
template bool fused_supported<float>(const axp_grid *);
template cudaError_t fused_step<double>(axp_grid *, int64_t, bool *);
template cudaError_t fused_step<float>(axp_grid *, int64_t, bool *);

}  // namespace axp

// kernels_diag.cu -- FP64 diagnostics (arXiv 2406.16796 Sec. 3.2-3.4 energy
// densities, conversion probabilities and laser centroid; Sec. 2.2 Gauss law).
//
// Deterministic two-stage reduction: a fixed grid of blocks writes one FP64
// partial per quantity per block (fixed tree order inside the block), then one
// block sums the partials in fixed order.  The result depends only on the
// grid size, never on scheduling, so a grid's diagnostics are bit-identical
// however the work around it is arranged.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "device_common.cuh"

namespace axp {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kQ = 7;  // H_phi, H_g0, H_g1, cross, sum x B1z^2, sum B1z^2, gauss

template <typename T, bool INCR>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(View<T> v, PhiPair<T, INCR> q, double *partials)
{
    double acc[kQ];
#pragma unroll
    for (int s = 0; s < kQ; s++) acc[s] = 0.0;
    const double dV = (double)v.d[0] * (double)v.d[1] * (double)v.d[2];
    const double m2 = (double)v.m2;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < v.N; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        cell_of(c, v.n, &i, &j, &k);
        if (i < v.region_lo[0] || i >= v.region_hi[0] || j < v.region_lo[1] || j >= v.region_hi[1] ||
            k < v.region_lo[2] || k >= v.region_hi[2])
            continue;
        T midT, DtT;
        phi_mid_dt<T, INCR>(v, q, i, j, k, &midT, &DtT);
        const double mid = midT, Dt = DtT;
        double g2 = 0.0, R = 0.0, bg = 0.0;
        // divisions by d and 2d (a multiplication where the reciprocal is exact)
        auto od = [&](double x, int a) { return v.rd[a] != T(0) ? x * (double)v.rd[a] : x / (double)v.d[a]; };
        auto o2d = [&](double x, int a) {
            return v.rd2[a] != T(0) ? x * (double)v.rd2[a] : x / (2.0 * (double)v.d[a]);
        };
        for (int a = 0; a < 3; a++) {
            int64_t u[3];
            unit(a, u);
            const double up = (double)phi_mid<T, INCR>(v, q, i + u[0], j + u[1], k + u[2]);
            const double dn = (double)phi_mid<T, INCR>(v, q, i - u[0], j - u[1], k - u[2]);
            const double fw = od(up - mid, a);
            g2 += fw * fw;
            const T *E1 = v.f[kE1 + a];
            R += od((double)E1[c] - (double)ld(v, E1, i - u[0], j - u[1], k - u[2]), a);
            bg += (double)b0_bar(v, a, i, j, k) * o2d(up - dn, a);
        }
        R += (double)v.g * bg;
        acc[0] += 0.5 * ((Dt * Dt + g2) + m2 * mid * mid) * dV;
        double e0 = 0.0, e1 = 0.0, x = 0.0;
        for (int a = 0; a < 3; a++) {
            const double E0a = v.f[kE0 + a][c], B0a = v.f[kB0 + a][c];
            const double E1a = v.f[kE1 + a][c], B1a = v.f[kB1 + a][c];
            e0 += E0a * E0a + B0a * B0a;
            e1 += E1a * E1a + B1a * B1a;
            x += (E0a + (double)v.Eext[a]) * E1a + (B0a + (double)v.Bext[a]) * B1a;
        }
        acc[1] += 0.5 * e0 * dV;
        acc[2] += 0.5 * e1 * dV;
        acc[3] += x * dV;
        const double xb = (double)v.lo[0] + (double)(i + 1) * (double)v.d[0];
        const double b1z = v.f[kB1 + 2][c];
        const double bz2 = b1z * b1z * dV;
        acc[4] += xb * bz2;
        acc[5] += bz2;
        acc[6] += R * R * dV;
    }
    __shared__ double sh[kQ][kDiagThreads];
#pragma unroll
    for (int s = 0; s < kQ; s++) sh[s][threadIdx.x] = acc[s];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int s = 0; s < kQ; s++) sh[s][threadIdx.x] += sh[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kQ) partials[(int64_t)blockIdx.x * kQ + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double *partials, int nblocks, axp_diag *out,
                                                             int64_t step, double t)
{
    __shared__ double sh[kQ][kDiagThreads];
    double acc[kQ];
#pragma unroll
    for (int s = 0; s < kQ; s++) acc[s] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kDiagThreads)
#pragma unroll
        for (int s = 0; s < kQ; s++) acc[s] += partials[(int64_t)b * kQ + s];
#pragma unroll
    for (int s = 0; s < kQ; s++) sh[s][threadIdx.x] = acc[s];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int s = 0; s < kQ; s++) sh[s][threadIdx.x] += sh[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        axp_diag d;
        d.step = step;
        d.t = t;
        d.H_phi = sh[0][0];
        d.H_g0 = sh[1][0];
        d.H_g1 = sh[2][0];
        d.P_g2a = d.H_g0 > 0 ? d.H_phi / d.H_g0 : 0.0;
        d.P_a2g = d.H_phi > 0 ? d.H_g1 / d.H_phi : 0.0;
        d.W = d.H_phi + sh[3][0];
        d.sum_xB1z2 = sh[4][0];
        d.sum_B1z2 = sh[5][0];
        d.gauss_l2 = sh[6][0];
        *out = d;
    }
}

}  // namespace

template <typename T>
static Ghosts<T> ghosts_lvl(axp_grid *g, int level)
{
    Ghosts<T> G;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) {
            const size_t off = g->layout.off_ghost[a][s][g->ghost_level_slot[level]];
            G.p[a][s] = off ? (T *)(g->ws + off) : nullptr;
        }
    return G;
}

template <typename T>
cudaError_t diag_compute(axp_grid *g, axp_diag *dev_dst)
{
    return diag_compute_rows<T>(g, dev_dst, -1, 0, 0);
}

// E^n from the two E levels a single-pass step leaves (Sec. 2.3): both E
// half-steps of the step from n-1/2 read the same X = curl B^n - g J^n, so
// E^n = a E^{n-1/2} + b X and E^{n+1/2} = a E^n + b X, where a, b are the
// half-step's layer coefficients (a = 1, b = h outside the layers; the smallest
// a of the axes at a corner).  Hence E^n = (E^{n+1/2} + a E^{n-1/2}) / (1 + a),
// the mean of the two levels outside the layers.  Written over E^{n-1/2} (the
// other field set); the active E arrays only (the others are zero in both sets).
template <typename T>
struct ELevels {
    T *lo[6];        // E^{n-1/2}, overwritten with E^n (order 0 xyz, order 1 xyz)
    const T *hi[6];  // E^{n+1/2}
    const T *a1[3];  // per axis, the one-half-step layer coefficient a (null: no layer along the axis)
    unsigned mask;   // arrays to form
    int64_t n0, n1, n2;
};

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_e_level(ELevels<T> L)
{
    const int64_t rows = L.n1 * L.n2;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const int64_t j = r % L.n1, k = r / L.n1;
        T ayz = T(1);
        if (L.a1[1] && L.a1[1][j] < ayz) ayz = L.a1[1][j];
        if (L.a1[2] && L.a1[2][k] < ayz) ayz = L.a1[2][k];
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.n0; i += (int64_t)gridDim.x * blockDim.x) {
            T a = ayz;
            if (L.a1[0] && L.a1[0][i] < a) a = L.a1[0][i];
            const int64_t c = i + L.n0 * r;
#pragma unroll
            for (int f = 0; f < 6; f++) {
                if (!(L.mask >> f & 1u)) continue;
                L.lo[f][c] = a == T(1) ? T(0.5) * (L.hi[f][c] + L.lo[f][c]) : (L.hi[f][c] + a * L.lo[f][c]) / (T(1) + a);
            }
        }
    }
}

template <typename T>
cudaError_t e_level_from_halves(axp_grid *g)
{
    ELevels<T> L;
    const Workspace &w = g->layout;
    const int oset = 1 - g->fset;
    const int fe[6] = {kE0, kE0 + 1, kE0 + 2, kE1, kE1 + 1, kE1 + 2};
    L.mask = 0;
    for (int f = 0; f < 6; f++) {
        L.lo[f] = (T *)(g->ws + w.off_fields[oset][fe[f]]);
        L.hi[f] = (const T *)(g->ws + w.off_fields[g->fset][fe[f]]);
        if (f >= 3 || (g->active >> fe[f] & 1u)) L.mask |= 1u << f;
    }
    for (int a = 0; a < 3; a++) {
        const bool lay = g->desc.em_bc[a][0] != AXP_BC_PERIODIC && g->desc.pml_cells > 0 && g->desc.pml_sigma_max_dt > 0;
        L.a1[a] = lay ? (const T *)(g->ws + w.off_pml_tab[a]) : nullptr;
    }
    L.n0 = g->desc.n[0];
    L.n1 = g->desc.n[1];
    L.n2 = g->desc.n[2];
    const int64_t rows = L.n1 * L.n2;
    dim3 grid((unsigned)((L.n0 + kDiagThreads - 1) / kDiagThreads), (unsigned)(rows < 65535 ? rows : 65535), 1);
    if (grid.x > 64) grid.x = 64;
    k_e_level<T><<<grid, kDiagThreads, 0, g->stream>>>(L);
    g->launches++;
    g->half_prev = false;  // the other set now holds E^n
    return cudaGetLastError();
}

// The sums over the cells whose index along `axis` lies in [lo, hi) as well as in
// the physical region (axis < 0: no restriction).  A slab of a decomposed grid
// sums its owned rows this way; the records' sums add up across slabs.
template <typename T>
cudaError_t diag_compute_rows(axp_grid *g, axp_diag *dev_dst, int axis, int64_t lo, int64_t hi)
{
    // staggered (fused-path) state: reconstruct E^n into the spare field set first,
    // from the two levels of the last single-pass step where the other set holds
    // them, else by the general kernels' inverse half-step
    View<T> v;
    if (g->staggered) {
        const bool halves = g->half_prev && g->half_prev_cfg == g->cfg_version;
        const cudaError_t e = halves ? e_level_from_halves<T>(g) : exit_staggered<T>(g, false);
        if (e != cudaSuccess) return e;
        v = make_view_eset<T>(g, 1 - g->fset);
    } else {
        v = make_view<T>(g);
    }
    if (axis >= 0) {
        if (lo > v.region_lo[axis]) v.region_lo[axis] = (int)lo;
        if (hi < v.region_hi[axis]) v.region_hi[axis] = (int)hi;
    }
    double *partials = (double *)(g->ws + g->layout.off_partials);
    const int nb = g->layout.diag_blocks;
    if (g->desc.precision == AXP_FP32_SPLIT) {
        PhiPair<T, true> q{v.phi_cur, v.phi_b, ghosts_lvl<T>(g, 0), ghosts_lvl<T>(g, 1)};
        k_diag_partial<T, true><<<nb, kDiagThreads, 0, g->stream>>>(v, q, partials);
    } else {
        PhiPair<T, false> q{v.phi_cur, v.phi_b, ghosts_lvl<T>(g, 0), ghosts_lvl<T>(g, 1)};
        k_diag_partial<T, false><<<nb, kDiagThreads, 0, g->stream>>>(v, q, partials);
    }
    k_diag_final<<<1, kDiagThreads, 0, g->stream>>>(partials, nb, dev_dst, g->step, (double)g->step * g->desc.dt);
    g->launches += 2;
    return cudaGetLastError();
}

template cudaError_t diag_compute<double>(axp_grid *, axp_diag *);
template cudaError_t diag_compute<float>(axp_grid *, axp_diag *);
template cudaError_t diag_compute_rows<double>(axp_grid *, axp_diag *, int, int64_t, int64_t);
template cudaError_t diag_compute_rows<float>(axp_grid *, axp_diag *, int, int64_t, int64_t);

// ---------------------------------------------------------------------------
// Diagnostics for callers that cannot allocate device memory.
//
// The per-block partial sums and the result record live in file-scope static
// device arrays instead of a workspace, so this entry point needs no
// allocation at all.  Every GPU that loads the library holds these arrays
// (kNoallocBlocks x 7 doubles + one record, about 230 KB) until the process
// exits.  The arrays are shared by every call: each call rewrites all the
// partials it uses and the result record, so nothing carries over between
// calls, but calls that overlap on the GPU (other host threads or streams)
// race on the shared arrays.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoallocBlocks = 4096;         // partial sums: one block of 256 threads ...
constexpr int kNoallocCellsPerBlock = 2048;  // ... covers 2048 cells (8 per thread)
constexpr int64_t kNoallocMaxCells = (int64_t)kNoallocBlocks * kNoallocCellsPerBlock;  // 8,388,608
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocBlocks * kQ];
static __device__ __align__(256) axp_diag g_noalloc_result;

std::mutex g_noalloc_mutex;
double *g_noalloc_partials_addr[kNoallocMaxDevices];
axp_diag *g_noalloc_result_addr[kNoallocMaxDevices];

// Device addresses of the static arrays for the current device.  In host code
// the array names are host-side stand-ins, never device addresses, so the
// real addresses are looked up once per device with that device current.
cudaError_t noalloc_setup(int dev, double **partials, axp_diag **result)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_partials_addr[dev]) {
        void *p = nullptr, *r = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&r, g_noalloc_result);
        if (e != cudaSuccess) return e;
        g_noalloc_partials_addr[dev] = (double *)p;
        g_noalloc_result_addr[dev] = (axp_diag *)r;
    }
    *partials = g_noalloc_partials_addr[dev];
    *result = g_noalloc_result_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace axp

extern "C" axp_status axp_diagnostics_noalloc(const axp_grid_desc *desc, const double *const dev_fields[14],
                                              const double B_ext[3], const double E_ext[3], int64_t step,
                                              void *cuda_stream, axp_diag *host_out)
{
    using namespace axp;
    if (!desc || !dev_fields || !B_ext || !E_ext || !host_out) return AXP_E_INVAL;
    for (int f = 0; f < 14; f++)
        if (!dev_fields[f]) return AXP_E_INVAL;
    size_t ws = 0;
    const axp_status st = axp_workspace_bytes(desc, &ws);  // host-side validation only
    if (st != AXP_OK) return st;
    if (desc->precision != AXP_FP64) {
        fprintf(stderr, "axp_diagnostics_noalloc: only FP64 fields are accepted\n");
        return AXP_E_INVAL;
    }
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++)
            if (desc->axion_bc[a][s] == AXP_BC_OUTFLOW) {
                fprintf(stderr, "axp_diagnostics_noalloc: outflow faces need ghost planes; use axp_compute_diagnostics\n");
                return AXP_E_INVAL;
            }
    const int64_t N = desc->n[0] * desc->n[1] * desc->n[2];
    if (N > kNoallocMaxCells) {
        fprintf(stderr, "axp_diagnostics_noalloc: %lld cells exceed the maximum of %lld\n", (long long)N,
                (long long)kNoallocMaxCells);
        return AXP_E_INVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return AXP_E_CUDA;
    double *partials = nullptr;
    axp_diag *result = nullptr;
    if (noalloc_setup(dev, &partials, &result) != cudaSuccess) return AXP_E_CUDA;

    View<double> v;
    memset(&v, 0, sizeof(v));
    for (int f = 0; f < kFields; f++) v.f[f] = const_cast<double *>(dev_fields[f]);
    v.phi_cur = const_cast<double *>(dev_fields[12]);
    v.phi_b = const_cast<double *>(dev_fields[13]);
    for (int a = 0; a < 3; a++) {
        v.n[a] = desc->n[a];
        v.d[a] = desc->d[a];
        v.lo[a] = desc->lo[a];
        v.Bext[a] = B_ext[a];
        v.Eext[a] = E_ext[a];
        v.periodic[a] = desc->em_bc[a][0] == AXP_BC_PERIODIC;
        for (int s = 0; s < 2; s++) v.axbc[a][s] = desc->axion_bc[a][s];
        int rlo = 0, rhi = (int)desc->n[a];
        if (desc->n[a] > 1 && !v.periodic[a]) {
            if (desc->em_bc[a][0] == AXP_BC_PML || desc->axion_bc[a][0] == AXP_BC_PML) rlo = desc->pml_cells;
            if (desc->em_bc[a][1] == AXP_BC_PML || desc->axion_bc[a][1] == AXP_BC_PML) rhi = (int)desc->n[a] - desc->pml_cells;
        }
        v.region_lo[a] = rlo;
        v.region_hi[a] = rhi;
    }
    v.N = N;
    v.dt = desc->dt;
    v.h = desc->dt / 2.0;
    v.g = desc->g;
    v.m2 = desc->m * desc->m;
    set_reciprocals(v);
    PhiPair<double, false> q;
    memset(&q, 0, sizeof(q));
    q.hi = v.phi_cur;
    q.b = v.phi_b;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int nb = (int)((N + kNoallocCellsPerBlock - 1) / kNoallocCellsPerBlock);
    if (nb < 1) nb = 1;
    k_diag_partial<double, false><<<nb, kDiagThreads, 0, stream>>>(v, q, partials);
    k_diag_final<<<1, kDiagThreads, 0, stream>>>(partials, nb, result, step, (double)step * desc->dt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, result, sizeof(axp_diag), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        fprintf(stderr, "axp: CUDA error %s\n", cudaGetErrorString(e));
        return AXP_E_CUDA;
    }
    const double vals[] = {host_out->H_phi, host_out->H_g0, host_out->H_g1, host_out->W, host_out->gauss_l2};
    for (double x : vals)
        if (!std::isfinite(x)) return AXP_E_NONFINITE;
    return AXP_OK;
}


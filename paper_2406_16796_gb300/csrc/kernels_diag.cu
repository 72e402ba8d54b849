// kernels_diag.cu -- FP64 diagnostics (arXiv 2406.16796 Sec. 3.2-3.4 energy
// densities, conversion probabilities and laser centroid; Sec. 2.2 Gauss law).
//
// Deterministic two-stage reduction: a fixed grid of blocks writes one FP64
// partial per quantity per block (fixed tree order inside the block), then one
// block sums the partials in fixed order.  The result depends only on the
// grid size, never on scheduling, so a grid's diagnostics are bit-identical
// however the work around it is arranged.
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
        for (int a = 0; a < 3; a++) {
            int64_t u[3];
            unit(a, u);
            const double up = (double)phi_mid<T, INCR>(v, q, i + u[0], j + u[1], k + u[2]);
            const double dn = (double)phi_mid<T, INCR>(v, q, i - u[0], j - u[1], k - u[2]);
            const double fw = (up - mid) / (double)v.d[a];
            g2 += fw * fw;
            const T *E1 = v.f[kE1 + a];
            R += ((double)E1[c] - (double)ld(v, E1, i - u[0], j - u[1], k - u[2])) / (double)v.d[a];
            bg += (double)b0_bar(v, a, i, j, k) * ((up - dn) / (2.0 * (double)v.d[a]));
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
    // staggered (fused-path) state: reconstruct E^n into the spare field set first
    View<T> v;
    if (g->staggered) {
        const cudaError_t e = exit_staggered<T>(g, false);
        if (e != cudaSuccess) return e;
        v = make_view_eset<T>(g, 1 - g->fset);
    } else {
        v = make_view<T>(g);
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

}  // namespace axp

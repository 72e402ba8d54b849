// kernels_init.cu -- initial conditions: laser placement and axion seeding.
//
// Laser: E0 = A pol env cos(k.(x - x_c) + phase) at integer time 0 and
// B0 = curl_h(pol F), F = (A / cos(theta/2)) env sin(...) / |K|, the discrete
// eigenmode of the half-step Yee scheme for a CW wave (B divergence-free by
// construction).  Axion: phi at t = +dt/2 and -dt/2, as arXiv 2406.16796
// Sec. 3.1 seeds its test pulse, with the discrete Klein-Gordon frequency.
// All profiles are evaluated in double and rounded once to the storage type.
#include "device_common.cuh"

namespace axp {
namespace {

struct Wave {
    double amp, k[3], dir[3], centre[3], waist, len, shift, phase, w, t;
    double pol[3];
    double fscale;  // laser: A / (cos(theta/2) |K|)
};

__device__ double envelope(const Wave &W, const double x[3], double shift)
{
    const double dx0 = x[0] - W.centre[0], dx1 = x[1] - W.centre[1], dx2 = x[2] - W.centre[2];
    const double xi = W.dir[0] * dx0 + W.dir[1] * dx1 + W.dir[2] * dx2;
    const double r2 = dx0 * dx0 + dx1 * dx1 + dx2 * dx2 - xi * xi;
    double e = 1.0;
    if (W.waist > 0) e *= exp(-r2 / (W.waist * W.waist));
    if (W.len > 0) e *= exp(-((xi - shift) * (xi - shift)) / (W.len * W.len));
    return e;
}

__device__ double phase_of(const Wave &W, const double x[3])
{
    return W.k[0] * (x[0] - W.centre[0]) + W.k[1] * (x[1] - W.centre[1]) + W.k[2] * (x[2] - W.centre[2]) + W.phase;
}

// Position of sample (i,j,k) of a staggered quantity: kind 0 = cell centre, 1 = E_a.
template <typename T>
__device__ void pos_of(const View<T> &v, const double lo[3], const double d[3], int kind, int a, int64_t i,
                       int64_t j, int64_t k, double x[3])
{
    const int64_t c[3] = {i, j, k};
    for (int b = 0; b < 3; b++) x[b] = lo[b] + ((double)c[b] + ((kind == 1 && b == a) ? 1.0 : 0.5)) * d[b];
}

// F_a at E-sample (i,j,k) with the field closure: periodic wrap, zero outside.
template <typename T>
__device__ double laser_F(const View<T> &v, const Wave &W, const double lo[3], const double d[3], int a, int64_t i,
                          int64_t j, int64_t k)
{
    if (W.pol[a] == 0.0) return 0.0;
    const int64_t c = lin_em(v, i, j, k);
    if (c < 0) return 0.0;
    int64_t ii, jj, kk;
    cell_of(c, v.n, &ii, &jj, &kk);
    double x[3];
    pos_of(v, lo, d, 1, a, ii, jj, kk, x);
    return W.fscale * W.pol[a] * envelope(W, x, 0.0) * sin(phase_of(W, x));
}

template <typename T>
__global__ void k_laser(View<T> v, Wave W, double lo0, double lo1, double lo2, double d0, double d1, double d2)
{
    const double lo[3] = {lo0, lo1, lo2}, d[3] = {d0, d1, d2};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < v.N; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        cell_of(c, v.n, &i, &j, &k);
        for (int a = 0; a < 3; a++) {
            if (W.pol[a] == 0.0) continue;
            double x[3];
            pos_of(v, lo, d, 1, a, i, j, k, x);
            const double e = W.amp * W.pol[a] * envelope(W, x, 0.0) * cos(phase_of(W, x));
            v.f[kE0 + a][c] = (T)((double)v.f[kE0 + a][c] + e);
        }
        // B = curl_h(pol F): forward differences as for curl E
        const double bx = (laser_F(v, W, lo, d, 2, i, j + 1, k) - laser_F(v, W, lo, d, 2, i, j, k)) / d1 -
                          (laser_F(v, W, lo, d, 1, i, j, k + 1) - laser_F(v, W, lo, d, 1, i, j, k)) / d2;
        const double by = (laser_F(v, W, lo, d, 0, i, j, k + 1) - laser_F(v, W, lo, d, 0, i, j, k)) / d2 -
                          (laser_F(v, W, lo, d, 2, i + 1, j, k) - laser_F(v, W, lo, d, 2, i, j, k)) / d0;
        const double bz = (laser_F(v, W, lo, d, 1, i + 1, j, k) - laser_F(v, W, lo, d, 1, i, j, k)) / d0 -
                          (laser_F(v, W, lo, d, 0, i, j + 1, k) - laser_F(v, W, lo, d, 0, i, j, k)) / d1;
        v.f[kB0][c] = (T)((double)v.f[kB0][c] + bx);
        v.f[kB0 + 1][c] = (T)((double)v.f[kB0 + 1][c] + by);
        v.f[kB0 + 2][c] = (T)((double)v.f[kB0 + 2][c] + bz);
    }
}

__device__ double axion_at(const Wave &W, const double x[3], double t)
{
    return W.amp * envelope(W, x, W.shift * t) * sin(phase_of(W, x) - W.w * t);
}

template <typename T, bool INCR>
__global__ void k_axion_seed(View<T> v, Wave W, double dt, double lo0, double lo1, double lo2, double d0, double d1,
                             double d2)
{
    const double lo[3] = {lo0, lo1, lo2}, d[3] = {d0, d1, d2};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < v.N; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        cell_of(c, v.n, &i, &j, &k);
        double x[3];
        pos_of(v, lo, d, 0, 0, i, j, k, x);
        const double p = axion_at(W, x, 0.5 * dt), q = axion_at(W, x, -0.5 * dt);
        v.phi_cur[c] = (T)((double)v.phi_cur[c] + p);
        if (INCR)
            v.phi_b[c] = (T)((double)v.phi_b[c] + (p - q));
        else
            v.phi_b[c] = (T)((double)v.phi_b[c] + q);
    }
}

template <typename T>
__global__ void k_axion_seed_ghost(View<T> v, Wave W, double dt, int ax, int side, T *g_cur, T *g_old, double lo0,
                                   double lo1, double lo2, double d0, double d1, double d2)
{
    const double lo[3] = {lo0, lo1, lo2}, d[3] = {d0, d1, d2};
    const int b = (ax + 1) % 3, cc = (ax + 2) % 3;
    const int64_t nb = v.n[b], nc = v.n[cc];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb * nc; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ca[3];
        ca[b] = t % nb;
        ca[cc] = t / nb;
        ca[ax] = side ? v.n[ax] : -1;
        double x[3];
        pos_of(v, lo, d, 0, 0, ca[0], ca[1], ca[2], x);
        const int64_t pi = ax == 0 ? ca[1] + v.n[1] * ca[2] : (ax == 1 ? ca[0] + v.n[0] * ca[2] : ca[0] + v.n[0] * ca[1]);
        g_cur[pi] = (T)((double)g_cur[pi] + axion_at(W, x, 0.5 * dt));
        g_old[pi] = (T)((double)g_old[pi] + axion_at(W, x, -0.5 * dt));
    }
}

inline int blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t inject_laser(axp_grid *g, const axp_laser_desc &L)
{
    const axp_grid_desc &D = g->desc;
    Wave W{};
    double K2 = 0, kk = 0;
    for (int a = 0; a < 3; a++) {
        const double Ka = (2.0 / D.d[a]) * sin(L.k[a] * D.d[a] / 2.0);
        K2 += Ka * Ka;
        kk += L.k[a] * L.k[a];
        W.k[a] = L.k[a];
        W.pol[a] = L.pol[a];
        W.centre[a] = L.centre[a];
    }
    const double Kmag = sqrt(K2), kmag = sqrt(kk);
    if (!(Kmag > 0)) return cudaErrorInvalidValue;
    const double sh = D.dt * Kmag / 2.0;
    const double ch = sqrt(1.0 - sh * sh);
    for (int a = 0; a < 3; a++) W.dir[a] = L.k[a] / kmag;
    W.amp = L.amplitude;
    W.waist = L.waist;
    W.len = L.duration > 0 ? L.duration / sqrt(2.0 * log(2.0)) : 0.0;
    W.phase = L.phase;
    W.fscale = L.amplitude / (ch * Kmag);
    View<T> v = make_view<T>(g);
    k_laser<T><<<blocks_for(v.N), 256, 0, g->stream>>>(v, W, lo_of(g, 0), lo_of(g, 1), lo_of(g, 2), D.d[0], D.d[1], D.d[2]);
    g->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t inject_axion(axp_grid *g, const axp_axion_desc &A)
{
    const axp_grid_desc &D = g->desc;
    Wave W{};
    double K2 = 0, kk = 0;
    for (int a = 0; a < 3; a++) {
        const double Ka = (2.0 / D.d[a]) * sin(A.k[a] * D.d[a] / 2.0);
        K2 += Ka * Ka;
        kk += A.k[a] * A.k[a];
        W.k[a] = A.k[a];
        W.centre[a] = A.centre[a];
    }
    const double cw = 1.0 - D.dt * D.dt * (K2 + D.m * D.m) / 2.0;
    W.w = acos(cw) / D.dt;
    const double kmag = sqrt(kk);
    for (int a = 0; a < 3; a++) W.dir[a] = kmag > 0 ? A.k[a] / kmag : 0.0;
    W.amp = A.amplitude;
    W.waist = A.waist;
    W.len = A.length;
    W.shift = A.speed;
    W.phase = A.phase;
    View<T> v = make_view<T>(g);
    if (D.precision == AXP_FP32_SPLIT)
        k_axion_seed<T, true><<<blocks_for(v.N), 256, 0, g->stream>>>(v, W, D.dt, lo_of(g, 0), lo_of(g, 1), lo_of(g, 2), D.d[0],
                                                                       D.d[1], D.d[2]);
    else
        k_axion_seed<T, false><<<blocks_for(v.N), 256, 0, g->stream>>>(v, W, D.dt, lo_of(g, 0), lo_of(g, 1), lo_of(g, 2), D.d[0],
                                                                        D.d[1], D.d[2]);
    g->launches++;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) {
            if (D.axion_bc[a][s] != AXP_BC_OUTFLOW) continue;
            T *gc = (T *)(g->ws + g->layout.off_ghost[a][s][g->ghost_level_slot[0]]);
            T *go = (T *)(g->ws + g->layout.off_ghost[a][s][g->ghost_level_slot[1]]);
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            k_axion_seed_ghost<T><<<blocks_for(D.n[b] * D.n[c]), 256, 0, g->stream>>>(
                v, W, D.dt, a, s, gc, go, lo_of(g, 0), lo_of(g, 1), lo_of(g, 2), D.d[0], D.d[1], D.d[2]);
            g->launches++;
        }
    return cudaGetLastError();
}

template cudaError_t inject_laser<double>(axp_grid *, const axp_laser_desc &);
template cudaError_t inject_laser<float>(axp_grid *, const axp_laser_desc &);
template cudaError_t inject_axion<double>(axp_grid *, const axp_axion_desc &);
template cudaError_t inject_axion<float>(axp_grid *, const axp_axion_desc &);

}  // namespace axp

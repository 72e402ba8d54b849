// kernels_general.cu -- the general multi-pass step (arXiv 2406.16796 Sec. 2.3-2.4).
//
// One kernel per stage of the half-step scheme, one thread per cell, every
// stencil access through the boundary-aware accessors of device_common.cuh.
// Covers every dimension, boundary kind and field component.  Each stage
// evaluates its expressions in the order the scheme states them; this
// translation unit is compiled without multiply-add contraction, so the FP64
// instantiation reproduces a literal double-precision evaluation of the scheme.
//
// Stage order of one step n -> n+1 (order 0 always before order 1):
//   [J^n if not cached] -> E half (both orders, J^n) -> B half (both orders)
//   -> S^{n+1/2} and phi^{n+3/2} (PML form in the layer) -> outflow ghosts
//   -> B half (both orders) -> E0 half -> J^{n+1} -> E1 half (J^{n+1}).
#include <utility>
#include "device_common.cuh"

namespace axp {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work)
{
    int64_t b = (work + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// P_a = (D_t phi) Bbar0_a - (Ebar0 x grad_c phi)_a at one cell centre, (a, b, c) cyclic.
template <typename T, bool INCR>
__device__ T p_comp(const View<T> &v, const PhiPair<T, INCR> &q, int a, int64_t i, int64_t j, int64_t k)
{
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    int64_t ub[3], uc[3];
    unit(b, ub);
    unit(c, uc);
    T mid, Dt;
    phi_mid_dt<T, INCR>(v, q, i, j, k, &mid, &Dt);
    const T dphi_c = over_2d(v,
                             phi_mid<T, INCR>(v, q, i + uc[0], j + uc[1], k + uc[2]) -
                                 phi_mid<T, INCR>(v, q, i - uc[0], j - uc[1], k - uc[2]),
                             c);
    const T dphi_b = over_2d(v,
                             phi_mid<T, INCR>(v, q, i + ub[0], j + ub[1], k + ub[2]) -
                                 phi_mid<T, INCR>(v, q, i - ub[0], j - ub[1], k - ub[2]),
                             b);
    const T cross = e0_bar(v, b, i, j, k) * dphi_c - e0_bar(v, c, i, j, k) * dphi_b;
    return Dt * b0_bar(v, a, i, j, k) - cross;
}

template <typename T>
struct PBuf {
    T *p[3];
};

// Soft-source sheet for one half-step (Sec. 3.2 injection, read as a pair of
// current sheets on an x-plane): the plane index (-1: no source), the sheet
// weights A pol_a f/dx of E_y, E_z over (j, k), and the incident wave's factor
// tau at this half-step's position and time.
template <typename T>
struct Sheet {
    int64_t plane;
    const T *w[2];
    T tau;
};

template <typename T>
Sheet<T> sheet_at(const axp_grid *g, double x, double t)
{
    Sheet<T> s;
    s.plane = g->src_on ? g->src.plane : -1;
    s.w[0] = (const T *)(g->ws + g->layout.off_src[0]);
    s.w[1] = (const T *)(g->ws + g->layout.off_src[1]);
    s.tau = g->src_on ? (T)source_wave(g, x, t) : T(0);
    return s;
}
// the electric sheet reads B at time t; the magnetic sheet E at t_{n+1/2}
template <typename T>
Sheet<T> e_sheet(const axp_grid *g, double t)
{
    return sheet_at<T>(g, g->src_on ? source_x_b(g) : 0.0, t);
}
template <typename T>
Sheet<T> b_sheet(const axp_grid *g, double t)
{
    return sheet_at<T>(g, g->src_on ? source_x_e(g) : 0.0, t);
}

// P at every cell centre, into scratch (one evaluation per cell and component).
// Each stage's work at one cell is a device function; the general kernels loop
// it over the grid, and the time-blocked 1D kernel over a window in shared memory.
template <typename T, bool INCR>
__device__ __forceinline__ void pcell_at(const View<T> &v, const PhiPair<T, INCR> &q, const PBuf<T> &P, int64_t c,
                                         int64_t i, int64_t j, int64_t k)
{
    for (int a = 0; a < 3; a++) P.p[a][c] = p_comp<T, INCR>(v, q, a, i, j, k);
}

// The same three components at a cell of a 2D grid (one cell along z,
// periodic) whose x and y neighbours all lie inside the grid: every accessor of
// p_comp then reads the array element itself (a z neighbour is the cell), so
// the loads are taken directly and the expressions are p_comp's, in its order.
template <typename T, bool INCR>
__device__ __forceinline__ void pcell_interior_2d(const View<T> &v, const PhiPair<T, INCR> &q, const PBuf<T> &P,
                                                  int64_t c)
{
    const int64_t sy = v.n[0];
    auto mid_dt = [&](int64_t x, T *mid, T *dtv) {
        const T hi = q.hi[x];
        if (INCR) {
            const T inc = q.b[x];
            *mid = hi - T(0.5) * inc;
            *dtv = inc / v.dt;
            return;
        }
        const T lo = q.b[x];
        *mid = T(0.5) * (hi + lo);
        *dtv = (hi - lo) / v.dt;
    };
    auto mid_of = [&](int64_t x) {
        T m, t;
        mid_dt(x, &m, &t);
        return m;
    };
    T mid, Dt;
    mid_dt(c, &mid, &Dt);
    // central differences of phi^n: along z the two neighbours are the cell itself
    const T dx = over_2d(v, mid_of(c + 1) - mid_of(c - 1), 0);
    const T dy = over_2d(v, mid_of(c + sy) - mid_of(c - sy), 1);
    const T dz = over_2d(v, mid - mid, 2);
    const T *E0x = v.f[kE0], *E0y = v.f[kE0 + 1], *E0z = v.f[kE0 + 2];
    const T *B0x = v.f[kB0], *B0y = v.f[kB0 + 1], *B0z = v.f[kB0 + 2];
    const T ex = T(0.5) * (E0x[c] + E0x[c - 1]) + v.Eext[0];
    const T ey = T(0.5) * (E0y[c] + E0y[c - sy]) + v.Eext[1];
    const T ez = T(0.5) * (E0z[c] + E0z[c]) + v.Eext[2];
    T s;
    s = B0x[c];
    s = s + B0x[c];
    s = s + B0x[c - sy];
    s = s + B0x[c - sy];
    const T bx = T(0.25) * s + v.Bext[0];
    s = B0y[c];
    s = s + B0y[c - 1];
    s = s + B0y[c];
    s = s + B0y[c - 1];
    const T by = T(0.25) * s + v.Bext[1];
    s = B0z[c];
    s = s + B0z[c - sy];
    s = s + B0z[c - 1];
    s = s + B0z[c - 1 - sy];
    const T bz = T(0.25) * s + v.Bext[2];
    // P_a = Dt Bbar_a - (Ebar_b dphi_c - Ebar_c dphi_b), (a, b, c) cyclic
    P.p[0][c] = Dt * bx - (ey * dz - ez * dy);
    P.p[1][c] = Dt * by - (ez * dx - ex * dz);
    P.p[2][c] = Dt * bz - (ex * dy - ey * dx);
}

template <typename T, bool INCR>
__global__ void __launch_bounds__(kThreads) k_pcell(View<T> v, PhiPair<T, INCR> q, PBuf<T> P)
{
    const bool flat = v.n[2] == 1 && v.periodic[2] && v.n[0] >= 3 && v.n[1] >= 3;
    for (int64_t qv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qv < v.Nv; qv += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        const int64_t c = visit(v, qv, &i, &j, &k);
        if (flat && i >= 1 && i <= v.n[0] - 2 && j >= 1 && j <= v.n[1] - 2)
            pcell_interior_2d<T, INCR>(v, q, P, c);
        else
            pcell_at<T, INCR>(v, q, P, c, i, j, k);
    }
}

// J_a(c + a/2) = (P_a(c) + P_a(c + a)) / 2, all three components; P(c + a) comes
// from the scratch where c + a is a grid cell (its periodic image included) and
// is evaluated in place beyond a non-periodic edge (ghost rules).
template <typename T, bool INCR>
__device__ __forceinline__ void current_at(const View<T> &v, const PhiPair<T, INCR> &q, const PBuf<T> &P, int64_t c,
                                           int64_t i, int64_t j, int64_t k)
{
    for (int a = 0; a < 3; a++) {
        int64_t u[3];
        unit(a, u);
        const T p0 = P.p[a][c];
        int64_t w[3] = {i + u[0], j + u[1], k + u[2]};
        bool in = true;
        if (w[a] >= v.n[a]) {
            // the periodic image is the same evaluation only when both the fields
            // and the axion wrap along a
            if (v.periodic[a] && v.axbc[a][0] == AXP_BC_PERIODIC && v.axbc[a][1] == AXP_BC_PERIODIC)
                w[a] -= v.n[a];
            else
                in = false;
        }
        const T p1 = in ? P.p[a][lin3(v.n, w[0], w[1], w[2])] : p_comp<T, INCR>(v, q, a, w[0], w[1], w[2]);
        v.J[a][c] = T(0.5) * (p0 + p1);
    }
}

template <typename T, bool INCR>
__global__ void __launch_bounds__(kThreads) k_current(View<T> v, PhiPair<T, INCR> q, PBuf<T> P)
{
    for (int64_t qv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qv < v.Nv; qv += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        const int64_t c = visit(v, qv, &i, &j, &k);
        current_at<T, INCR>(v, q, P, c, i, j, k);
    }
}

// (curl B)_a at the E_a location: backward differences.
template <typename T>
__device__ __forceinline__ T curl_b(const View<T> &v, T *const B[3], int a, int64_t i, int64_t j, int64_t k)
{
    if (a == 0)
        return over_d(v, ld(v, B[2], i, j, k) - ld(v, B[2], i, j - 1, k), 1) -
               over_d(v, ld(v, B[1], i, j, k) - ld(v, B[1], i, j, k - 1), 2);
    if (a == 1)
        return over_d(v, ld(v, B[0], i, j, k) - ld(v, B[0], i, j, k - 1), 2) -
               over_d(v, ld(v, B[2], i, j, k) - ld(v, B[2], i - 1, j, k), 0);
    return over_d(v, ld(v, B[1], i, j, k) - ld(v, B[1], i - 1, j, k), 0) -
           over_d(v, ld(v, B[0], i, j, k) - ld(v, B[0], i, j - 1, k), 1);
}

// (curl E)_a at the B_a location: forward differences.
template <typename T>
__device__ __forceinline__ T curl_e(const View<T> &v, T *const E[3], int a, int64_t i, int64_t j, int64_t k)
{
    if (a == 0)
        return over_d(v, ld(v, E[2], i, j + 1, k) - ld(v, E[2], i, j, k), 1) -
               over_d(v, ld(v, E[1], i, j, k + 1) - ld(v, E[1], i, j, k), 2);
    if (a == 1)
        return over_d(v, ld(v, E[0], i, j, k + 1) - ld(v, E[0], i, j, k), 2) -
               over_d(v, ld(v, E[2], i + 1, j, k) - ld(v, E[2], i, j, k), 0);
    return over_d(v, ld(v, E[1], i + 1, j, k) - ld(v, E[1], i, j, k), 0) -
           over_d(v, ld(v, E[0], i, j + 1, k) - ld(v, E[0], i, j, k), 1);
}

// E half-step: orders selected by the mask (bit 0 = order 0, bit 1 = order 1);
// order 1 includes the axion current: X = curl B1 - g J.
// Order 0 may carry the electric sheet: E_y, E_z of the cells at the plane add
// w tau to their curl.
template <typename T>
__device__ __forceinline__ void e_half_at(const View<T> &v, int orders, const Sheet<T> &s, int64_t c, int64_t i,
                                          int64_t j, int64_t k)
{
    const T sig = sigma_of<T>(v.sig_em, i, j, k);
    if (orders & 1) {
        T *const B[3] = {v.f[kB0], v.f[kB0 + 1], v.f[kB0 + 2]};
        for (int a = 0; a < 3; a++) {
            T X = curl_b(v, B, a, i, j, k);
            if (i == s.plane && a > 0) X = X + s.w[a - 1][j + v.n[1] * k] * s.tau;
            if (v.jp[0][a]) X = X - v.jp[0][a][c];  // macroparticle current j0 (Ampere's law)
            v.f[kE0 + a][c] = half_update(v.f[kE0 + a][c], X, sig, v.h);
        }
    }
    if (orders & 2) {
        T *const B[3] = {v.f[kB1], v.f[kB1 + 1], v.f[kB1 + 2]};
        for (int a = 0; a < 3; a++) {
            T X = curl_b(v, B, a, i, j, k);
            X = X - v.g * v.J[a][c];
            if (v.jp[1][a]) X = X - v.jp[1][a][c];  // first-order particle current j1
            v.f[kE1 + a][c] = half_update(v.f[kE1 + a][c], X, sig, v.h);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_e_half(View<T> v, int orders, Sheet<T> s)
{
    for (int64_t qv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qv < v.Nv; qv += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        const int64_t c = visit(v, qv, &i, &j, &k);
        e_half_at<T>(v, orders, s, c, i, j, k);
    }
}

// B half-step of both orders: B <- B - h curl E.  Order 0 may carry the magnetic
// sheet on the faces at the plane (index plane - 1): B_y adds -w_z tau, B_z +w_y tau.
template <typename T>
__device__ __forceinline__ void b_half_at(const View<T> &v, const Sheet<T> &s, int64_t c, int64_t i, int64_t j,
                                          int64_t k)
{
    const T sig = sigma_of<T>(v.sig_em, i, j, k);
    T *const E0[3] = {v.f[kE0], v.f[kE0 + 1], v.f[kE0 + 2]};
    T *const E1[3] = {v.f[kE1], v.f[kE1 + 1], v.f[kE1 + 2]};
    for (int a = 0; a < 3; a++) {
        T X = -curl_e(v, E0, a, i, j, k);
        if (i == s.plane - 1 && a > 0) {
            const int64_t jk = j + v.n[1] * k;
            X = X + (a == 1 ? -(s.w[1][jk] * s.tau) : s.w[0][jk] * s.tau);
        }
        v.f[kB0 + a][c] = half_update(v.f[kB0 + a][c], X, sig, v.h);
    }
    for (int a = 0; a < 3; a++) v.f[kB1 + a][c] = half_update(v.f[kB1 + a][c], -curl_e(v, E1, a, i, j, k), sig, v.h);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_b_half(View<T> v, Sheet<T> s)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < v.N; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        cell_of(c, v.n, &i, &j, &k);
        b_half_at<T>(v, s, c, i, j, k);
    }
}

// Axion leapfrog (Eq. update_axion) with the source S^{n+1/2} = g Ebar0 . Bbar0,
// and the damped form of Sec. 2.4 item 4 inside the PML.
//   FP64 (two levels): phi^{n+3/2} is written over phi^{n-1/2}.
//   FP32 split: pi^{n+1} = phi^{n+3/2} - phi^{n+1/2} replaces pi^n in place and
//   phi^{n+3/2} = phi^{n+1/2} + pi^{n+1} goes to phi_next.
template <typename T, bool INCR>
__device__ __forceinline__ void axion_at(const View<T> &v, const Ghosts<T> &gcur, T dt2, int64_t c, int64_t i,
                                         int64_t j, int64_t k)
{
    {
        const T S = source_at(v, i, j, k);
        const T ph = v.phi_cur[c];
        T lap = T(0);
        for (int a = 0; a < 3; a++) {
            int64_t u[3];
            unit(a, u);
            const T up = ld_phi(v, v.phi_cur, gcur, i + u[0], j + u[1], k + u[2]);
            const T dn = ld_phi(v, v.phi_cur, gcur, i - u[0], j - u[1], k - u[2]);
            // FP32 split: from neighbour differences, which do not round against 2*phi
            const T d2 = INCR ? (up - ph) + (dn - ph) : (up + dn) - T(2) * ph;
            lap = lap + over_dd(v, d2, a);
        }
        const T sig = sigma_of<T>(v.sig_ax, i, j, k);
        if (!INCR) {
            const T old = v.phi_b[c];
            T nw;
            if (sig == T(0)) {
                nw = T(2) * ph - old + dt2 * ((lap - v.m2 * ph) + S);
            } else {
                const T Y = ((S - v.m2 * ph) + lap) - sig * sig * ph;
                nw = (dt2 * Y + sig * v.dt * old + T(2) * ph - old) / (T(1) + sig * v.dt);
            }
            v.phi_b[c] = nw;
        } else {
            const T inc = v.phi_b[c];
            T nin;
            if (sig == T(0)) {
                nin = inc + dt2 * ((lap - v.m2 * ph) + S);
            } else {
                const T Y = ((S - v.m2 * ph) + lap) - sig * sig * ph;
                nin = (dt2 * Y + (T(1) - sig * v.dt) * inc) / (T(1) + sig * v.dt);
            }
            v.phi_b[c] = nin;
            v.phi_next[c] = ph + nin;
        }
    }
}

template <typename T, bool INCR>
__global__ void __launch_bounds__(kThreads) k_axion(View<T> v, Ghosts<T> gcur)
{
    const T dt2 = v.dt * v.dt;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < v.N; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        cell_of(c, v.n, &i, &j, &k);
        axion_at<T, INCR>(v, gcur, dt2, c, i, j, k);
    }
}

// Outflow ghosts at the new level for one face (Sec. 2.4 item 3): solve the
// one-way wave equation and the wave equation at the ghost for
// V = phi^{cur}_{-3/2} and U = phi^{new}_{-1/2}.
template <typename T>
__global__ void k_outflow(View<T> v, int ax, int side, const T *g_cur, const T *g_old, T *g_new)
{
    const int b = (ax + 1) % 3, cc = (ax + 2) % 3;
    const int64_t nb = v.n[b], nc = v.n[cc];
    const T r = v.dt / v.d[ax];
    const T r2 = (v.dt * v.dt) / (v.d[ax] * v.d[ax]);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb * nc; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ca[3];
        ca[b] = t % nb;
        ca[cc] = t / nb;
        ca[ax] = side ? v.n[ax] : -1;
        const int64_t pi = ax == 0 ? ca[1] + v.n[1] * ca[2] : (ax == 1 ? ca[0] + v.n[0] * ca[2] : ca[0] + v.n[0] * ca[1]);
        const T Sg = source_at(v, ca[0], ca[1], ca[2]);
        int64_t ci[3] = {ca[0], ca[1], ca[2]};
        ci[ax] = side ? v.n[ax] - 1 : 0;
        const T p0 = v.phi_cur[lin3(v.n, ci[0], ci[1], ci[2])];
        const T gc = g_cur[pi], go = g_old[pi];
        const T rhs = T(-2) * gc + T(2) * go - (v.dt * v.dt) * (Sg - v.m2 * gc) + r * p0 - r2 * (p0 - T(2) * gc);
        const T V = rhs / (r + r2);
        g_new[pi] = go + r * (p0 - V);
    }
}

// Inverse of half_update: the field a half-step h earlier, given X.
template <typename T>
__device__ __forceinline__ T half_inverse(T Fh, T X, T sig, T h)
{
    if (sig == T(0)) return Fh - h * X;
    return ((T(1) + sig * h / T(2)) * Fh - h * X) / (T(1) - sig * h / T(2));
}

template <typename T>
struct EOut {
    T *p[3];
};

// E^n from E^{n+1/2} of one order: E^n = E^{n+1/2} - h (curl B^n - g J^n) (order 1)
// or - h curl B^n (order 0), written to `out` (which may alias the input).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_e_unhalf(View<T> v, int order, EOut<T> out, Sheet<T> s)
{
    for (int64_t qv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qv < v.Nv; qv += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        const int64_t c = visit(v, qv, &i, &j, &k);
        const T sig = sigma_of<T>(v.sig_em, i, j, k);
        const int fb = order ? kB1 : kB0, fe = order ? kE1 : kE0;
        T *const B[3] = {v.f[fb], v.f[fb + 1], v.f[fb + 2]};
        for (int a = 0; a < 3; a++) {
            T X = curl_b(v, B, a, i, j, k);
            if (order) X = X - v.g * v.J[a][c];
            else if (i == s.plane && a > 0) X = X + s.w[a - 1][j + v.n[1] * k] * s.tau;
            out.p[a][c] = half_inverse(v.f[fe + a][c], X, sig, v.h);
        }
    }
}

// Moving window: dst = src shifted by s cells towards lower index along `axis`;
// the s cells entering at the high end are vacuum.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_shift(const T *__restrict__ src, T *__restrict__ dst, int64_t N,
                                                     int64_t stride, int64_t na, int64_t s)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ca = (c / stride) % na;
        dst[c] = ca + s < na ? src[c + s * stride] : T(0);
    }
}

}  // namespace

template <typename T>
static Ghosts<T> ghosts_at(axp_grid *g, int level)
{
    Ghosts<T> G;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) {
            const size_t off = g->layout.off_ghost[a][s][g->ghost_level_slot[level]];
            G.p[a][s] = off ? (T *)(g->ws + off) : nullptr;
        }
    return G;
}

template <typename T, bool INCR>
static cudaError_t launch_current(axp_grid *g, const View<T> &v, const T *hi, const T *b, int lev_hi, int lev_lo)
{
    PhiPair<T, INCR> q;
    q.hi = hi;
    q.b = b;
    q.ghi = ghosts_at<T>(g, lev_hi);
    q.glo = ghosts_at<T>(g, lev_lo);
    // P at the cell centres goes to its own workspace arrays (the field sets may
    // not be written: the fused kernels leave inactive arrays untouched, so any
    // value left in one would become part of the state)
    PBuf<T> P;
    for (int a = 0; a < 3; a++) P.p[a] = (T *)(g->ws + g->layout.off_P[a]);
    // J at a cell averages P there and one cell up along each axis: on a slab, P is
    // formed one cell further along the slab's axis
    View<T> vp = v;
    if (v.vaxis >= 0 && v.vhi < v.n[v.vaxis]) {
        vp.vhi = v.vhi + 1;
        vp.Nv = v.Nv / (v.vhi - v.vlo) * (vp.vhi - vp.vlo);
    }
    k_pcell<T, INCR><<<grid_for(vp.Nv), kThreads, 0, g->stream>>>(vp, q, P);
    k_current<T, INCR><<<grid_for(v.Nv), kThreads, 0, g->stream>>>(v, q, P);
    g->launches += 2;
    return cudaGetLastError();
}

template <typename T>
cudaError_t general_current(axp_grid *g)
{
    View<T> v = make_view<T>(g);
    if (g->desc.precision == AXP_FP32_SPLIT) return launch_current<T, true>(g, v, v.phi_cur, v.phi_b, 0, 1);
    return launch_current<T, false>(g, v, v.phi_cur, v.phi_b, 0, 1);
}

template <typename T>
cudaError_t general_step(axp_grid *g, int64_t nsteps)
{
    const bool incr = g->desc.precision == AXP_FP32_SPLIT;
    const int nb = grid_for(g->layout.total ? (int64_t)(g->desc.n[0] * g->desc.n[1] * g->desc.n[2]) : 1);
    for (int64_t it = 0; it < nsteps; it++) {
        cudaError_t e;
        if (!g->J_valid) {
            if ((e = general_current<T>(g)) != cudaSuccess) return e;
            g->J_valid = true;
        }
        View<T> v = make_view<T>(g);
        const Sheet<T> se0 = e_sheet<T>(g, time_n(g, g->step)), sb = b_sheet<T>(g, time_half(g, g->step));
        const Sheet<T> se1 = e_sheet<T>(g, time_n(g, g->step + 1));
        k_e_half<T><<<nb, kThreads, 0, g->stream>>>(v, 3, se0);
        k_b_half<T><<<nb, kThreads, 0, g->stream>>>(v, sb);
        Ghosts<T> gcur = ghosts_at<T>(g, 0);
        if (incr)
            k_axion<T, true><<<nb, kThreads, 0, g->stream>>>(v, gcur);
        else
            k_axion<T, false><<<nb, kThreads, 0, g->stream>>>(v, gcur);
        g->launches += 3;
        Ghosts<T> gold = ghosts_at<T>(g, 1), gnew = ghosts_at<T>(g, 2);
        for (int a = 0; a < 3; a++)
            for (int s = 0; s < 2; s++) {
                if (g->desc.axion_bc[a][s] != AXP_BC_OUTFLOW) continue;
                const int b = (a + 1) % 3, c = (a + 2) % 3;
                const int64_t plane = g->desc.n[b] * g->desc.n[c];
                k_outflow<T><<<grid_for(plane), kThreads, 0, g->stream>>>(v, a, s, gcur.p[a][s], gold.p[a][s],
                                                                           gnew.p[a][s]);
                g->launches++;
            }
        // macroparticles pushed by the fields of both orders at t_{n+1/2}; they
        // deposit j^{n+1}, which the second E half-steps (and the next step's first) read
        if constexpr (sizeof(T) == sizeof(double)) {
            if (g->parts && (e = particles_push(g, v)) != cudaSuccess) return e;
        }
        k_b_half<T><<<nb, kThreads, 0, g->stream>>>(v, sb);
        k_e_half<T><<<nb, kThreads, 0, g->stream>>>(v, 1, se1);
        g->launches += 2;
        // J^{n+1} from phi^{n+3/2} (hi) and phi^{n+1/2}
        if (incr) {
            e = launch_current<T, true>(g, v, v.phi_next, v.phi_b, 2, 0);
        } else {
            e = launch_current<T, false>(g, v, v.phi_b, v.phi_cur, 2, 0);
        }
        if (e != cudaSuccess) return e;
        k_e_half<T><<<nb, kThreads, 0, g->stream>>>(v, 2, se1);
        g->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // rotate the axion levels and the ghost planes
        if (incr) {
            const int t = g->phi_cur_slot;
            g->phi_cur_slot = g->phi_next_slot;
            g->phi_next_slot = t;
        } else {
            const int t = g->phi_cur_slot;
            g->phi_cur_slot = g->phi_b_slot;
            g->phi_b_slot = t;
        }
        const int s0 = g->ghost_level_slot[0], s1 = g->ghost_level_slot[1], s2 = g->ghost_level_slot[2];
        g->ghost_level_slot[0] = s2;
        g->ghost_level_slot[1] = s0;
        g->ghost_level_slot[2] = s1;
        g->step++;
        if (g->desc.diag_every > 0 && g->step % g->desc.diag_every == 0) {
            axp_diag *dst = ring_slot(g, g->ring_written);
            if ((e = diag_compute<T>(g, dst)) != cudaSuccess) return e;
            g->ring_written++;
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t enter_staggered(axp_grid *g)
{
    if (g->staggered) return cudaSuccess;
    g->half_prev = false;
    cudaError_t e = general_current<T>(g);
    if (e != cudaSuccess) return e;
    View<T> v = make_view<T>(g);
    const int nb = grid_for(v.N);
    k_e_half<T><<<nb, kThreads, 0, g->stream>>>(v, 3, e_sheet<T>(g, time_n(g, g->step)));
    g->launches++;
    g->staggered = true;
    g->J_valid = false;
    return cudaGetLastError();
}

template <typename T>
cudaError_t exit_staggered(axp_grid *g, bool in_place)
{
    if (!g->staggered) return cudaSuccess;
    g->half_prev = false;
    const int oset = in_place ? g->fset : 1 - g->fset;
    View<T> vin = make_view<T>(g);
    View<T> vout = make_view_eset<T>(g, oset);
    const int nb = grid_for(vin.N);
    EOut<T> o0{{vout.f[kE0], vout.f[kE0 + 1], vout.f[kE0 + 2]}};
    const Sheet<T> se = e_sheet<T>(g, time_n(g, g->step));
    k_e_unhalf<T><<<nb, kThreads, 0, g->stream>>>(vin, 0, o0, se);
    g->launches++;
    cudaError_t e;
    // J^n from E0^n (in vout), B0^n and the axion levels
    if (g->desc.precision == AXP_FP32_SPLIT)
        e = launch_current<T, true>(g, vout, vout.phi_cur, vout.phi_b, 0, 1);
    else
        e = launch_current<T, false>(g, vout, vout.phi_cur, vout.phi_b, 0, 1);
    if (e != cudaSuccess) return e;
    EOut<T> o1{{vout.f[kE1], vout.f[kE1 + 1], vout.f[kE1 + 2]}};
    k_e_unhalf<T><<<nb, kThreads, 0, g->stream>>>(vin, 1, o1, se);
    g->launches++;
    if (in_place) {
        g->staggered = false;
        g->J_valid = true;
    } else {
        g->J_valid = false;
    }
    return cudaGetLastError();
}

// View of the cells whose index along `axis` lies in [lo, hi).
template <typename T>
static View<T> slab_view(axp_grid *g, int axis, int64_t lo, int64_t hi)
{
    View<T> v = make_view<T>(g);
    v.vaxis = axis;
    v.vlo = lo;
    v.vhi = hi;
    v.Nv = v.N / g->desc.n[axis] * (hi - lo);
    return v;
}

template <typename T>
static cudaError_t slab_current(axp_grid *g, const View<T> &v)
{
    if (g->desc.precision == AXP_FP32_SPLIT) return launch_current<T, true>(g, v, v.phi_cur, v.phi_b, 0, 1);
    return launch_current<T, false>(g, v, v.phi_cur, v.phi_b, 0, 1);
}

// E^{n+1/2} -> E^n in place on a slab, the other cells left as they are.
template <typename T>
static cudaError_t exit_slab(axp_grid *g, int axis, int64_t lo, int64_t hi)
{
    const View<T> v = slab_view<T>(g, axis, lo, hi);
    const Sheet<T> se = e_sheet<T>(g, time_n(g, g->step));
    EOut<T> o0{{v.f[kE0], v.f[kE0 + 1], v.f[kE0 + 2]}};
    k_e_unhalf<T><<<grid_for(v.Nv), kThreads, 0, g->stream>>>(v, 0, o0, se);
    g->launches++;
    cudaError_t e = slab_current<T>(g, v);
    if (e != cudaSuccess) return e;
    EOut<T> o1{{v.f[kE1], v.f[kE1 + 1], v.f[kE1 + 2]}};
    k_e_unhalf<T><<<grid_for(v.Nv), kThreads, 0, g->stream>>>(v, 1, o1, se);
    g->launches++;
    return cudaGetLastError();
}

// E^n -> E^{n+1/2} in place on a slab.
template <typename T>
static cudaError_t enter_slab(axp_grid *g, int axis, int64_t lo, int64_t hi)
{
    const View<T> v = slab_view<T>(g, axis, lo, hi);
    cudaError_t e = slab_current<T>(g, v);
    if (e != cudaSuccess) return e;
    k_e_half<T><<<grid_for(v.Nv), kThreads, 0, g->stream>>>(v, 3, e_sheet<T>(g, time_n(g, g->step)));
    g->launches++;
    return cudaGetLastError();
}

// Moving-window shift of the staggered state (E^{n+1/2}, B^n, phi) without a
// round trip of the whole grid through integer time.  Away from the ends of the
// window axis the shift commutes with the local conversion E^{n+1/2} = E^n +
// h X(E0^n, B^n, phi) (X = curl B - g J, boundary closure included: the cells
// entering at the high end are vacuum, as the zero closure outside the grid
// was).  It does not commute where the absorbing layer's sigma differs between a
// cell's old and new position, nor at the low end, where a cell loses its lower
// neighbour.  So only the bands there go through integer time: the source
// bands are converted to E^n in place, everything is shifted, and the
// destination bands are converted back.  The bands reach r = 2 cells beyond the
// layers (the current's stencil) and m = 3 more; at a band's inner edge both
// conversions read the same (translated) neighbours outside the band, so they
// cancel there.  Returns false (and does nothing) where the bands would meet or
// a soft source is set (its sheet cells would need bands of their own): the
// caller then converts the whole grid.
template <typename T>
cudaError_t shift_staggered(axp_grid *g, int axis, int64_t s, bool *done)
{
    *done = false;
    const axp_grid_desc &d = g->desc;
    const int64_t n = d.n[axis];
    if (!g->staggered || g->src_on || s <= 0 || s >= n) return cudaSuccess;
    auto layer = [&](int side) -> int64_t {
        return (d.em_bc[axis][side] == AXP_BC_PML || d.axion_bc[axis][side] == AXP_BC_PML) ? d.pml_cells : 0;
    };
    const int64_t r = 2, m = 3;
    const int64_t d0_hi = layer(0) + r + m;          // destination band at the low end: [0, d0_hi)
    const int64_t d1_lo = n - layer(1) - s - r - m;  // at the high end, with the entering cells: [d1_lo, n)
    const int64_t s0_lo = std::max<int64_t>(0, s - r), s0_hi = d0_hi + s;  // their sources
    const int64_t s1_lo = d1_lo + s;
    if (d1_lo < d0_hi + 4 || s1_lo < s0_hi + 4) return cudaSuccess;
    cudaError_t e = exit_slab<T>(g, axis, s0_lo, s0_hi);
    if (e == cudaSuccess) e = exit_slab<T>(g, axis, s1_lo, n);
    if (e == cudaSuccess) e = shift_window<T>(g, axis, s);
    if (e == cudaSuccess) e = enter_slab<T>(g, axis, 0, d0_hi);
    if (e == cudaSuccess) e = enter_slab<T>(g, axis, d1_lo, n);
    g->J_valid = false;
    *done = e == cudaSuccess;
    return e;
}

// Shift the integer-time state (every field array and both axion levels) by s
// cells along `axis`, out of place into the spare field set and axion buffers.
template <typename T>
cudaError_t shift_window(axp_grid *g, int axis, int64_t s)
{
    const int64_t *n = g->desc.n;
    const int64_t N = n[0] * n[1] * n[2];
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n[0] : n[0] * n[1]);
    const int nb = grid_for(N);
    const Workspace &w = g->layout;
    const int in = g->fset, out = 1 - g->fset;
    auto at = [&](size_t off) { return (T *)(g->ws + off); };
    for (int f = 0; f < kFields; f++) {
        k_shift<T><<<nb, kThreads, 0, g->stream>>>(at(w.off_fields[in][f]), at(w.off_fields[out][f]), N, stride,
                                                  n[axis], s);
        g->launches++;
    }
    g->fset = out;
    const int cur = g->phi_cur_slot, b = g->phi_b_slot, nxt = g->phi_next_slot;
    k_shift<T><<<nb, kThreads, 0, g->stream>>>(at(w.off_phi[cur]), at(w.off_phi[nxt]), N, stride, n[axis], s);
    if (g->desc.precision == AXP_FP32_SPLIT) {
        const int nb2 = g->phi_next_b_slot;
        k_shift<T><<<nb, kThreads, 0, g->stream>>>(at(w.off_phi[b]), at(w.off_phi[nb2]), N, stride, n[axis], s);
        std::swap(g->phi_cur_slot, g->phi_next_slot);
        std::swap(g->phi_b_slot, g->phi_next_b_slot);
    } else {
        // three buffers: the second level goes into the buffer phi^{n+1/2} just left
        k_shift<T><<<nb, kThreads, 0, g->stream>>>(at(w.off_phi[b]), at(w.off_phi[cur]), N, stride, n[axis], s);
        g->phi_cur_slot = nxt;
        g->phi_b_slot = cur;
        g->phi_next_slot = b;
    }
    g->launches += 2;
    g->J_valid = false;
    return cudaGetLastError();
}

template cudaError_t shift_staggered<double>(axp_grid *, int, int64_t, bool *);
template cudaError_t shift_staggered<float>(axp_grid *, int, int64_t, bool *);
template cudaError_t shift_window<double>(axp_grid *, int, int64_t);
template cudaError_t shift_window<float>(axp_grid *, int, int64_t);
template cudaError_t enter_staggered<double>(axp_grid *);
template cudaError_t enter_staggered<float>(axp_grid *);
template cudaError_t exit_staggered<double>(axp_grid *, bool);
template cudaError_t exit_staggered<float>(axp_grid *, bool);
template cudaError_t general_step<double>(axp_grid *, int64_t);
template cudaError_t general_step<float>(axp_grid *, int64_t);
template cudaError_t general_current<double>(axp_grid *);
template cudaError_t general_current<float>(axp_grid *);

}  // namespace axp

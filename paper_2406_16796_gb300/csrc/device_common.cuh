// device_common.cuh -- boundary-aware device accessors of the general kernels.
//
// Index closure (arXiv 2406.16796 Sec. 2.3-2.4 and the readings of this
// library): periodic axes wrap; along a non-periodic axis E and B are zero
// outside the grid; the axion has one ghost cell per face -- reflect mirrors
// the first interior cell (phi_{-1/2} = phi_{1/2}), PML gives 0, outflow
// reads the stored ghost plane -- and 0 in cells outside along two axes.
#pragma once

#include "axp_internal.h"

namespace axp {

template <typename T>
struct Ghosts {
    T *p[3][2];
};

// Axion time-level pair around an integer time.  Two-level storage (FP64):
// b = earlier level.  Increment storage (FP32 split): b = hi - earlier level.
template <typename T, bool INCR>
struct PhiPair {
    const T *hi;
    const T *b;
    Ghosts<T> ghi, glo;
};

__host__ __device__ inline int64_t lin3(const int64_t n[3], int64_t i, int64_t j, int64_t k)
{
    return i + n[0] * (j + n[1] * k);
}

// x / d_a, x / (2 d_a) and x / d_a^2: a multiplication by the exact reciprocal
// where the view holds one (d_a a power of two: the same correctly rounded
// value as the division), else the division itself.
template <typename T>
__device__ __forceinline__ T over_d(const View<T> &v, T x, int a)
{
    return v.rd[a] != T(0) ? x * v.rd[a] : x / v.d[a];
}
template <typename T>
__device__ __forceinline__ T over_2d(const View<T> &v, T x, int a)
{
    return v.rd2[a] != T(0) ? x * v.rd2[a] : x / (T(2) * v.d[a]);
}
template <typename T>
__device__ __forceinline__ T over_dd(const View<T> &v, T x, int a)
{
    return v.rdd[a] != T(0) ? x * v.rdd[a] : x / (v.d[a] * v.d[a]);
}

// Linear index after periodic wrap (offsets of at most one period), or -1 when
// the point lies outside the grid along a non-periodic axis.
template <typename T>
__device__ __forceinline__ int64_t lin_em(const View<T> &v, int64_t i, int64_t j, int64_t k)
{
    if (i < 0 || i >= v.n[0]) {
        if (!v.periodic[0]) return -1;
        i += i < 0 ? v.n[0] : -v.n[0];
    }
    if (j < 0 || j >= v.n[1]) {
        if (!v.periodic[1]) return -1;
        j += j < 0 ? v.n[1] : -v.n[1];
    }
    if (k < 0 || k >= v.n[2]) {
        if (!v.periodic[2]) return -1;
        k += k < 0 ? v.n[2] : -v.n[2];
    }
    return lin3(v.n, i, j, k);
}

template <typename T>
__device__ __forceinline__ T ld(const View<T> &v, const T *F, int64_t i, int64_t j, int64_t k)
{
    const int64_t c = lin_em(v, i, j, k);
    return c < 0 ? T(0) : F[c];
}

// Where an axion sample lives: an interior index, a ghost plane entry, or zero.
struct PhiLoc {
    int kind;  // 0 interior, 1 zero, 2 outflow ghost plane
    int ax, side;
    int64_t idx;
};

template <typename T>
__device__ __forceinline__ PhiLoc resolve_phi(const View<T> &v, int64_t i, int64_t j, int64_t k)
{
    int64_t c[3] = {i, j, k};
    int nout = 0, ax = -1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= v.n[a]) {
            if (v.periodic[a]) {
                c[a] += c[a] < 0 ? v.n[a] : -v.n[a];
            } else {
                nout++;
                ax = a;
            }
        }
    }
    PhiLoc L;
    L.ax = ax;
    L.side = 0;
    if (nout == 0) {
        L.kind = 0;
        L.idx = lin3(v.n, c[0], c[1], c[2]);
        return L;
    }
    L.kind = 1;
    L.idx = 0;
    if (nout > 1) return L;
    const int side = c[ax] < 0 ? 0 : 1;
    L.side = side;
    const int bc = v.axbc[ax][side];
    if (bc == AXP_BC_REFLECT) {
        c[ax] = side ? v.n[ax] - 1 : 0;
        L.kind = 0;
        L.idx = lin3(v.n, c[0], c[1], c[2]);
    } else if (bc == AXP_BC_OUTFLOW) {
        L.kind = 2;
        L.idx = ax == 0 ? c[1] + v.n[1] * c[2] : (ax == 1 ? c[0] + v.n[0] * c[2] : c[0] + v.n[0] * c[1]);
    }
    return L;
}

// phi of one stored level (array + its ghost planes) at a possibly-ghost cell.
template <typename T>
__device__ __forceinline__ T ld_phi(const View<T> &v, const T *P, const Ghosts<T> &G, int64_t i, int64_t j,
                                    int64_t k)
{
    const PhiLoc L = resolve_phi(v, i, j, k);
    if (L.kind == 0) return P[L.idx];
    if (L.kind == 2) return G.p[L.ax][L.side][L.idx];
    return T(0);
}

// Time-centred value phi^n = (phi^{n+1/2} + phi^{n-1/2})/2 and D_t phi^n at a cell.
template <typename T, bool INCR>
__device__ __forceinline__ void phi_mid_dt(const View<T> &v, const PhiPair<T, INCR> &q, int64_t i, int64_t j,
                                           int64_t k, T *mid, T *dtv)
{
    const PhiLoc L = resolve_phi(v, i, j, k);
    T hi, lo;
    if (L.kind == 0) {
        hi = q.hi[L.idx];
        if (INCR) {
            const T inc = q.b[L.idx];
            *mid = hi - T(0.5) * inc;
            *dtv = inc / v.dt;
            return;
        }
        lo = q.b[L.idx];
    } else if (L.kind == 2) {
        hi = q.ghi.p[L.ax][L.side][L.idx];
        lo = q.glo.p[L.ax][L.side][L.idx];
    } else {
        *mid = T(0);
        *dtv = T(0);
        return;
    }
    *mid = T(0.5) * (hi + lo);
    *dtv = (hi - lo) / v.dt;
}

template <typename T, bool INCR>
__device__ __forceinline__ T phi_mid(const View<T> &v, const PhiPair<T, INCR> &q, int64_t i, int64_t j, int64_t k)
{
    T m, t;
    phi_mid_dt<T, INCR>(v, q, i, j, k, &m, &t);
    return m;
}

__device__ __forceinline__ void unit(int a, int64_t u[3])
{
    u[0] = a == 0;
    u[1] = a == 1;
    u[2] = a == 2;
}

// 2-point average of E0_a at the cell centre plus the background (Sec. 2.3).
template <typename T>
__device__ __forceinline__ T e0_bar(const View<T> &v, int a, int64_t i, int64_t j, int64_t k)
{
    int64_t u[3];
    unit(a, u);
    const T *E = v.f[kE0 + a];
    return T(0.5) * (ld(v, E, i, j, k) + ld(v, E, i - u[0], j - u[1], k - u[2])) + v.Eext[a];
}

// 4-point average of B0_a at the cell centre plus the background (Sec. 2.3);
// for a = x the offsets are (0,0), (0,-z), (-y,0), (-y,-z), cyclic for y, z.
template <typename T>
__device__ __forceinline__ T b0_bar(const View<T> &v, int a, int64_t i, int64_t j, int64_t k)
{
    int64_t ub[3], uc[3];
    unit((a + 1) % 3, ub);
    unit((a + 2) % 3, uc);
    const T *B = v.f[kB0 + a];
    T s = ld(v, B, i, j, k);
    s = s + ld(v, B, i - uc[0], j - uc[1], k - uc[2]);
    s = s + ld(v, B, i - ub[0], j - ub[1], k - ub[2]);
    s = s + ld(v, B, i - ub[0] - uc[0], j - ub[1] - uc[1], k - ub[2] - uc[2]);
    return T(0.25) * s + v.Bext[a];
}

template <typename T>
__device__ __forceinline__ T source_at(const View<T> &v, int64_t i, int64_t j, int64_t k)
{
    T s = e0_bar(v, 0, i, j, k) * b0_bar(v, 0, i, j, k);
    s = s + e0_bar(v, 1, i, j, k) * b0_bar(v, 1, i, j, k);
    s = s + e0_bar(v, 2, i, j, k) * b0_bar(v, 2, i, j, k);
    return v.g * s;
}

template <typename T>
__device__ __forceinline__ T sigma_of(const T *const tab[3], int64_t i, int64_t j, int64_t k)
{
    T s = tab[0][i];
    const T s1 = tab[1][j], s2 = tab[2][k];
    if (s1 > s) s = s1;
    if (s2 > s) s = s2;
    return s;
}

// dF/dt = X - sigma F over a half-step h, trapezoidal in time.
template <typename T>
__device__ __forceinline__ T half_update(T F, T X, T sig, T h)
{
    if (sig == T(0)) return F + h * X;
    return ((T(1) - sig * h / T(2)) * F + h * X) / (T(1) + sig * h / T(2));
}

__device__ __forceinline__ void cell_of(int64_t c, const int64_t n[3], int64_t *i, int64_t *j, int64_t *k)
{
    if (c < 0xffffffffLL && n[0] < 0xffffffffLL && n[1] < 0xffffffffLL) {
        // 32-bit division where the index fits (64-bit division is a long sequence)
        const uint32_t cc = (uint32_t)c, n0 = (uint32_t)n[0], n1 = (uint32_t)n[1];
        const uint32_t r = cc / n0;
        *i = cc - r * n0;
        *j = r % n1;
        *k = r / n1;
        return;
    }
    *i = c % n[0];
    const int64_t r = c / n[0];
    *j = r % n[1];
    *k = r / n[1];
}

// The q-th cell a general kernel visits (x fastest): every cell, or only those
// with vlo <= index < vhi along vaxis.  Returns the cell's linear index.
template <typename T>
__device__ __forceinline__ int64_t visit(const View<T> &v, int64_t q, int64_t *i, int64_t *j, int64_t *k)
{
    if (v.vaxis < 0) {
        cell_of(q, v.n, i, j, k);
        return q;
    }
    int64_t m[3] = {v.n[0], v.n[1], v.n[2]};
    m[v.vaxis] = v.vhi - v.vlo;
    cell_of(q, m, i, j, k);
    if (v.vaxis == 0) *i += v.vlo;
    else if (v.vaxis == 1) *j += v.vlo;
    else *k += v.vlo;
    return lin3(v.n, *i, *j, *k);
}

}  // namespace axp

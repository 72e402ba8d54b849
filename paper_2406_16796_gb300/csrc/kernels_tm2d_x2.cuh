// kernels_tm2d_x2.cuh -- the 2D step of kernels_tm2d.cuh for FP32-split grids,
// two adjacent x columns per thread (arXiv 2406.16796 Sec. 2.3; the 2D pulse
// workload in FP32 split).
//
// Same scheme, same staggered state and the same four stages per plane as
// tm2d::tile (see kernels_tm2d.cuh).  What changes is the work unit: a thread
// owns the column pair (2t, 2t+1) of its tile and carries the pair's history
// along y as float2 values, so
//   * each input and output moves as one 8-byte access (cp.async of 8 bytes,
//     64-bit stores) for two cells, and one address serves both;
//   * the arithmetic runs on the packed FP32 pipe (__ffma2_rn, __fadd2_rn,
//     __fmul2_rn): one instruction for two cells;
//   * a published row holds pairs; a stage that needs the x neighbour of a pair
//     forms the shifted pair from its own other column and one float of the
//     neighbouring thread's pair.
// The pair starts at an even column: the tile keeps 2 halo columns below and 4
// above (an even number of written columns), and the grid's width is even, so
// a pair is always wholly inside or wholly outside the grid and always 8-byte
// aligned.  Grids of odd width, soft sources and groups take tm2d::tile.
#pragma once

#include "kernels_tm2d.cuh"

namespace axp {
namespace tm2d_x2 {

constexpr int NTX = 128;            // threads per block (largest); columns = 2 x threads
constexpr int HL = 2, HR = 4;       // halo columns below / above
constexpr int RS = NTX + 2;         // row stride in pairs: one guard pair on each side
constexpr int NS = 4;               // staging ring depth (planes, power of two)
constexpr int NIN = tm2d::NIN;      // input arrays per plane

constexpr size_t stage_bytes(int ntx = NTX) { return (size_t)NS * NIN * ntx * sizeof(float2); }

__device__ __forceinline__ void cp_pair(float2 *dst, const float *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}

__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
// the pair one column to the right / left: (own.y, right.x) and (left.y, own.x)
__device__ __forceinline__ float2 right_of(float2 own, const float2 *row, int t) { return make_float2(own.y, row[t + 2].x); }
__device__ __forceinline__ float2 left_of(float2 own, const float2 *row, int t) { return make_float2(row[t].y, own.x); }

enum { R_E0Z, R_E1Y, R_E1Z, R_PHI, R_N0Y2, R_MID3, R_N0Y3, R_PX4, R_N1Z4, R_N1Y4, R_N0Y4, NROWS };

__device__ __forceinline__ void tile(const fused::Params<float> &P, const int bx, const int by,
                                     float2 (&rows)[2][NROWS][RS], float2 *stage)
{
    const int ntx = (int)blockDim.x, vx = 2 * ntx - HL - HR;  // written columns of this launch's tiles
    for (int i = threadIdx.x; i < 2 * NROWS * RS; i += ntx) (&rows[0][0][0])[i] = make_float2(0.f, 0.f);

    const int tx = threadIdx.x;
    const int nx = P.n[0], ny = P.n[1];
    const bool perx = P.per[0], pery = P.per[1];
    const int gx = bx * vx - HL + 2 * tx;  // first column of the pair (even)
    int wx = gx;
    if (wx < 0 || wx >= nx) wx = perx ? ((wx % nx) + nx) % nx : -1;
    const bool write_col = 2 * tx >= HL && 2 * tx < 2 * ntx - HR && gx >= 0 && gx < nx;
    const int nstrips = (nx + vx - 1) / vx;
    const bool xstrip = !perx && (bx == 0 || bx == nstrips - 1);
    const int chunk = xstrip ? P.chunk_edge : P.chunk;
    const int first = xstrip ? P.chunk_edge : P.chunk_first;
    const int m0 = by == 0 ? 0 : first + (by - 1) * chunk;
    if (m0 >= ny) return;
    const int m1 = min(ny, by == 0 ? first : m0 + chunk);
    const int gx0 = bx * vx - HL;
    const int wx0 = gx0 + 2 * (tx & ~31), wx1 = wx0 + 63;  // columns of this warp
    const bool tile_fast = perx || (wx0 - 1 >= P.lay[0][0] && wx1 + 1 <= nx - 1 - P.lay[0][1]);
    // A warp whose columns all lie beyond the last column of a non-periodic grid
    // would compute the closure's zeros (the edge body sets every value it keeps or
    // publishes to zero outside the grid): it keeps the zeros of its registers and
    // of the zeroed rows instead, meeting every barrier with the other warps.
    const bool dead = !perx && wx0 >= nx;
    const int ylo = P.lay[1][0], yhi = ny - 1 - P.lay[1][1];

    const float h = P.h, g = P.g, idx = P.idx[0], idy = P.idx[1], hidx = P.hidx[0], hidy = P.hidx[1];
    const float hx = h * idx, hy = h * idy, h2x = 2.f * hx, h2y = 2.f * hy, hg = h * g;
    const float cx = P.lap_c[0], cy = P.lap_c[1], c0 = P.lap_0, dt2g = P.dt2g, inv_dt = P.inv_dt;
    const float Bz = P.Bext[2];
    const float qidx = 0.5f * hidx, qidy = 0.5f * hidy, hinv_dt = 0.5f * inv_dt;
    const float Bxi = P.Bext[0] * inv_dt, Byi = P.Bext[1] * inv_dt, dt2gBz = dt2g * Bz, gBzi = g * Bz * inv_dt;
    const float h2gBzi = 2.f * hg * Bz * inv_dt;
    const bool xl = wx >= 0 && P.has_pml;
    // this pair's layer coefficients (the plain update's where there is no layer)
    auto colcoef = [&](int k, float plain) {
        return xl ? make_float2(P.pml_tab[0][k * nx + wx], P.pml_tab[0][k * nx + wx + 1]) : f2(plain);
    };
    const float2 ax1 = colcoef(0, 1.f), bx1 = colcoef(1, h), ax2 = colcoef(2, 1.f), bx2 = colcoef(3, 2.f * h);
    const float2 kx1 = colcoef(4, P.dt2), kx2 = colcoef(5, 1.f);
    const float2 sxa = xl ? make_float2(P.sig_ax[0][wx], P.sig_ax[0][wx + 1]) : f2(0.f);

    enum { Y_A1, Y_B1, Y_A2, Y_B2, Y_K1, Y_K2, Y_SA, NY };
    constexpr int YR = 16;
    __shared__ __align__(16) float yring[YR][NY + 1];
    auto fill_y = [&](int p) {
        if (tx < NY) {
            float *dst = &yring[p & (YR - 1)][tx];
            if (!pery && P.has_pml && p >= 0 && p < ny) {
                tm2d::cp_elem(dst, tx < Y_SA ? P.pml_tab[1] + (tx * ny + p) : P.sig_ax[1] + p, true);
            } else {
                *dst = (tx == Y_A1 || tx == Y_A2 || tx == Y_K2) ? 1.f
                       : tx == Y_B1                              ? h
                       : tx == Y_B2                              ? 2.f * h
                       : tx == Y_K1                              ? P.dt2
                                                                 : 0.f;
            }
        }
    };

    const float2 z2 = make_float2(0.f, 0.f);
    float2 E0z0 = z2, E0z1 = z2, E0z2 = z2, E0z3 = z2, E0z4 = z2;
    float2 E1x0 = z2, E1x1 = z2, E1x2 = z2, E1x3 = z2, E1x4 = z2;
    float2 E1y0 = z2, E1y1 = z2, E1y2 = z2, E1y3 = z2, E1y4 = z2;
    float2 E1z0 = z2, E1z1 = z2, E1z2 = z2, E1z3 = z2, E1z4 = z2;
    float2 B0x0 = z2, B0x1 = z2, B0y0 = z2, B0y1 = z2, B1x0 = z2, B1x1 = z2, B1y0 = z2, B1y1 = z2, B1z0 = z2,
           B1z1 = z2;
    float2 ph0 = z2, ph1 = z2, ph2 = z2, ph3 = z2, pb0 = z2, pb1 = z2, pb2 = z2;
    float2 N0x1 = z2, N0x2 = z2, N0x3 = z2, N0x4 = z2, N0x5 = z2;
    float2 N0y1 = z2, N0y2 = z2, N0y3 = z2, N0y4 = z2;
    float2 N1x1 = z2, N1x2 = z2, N1x3 = z2, N1x4 = z2, N1x5 = z2;
    float2 N1y1 = z2, N1y2 = z2, N1y3 = z2, N1y4 = z2;
    float2 N1z1 = z2, N1z2 = z2, N1z3 = z2, N1z4 = z2, N1z5 = z2;
    float2 SM2 = z2, SM3 = z2, SM4 = z2, DF2 = z2, DF3 = z2, DF4 = z2;
    float2 EN2 = z2, EN3 = z2, EN4 = z2;
    float2 PX3 = z2, PX4 = z2, PY3 = z2, PY4 = z2;
    const int t0 = m0 - 2, t1 = m1 + 3;

    // element offsets within an array are 32-bit (grids of at most 2^32 cells)
    auto prefetch = [&](int p) {
        fill_y(p);
        int wp = p;
        if (wp < 0 || wp >= ny) wp = pery ? ((wp % ny) + ny) % ny : -1;
        const bool ok = wx >= 0 && wp >= 0;
        const unsigned o = ok ? (unsigned)wx + (unsigned)nx * (unsigned)wp : 0u;
        float2 *st = stage + ((p - t0) & (NS - 1)) * (NIN * ntx) + tx;
        cp_pair(st + 0 * ntx, P.Ein[2] + o, ok);
        cp_pair(st + 1 * ntx, P.Ein[3] + o, ok);
        cp_pair(st + 2 * ntx, P.Ein[4] + o, ok);
        cp_pair(st + 3 * ntx, P.Ein[5] + o, ok);
        cp_pair(st + 4 * ntx, P.Bin[0] + o, ok);
        cp_pair(st + 5 * ntx, P.Bin[1] + o, ok);
        cp_pair(st + 6 * ntx, P.Bin[3] + o, ok);
        cp_pair(st + 7 * ntx, P.Bin[4] + o, ok);
        cp_pair(st + 8 * ntx, P.Bin[5] + o, ok);
        cp_pair(st + 9 * ntx, P.phi + o, ok);
        cp_pair(st + 10 * ntx, P.phib + o, ok);
    };
    auto take = [&](int p) {
        const float2 *st = stage + ((p - t0) & (NS - 1)) * (NIN * ntx) + tx;
        E0z0 = st[0 * ntx];
        E1x0 = st[1 * ntx];
        E1y0 = st[2 * ntx];
        E1z0 = st[3 * ntx];
        B0x0 = st[4 * ntx];
        B0y0 = st[5 * ntx];
        B1x0 = st[6 * ntx];
        B1y0 = st[7 * ntx];
        B1z0 = st[8 * ntx];
        ph0 = st[9 * ntx];
        pb0 = st[10 * ntx];
    };
    auto lay = [&](bool in, int p, float2 &a1, float2 &b1, float2 &a2, float2 &b2) {
        a1 = ax1;
        b1 = bx1;
        a2 = ax2;
        b2 = bx2;
        if (in && !pery) {
            const float *y = yring[p & (YR - 1)];
            a1 = min2(a1, f2(y[Y_A1]));
            b1 = min2(b1, f2(y[Y_B1]));
            a2 = min2(a2, f2(y[Y_A2]));
            b2 = min2(b2, f2(y[Y_B2]));
        }
    };
    auto inside = [&](int p) { return wx >= 0 && (pery || (p >= 0 && p < ny)); };
    auto store = [](float *base, unsigned gi, float2 v) { *reinterpret_cast<float2 *>(base + gi) = v; };

    auto body = [&](auto edge_tag, int t, int b) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        float2(*R)[RS] = rows[b];
        // ---- stage 1: B^{n+1} on plane t-1 ----
        {
            const int p = t - 1;
            const bool in = !EDGE || inside(p);
            const float2 d0y = sub2(E0z0, E0z1), d0x = sub2(right_of(E0z1, R[R_E0Z], tx), E0z1);
            const float2 d1zy = sub2(E1z0, E1z1), d1zx = sub2(right_of(E1z1, R[R_E1Z], tx), E1z1);
            const float2 d1yx = sub2(right_of(E1y1, R[R_E1Y], tx), E1y1), d1xy = sub2(E1x0, E1x1);
            auto plain = [&]() {
                N0x1 = fma2(f2(-h2y), d0y, B0x1);
                N0y1 = fma2(f2(h2x), d0x, B0y1);
                N1x1 = fma2(f2(-h2y), d1zy, B1x1);
                N1y1 = fma2(f2(h2x), d1zx, B1y1);
                N1z1 = fma2(f2(-h2x), d1yx, fma2(f2(h2y), d1xy, B1z1));
            };
            if (!EDGE) {
                plain();
            } else {
                float2 a1, b1, a2, b2;
                lay(in, p, a1, b1, a2, b2);
                if (a2.x == 1.f && a2.y == 1.f) {
                    plain();
                } else {
                    const float2 c0x = mul2(d0y, f2(idy)), c0y = mul2(d0x, f2(-idx));
                    const float2 c1x = mul2(d1zy, f2(idy)), c1y = mul2(d1zx, f2(-idx));
                    const float2 c1z = fma2(d1yx, f2(idx), mul2(d1xy, f2(-idy)));
                    const float2 nb2 = mul2(b2, f2(-1.f));
                    N0x1 = fma2(nb2, c0x, mul2(a2, B0x1));
                    N0y1 = fma2(nb2, c0y, mul2(a2, B0y1));
                    N1x1 = fma2(nb2, c1x, mul2(a2, B1x1));
                    N1y1 = fma2(nb2, c1y, mul2(a2, B1y1));
                    N1z1 = fma2(nb2, c1z, mul2(a2, B1z1));
                }
            }
            if (EDGE && !in) N0x1 = N0y1 = N1x1 = N1y1 = N1z1 = z2;
            if (write_col && p >= m0 && p < m1) {
                const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                store(P.Bout[0], gi, N0x1);
                store(P.Bout[1], gi, N0y1);
                store(P.Bout[3], gi, N1x1);
                store(P.Bout[4], gi, N1y1);
                store(P.Bout[5], gi, N1z1);
            }
        }
        // ---- stage 2: axion on plane t-2, E0z^{n+1} ----
        {
            const int p = t - 2;
            const bool in = !EDGE || inside(p);
            const float2 spx = add2(sub2(right_of(ph2, R[R_PHI], tx), ph2), sub2(left_of(ph2, R[R_PHI], tx), ph2));
            const float2 spy = add2(sub2(ph1, ph2), sub2(ph3, ph2));
            float2 sa = z2;
            if (EDGE && in && P.has_pml) sa = pery ? sxa : max2(sxa, f2(yring[p & (YR - 1)][Y_SA]));
            float2 pin;
            if (!EDGE || (sa.x == 0.f && sa.y == 0.f)) {
                float2 acc = fma2(f2(c0), ph2, pb2);
                acc = fma2(f2(cx), spx, acc);
                acc = fma2(f2(cy), spy, acc);
                pin = fma2(f2(dt2gBz), E0z2, acc);
            } else {
                const float2 lap = fma2(spx, f2(P.idx2[0]), mul2(spy, f2(P.idx2[1])));
                const float2 S = mul2(E0z2, f2(Bz));
                // ((g S - m^2 phi) + lap) - s^2 phi, per column
                const float2 gS = fma2(f2(-P.m2), ph2, mul2(f2(g), S));
                const float2 Y = sub2(add2(gS, lap), mul2(mul2(sa, sa), ph2));
                float2 c1 = kx1, c2 = kx2;
                if (!pery) {
                    c1 = min2(c1, f2(yring[p & (YR - 1)][Y_K1]));
                    c2 = min2(c2, f2(yring[p & (YR - 1)][Y_K2]));
                }
                pin = fma2(c1, Y, mul2(c2, pb2));
            }
            const float2 nw = add2(ph2, pin);
            SM2 = fma2(f2(2.f), ph2, pin);
            DF2 = pin;
            if (write_col && p >= m0 && p < m1) {
                const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                store(P.phi_out, gi, nw);
                store(P.phib_out, gi, pin);
            }
            // E0z^{n+1} = E0z^{n+1/2} + h (curl B0)_z, backward differences
            const float2 dbx = sub2(N0y2, left_of(N0y2, R[R_N0Y2], tx)), dby = sub2(N0x2, N0x3);
            if (!EDGE) {
                EN2 = fma2(f2(hx), dbx, fma2(f2(-hy), dby, E0z2));
            } else {
                float2 a1, b1, a2, b2;
                lay(in, p, a1, b1, a2, b2);
                EN2 = (a1.x == 1.f && a1.y == 1.f)
                          ? fma2(f2(hx), dbx, fma2(f2(-hy), dby, E0z2))
                          : fma2(b1, fma2(dbx, f2(idx), mul2(dby, f2(-idy))), mul2(a1, E0z2));
            }
            if (EDGE && !in) SM2 = DF2 = EN2 = z2;
        }
        // ---- stage 3: P^{n+1} on plane t-3 ----
        {
            const int p = t - 3;
            const float2 bbx = fma2(f2(hinv_dt), add2(N0x3, N0x4), f2(Bxi));
            const float2 bby = fma2(f2(hinv_dt), add2(N0y3, left_of(N0y3, R[R_N0Y3], tx)), f2(Byi));
            const float2 dpy = mul2(sub2(SM2, SM4), f2(qidy));
            const float2 dpx = mul2(sub2(right_of(SM3, R[R_MID3], tx), left_of(SM3, R[R_MID3], tx)), f2(qidx));
            PX3 = fma2(EN3, dpy, mul2(DF3, bbx));
            PY3 = fma2(mul2(EN3, f2(-1.f)), dpx, mul2(DF3, bby));
            if (EDGE && !inside(p)) PX3 = PY3 = z2;
        }
        // ---- stage 4: J^{n+1}, E^{n+3/2} on plane t-4 ----
        {
            const int p = t - 4;
            if (p >= m0 && p < m1) {
                const bool in = !EDGE || inside(p);
                const float2 sjx = add2(PX4, right_of(PX4, R[R_PX4], tx)), sjy = add2(PY4, PY3);
                const float2 e1zy = sub2(N1z4, N1z5), e1zx = sub2(N1z4, left_of(N1z4, R[R_N1Z4], tx));
                const float2 e1yx = sub2(N1y4, left_of(N1y4, R[R_N1Y4], tx)), e1xy = sub2(N1x4, N1x5);
                float2 ex, ey, ez, e0;
                auto plain = [&]() {
                    ex = fma2(f2(h2y), e1zy, fma2(f2(-hg), sjx, E1x4));
                    ey = fma2(f2(-h2x), e1zx, fma2(f2(-hg), sjy, E1y4));
                    ez = fma2(f2(h2x), e1yx, fma2(f2(-h2y), e1xy, fma2(f2(-h2gBzi), DF4, E1z4)));
                    e0 = fma2(f2(2.f), EN4, mul2(E0z4, f2(-1.f)));
                };
                if (!EDGE) {
                    plain();
                } else {
                    float2 a1, b1, a2, b2;
                    lay(in, p, a1, b1, a2, b2);
                    if (a2.x == 1.f && a2.y == 1.f) {
                        plain();
                    } else {
                        const float2 xx = fma2(f2(-g), mul2(f2(0.5f), sjx), mul2(e1zy, f2(idy)));
                        const float2 xy = fma2(f2(-g), mul2(f2(0.5f), sjy), mul2(e1zx, f2(-idx)));
                        const float2 xz = fma2(f2(-gBzi), DF4, fma2(e1yx, f2(idx), mul2(e1xy, f2(-idy))));
                        const float2 e0yx = sub2(N0y4, left_of(N0y4, R[R_N0Y4], tx)), e0xy = sub2(N0x4, N0x5);
                        ex = fma2(b2, xx, mul2(a2, E1x4));
                        ey = fma2(b2, xy, mul2(a2, E1y4));
                        ez = fma2(b2, xz, mul2(a2, E1z4));
                        e0 = fma2(b1, fma2(e0yx, f2(idx), mul2(e0xy, f2(-idy))), mul2(a1, EN4));
                    }
                }
                if (write_col) {
                    const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                    store(P.Eout[3], gi, ex);
                    store(P.Eout[4], gi, ey);
                    store(P.Eout[5], gi, ez);
                    store(P.Eout[2], gi, e0);
                }
            }
        }
    };

    for (int p = t0 - 4; p < t0; p++) fill_y(p);
    for (int j = 0; j < NS - 1; j++) {
        if (!dead && t0 + j <= t1) prefetch(t0 + j);
        tm2d::cp_commit();
    }
    tm2d::cp_wait<NS - 2>();
    if (!dead) take(t0);
    __syncthreads();
#pragma unroll 2
    for (int t = t0; t <= t1; ++t) {
        if (!dead && t + NS - 1 <= t1) prefetch(t + NS - 1);
        tm2d::cp_commit();
        const int b = (t - t0) & 1;
        if (!dead) {
        rows[b][R_E0Z][tx + 1] = E0z1;
        rows[b][R_E1Y][tx + 1] = E1y1;
        rows[b][R_E1Z][tx + 1] = E1z1;
        rows[b][R_PHI][tx + 1] = ph2;
        rows[b][R_N0Y2][tx + 1] = N0y2;
        rows[b][R_MID3][tx + 1] = SM3;
        rows[b][R_N0Y3][tx + 1] = N0y3;
        rows[b][R_PX4][tx + 1] = PX4;
        rows[b][R_N1Z4][tx + 1] = N1z4;
        rows[b][R_N1Y4][tx + 1] = N1y4;
        rows[b][R_N0Y4][tx + 1] = N0y4;
        }
        __syncthreads();
        const bool fast = tile_fast && (pery || (t - 6 >= ylo && t + 1 <= yhi));
        if (dead) {
        } else if (fast) {
            body(std::false_type{}, t, b);
        } else {
            body(std::true_type{}, t, b);
        }
        E0z4 = E0z3; E0z3 = E0z2; E0z2 = E0z1; E0z1 = E0z0;
        E1x4 = E1x3; E1x3 = E1x2; E1x2 = E1x1; E1x1 = E1x0;
        E1y4 = E1y3; E1y3 = E1y2; E1y2 = E1y1; E1y1 = E1y0;
        E1z4 = E1z3; E1z3 = E1z2; E1z2 = E1z1; E1z1 = E1z0;
        B0x1 = B0x0; B0y1 = B0y0; B1x1 = B1x0; B1y1 = B1y0; B1z1 = B1z0;
        ph3 = ph2; ph2 = ph1; ph1 = ph0; pb2 = pb1; pb1 = pb0;
        N0x5 = N0x4; N0x4 = N0x3; N0x3 = N0x2; N0x2 = N0x1;
        N0y4 = N0y3; N0y3 = N0y2; N0y2 = N0y1;
        N1x5 = N1x4; N1x4 = N1x3; N1x3 = N1x2; N1x2 = N1x1;
        N1y4 = N1y3; N1y3 = N1y2; N1y2 = N1y1;
        N1z5 = N1z4; N1z4 = N1z3; N1z3 = N1z2; N1z2 = N1z1;
        SM4 = SM3; SM3 = SM2; DF4 = DF3; DF3 = DF2; EN4 = EN3; EN3 = EN2;
        PX4 = PX3; PY4 = PY3;
        tm2d::cp_wait<NS - 2>();
        if (!dead && t < t1) take(t + 1);
    }
    tm2d::cp_wait<0>();
}

// (a template, so that every unit including this header may instantiate it)
template <int UNUSED = 0>
__global__ void __launch_bounds__(NTX, 2) k_tm2d_x2(fused::Params<float> P)
{
    __shared__ float2 rows[2][NROWS][RS];
    extern __shared__ __align__(16) unsigned char tm2d_x2_dyn[];
    tile(P, (int)blockIdx.x, (int)blockIdx.y, rows, reinterpret_cast<float2 *>(tm2d_x2_dyn));
}

}  // namespace tm2d_x2
}  // namespace axp

namespace axp {
namespace tm2d_x2 {

// Launch over tiles of `cols` columns (cols / 2 threads, a multiple of 64 columns
// up to 2 NTX); nchunks = 0 only reports the resident blocks per SM.
inline cudaError_t launch(const fused::Params<float> &P, int nchunks, cudaStream_t stream, int *occupancy, int cols)
{
    static int occ[NTX / 32 + 1] = {};
    const int ntx = cols / 2;
    if (cols % 64 || ntx < 32 || ntx > NTX) return cudaErrorInvalidValue;
    const size_t dyn = stage_bytes(ntx);
    if (occ[ntx / 32] == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_tm2d_x2<>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes());
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[ntx / 32], k_tm2d_x2<>, ntx, dyn);
        if (e != cudaSuccess) return e;
    }
    if (occupancy) *occupancy = occ[ntx / 32];
    if (nchunks <= 0) return cudaSuccess;
    const int vx = cols - HL - HR;
    dim3 grid((P.n[0] + vx - 1) / vx, nchunks, 1);
    k_tm2d_x2<><<<grid, ntx, dyn, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace tm2d_x2
}  // namespace axp

// kernels_tm2d.cuh -- fused step specialised for 2D grids whose laser is the
// (E0z; B0x, B0y) polarisation (arXiv 2406.16796 Sec. 2.3; the 2D pulse
// workload), with periodic or absorbing (PML) edges.
//
// Same scheme and staggered state as kernels_fused.cuh: per step
//   1. B^{n+1} = B^n - h curl E^{n+1/2} (twice)
//   2. S^{n+1/2}/g = E0z B_ext,z; phi^{n+3/2}; 2 phi^{n+1}, dt D_t phi^{n+1}; E0z^{n+1}
//   3. P^{n+1} = (D_t phi) Bbar0 - Ebar0 x grad_c phi
//   4. J^{n+1}; E^{n+3/2} = E^{n+1/2} + 2 x h (curl B^{n+1} - g J^{n+1}); E0z^{n+3/2}
// A thread owns one x column of a tile (2 halo columns below, 3 above) and
// marches along y; stage k works on plane t - k while plane t is loaded.  Every
// neighbour value a stage reads along x was produced in an earlier iteration,
// so each thread keeps its column's history along y in registers and publishes
// only the values its x neighbours need into double-buffered shared rows at the
// start of an iteration: one barrier per plane, and no shared-memory rings for
// the stages' results (the inputs and the y layer coefficients are staged ahead
// in rings of their own, below).
//
// On the PML edges every quantity outside the grid is zero (the E/B closure and
// the PML ghost of phi), so the edge version of the body only zeroes what it
// computes outside and applies the damped updates inside the layer.
#pragma once

#include <type_traits>

#include "kernels_fused.cuh"

namespace axp {
namespace tm2d {

constexpr int TX = 256;     // largest block (tile) width; a launch may use a narrower multiple of 32
constexpr int HL = 2, HR = 3;
constexpr int VX = TX - HL - HR;
constexpr int RS = TX + 2;  // row stride: one guard element on each side

// Input staging: each thread copies its own column's 11 input values of a plane
// into shared memory with asynchronous copies (cp.async, zero-filled outside
// the grid), NS planes deep, and reads them back when the plane is taken.  No
// registers hold loads in flight and no barrier is needed for the staging (a
// thread reads only what it copied itself).  A plane's slot is thread-major (a
// thread's 11 values together: an odd stride, so a warp's accesses fall in
// distinct banks) and sized for the launch's tile width.
//
// Planes in the staging ring (a power of two): 3 planes of loads in flight.  In
// FP32 that is with two 256-wide blocks per SM (16 warps); 7 planes took 226 KB
// of shared memory per SM for two such blocks, leaving too little L1, and ran
// 13% slower than 3.
template <typename T>
__host__ __device__ constexpr int ns()
{
    return 4;
}
constexpr int NIN = 11;  // input arrays per plane

template <typename T>
constexpr size_t stage_bytes(int tx = TX)
{
    return (size_t)ns<T>() * NIN * tx * sizeof(T);
}

__device__ __forceinline__ void cp_elem(float *dst, const float *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_elem(double *dst, const double *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// rows published each iteration (all at x offset +1 in the row)
enum { R_E0Z, R_E1Y, R_E1Z, R_PHI, R_N0Y2, R_MID3, R_N0Y3, R_PX4, R_N1Z4, R_N1Y4, R_N0Y4, NROWS };

// One tile: x strip bx (VX written columns), planes [m0, m1) of the grid P
// describes.  `rows` is the block's shared staging; the caller separates
// consecutive tiles of one block with a barrier.  SRC compiles in the soft
// source's sheets (P.src_x >= 0); without it the body has no trace of them.
// FOLDP: square cells (dx = dy) and no uniform background B along x or y, the
// 2D pulse's case.  The axion current is then carried as P / (1/(2 dt)): the
// factor meets the gradient's 1/(4 dx) in one constant and the current's
// coefficient in the E updates, three operations fewer per cell.
template <typename T, bool INCR, bool SRC = false, bool FOLDP = false>
__device__ __forceinline__ void tile_span(const fused::Params<T> &P, const int bx, const int m0, const int m1,
                                          T (&rows)[2][NROWS][RS], T *stage)
{
    constexpr int NS = ns<T>();
    const int ntx = (int)blockDim.x, vx = ntx - HL - HR;  // this launch's tile width
    for (int i = threadIdx.x; i < 2 * NROWS * RS; i += ntx) (&rows[0][0][0])[i] = T(0);

    const int tx = threadIdx.x;
    const int nx = P.n[0], ny = P.n[1];
    const bool perx = P.per[0], pery = P.per[1];
    const int gx = bx * vx - HL + tx;
    int wx = gx;
    if (wx < 0 || wx >= nx) wx = perx ? ((wx % nx) + nx) % nx : -1;
    const bool write_col = tx >= HL && tx < ntx - HR && gx >= 0 && gx < nx;
    const int gx0 = bx * vx - HL;
    // The plain body is exact for a column inside the grid with no x layer (the
    // edge body adds nothing there), so the choice is made per warp: in a tile
    // at an x edge only the warps over the layer take the edge body.
    const int wx0 = gx0 + (tx & ~31), wx1 = wx0 + 31;
    const bool tile_fast = perx || (wx0 - 1 >= P.lay[0][0] && wx1 + 1 <= nx - 1 - P.lay[0][1]);
    // A warp whose columns all lie beyond the last column of a non-periodic grid
    // would compute the closure's zeros (the edge body sets every value it keeps or
    // publishes to zero outside the grid): it keeps the zeros of its registers and
    // of the zeroed rows instead, and leaves the pipes to the other warps.
    const bool dead = !perx && wx0 >= nx;
    const int ylo = P.lay[1][0], yhi = ny - 1 - P.lay[1][1];

    const T h = P.h, g = P.g, idx = P.idx[0], idy = P.idx[1], hidx = P.hidx[0], hidy = P.hidx[1];
    // step constants of the folded updates
    const T hx = h * idx, hy = h * idy, h2x = T(2) * hx, h2y = T(2) * hy, hg = h * g, h2g = T(2) * hg;
    const T cx = P.lap_c[0], cy = P.lap_c[1], c0 = P.lap_0, dt2g = P.dt2g, inv_dt = P.inv_dt;
    const T Bx = P.Bext[0], By = P.Bext[1], Bz = P.Bext[2];
    // The axion is carried as SM = 2 phi^{n+1} and DF = dt D_t phi^{n+1} (sum and
    // difference of its two levels), with 1/2 and 1/dt folded into the constants
    // that meet them: qidx = hidx/2 (exact), Bbar/dt as (N + N')(1/(2dt)) + B_ext/dt,
    // and B_ext,z folded into the source and J_z coefficients.
    const T qidx = T(0.5) * hidx, qidy = T(0.5) * hidy, hinv_dt = T(0.5) * inv_dt;
    const T Bxi = Bx * inv_dt, Byi = By * inv_dt, dt2gBz = dt2g * Bz, gBzi = g * Bz * inv_dt;
    const T h2gBzi = h2g * Bz * inv_dt;
    // FOLDP: P_x, P_y carried divided by 1/(2 dt); the gradient's factor and the
    // current's coefficients absorb it
    const T qq = qidx / hinv_dt;
    const T hgP = FOLDP ? hg * hinv_dt : hg, gP = FOLDP ? g * hinv_dt : g;
    // soft source: this column holds the sheet's E cells (electric sheet) or the
    // B faces on the plane (magnetic sheet)
    const bool src_e_col = SRC && wx == P.src_x;
    const bool src_b_col = SRC && wx >= 0 && wx == P.src_x - 1;
    const bool xl = wx >= 0 && P.has_pml;
    const T sxa = xl ? P.sig_ax[0][wx] : T(0);
    // this column's layer coefficients (the plain update's where there is no layer):
    // one half-step a, b; two half-steps a^2, b (1 + a); axion k1, k2
    const T ax1 = xl ? P.pml_tab[0][wx] : T(1);
    const T bx1 = xl ? P.pml_tab[0][nx + wx] : h;
    const T ax2 = xl ? P.pml_tab[0][2 * nx + wx] : T(1);
    const T bx2 = xl ? P.pml_tab[0][3 * nx + wx] : T(2) * h;
    const T kx1 = xl ? P.pml_tab[0][4 * nx + wx] : P.dt2;
    const T kx2 = xl ? P.pml_tab[0][5 * nx + wx] : T(1);
    auto smax = [](T a, T b) { return a > b ? a : b; };
    auto smin = [](T a, T b) { return a < b ? a : b; };
    // The y values of the same coefficients (and the axion sigma) are the same for
    // a whole plane: a ring of planes in shared memory, copied asynchronously
    // with the plane's inputs (NS - 1 planes ahead), keeps their loads off the
    // per-plane critical path.
    // The ring's last slot holds the soft source's electric-sheet weight of the
    // plane (zero without a source).
    enum { Y_A1, Y_B1, Y_A2, Y_B2, Y_K1, Y_K2, Y_SA, NY, Y_W = NY };
    // Ring depth: a block's threads are at most one iteration apart (one barrier per
    // iteration), and the fill for plane t+NS-1 at the top of iteration t happens
    // before that iteration's barrier, while a thread still in iteration t-1 may
    // read planes down to t-5: 9 planes live at once, so 16 slots.
    constexpr int YR = 16;
    __shared__ __align__(16) T yring[YR][NY + 1];
    auto fill_y = [&](int p) {
        if (SRC && tx == Y_W) {
            const int pw = pery ? ((p % ny) + ny) % ny : p;
            T *dst = &yring[p & (YR - 1)][Y_W];
            if (P.src_x >= 0 && pw >= 0 && pw < ny) cp_elem(dst, P.src_w + pw, true);
            else *dst = T(0);
        } else if (tx < NY) {
            T *dst = &yring[p & (YR - 1)][tx];
            if (!pery && P.has_pml && p >= 0 && p < ny) {
                cp_elem(dst, tx < Y_SA ? P.pml_tab[1] + (tx * ny + p) : P.sig_ax[1] + p, true);
            } else {  // no layer: the plain update's coefficients
                *dst = (tx == Y_A1 || tx == Y_A2 || tx == Y_K2) ? T(1)
                       : tx == Y_B1                              ? h
                       : tx == Y_B2                              ? T(2) * h
                       : tx == Y_K1                              ? P.dt2
                                                                 : T(0);
            }
        }
    };

    // column history along y; suffix k = plane t - k of the current iteration
    T E0z0 = 0, E0z1 = 0, E0z2 = 0, E0z3 = 0, E0z4 = 0;
    T E1x0 = 0, E1x1 = 0, E1x2 = 0, E1x3 = 0, E1x4 = 0;
    T E1y0 = 0, E1y1 = 0, E1y2 = 0, E1y3 = 0, E1y4 = 0;
    T E1z0 = 0, E1z1 = 0, E1z2 = 0, E1z3 = 0, E1z4 = 0;
    T B0x0 = 0, B0x1 = 0, B0y0 = 0, B0y1 = 0, B1x0 = 0, B1x1 = 0, B1y0 = 0, B1y1 = 0, B1z0 = 0, B1z1 = 0;
    T ph0 = 0, ph1 = 0, ph2 = 0, ph3 = 0, pb0 = 0, pb1 = 0, pb2 = 0;
    T N0x1 = 0, N0x2 = 0, N0x3 = 0, N0x4 = 0, N0x5 = 0;  // B^{n+1}
    T N0y1 = 0, N0y2 = 0, N0y3 = 0, N0y4 = 0;
    T N1x1 = 0, N1x2 = 0, N1x3 = 0, N1x4 = 0, N1x5 = 0;
    T N1y1 = 0, N1y2 = 0, N1y3 = 0, N1y4 = 0;
    T N1z1 = 0, N1z2 = 0, N1z3 = 0, N1z4 = 0, N1z5 = 0;
    T SM2 = 0, SM3 = 0, SM4 = 0, DF2 = 0, DF3 = 0, DF4 = 0;  // 2 phi^{n+1}, dt D_t phi^{n+1}
    T EN2 = 0, EN3 = 0, EN4 = 0;                        // E0z^{n+1}
    T PX3 = 0, PX4 = 0, PY3 = 0, PY4 = 0;
    const int t0 = m0 - 2, t1 = m1 + 3;

    // Element offsets within an array are 32-bit: the host takes this kernel only
    // for grids of at most 2^32 cells.
    auto prefetch = [&](int p) {
        fill_y(p);
        int wp = p;
        if (wp < 0 || wp >= ny) wp = pery ? ((wp % ny) + ny) % ny : -1;
        const bool ok = wx >= 0 && wp >= 0;
        const unsigned o = ok ? (unsigned)wx + (unsigned)nx * (unsigned)wp : 0u;
        T *st = stage + ((p - t0) & (NS - 1)) * (NIN * ntx) + tx * NIN;
        cp_elem(st + 0, P.Ein[2] + o, ok);
        cp_elem(st + 1, P.Ein[3] + o, ok);
        cp_elem(st + 2, P.Ein[4] + o, ok);
        cp_elem(st + 3, P.Ein[5] + o, ok);
        cp_elem(st + 4, P.Bin[0] + o, ok);
        cp_elem(st + 5, P.Bin[1] + o, ok);
        cp_elem(st + 6, P.Bin[3] + o, ok);
        cp_elem(st + 7, P.Bin[4] + o, ok);
        cp_elem(st + 8, P.Bin[5] + o, ok);
        cp_elem(st + 9, P.phi + o, ok);
        cp_elem(st + 10, P.phib + o, ok);
    };
    auto take = [&](int p) {
        const T *st = stage + ((p - t0) & (NS - 1)) * (NIN * ntx) + tx * NIN;
        E0z0 = st[0];
        E1x0 = st[1];
        E1y0 = st[2];
        E1z0 = st[3];
        B0x0 = st[4];
        B0y0 = st[5];
        B1x0 = st[6];
        B1y0 = st[7];
        B1z0 = st[8];
        ph0 = st[9];
        pb0 = st[10];
    };
    // Absorbing-layer half-step F <- ((1 - s h/2) F + h X) / (1 + s h/2) written as
    // a F + b X, and two of them as a^2 F + b (1 + a) X, with per-axis tables; at a
    // corner s is the largest of the axes' values and every coefficient decreases
    // with s, so the corner's coefficients are the smallest of the axes'.  Where
    // a = 1 (no layer) the plain half-steps are taken, bit for bit.
    auto lay = [&](bool in, int p, T &a1, T &b1, T &a2, T &b2) {
        a1 = ax1;
        b1 = bx1;
        a2 = ax2;
        b2 = bx2;
        if (in && !pery) {
            const T *y = yring[p & (YR - 1)];
            a1 = smin(a1, y[Y_A1]);
            b1 = smin(b1, y[Y_B1]);
            a2 = smin(a2, y[Y_A2]);
            b2 = smin(b2, y[Y_B2]);
        }
    };
    auto inside = [&](int p) { return wx >= 0 && (pery || (p >= 0 && p < ny)); };

    // one iteration's four stages; EDGE adds the closure zeros and the layer damping
    auto body = [&](auto edge_tag, int t, int b) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        T(*R)[RS] = rows[b];
        // ---- stage 1: B^{n+1} on plane t-1 ----
        {
            const int p = t - 1;
            const bool in = !EDGE || inside(p);
            // differences of E^{n+1/2} (times the cell size)
            const T d0y = E0z0 - E0z1, d0x = R[R_E0Z][tx + 2] - E0z1;
            const T d1zy = E1z0 - E1z1, d1zx = R[R_E1Z][tx + 2] - E1z1;
            const T d1yx = R[R_E1Y][tx + 2] - E1y1, d1xy = E1x0 - E1x1;
            // B^{n+1} = B^n - 2h curl E^{n+1/2}: the two half-steps as one multiply-add
            // per difference, (curl E0)_x = D_y E0z, (curl E0)_y = -D_x E0z,
            // (curl E1)_z = D_x E1y - D_y E1x
            auto plain = [&]() {
                N0x1 = fma(-h2y, d0y, B0x1);
                N0y1 = fma(h2x, d0x, B0y1);
                N1x1 = fma(-h2y, d1zy, B1x1);
                N1y1 = fma(h2x, d1zx, B1y1);
                N1z1 = fma(-h2x, d1yx, fma(h2y, d1xy, B1z1));
            };
            if (!EDGE) {
                plain();
            } else {
                T a1, b1, a2, b2;
                lay(in, p, a1, b1, a2, b2);
                if (a2 == T(1)) {
                    plain();
                } else {
                    const T c0x = d0y * idy, c0y = -d0x * idx, c1x = d1zy * idy, c1y = -d1zx * idx;
                    const T c1z = d1yx * idx - d1xy * idy;
                    N0x1 = fma(-b2, c0x, a2 * B0x1);
                    N0y1 = fma(-b2, c0y, a2 * B0y1);
                    N1x1 = fma(-b2, c1x, a2 * B1x1);
                    N1y1 = fma(-b2, c1y, a2 * B1y1);
                    N1z1 = fma(-b2, c1z, a2 * B1z1);
                }
            }
            // magnetic sheet on the B0y faces at the plane: -w tau in each of the two
            // half-steps (the sheet stops at the transverse layers: w = 0 there)
            if (src_b_col) N0y1 = fma(-yring[p & (YR - 1)][Y_W], P.src_b, N0y1);
            if (EDGE && !in) N0x1 = N0y1 = N1x1 = N1y1 = N1z1 = T(0);
            if (write_col && p >= m0 && p < m1) {
                const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                P.Bout[0][gi] = N0x1;
                P.Bout[1][gi] = N0y1;
                P.Bout[3][gi] = N1x1;
                P.Bout[4][gi] = N1y1;
                P.Bout[5][gi] = N1z1;
            }
        }
        // ---- stage 2: axion on plane t-2, E0z^{n+1} ----
        {
            const int p = t - 2;
            const bool in = !EDGE || inside(p);
            // S/g = Ebar0 . Bbar0 = E0z B_ext,z (only E0z and the background along z)
            // FP32 split: second differences formed from neighbour differences and the
            // mass term kept apart, so that neither rounds against the 2*phi terms
            const T spx = INCR ? (R[R_PHI][tx + 2] - ph2) + (R[R_PHI][tx] - ph2) : R[R_PHI][tx + 2] + R[R_PHI][tx];
            const T spy = INCR ? (ph1 - ph2) + (ph3 - ph2) : ph1 + ph3;
            const T sa = (EDGE && in && P.has_pml) ? (pery ? sxa : smax(sxa, yring[p & (YR - 1)][Y_SA])) : T(0);
            T nw, pin = T(0);
            if (!EDGE || sa == T(0)) {
                T acc = INCR ? fma(c0, ph2, pb2) : fma(c0, ph2, -pb2);
                acc = fma(cx, spx, acc);
                acc = fma(cy, spy, acc);
                acc = fma(dt2gBz, E0z2, acc);
                if (INCR) {
                    pin = acc;
                    nw = ph2 + pin;
                } else {
                    nw = acc;
                }
            } else {
                const T lap = INCR ? spx * P.idx2[0] + spy * P.idx2[1]
                                   : (spx - T(2) * ph2) * P.idx2[0] + (spy - T(2) * ph2) * P.idx2[1];
                const T S = E0z2 * Bz;
                const T Y = ((g * S - P.m2 * ph2) + lap) - sa * sa * ph2;
                // damped leapfrog (1 + s dt) pi^{n+1} = dt^2 Y + (1 - s dt) pi^n as
                // pi^{n+1} = c1 Y + c2 pi^n, with the corner's (smallest) coefficients
                T c1 = kx1, c2 = kx2;
                if (!pery) {
                    c1 = smin(c1, yring[p & (YR - 1)][Y_K1]);
                    c2 = smin(c2, yring[p & (YR - 1)][Y_K2]);
                }
                if (INCR) {
                    pin = fma(c1, Y, c2 * pb2);
                    nw = ph2 + pin;
                } else {
                    nw = ph2 + fma(c1, Y, c2 * (ph2 - pb2));
                }
            }
            if (INCR) {
                SM2 = fma(T(2), ph2, pin);
                DF2 = pin;
            } else {
                SM2 = nw + ph2;
                DF2 = nw - ph2;
            }
            if (write_col && p >= m0 && p < m1) {
                const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                P.phi_out[gi] = nw;
                if (INCR) P.phib_out[gi] = pin;
            }
            // E0z^{n+1} = E0z^{n+1/2} + h (curl B0)_z, (curl B0)_z = D_x B0y - D_y B0x at the
            // E0z location (backward differences)
            const T dbx = N0y2 - R[R_N0Y2][tx], dby = N0x2 - N0x3;
            if (!EDGE) {
                EN2 = fma(hx, dbx, fma(-hy, dby, E0z2));
            } else {
                T a1, b1, a2, b2;
                lay(in, p, a1, b1, a2, b2);
                EN2 = a1 == T(1) ? fma(hx, dbx, fma(-hy, dby, E0z2)) : fma(b1, dbx * idx - dby * idy, a1 * E0z2);
            }
            if (src_e_col) EN2 = fma(yring[p & (YR - 1)][Y_W], P.src_e, EN2);  // electric sheet
            if (EDGE && !in) SM2 = DF2 = EN2 = T(0);
        }
        // ---- stage 3: P^{n+1} on plane t-3 ----
        {
            const int p = t - 3;
            if constexpr (FOLDP) {
                // P / (1/(2 dt)) = DF (N + N') + (E0z q) dphi, q = (1/(4 dx)) / (1/(2 dt))
                const T ENq = EN3 * qq;
                PX3 = fma(ENq, SM2 - SM4, DF3 * (N0x3 + N0x4));
                PY3 = fma(-ENq, R[R_MID3][tx + 2] - R[R_MID3][tx], DF3 * (N0y3 + R[R_N0Y3][tx]));
            } else {
            const T bbx = fma(hinv_dt, N0x3 + N0x4, Bxi);  // Bbar_x / dt
            const T bby = fma(hinv_dt, N0y3 + R[R_N0Y3][tx], Byi);
            const T dpy = (SM2 - SM4) * qidy;
            const T dpx = (R[R_MID3][tx + 2] - R[R_MID3][tx]) * qidx;
            PX3 = fma(EN3, dpy, DF3 * bbx);   // Dt Bbar_x - (Ebar_y dphi_z - Ebar_z dphi_y)
            PY3 = fma(-EN3, dpx, DF3 * bby);  // Dt Bbar_y - (Ebar_z dphi_x - Ebar_x dphi_z)
            }
            // P_z = Dt B_ext,z (no laser B0z, no Ebar_x, Ebar_y): DF B_ext,z/dt, folded into E1z
            if (EDGE && !inside(p)) PX3 = PY3 = T(0);
        }
        // ---- stage 4: J^{n+1}, E^{n+3/2} on plane t-4 ----
        {
            const int p = t - 4;
            if (p >= m0 && p < m1) {
                const bool in = !EDGE || inside(p);
                // J^{n+1} = face averages of P; E^{n+3/2} = E^{n+1/2} + 2h (curl B1^{n+1} - g J^{n+1})
                // with (curl B1)_x = D_y B1z, (curl B1)_y = -D_x B1z, (curl B1)_z = D_x B1y - D_y B1x,
                // and E0z^{n+3/2} = E0z^{n+1} + h (curl B0^{n+1})_z
                const T sjx = PX4 + R[R_PX4][tx + 2], sjy = PY4 + PY3;  // 2 J_x, 2 J_y
                const T e1zy = N1z4 - N1z5, e1zx = N1z4 - R[R_N1Z4][tx];
                const T e1yx = N1y4 - R[R_N1Y4][tx], e1xy = N1x4 - N1x5;
                T ex, ey, ez, e0;
                // E0z's two half-steps read the same curl of B0^{n+1}: E0z^{n+3/2} =
                // 2 E0z^{n+1} - E0z^{n+1/2} (an electric sheet's term is in it twice, too)
                auto plain = [&]() {
                    ex = fma(h2y, e1zy, fma(-hgP, sjx, E1x4));
                    ey = fma(-h2x, e1zx, fma(-hgP, sjy, E1y4));
                    ez = fma(h2x, e1yx, fma(-h2y, e1xy, fma(-h2gBzi, DF4, E1z4)));
                    e0 = fma(T(2), EN4, -E0z4);
                };
                if (!EDGE) {
                    plain();
                } else {
                    T a1, b1, a2, b2;
                    lay(in, p, a1, b1, a2, b2);
                    if (a2 == T(1)) {
                        plain();
                    } else {
                        const T xx = fma(-gP, T(0.5) * sjx, e1zy * idy);
                        const T xy = fma(-gP, T(0.5) * sjy, -e1zx * idx);
                        const T xz = fma(-gBzi, DF4, e1yx * idx - e1xy * idy);
                        const T e0yx = N0y4 - R[R_N0Y4][tx], e0xy = N0x4 - N0x5;
                        ex = fma(b2, xx, a2 * E1x4);
                        ey = fma(b2, xy, a2 * E1y4);
                        ez = fma(b2, xz, a2 * E1z4);
                        e0 = fma(b1, e0yx * idx - e0xy * idy, a1 * EN4);
                    }
                }
                if (write_col) {
                    const unsigned gi = (unsigned)gx + (unsigned)nx * (unsigned)p;
                    P.Eout[3][gi] = ex;
                    P.Eout[4][gi] = ey;
                    P.Eout[5][gi] = ez;
                    P.Eout[2][gi] = e0;
                }
            }
        }
    };

    // planes t0 .. t0+NS-2 in flight, then one more per iteration; after the
    // wait at the end of iteration t everything up to plane t+1 has landed
    for (int p = t0 - 4; p < t0; p++) fill_y(p);  // joins the first group (plane t0)
    for (int j = 0; j < NS - 1; j++) {
        if (!dead && t0 + j <= t1) prefetch(t0 + j);
        cp_commit();
    }
    cp_wait<NS - 2>();
    if (!dead) take(t0);
    __syncthreads();
    // FP32: unrolled by 4, so that the column history shifts become register
    // renaming and the row buffer and staging slot indices (taken relative to t0)
    // become constants; FP64 is bound by its FP64 pipe and keeps the rolled loop
    // (its registers are at the limit)
#pragma unroll(sizeof(T) == 4 ? 4 : 1)
    for (int t = t0; t <= t1; ++t) {
        if (!dead && t + NS - 1 <= t1) prefetch(t + NS - 1);
        cp_commit();
        const int b = (t - t0) & 1;
        // publish what the x neighbours read in this iteration (a dead warp's slots
        // keep their zeros; fill_y is warp 0's, which always holds a column of the grid)
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
        // advance the column history by one plane
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
        cp_wait<NS - 2>();
        if (!dead && t < t1) take(t + 1);
    }
    cp_wait<0>();
}

// The tile of strip bx and march chunk by of the uniform launch grid.  The strips
// at a non-periodic x edge (which carry the x layers and run the edge body) may
// march shorter chunks than the others; the others' first chunk (and, by the
// host's choice of sizes, about the last) may be shorter than the rest, since they
// run the edge body over the y layers.
template <typename T, bool INCR, bool SRC = false, bool FOLDP = false>
__device__ __forceinline__ void tile(const fused::Params<T> &P, const int bx, const int by, T (&rows)[2][NROWS][RS],
                                     T *stage)
{
    const int ntx = (int)blockDim.x, vx = ntx - HL - HR;
    const int nx = P.n[0], ny = P.n[1];
    const int nstrips = (nx + vx - 1) / vx;
    const bool xstrip = !P.per[0] && (bx == 0 || bx == nstrips - 1);
    const int chunk = xstrip ? P.chunk_edge : P.chunk;
    const int first = xstrip ? P.chunk_edge : P.chunk_first;
    const int m0 = by == 0 ? 0 : first + (by - 1) * chunk;
    if (m0 >= ny) return;  // (the whole block: more chunk rows than this strip uses)
    const int m1 = min(ny, by == 0 ? first : m0 + chunk);
    tile_span<T, INCR, SRC, FOLDP>(P, bx, m0, m1, rows, stage);
}

template <typename T, bool INCR, bool SRC, bool FOLDP = false>
__global__ void __launch_bounds__(TX, sizeof(T) == 4 ? 2 : 1) k_tm2d(fused::Params<T> P)
{
    __shared__ T rows[2][NROWS][RS];
    extern __shared__ __align__(16) unsigned char tm2d_dyn[];
    tile<T, INCR, SRC, FOLDP>(P, (int)blockIdx.x, (int)blockIdx.y, rows, reinterpret_cast<T *>(tm2d_dyn));
}

template <typename T, bool INCR, bool SRC, bool FOLDP = false>
cudaError_t launch_variant(const fused::Params<T> &P, int nchunks, cudaStream_t stream, int *occupancy, int tx)
{
    // resident blocks per SM for each tile width (multiples of 32 up to TX)
    static int occ[TX / 32 + 1] = {};
    auto kern = k_tm2d<T, INCR, SRC, FOLDP>;
    // the staging ring is sized for the launch's tile width
    const size_t dyn = stage_bytes<T>(tx);
    if (tx < 64 || tx > TX || tx % 32) return cudaErrorInvalidValue;
    if (occ[tx / 32] == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes<T>());
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[tx / 32], kern, tx, dyn);
        if (e != cudaSuccess) return e;
    }
    if (occupancy) *occupancy = occ[tx / 32];
    if (nchunks <= 0) return cudaSuccess;
    const int vx = tx - HL - HR;
    dim3 grid((P.n[0] + vx - 1) / vx, nchunks, 1);
    kern<<<grid, tx, dyn, stream>>>(P);
    return cudaGetLastError();
}

// Work-list form: block b runs the tiles items[b * per_block + j], j < per_block,
// one after the other (x: strip, y and z: planes [y, z); an item with z <= y is
// empty).  The host balances the lists so that every block's tiles cost about
// the same, with all blocks resident at once.
template <typename T, bool INCR, bool FOLDP>
__global__ void __launch_bounds__(TX, sizeof(T) == 4 ? 2 : 1)
    k_tm2d_list(fused::Params<T> P, const int4 *__restrict__ items, int per_block)
{
    __shared__ T rows[2][NROWS][RS];
    extern __shared__ __align__(16) unsigned char tm2d_dyn[];
    for (int j = 0; j < per_block; j++) {
        const int4 it = items[(size_t)blockIdx.x * per_block + j];
        if (it.z <= it.y) continue;  // (the same item for the whole block)
        if (j > 0) __syncthreads();  // the previous tile's last reads of rows and yring
        tile_span<T, INCR, false, FOLDP>(P, it.x, it.y, it.z, rows, reinterpret_cast<T *>(tm2d_dyn));
    }
}

template <typename T, bool INCR, bool FOLDP>
cudaError_t launch_list_variant(const fused::Params<T> &P, const int4 *items, int nblocks, int per_block,
                                cudaStream_t stream, int *occupancy, int tx)
{
    static int occ[TX / 32 + 1] = {};
    auto kern = k_tm2d_list<T, INCR, FOLDP>;
    const size_t dyn = stage_bytes<T>(tx);
    if (tx < 64 || tx > TX || tx % 32) return cudaErrorInvalidValue;
    if (occ[tx / 32] == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes<T>());
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[tx / 32], kern, tx, dyn);
        if (e != cudaSuccess) return e;
    }
    if (occupancy) *occupancy = occ[tx / 32];
    if (nblocks <= 0) return cudaSuccess;
    kern<<<nblocks, tx, dyn, stream>>>(P, items, per_block);
    return cudaGetLastError();
}

// The work-list form takes grids without a soft source.
template <typename T, bool INCR>
cudaError_t launch_list(const fused::Params<T> &P, const int4 *items, int nblocks, int per_block, cudaStream_t stream,
                        int *occupancy, int tx)
{
    if (P.src_x >= 0) return cudaErrorInvalidValue;
#ifndef AXP_TM2D_NO_FOLDP
    if (sizeof(T) == 8 && P.Bext[0] == T(0) && P.Bext[1] == T(0) && P.idx[0] == P.idx[1])
        return launch_list_variant<T, INCR, true>(P, items, nblocks, per_block, stream, occupancy, tx);
#endif
    return launch_list_variant<T, INCR, false>(P, items, nblocks, per_block, stream, occupancy, tx);
}

template <typename T, bool INCR>
cudaError_t launch(const fused::Params<T> &P, int nchunks, cudaStream_t stream, int *occupancy, int tx = TX)
{
    if (P.src_x >= 0) return launch_variant<T, INCR, true>(P, nchunks, stream, occupancy, tx);
#ifndef AXP_TM2D_NO_FOLDP
    // FP64 with square cells and no uniform B along x or y: the folded current
    if (sizeof(T) == 8 && P.Bext[0] == T(0) && P.Bext[1] == T(0) && P.idx[0] == P.idx[1])
        return launch_variant<T, INCR, false, true>(P, nchunks, stream, occupancy, tx);
#endif
    return launch_variant<T, INCR, false>(P, nchunks, stream, occupancy, tx);
}

}  // namespace tm2d
}  // namespace axp

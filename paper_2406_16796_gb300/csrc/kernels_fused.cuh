// kernels_fused.cuh -- single-pass fused step (arXiv 2406.16796 Sec. 2.3-2.4).
//
// One launch advances every field one full time step.  The kernel keeps the
// leapfrog-staggered state (E^{n+1/2}, B^n, phi^{n+1/2}, phi^{n-1/2}): the two
// E half-steps of consecutive steps share the same curl B^{n+1} - g J^{n+1},
// so the axion current is formed exactly once per step and never stored.
// Per step (order 0 always before order 1, as in the half-step scheme):
//   1. B^{n+1/2}, B^{n+1}   = B^n - h curl E^{n+1/2} (twice)
//   2. S^{n+1/2} = Ebar0 . Bbar0 (without g),  phi^{n+3/2}  (PML form in the layer),
//      phi^{n+1} and D_t phi^{n+1},  E0^{n+1} = E0^{n+1/2} + h curl B0^{n+1}
//   3. P^{n+1} = (D_t phi) Bbar0 - Ebar0 x grad_c phi at cell centres
//   4. J^{n+1} = face average of P;  E1^{n+3/2} = E1^{n+1/2} + 2 x h (curl B1^{n+1} - g J^{n+1}),
//      E0^{n+3/2} = E0^{n+1} + h curl B0^{n+1}
//
// Geometry: a CTA owns a transverse tile (x in 1D/2D; x-y in 3D) including a
// halo of 2 cells below and 3 above, and marches along the last grid axis
// (y in 2D, z in 3D) plane by plane.  Each stage runs one plane behind the
// previous one, so every plane of every intermediate is computed once per
// CTA and kept in a small shared-memory ring (5 planes deep at most).  Inputs
// are read once from HBM (halo columns from L2) and outputs written once, to
// the other field set (no in-place update: neighbouring CTAs still read the
// old values).
//
// Boundaries: periodic axes are loaded wrapped.  On non-periodic axes E and B
// are zero outside the grid (written as zero when an intermediate lands
// outside), and axion reads outside the grid are redirected at read time to
// the mirror cell (reflect) or read as zero (PML, and cells outside along two
// axes).  Absorbing layers damp E/B and phi with the profiles of the general
// path.  Outflow axion boundaries and a uniform background E are left to the
// general kernels.
#pragma once

#include <type_traits>
#include <utility>

#include "device_common.cuh"

namespace axp {
namespace fused {

constexpr int HL = 2, HR = 3;

template <typename T, int MODE>
struct Tile {
    // 1D grids are short (the state of a 4096-cell run is 256 KB): narrow tiles
    // spread one step over more SMs
    static constexpr int TX = MODE == 3 ? 32 : (MODE == 1 ? (sizeof(T) == 8 ? 32 : 64) : (sizeof(T) == 8 ? 128 : 256));
    static constexpr int TY = MODE == 3 ? 16 : 1;
    static constexpr int NT = TX * TY;
    static constexpr int VX = TX - HL - HR;  // valid outputs per tile along x
    static constexpr int VY = MODE == 3 ? TY - HL - HR : 1;
    static constexpr bool MARCH = MODE >= 2;
};

__host__ __device__ constexpr bool axis_on(int MODE, int a) { return a == 0 || (a == 1 && MODE >= 2) || (a == 2 && MODE == 3); }

// Shared-memory ring layout (in planes of NT cells) for the active component sets.
template <int MODE, int E0M, int B0M>
struct Lay {
    static constexpr bool M = MODE >= 2;
    static constexpr int DE = M ? 6 : 1, DB = M ? 2 : 1, DPHI = M ? 4 : 1, DPB = M ? 3 : 1, DBH = M ? 3 : 1,
                         DBN = M ? 5 : 1, DMID = M ? 3 : 1, DDT = M ? 3 : 1, DE0N = M ? 3 : 1, DP = M ? 2 : 1;
    __host__ __device__ static constexpr bool e_on(int q) { return q >= 3 || ((E0M >> q) & 1); }  // q: 0-2 order 0, 3-5 order 1
    __host__ __device__ static constexpr bool b_on(int q) { return q >= 3 || ((B0M >> q) & 1); }
    __host__ __device__ static constexpr int base_E(int q)
    {
        int o = 0;
        for (int i = 0; i < q; i++) o += e_on(i) ? DE : 0;
        return o;
    }
    __host__ __device__ static constexpr int base_B(int q)
    {
        int o = base_E(6);
        for (int i = 0; i < q; i++) o += b_on(i) ? DB : 0;
        return o;
    }
    static constexpr int PHI = base_B(6);
    static constexpr int PB = PHI + DPHI;
    __host__ __device__ static constexpr int base_BH(int a)
    {
        int o = PB + DPB;
        for (int i = 0; i < a; i++) o += ((B0M >> i) & 1) ? DBH : 0;
        return o;
    }
    __host__ __device__ static constexpr int base_BN(int q)
    {
        int o = base_BH(3);
        for (int i = 0; i < q; i++) o += b_on(i) ? DBN : 0;
        return o;
    }
    static constexpr int MID = base_BN(6);
    static constexpr int DTQ = MID + DMID;
    __host__ __device__ static constexpr int base_E0N(int a)
    {
        int o = DTQ + DDT;
        for (int i = 0; i < a; i++) o += ((E0M >> i) & 1) ? DE0N : 0;
        return o;
    }
    __host__ __device__ static constexpr int base_P(int a) { return base_E0N(3) + a * DP; }
    static constexpr int PLANES = base_P(3);
};

template <typename T>
struct Params {
    const T *Ein[6], *Bin[6];  // order-0 xyz then order-1 xyz: E^{n+1/2}, B^n
    const T *phi, *phib;       // phi^{n+1/2}; phi^{n-1/2} (two levels) or the increment pi^n
    T *Eout[6], *Bout[6];
    T *phi_out, *phib_out;     // phi^{n+3/2}; pi^{n+1} (increment storage only)
    const T *sig_em[3], *sig_ax[3];
    const T *pml_tab[3];  // per axis 6 x n: layer coefficients a, b, a^2, b(1+a) (E/B) and c1, c2 (axion)
    int n[3];
    int per[3];
    int axbc[3][2];
    int chunk;
    int chunk_edge;   // march chunk of the strips at a non-periodic x edge (2D TM kernel)
    int chunk_first;  // first (and about the last) chunk of the other strips (2D TM kernel)
    int has_pml;
    int lay[3][2];  // cells of absorbing layer at each side (0 where none)
    T idx[3], hidx[3], idx2[3];  // 1/d, 1/(2d), 1/d^2
    T lap_c[3];                  // dt^2/d^2
    T lap_0;                     // two levels: 2 - dt^2 (m^2 + 2 sum 1/d^2); increment: -dt^2 m^2
    T dt2g;                      // dt^2 g
    T h, dt, dt2, inv_dt, g, m2;
    T Bext[3];
    // soft source (2D TM kernel): the x column of the sheet's E cells (-1: none), the
    // electric sheet's weight per row (A pol_z f/dx), and this step's factors
    // src_b = 2h tau(x_p + dx/2, t_{n+1/2}) (magnetic sheet, both B half-steps) and
    // src_e = h tau(x_p, t_{n+1}) (electric sheet, each E half-step that reads B^{n+1})
    int src_x;
    const T *src_w;
    T src_b, src_e;
};

// Compile-time loop: f(integral_constant<int, I>) for I = 0 .. N-1.
template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

template <int D>
__device__ __forceinline__ int slot(int p)
{
    return (p + 600 * D) % D;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T, bool INCR, int MODE, int E0M, int B0M>
struct Kernel {
    using TL = Tile<T, MODE>;
    using L = Lay<MODE, E0M, B0M>;
    static constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT;
    static constexpr int MA = MODE == 3 ? 2 : 1;  // march axis (unused in 1D)

    const Params<T> &P;
    T *sm;
    int tx, ty, gx, gy, nm;

    __device__ Kernel(const Params<T> &p, T *s) : P(p), sm(s) {}

    // generic offset (dx, dy, dz) -> transverse tile offsets and march-plane offset
    __device__ static constexpr int ox(int dx, int, int) { return dx; }
    __device__ static constexpr int oy(int, int dy, int) { return MODE == 3 ? dy : 0; }
    __device__ static constexpr int op(int, int dy, int dz) { return MODE == 2 ? dy : (MODE == 3 ? dz : 0); }

    // Ring access.  Away from the grid edges (E = false) neighbour offsets stay
    // within one cell of the tile and land in the guard band around the ring,
    // so no clamping is needed; near edges (E = true) indices are clamped.
    template <int D, bool E = true>
    __device__ __forceinline__ T &at(int base, int p, int x, int y)
    {
        if (E) return sm[(base + slot<D>(p)) * NT + clampi(y, 0, TY - 1) * TX + clampi(x, 0, TX - 1)];
        return sm[(base + slot<D>(p)) * NT + y * TX + x];
    }

    // plain ring read (E/B-type quantities) at generic offset
    template <int D, bool E = true>
    __device__ __forceinline__ T rd(int base, int p, int dx, int dy, int dz)
    {
        return at<D, E>(base, p + op(dx, dy, dz), tx + ox(dx, dy, dz), ty + oy(dx, dy, dz));
    }

    // axion-type ring read; near edges the ghost rules are applied at read time
    template <int D, bool E = true>
    __device__ __forceinline__ T rdphi(int base, int p, int dx, int dy, int dz)
    {
        if (!E) return rd<D, false>(base, p, dx, dy, dz);
        int c[3] = {gx + ox(dx, dy, dz), gy + oy(dx, dy, dz), p + op(dx, dy, dz)};
        const int ax_of[3] = {0, 1, MA};
        const int lim[3] = {P.n[0], MODE == 3 ? P.n[1] : 1, nm};
        int nout = 0, which = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if ((k == 1 && MODE != 3) || (k == 2 && MODE == 1)) continue;
            const int a = ax_of[k];
            if (!P.per[a] && (c[k] < 0 || c[k] >= lim[k])) {
                nout++;
                which = k;
            }
        }
        if (nout > 1) return T(0);
        if (nout == 1) {
            const int a = ax_of[which];
            const int side = c[which] < 0 ? 0 : 1;
            if (P.axbc[a][side] != AXP_BC_REFLECT) return T(0);
            c[which] = clampi(side ? 2 * lim[which] - 1 - c[which] : -1 - c[which], 0, lim[which] - 1);
        }
        return at<D>(base, c[2], tx + (c[0] - gx), ty + (c[1] - gy));
    }

    __device__ __forceinline__ bool inside(int p) const
    {
        if (!P.per[0] && (gx < 0 || gx >= P.n[0])) return false;
        if (MODE == 3 && !P.per[1] && (gy < 0 || gy >= P.n[1])) return false;
        if (MODE >= 2 && !P.per[MA] && (p < 0 || p >= nm)) return false;
        return true;
    }

    __device__ __forceinline__ int wrap(int c, int n, int per) const
    {
        if (c >= 0 && c < n) return c;
        if (!per) return -1;
        c %= n;
        return c < 0 ? c + n : c;
    }

    // global linear index of the tile cell on plane p, or -1 outside the grid
    __device__ __forceinline__ int64_t gidx(int p) const
    {
        const int wx = wrap(gx, P.n[0], P.per[0]);
        const int wy = MODE == 3 ? wrap(gy, P.n[1], P.per[1]) : 0;
        const int wm = MODE >= 2 ? wrap(p, nm, P.per[MA]) : 0;
        if (wx < 0 || wy < 0 || wm < 0) return -1;
        if (MODE == 1) return wx;
        if (MODE == 2) return wx + (int64_t)P.n[0] * wm;
        return wx + (int64_t)P.n[0] * (wy + (int64_t)P.n[1] * wm);
    }

    __device__ __forceinline__ T sigma(const T *const tab[3], int p) const
    {
        const int wx = wrap(gx, P.n[0], P.per[0]);
        T s = tab[0][wx < 0 ? 0 : wx];
        if (MODE >= 2) {
            const int wy = MODE == 3 ? wrap(gy, P.n[1], P.per[1]) : wrap(p, nm, P.per[1]);
            const T s1 = tab[1][wy < 0 ? 0 : wy];
            if (s1 > s) s = s1;
        }
        if (MODE == 3) {
            const int wz = wrap(p, nm, P.per[2]);
            const T s2 = tab[2][wz < 0 ? 0 : wz];
            if (s2 > s) s = s2;
        }
        return s;
    }

    __device__ __forceinline__ T half(T F, T X, T sig) const
    {
        if (sig == T(0)) return fma(P.h, X, F);
        return ((T(1) - sig * P.h / T(2)) * F + P.h * X) / (T(1) + sig * P.h / T(2));
    }

    // 4-point average of order-0 B component A to the cell centre (Sec. 2.3);
    // an invariant axis folds its two coinciding samples.  Plus the background.
    template <int D, bool E, int A>
    __device__ __forceinline__ T bbar_c(int base, int p)
    {
        constexpr int b = (A + 1) % 3, c = (A + 2) % 3;
        constexpr bool ab = axis_on(MODE, b), ac = axis_on(MODE, c);
        constexpr int bx = b == 0, by = b == 1, bz = b == 2, cx = c == 0, cy = c == 1, cz = c == 2;
        const T B0 = rd<D, E>(base, p, 0, 0, 0);
        T s;
        if constexpr (ab && ac)
            s = T(0.25) * (((B0 + rd<D, E>(base, p, -cx, -cy, -cz)) + rd<D, E>(base, p, -bx, -by, -bz)) +
                           rd<D, E>(base, p, -bx - cx, -by - cy, -bz - cz));
        else if constexpr (ab)
            s = T(0.5) * (B0 + rd<D, E>(base, p, -bx, -by, -bz));
        else if constexpr (ac)
            s = T(0.5) * (B0 + rd<D, E>(base, p, -cx, -cy, -cz));
        else
            s = B0;
        return s + P.Bext[A];
    }

    // 2-point average of order-0 E component A to the cell centre
    template <int D, bool E, int A>
    __device__ __forceinline__ T ebar_c(int base, int p)
    {
        const T E0 = rd<D, E>(base, p, 0, 0, 0);
        if constexpr (!axis_on(MODE, A)) return E0;
        else return T(0.5) * (E0 + rd<D, E>(base, p, -(A == 0), -(A == 1), -(A == 2)));
    }

    // (curl B)_A at the E_A location from the B^{n+1} ring of order O (backward differences)
    template <int O, int A>
    __host__ __device__ static constexpr bool curl_b_t1()
    {
        return axis_on(MODE, (A + 1) % 3) && L::b_on(3 * O + (A + 2) % 3);
    }
    template <int O, int A>
    __host__ __device__ static constexpr bool curl_b_t2()
    {
        return axis_on(MODE, (A + 2) % 3) && L::b_on(3 * O + (A + 1) % 3);
    }
    template <bool E, int O, int A>
    __device__ __forceinline__ T curl_b_new(int p)
    {
        constexpr int b = (A + 1) % 3, c = (A + 2) % 3;
        T v = T(0);
        if constexpr (curl_b_t1<O, A>()) {
            constexpr int base = L::base_BN(3 * O + c);
            v = (rd<L::DBN, E>(base, p, 0, 0, 0) - rd<L::DBN, E>(base, p, -(b == 0), -(b == 1), -(b == 2))) * P.idx[b];
        }
        if constexpr (curl_b_t2<O, A>()) {
            constexpr int base = L::base_BN(3 * O + b);
            const T t = (rd<L::DBN, E>(base, p, 0, 0, 0) - rd<L::DBN, E>(base, p, -(c == 0), -(c == 1), -(c == 2))) * P.idx[c];
            if constexpr (curl_b_t1<O, A>()) v = v - t;
            else v = -t;
        }
        return v;
    }

    // Inputs of one plane: fetched into registers one iteration ahead (so the
    // HBM latency overlaps the compute stages), then committed to the rings.
    T pre[14];

    __device__ __forceinline__ void prefetch(int t)
    {
        const int64_t gi = gidx(t);
        sfor<6>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            if constexpr (L::e_on(q)) pre[q] = gi >= 0 ? __ldg(P.Ein[q] + gi) : T(0);
            if constexpr (L::b_on(q)) pre[6 + q] = gi >= 0 ? __ldg(P.Bin[q] + gi) : T(0);
        });
        pre[12] = gi >= 0 ? __ldg(P.phi + gi) : T(0);
        pre[13] = gi >= 0 ? __ldg(P.phib + gi) : T(0);
    }

    __device__ __forceinline__ void commit(int t)
    {
        sfor<6>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            if constexpr (L::e_on(q)) at<L::DE, false>(L::base_E(q), t, tx, ty) = pre[q];
            if constexpr (L::b_on(q)) at<L::DB, false>(L::base_B(q), t, tx, ty) = pre[6 + q];
        });
        at<L::DPHI, false>(L::PHI, t, tx, ty) = pre[12];
        at<L::DPB, false>(L::PB, t, tx, ty) = pre[13];
    }

    __device__ __forceinline__ bool out_ok(int p, int m0, int m1) const
    {
        if (tx < HL || tx >= TX - HR) return false;
        if (MODE == 3 && (ty < HL || ty >= TY - HR)) return false;
        if (gx < 0 || gx >= P.n[0]) return false;
        if (MODE == 3 && (gy < 0 || gy >= P.n[1])) return false;
        if (MODE >= 2 && (p < m0 || p >= m1)) return false;
        return true;
    }

    // Stage 1: B^{n+1/2}, B^{n+1} on plane p
    // Stage 1: B^{n+1/2}, B^{n+1} on plane p
    template <bool E>
    __device__ void stage1(int p, int m0, int m1)
    {
        const bool in = !E || inside(p);
        const T sig = (E && in && P.has_pml) ? sigma(P.sig_em, p) : T(0);
        const bool wr = out_ok(p, m0, m1);
        const int64_t gi = wr ? gidx(p) : -1;
        sfor<6>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            if constexpr (L::b_on(q)) {
                constexpr int o = q / 3, a = q % 3, b = (a + 1) % 3, c = (a + 2) % 3;
                // (curl E)_a = D_b E_c - D_c E_b, forward differences
                constexpr bool t1 = axis_on(MODE, b) && L::e_on(3 * o + c);
                constexpr bool t2 = axis_on(MODE, c) && L::e_on(3 * o + b);
                T cE = T(0);
                if constexpr (t1) {
                    constexpr int base = L::base_E(3 * o + c);
                    cE = (rd<L::DE, E>(base, p, b == 0, b == 1, b == 2) - rd<L::DE, E>(base, p, 0, 0, 0)) * P.idx[b];
                }
                if constexpr (t2) {
                    constexpr int base = L::base_E(3 * o + b);
                    const T t = (rd<L::DE, E>(base, p, c == 0, c == 1, c == 2) - rd<L::DE, E>(base, p, 0, 0, 0)) * P.idx[c];
                    if constexpr (t1) cE = cE - t;
                    else cE = -t;
                }
                const T Bv = rd<L::DB, E>(L::base_B(q), p, 0, 0, 0);
                T Bh, Bn;
                if (!in) {
                    Bh = T(0);
                    Bn = T(0);
                } else if (sig == T(0)) {
                    if constexpr (t1 || t2) {
                        Bh = fma(-P.h, cE, Bv);
                        Bn = fma(-P.h, cE, Bh);
                    } else {
                        Bh = Bv;
                        Bn = Bv;
                    }
                } else {
                    Bh = half(Bv, -cE, sig);
                    Bn = half(Bh, -cE, sig);
                }
                if constexpr (o == 0) at<L::DBH, false>(L::base_BH(a), p, tx, ty) = Bh;
                at<L::DBN, false>(L::base_BN(q), p, tx, ty) = Bn;
                if (gi >= 0) P.Bout[q][gi] = Bn;
            }
        });
    }

    // Stage 2: source, axion leapfrog, phi^{n+1}, D_t phi^{n+1}, E0^{n+1} on plane p
    template <bool E>
    __device__ void stage2(int p, int m0, int m1)
    {
        const bool in = !E || inside(p);
        // S^{n+1/2} / g = Ebar0 . Bbar0 with B0^{n+1/2}
        constexpr bool hasS = E0M != 0;
        T S = T(0);
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr ((E0M >> a) & 1) {
                const T e = ebar_c<L::DE, E, a>(L::base_E(a), p);
                T bb;
                if constexpr ((B0M >> a) & 1) bb = bbar_c<L::DBH, E, a>(L::base_BH(a), p);
                else bb = P.Bext[a];
                if constexpr ((E0M & ((1 << a) - 1)) == 0) S = e * bb;
                else S = fma(e, bb, S);
            }
        });
        const T ph = rdphi<L::DPHI, E>(L::PHI, p, 0, 0, 0);
        const T pb = rd<L::DPB, E>(L::PB, p, 0, 0, 0);
        T sp[3];
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            // FP32 split (INCR): the second difference from neighbour differences, so
            // it does not round against 2*phi; FP64: the neighbour sum
            if constexpr (axis_on(MODE, a) && INCR)
                sp[a] = (rdphi<L::DPHI, E>(L::PHI, p, a == 0, a == 1, a == 2) - ph) +
                        (rdphi<L::DPHI, E>(L::PHI, p, -(a == 0), -(a == 1), -(a == 2)) - ph);
            else if constexpr (axis_on(MODE, a))
                sp[a] = rdphi<L::DPHI, E>(L::PHI, p, a == 0, a == 1, a == 2) +
                        rdphi<L::DPHI, E>(L::PHI, p, -(a == 0), -(a == 1), -(a == 2));
            else
                sp[a] = T(0);
        });
        const T sig = (E && in && P.has_pml) ? sigma(P.sig_ax, p) : T(0);
        T nw, pin = T(0);
        if (sig == T(0)) {
            T acc = INCR ? fma(P.lap_0, ph, pb) : fma(P.lap_0, ph, -pb);
            sfor<3>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (axis_on(MODE, a)) acc = fma(P.lap_c[a], sp[a], acc);
            });
            if constexpr (hasS) acc = fma(P.dt2g, S, acc);
            if constexpr (INCR) {
                pin = acc;
                nw = ph + pin;
            } else {
                nw = acc;
            }
        } else {
            T lap = T(0);
            sfor<3>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (axis_on(MODE, a)) lap = lap + (INCR ? sp[a] : sp[a] - T(2) * ph) * P.idx2[a];
            });
            const T Y = ((P.g * S - P.m2 * ph) + lap) - sig * sig * ph;
            if constexpr (INCR) {
                pin = (P.dt2 * Y + (T(1) - sig * P.dt) * pb) / (T(1) + sig * P.dt);
                nw = ph + pin;
            } else {
                nw = (P.dt2 * Y + sig * P.dt * pb + T(2) * ph - pb) / (T(1) + sig * P.dt);
            }
        }
        T mid, dtv;
        if constexpr (INCR) {
            mid = fma(T(0.5), pin, ph);
            dtv = pin * P.inv_dt;
        } else {
            mid = T(0.5) * (nw + ph);
            dtv = (nw - ph) * P.inv_dt;
        }
        at<L::DMID, false>(L::MID, p, tx, ty) = mid;
        at<L::DDT, false>(L::DTQ, p, tx, ty) = dtv;
        if (out_ok(p, m0, m1)) {
            const int64_t gi = gidx(p);
            P.phi_out[gi] = nw;
            if constexpr (INCR) P.phib_out[gi] = pin;
        }
        // E0^{n+1}
        const T sg = (E && in && P.has_pml) ? sigma(P.sig_em, p) : T(0);
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr ((E0M >> a) & 1) {
                constexpr bool any = curl_b_t1<0, a>() || curl_b_t2<0, a>();
                const T cB = curl_b_new<E, 0, a>(p);
                const T Eh = rd<L::DE, E>(L::base_E(a), p, 0, 0, 0);
                T En;
                if (!in) En = T(0);
                else if (sg == T(0)) En = any ? fma(P.h, cB, Eh) : Eh;
                else En = half(Eh, cB, sg);
                at<L::DE0N, false>(L::base_E0N(a), p, tx, ty) = En;
            }
        });
    }

    // Stage 3: P^{n+1} at cell centres on plane p
    template <bool E>
    __device__ void stage3(int p)
    {
        const T Dt = rdphi<L::DDT, E>(L::DTQ, p, 0, 0, 0);
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value, b = (a + 1) % 3, c = (a + 2) % 3;
            T Pa;
            if constexpr ((B0M >> a) & 1) Pa = Dt * bbar_c<L::DBN, E, a>(L::base_BN(a), p);
            else Pa = Dt * P.Bext[a];
            // -(Ebar_b dphi_c - Ebar_c dphi_b)
            if constexpr (((E0M >> b) & 1) && axis_on(MODE, c)) {
                const T eb = ebar_c<L::DE0N, E, b>(L::base_E0N(b), p);
                const T dc = (rdphi<L::DMID, E>(L::MID, p, c == 0, c == 1, c == 2) -
                              rdphi<L::DMID, E>(L::MID, p, -(c == 0), -(c == 1), -(c == 2))) * P.hidx[c];
                Pa = fma(-eb, dc, Pa);
            }
            if constexpr (((E0M >> c) & 1) && axis_on(MODE, b)) {
                const T ec = ebar_c<L::DE0N, E, c>(L::base_E0N(c), p);
                const T db = (rdphi<L::DMID, E>(L::MID, p, b == 0, b == 1, b == 2) -
                              rdphi<L::DMID, E>(L::MID, p, -(b == 0), -(b == 1), -(b == 2))) * P.hidx[b];
                Pa = fma(ec, db, Pa);
            }
            at<L::DP, false>(L::base_P(a), p, tx, ty) = Pa;
        });
    }

    // Stage 4: J^{n+1} and E^{n+3/2} on plane p
    template <bool E>
    __device__ void stage4(int p, int m0, int m1)
    {
        const bool in = !E || inside(p);
        const bool wr = out_ok(p, m0, m1) && in;
        const int64_t gi = wr ? gidx(p) : -1;
        const T sg = (E && in && P.has_pml) ? sigma(P.sig_em, p) : T(0);
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            constexpr int base = L::base_P(a);
            T J = rd<L::DP, E>(base, p, 0, 0, 0);
            if constexpr (axis_on(MODE, a)) J = T(0.5) * (J + rd<L::DP, E>(base, p, a == 0, a == 1, a == 2));
            constexpr bool any = curl_b_t1<1, a>() || curl_b_t2<1, a>();
            T X;
            if constexpr (any) X = fma(-P.g, J, curl_b_new<E, 1, a>(p));
            else X = -P.g * J;
            const T Eh = rd<L::DE, E>(L::base_E(3 + a), p, 0, 0, 0);
            T Enew;
            if (sg == T(0)) Enew = fma(P.h, X, fma(P.h, X, Eh));
            else Enew = half(half(Eh, X, sg), X, sg);
            if (gi >= 0) P.Eout[3 + a][gi] = Enew;
        });
        sfor<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr ((E0M >> a) & 1) {
                constexpr bool any = curl_b_t1<0, a>() || curl_b_t2<0, a>();
                const T cB = curl_b_new<E, 0, a>(p);
                const T En = rd<L::DE0N, E>(L::base_E0N(a), p, 0, 0, 0);
                T Enew;
                if (sg == T(0)) Enew = any ? fma(P.h, cB, En) : En;
                else Enew = half(En, cB, sg);
                if (gi >= 0) P.Eout[a][gi] = Enew;
            }
        });
    }

    // Does the transverse tile keep one cell clear of the grid edges and of
    // every absorbing layer (so that no boundary rule applies inside it)?
    __device__ bool tile_interior() const
    {
        const int gx0 = gx - tx, gx1 = gx0 + TX - 1;
        if (!P.per[0] && (gx0 - 1 < P.lay[0][0] || gx1 + 1 > P.n[0] - 1 - P.lay[0][1])) return false;
        if (MODE == 3) {
            const int gy0 = gy - ty, gy1 = gy0 + TY - 1;
            if (!P.per[1] && (gy0 - 1 < P.lay[1][0] || gy1 + 1 > P.n[1] - 1 - P.lay[1][1])) return false;
        }
        return true;
    }

    template <bool E>
    __device__ __forceinline__ void stages(int t, int m0, int m1)
    {
        if (t - 1 >= m0 - 2) stage1<E>(t - 1, m0, m1);
        __syncthreads();
        if (t - 2 >= m0 - 1) stage2<E>(t - 2, m0, m1);
        __syncthreads();
        if (t - 3 >= m0) stage3<E>(t - 3);
        __syncthreads();
    }

    __device__ void run()
    {
        tx = threadIdx.x;
        ty = threadIdx.y;
        gx = (int)blockIdx.x * TL::VX - HL + tx;
        gy = MODE == 3 ? (int)blockIdx.y * TL::VY - HL + ty : 0;
        nm = MODE == 3 ? P.n[2] : (MODE == 2 ? P.n[1] : 1);
        if (!TL::MARCH) {
            prefetch(0);
            commit(0);
            __syncthreads();
            stage1<true>(0, 0, 1);
            __syncthreads();
            stage2<true>(0, 0, 1);
            __syncthreads();
            stage3<true>(0);
            __syncthreads();
            stage4<true>(0, 0, 1);
            return;
        }
        const int chunk_id = MODE == 3 ? blockIdx.z : blockIdx.y;
        const int m0 = chunk_id * P.chunk;
        const int m1 = min(nm, m0 + P.chunk);
        const bool tin = tile_interior();
        const bool mper = P.per[MA];
        const int mlo = P.lay[MA][0], mhi = nm - 1 - P.lay[MA][1];
        const int t0 = m0 - 2, t1 = m1 + 3;
        prefetch(t0);
        commit(t0);
        __syncthreads();
        for (int t = t0; t <= t1; ++t) {
            if (t + 1 <= t1) prefetch(t + 1);
            // this iteration reads planes t-5 .. t; interior iff all of them are
            const bool edge = !tin || (!mper && (t - 5 - 1 < mlo || t + 1 > mhi));
            if (edge) stages<true>(t, m0, m1);
            else stages<false>(t, m0, m1);
            if (t + 1 <= t1) commit(t + 1);
            if (t - 4 >= m0 && t - 4 < m1) {
                if (edge) stage4<true>(t - 4, m0, m1);
                else stage4<false>(t - 4, m0, m1);
            }
            __syncthreads();
        }
    }
};

template <typename T, bool INCR, int MODE, int E0M, int B0M>
__global__ void __launch_bounds__(Tile<T, MODE>::NT) k_fused(Params<T> P)
{
    if (MODE == 1) {
        // 1D steps are launched as programmatic dependents of the step before:
        // the grid may be scheduled while that one drains, and waits here, before
        // touching any global memory, until it has completed and its writes are
        // visible; it then lets the next step's grid be scheduled in turn
        asm volatile("griddepcontrol.wait;\n" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    // the rings sit between two guard bands of kGuard elements, which absorb the
    // one-cell neighbour reads of the tile's outermost cells
    constexpr int guard = 2 * Tile<T, MODE>::TX;
    constexpr int total = Lay<MODE, E0M, B0M>::PLANES * Tile<T, MODE>::NT + 2 * guard;
    T *base = reinterpret_cast<T *>(smraw);
    // start from a defined ring: slots read before their first write only feed
    // halo/warm-up cells, which must still hold finite values
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int i = tid; i < total; i += Tile<T, MODE>::NT) base[i] = T(0);
    __syncthreads();
    Kernel<T, INCR, MODE, E0M, B0M> K(P, base + guard);
    K.run();
}

// Host launcher for one instantiation.
template <typename T, bool INCR, int MODE, int E0M, int B0M>
cudaError_t launch(const Params<T> &P, int nchunks, cudaStream_t stream, int *occupancy)
{
    using TL = Tile<T, MODE>;
    constexpr size_t smem = ((size_t)Lay<MODE, E0M, B0M>::PLANES * TL::NT + 4 * TL::TX) * sizeof(T);
    static bool configured = false;
    static int occ = 0;
    auto kern = k_fused<T, INCR, MODE, E0M, B0M>;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TL::NT, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (occupancy) *occupancy = occ;
    if (nchunks <= 0) return cudaSuccess;  // query only
    dim3 block(TL::TX, TL::TY, 1);
    dim3 grid((P.n[0] + TL::VX - 1) / TL::VX, 1, 1);
    if (MODE == 2) grid.y = nchunks;
    if (MODE == 3) {
        grid.y = (P.n[1] + TL::VY - 1) / TL::VY;
        grid.z = nchunks;
    }
    if (MODE == 1) {
        // a 1D step is a few microseconds of work: overlap its launch with the
        // previous step's tail (programmatic dependent launch, also inside graphs)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, P);
    }
    kern<<<grid, block, smem, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace fused
}  // namespace axp

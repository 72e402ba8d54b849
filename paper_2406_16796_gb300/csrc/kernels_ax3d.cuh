// kernels_ax3d.cuh -- fused step specialised for 3D periodic grids with no
// order-0 (laser) fields and no uniform background E: the axion box set-up
// (arXiv 2406.16796 Sec. 2.3 update; an axion wave converting in a uniform B).
//
// With E0 = B0 = 0 and E_ext = 0 the scheme reduces to
//   S = 0,  P = (D_t phi) B_ext,  J_a(c + a/2) = B_ext,a (D_t phi(c) + D_t phi(c + a)) / 2,
// and per step, in the leapfrog-staggered state (E^{n+1/2}, B^n, phi^{n+1/2}, pi^n):
//   1. B1^{n+1} = B1^n - h curl E1^{n+1/2} (twice)
//   2. phi^{n+3/2}, D_t phi^{n+1} = (phi^{n+3/2} - phi^{n+1/2}) / dt
//   3. E1^{n+3/2} = E1^{n+1/2} + 2 x h (curl B1^{n+1} - g J^{n+1})
// the same mathematics as the generic fused kernel for this component set, with
// the two half-steps of each curl folded into one multiply-add per difference.
//
// A block of TX x TY threads owns an (x, y) tile, one column per thread with a
// halo of one column below and two above along x and y, and marches along z.
// Stage 1 and 2 work on plane t-1 and stage 3 on plane t-2 while plane t is
// taken in.  Each thread keeps its column's history along z in registers; the
// values its y neighbours read are published into double-buffered shared planes
// at the start of an iteration (one barrier per plane); a warp is one x row of
// the tile, so x neighbours come by warp shuffles.  Inputs are
// staged NS planes ahead with cp.async, each thread copying and later reading
// only its own column.
#pragma once

#include "kernels_fused.cuh"
#include "kernels_tm2d.cuh"

namespace axp {
namespace ax3d {

constexpr int TX = 32;
constexpr int HL = 1, HR = 2;
constexpr int VX = TX - HL - HR;
constexpr int PX = TX + 2;  // published planes: one guard cell around the tile
// Tile height: FP32 takes 32 rows (one 1024-thread block per SM at <= 64
// registers; the y halo is 3 of 32 rows instead of 3 of 16), FP64 16 rows.
template <typename T>
struct Geo {
    static constexpr int TY = sizeof(T) == 4 ? 32 : 16, NT = TX * TY, VY = TY - HL - HR;
    static constexpr int PY = TY + 2, PLANE = PX * PY;
};
constexpr int NS = 4;                                     // input staging depth (power of two)
constexpr int NIN = 8;                                    // E1 xyz, B1 xyz, phi, second axion level
enum { P_EX, P_EZ, P_PHI, P_NX, P_NZ, P_DT, NPUB };  // values read by the y neighbours

template <typename T>
constexpr size_t smem_bytes()
{
    return ((size_t)2 * NPUB * Geo<T>::PLANE + (size_t)NS * NIN * Geo<T>::NT) * sizeof(T);
}

template <typename T, bool INCR>
__global__ void __launch_bounds__(Geo<T>::NT, 1) k_ax3d(fused::Params<T> P)
{
    constexpr int TY = Geo<T>::TY, NT = Geo<T>::NT, VY = Geo<T>::VY, PLANE = Geo<T>::PLANE;
    extern __shared__ __align__(16) unsigned char ax3d_dyn[];
    T *pub = reinterpret_cast<T *>(ax3d_dyn);  // [2][NPUB][PY][PX]
    T *stage = pub + 2 * NPUB * PLANE;         // [NS][NIN][NT]
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    for (int i = tid; i < 2 * NPUB * PLANE; i += NT) pub[i] = T(0);

    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int gx = (int)blockIdx.x * VX - HL + tx, gy = (int)blockIdx.y * VY - HL + ty;
    const int wx = ((gx % nx) + nx) % nx, wy = ((gy % ny) + ny) % ny;
    const bool write_col = tx >= HL && tx < TX - HR && ty >= HL && ty < TY - HR && gx < nx && gy < ny;
    const int64_t col = (int64_t)wx + (int64_t)nx * wy, plane_stride = (int64_t)nx * ny;
    const int m0 = (int)blockIdx.z * P.chunk, m1 = min(nz, m0 + P.chunk);
    const int t0 = m0 - 1, t1 = m1 + 1;

    const T h = P.h, g = P.g, inv_dt = P.inv_dt;
    const T idx = P.idx[0], idy = P.idx[1], idz = P.idx[2];
    const T cx = P.lap_c[0], cy = P.lap_c[1], cz = P.lap_c[2], c0 = P.lap_0;
    const T BEx = P.Bext[0], BEy = P.Bext[1], BEz = P.Bext[2];  // uniform background B
    // step constants of the folded updates: two half-steps of the curls as one
    // multiply-add per difference, and 2h g J_a = h g B_ext,a (D_t phi + neighbour)
    const T h2x = T(2) * h * idx, h2y = T(2) * h * idy, h2z = T(2) * h * idz;
    const T hgx = h * g * BEx, hgy = h * g * BEy, hgz = h * g * BEz;

    // column history along z; suffix k = plane t - k of the current iteration
    T Ex0 = 0, Ex1 = 0, Ex2 = 0, Ey0 = 0, Ey1 = 0, Ey2 = 0, Ez0 = 0, Ez1 = 0, Ez2 = 0;  // E^{n+1/2}
    T Bx0 = 0, Bx1 = 0, By0 = 0, By1 = 0, Bz0 = 0, Bz1 = 0;                             // B^n
    T Nx1 = 0, Nx2 = 0, Nx3 = 0, Ny1 = 0, Ny2 = 0, Ny3 = 0, Nz1 = 0, Nz2 = 0;           // B^{n+1}
    T ph0 = 0, ph1 = 0, ph2 = 0, pb0 = 0, pb1 = 0;                                       // phi^{n+1/2}, 2nd level
    T D1 = 0, D2 = 0;                                                                     // D_t phi^{n+1}

    // planes t0 - 1 .. t1 lie in [-1, nz]: at most one period off the grid
    auto gidx = [&](int p) -> int64_t {
        const int wp = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        return col + plane_stride * (int64_t)wp;
    };
    auto oidx = [&](int p) -> int64_t { return col + plane_stride * (int64_t)p; };  // p in [m0, m1)
    auto prefetch = [&](int p) {
        const int64_t o = gidx(p);
        T *st = stage + ((p - t0) & (NS - 1)) * (NIN * NT) + tid;
        tm2d::cp_elem(st + 0 * NT, P.Ein[3] + o, true);
        tm2d::cp_elem(st + 1 * NT, P.Ein[4] + o, true);
        tm2d::cp_elem(st + 2 * NT, P.Ein[5] + o, true);
        tm2d::cp_elem(st + 3 * NT, P.Bin[3] + o, true);
        tm2d::cp_elem(st + 4 * NT, P.Bin[4] + o, true);
        tm2d::cp_elem(st + 5 * NT, P.Bin[5] + o, true);
        tm2d::cp_elem(st + 6 * NT, P.phi + o, true);
        tm2d::cp_elem(st + 7 * NT, P.phib + o, true);
    };
    auto take = [&](int p) {
        const T *st = stage + ((p - t0) & (NS - 1)) * (NIN * NT) + tid;
        Ex0 = st[0 * NT];
        Ey0 = st[1 * NT];
        Ez0 = st[2 * NT];
        Bx0 = st[3 * NT];
        By0 = st[4 * NT];
        Bz0 = st[5 * NT];
        ph0 = st[6 * NT];
        pb0 = st[7 * NT];
    };
    const int me = (ty + 1) * PX + (tx + 1);  // this column's cell in a published plane

    // planes t0 .. t0+NS-2 in flight, then one more per iteration
    for (int j = 0; j < NS - 1; j++) {
        if (t0 + j <= t1) prefetch(t0 + j);
        tm2d::cp_commit();
    }
    tm2d::cp_wait<NS - 2>();
    take(t0);
    __syncthreads();
    for (int t = t0; t <= t1; ++t) {
        if (t + NS - 1 <= t1) prefetch(t + NS - 1);
        tm2d::cp_commit();
        T *Q = pub + (t & 1) * (NPUB * PLANE);
        // publish what the y neighbours (other warps) read in this iteration; a
        // warp is one x row of the tile, so x neighbours come by shuffles
        Q[P_EX * PLANE + me] = Ex1;
        Q[P_EZ * PLANE + me] = Ez1;
        Q[P_PHI * PLANE + me] = ph1;
        Q[P_NX * PLANE + me] = Nx2;
        Q[P_NZ * PLANE + me] = Nz2;
        Q[P_DT * PLANE + me] = D2;
        const unsigned all = 0xffffffffu;
        const T Ez_xp = __shfl_down_sync(all, Ez1, 1), Ey_xp = __shfl_down_sync(all, Ey1, 1);
        const T ph_xp = __shfl_down_sync(all, ph1, 1), ph_xm = __shfl_up_sync(all, ph1, 1);
        const T D_xp = __shfl_down_sync(all, D2, 1);
        const T Nz_xm = __shfl_up_sync(all, Nz2, 1), Ny_xm = __shfl_up_sync(all, Ny2, 1);
        __syncthreads();
        const T *qEx = Q + P_EX * PLANE + me, *qEz = Q + P_EZ * PLANE + me;
        const T *qph = Q + P_PHI * PLANE + me, *qNx = Q + P_NX * PLANE + me;
        const T *qNz = Q + P_NZ * PLANE + me, *qDt = Q + P_DT * PLANE + me;

        // ---- stage 1: B^{n+1} on plane t-1 (forward differences of E^{n+1/2}) ----
        {
            const int p = t - 1;
            // B^{n+1} = B^n - 2h curl E^{n+1/2}, (curl E)_x = D_y E_z - D_z E_y,
            // (curl E)_y = D_z E_x - D_x E_z, (curl E)_z = D_x E_y - D_y E_x
            Nx1 = fma(-h2y, qEz[PX] - Ez1, fma(h2z, Ey0 - Ey1, Bx1));
            Ny1 = fma(-h2z, Ex0 - Ex1, fma(h2x, Ez_xp - Ez1, By1));
            Nz1 = fma(-h2x, Ey_xp - Ey1, fma(h2y, qEx[PX] - Ex1, Bz1));
            if (write_col && p >= m0 && p < m1) {
                const int64_t gi = oidx(p);
                P.Bout[3][gi] = Nx1;
                P.Bout[4][gi] = Ny1;
                P.Bout[5][gi] = Nz1;
            }
        }
        // ---- stage 2: phi^{n+3/2} and D_t phi^{n+1} on plane t-1 ----
        {
            const int p = t - 1;
            T nw, pin = T(0);
            if (INCR) {
                // second differences from neighbour differences; the mass term apart
                const T spx = (ph_xp - ph1) + (ph_xm - ph1);
                const T spy = (qph[PX] - ph1) + (qph[-PX] - ph1);
                const T spz = (ph0 - ph1) + (ph2 - ph1);
                T acc = fma(c0, ph1, pb1);
                acc = fma(cx, spx, acc);
                acc = fma(cy, spy, acc);
                acc = fma(cz, spz, acc);
                pin = acc;
                nw = ph1 + pin;
                D1 = pin * inv_dt;
            } else {
                const T spx = ph_xp + ph_xm, spy = qph[PX] + qph[-PX], spz = ph0 + ph2;
                T acc = fma(c0, ph1, -pb1);
                acc = fma(cx, spx, acc);
                acc = fma(cy, spy, acc);
                acc = fma(cz, spz, acc);
                nw = acc;
                D1 = (nw - ph1) * inv_dt;
            }
            if (write_col && p >= m0 && p < m1) {
                const int64_t gi = oidx(p);
                P.phi_out[gi] = nw;
                if (INCR) P.phib_out[gi] = pin;
            }
        }
        // ---- stage 3: J^{n+1} and E^{n+3/2} on plane t-2 (backward differences of B^{n+1}) ----
        {
            const int p = t - 2;
            if (write_col && p >= m0 && p < m1) {
                // E^{n+3/2} = E^{n+1/2} + 2h (curl B^{n+1} - g J^{n+1}), J_a the face average of
                // P_a = D_t phi B_ext,a; (curl B)_x = D_y B_z - D_z B_y, (curl B)_y = D_z B_x - D_x B_z,
                // (curl B)_z = D_x B_y - D_y B_x (backward differences)
                const int64_t gi = oidx(p);
                P.Eout[3][gi] = fma(h2y, Nz2 - qNz[-PX], fma(-h2z, Ny2 - Ny3, fma(-hgx, D2 + D_xp, Ex2)));
                P.Eout[4][gi] = fma(h2z, Nx2 - Nx3, fma(-h2x, Nz2 - Nz_xm, fma(-hgy, D2 + qDt[PX], Ey2)));
                P.Eout[5][gi] = fma(h2x, Ny2 - Ny_xm, fma(-h2y, Nx2 - qNx[-PX], fma(-hgz, D2 + D1, Ez2)));
            }
        }
        // advance the column history by one plane
        Ex2 = Ex1; Ex1 = Ex0; Ey2 = Ey1; Ey1 = Ey0; Ez2 = Ez1; Ez1 = Ez0;
        Bx1 = Bx0; By1 = By0; Bz1 = Bz0;
        Nx3 = Nx2; Nx2 = Nx1; Ny3 = Ny2; Ny2 = Ny1; Nz2 = Nz1;
        ph2 = ph1; ph1 = ph0; pb1 = pb0;
        D2 = D1;
        tm2d::cp_wait<NS - 2>();
        if (t < t1) take(t + 1);
    }
    tm2d::cp_wait<0>();
}

// FP32 split with two adjacent x cells per thread: a block of 16 x 32 threads
// owns a 32 x 32-cell tile (halo of 2 columns on each side along x, one row
// below and two above along y), each thread the pair (2 tx, 2 tx + 1) of its
// row.  The pair's history moves as float2: 8-byte staging copies, stores and
// publishes, and the packed FP32 pipe for the arithmetic (one instruction for
// two cells).  A warp holds two tile rows of 16 pairs; x neighbours of a pair
// come from its own other cell and, across pairs, by 16-lane shuffles.  The
// pair starts at an even x (written columns per tile: 28), so with an even nx
// every pair lies inside the grid and is 8-byte aligned.
namespace x2 {
constexpr int TXP = 16;             // pairs per tile row (threads along x)
constexpr int TY = 32;              // tile rows (threads along y)
constexpr int NT = TXP * TY;        // 512 threads
constexpr int HLX = 2, HRX = 2;     // halo columns along x (even: pairs stay aligned)
constexpr int VXC = 2 * TXP - HLX - HRX;  // written columns per tile: 28
constexpr int VYR = TY - HL - HR;   // written rows per tile: 29
constexpr int PXP = TXP + 2;        // published row, in pairs, with a guard pair each side
constexpr int PYR = TY + 2;
constexpr int PLANE = PXP * PYR;
constexpr size_t smem_bytes() { return ((size_t)2 * NPUB * PLANE + (size_t)NS * NIN * NT) * sizeof(float2); }

__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void cp_pair(float2 *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
}  // namespace x2

template <typename T>
__global__ void __launch_bounds__(x2::NT, 1) k_ax3d_x2(fused::Params<T> P)
{
    static_assert(sizeof(T) == 4, "the pair form is the FP32-split kernel");
    using namespace x2;
    constexpr int PL = x2::PLANE;
    extern __shared__ __align__(16) unsigned char ax3d_x2_dyn[];
    float2 *pub = reinterpret_cast<float2 *>(ax3d_x2_dyn);  // [2][NPUB][PYR][PXP]
    float2 *stage = pub + 2 * NPUB * PL;                     // [NS][NIN][NT]
    const int tid = threadIdx.x, tx = tid % TXP, ty = tid / TXP;
    for (int i = tid; i < 2 * NPUB * PL; i += NT) pub[i] = make_float2(0.f, 0.f);

    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int gx = (int)blockIdx.x * VXC - HLX + 2 * tx, gy = (int)blockIdx.y * VYR - HL + ty;
    const int wx = ((gx % nx) + nx) % nx, wy = ((gy % ny) + ny) % ny;
    const bool write_col = tx >= HLX / 2 && tx < TXP - HRX / 2 && ty >= HL && ty < TY - HR && gx < nx && gy < ny;
    const int64_t col = (int64_t)wx + (int64_t)nx * wy, plane_stride = (int64_t)nx * ny;
    const int m0 = (int)blockIdx.z * P.chunk, m1 = min(nz, m0 + P.chunk);
    const int t0 = m0 - 1, t1 = m1 + 1;

    const float inv_dt = P.inv_dt;
    const float h = P.h, g = P.g, idx = P.idx[0], idy = P.idx[1], idz = P.idx[2];
    const float2 cx = f2(P.lap_c[0]), cy = f2(P.lap_c[1]), cz = f2(P.lap_c[2]), c0 = f2(P.lap_0);
    const float2 h2x = f2(2.f * h * idx), h2y = f2(2.f * h * idy), h2z = f2(2.f * h * idz);
    const float2 mh2x = f2(-2.f * h * idx), mh2y = f2(-2.f * h * idy), mh2z = f2(-2.f * h * idz);
    const float2 mhgx = f2(-h * g * P.Bext[0]), mhgy = f2(-h * g * P.Bext[1]), mhgz = f2(-h * g * P.Bext[2]);
    const float2 idt = f2(inv_dt);

    const float2 z = make_float2(0.f, 0.f);
    float2 Ex0 = z, Ex1 = z, Ex2 = z, Ey0 = z, Ey1 = z, Ey2 = z, Ez0 = z, Ez1 = z, Ez2 = z;
    float2 Bx0 = z, Bx1 = z, By0 = z, By1 = z, Bz0 = z, Bz1 = z;
    float2 Nx1 = z, Nx2 = z, Nx3 = z, Ny1 = z, Ny2 = z, Ny3 = z, Nz1 = z, Nz2 = z;
    float2 ph0 = z, ph1 = z, ph2 = z, pb0 = z, pb1 = z;
    float2 D1 = z, D2 = z;

    auto gidx = [&](int p) -> int64_t {
        const int wp = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        return col + plane_stride * (int64_t)wp;
    };
    auto prefetch = [&](int p) {
        const int64_t o = gidx(p);
        float2 *st = stage + ((p - t0) & (NS - 1)) * (NIN * NT) + tid;
        cp_pair(st + 0 * NT, P.Ein[3] + o);
        cp_pair(st + 1 * NT, P.Ein[4] + o);
        cp_pair(st + 2 * NT, P.Ein[5] + o);
        cp_pair(st + 3 * NT, P.Bin[3] + o);
        cp_pair(st + 4 * NT, P.Bin[4] + o);
        cp_pair(st + 5 * NT, P.Bin[5] + o);
        cp_pair(st + 6 * NT, P.phi + o);
        cp_pair(st + 7 * NT, P.phib + o);
    };
    auto take = [&](int p) {
        const float2 *st = stage + ((p - t0) & (NS - 1)) * (NIN * NT) + tid;
        Ex0 = st[0 * NT];
        Ey0 = st[1 * NT];
        Ez0 = st[2 * NT];
        Bx0 = st[3 * NT];
        By0 = st[4 * NT];
        Bz0 = st[5 * NT];
        ph0 = st[6 * NT];
        pb0 = st[7 * NT];
    };
    // the new state is read again only in the next step, after the whole box has
    // streamed through L2: stores are marked evict-first
    auto store = [](float *base, int64_t gi, float2 v) { __stcs(reinterpret_cast<float2 *>(base + gi), v); };
    const int me = (ty + 1) * PXP + (tx + 1);
    const unsigned all = 0xffffffffu;
    // the pair one cell along +x / -x: (own.y, next pair's x) and (previous pair's y, own.x)
    auto xp = [&](float2 v) { return make_float2(v.y, __shfl_down_sync(all, v.x, 1, TXP)); };
    auto xm = [&](float2 v) { return make_float2(__shfl_up_sync(all, v.y, 1, TXP), v.x); };

    for (int j = 0; j < NS - 1; j++) {
        if (t0 + j <= t1) prefetch(t0 + j);
        tm2d::cp_commit();
    }
    tm2d::cp_wait<NS - 2>();
    take(t0);
    __syncthreads();
    for (int t = t0; t <= t1; ++t) {
        if (t + NS - 1 <= t1) prefetch(t + NS - 1);
        tm2d::cp_commit();
        float2 *Q = pub + (t & 1) * (NPUB * PL);
        Q[P_EX * PL + me] = Ex1;
        Q[P_EZ * PL + me] = Ez1;
        Q[P_PHI * PL + me] = ph1;
        Q[P_NX * PL + me] = Nx2;
        Q[P_NZ * PL + me] = Nz2;
        Q[P_DT * PL + me] = D2;
        const float2 Ez_xp = xp(Ez1), Ey_xp = xp(Ey1), ph_xp = xp(ph1), ph_xm = xm(ph1), D_xp = xp(D2);
        const float2 Nz_xm = xm(Nz2), Ny_xm = xm(Ny2);
        __syncthreads();
        const float2 *qEx = Q + P_EX * PL + me, *qEz = Q + P_EZ * PL + me;
        const float2 *qph = Q + P_PHI * PL + me, *qNx = Q + P_NX * PL + me;
        const float2 *qNz = Q + P_NZ * PL + me, *qDt = Q + P_DT * PL + me;
        // ---- stage 1: B^{n+1} on plane t-1 ----
        {
            const int p = t - 1;
            Nx1 = fma2(mh2y, sub2(qEz[PXP], Ez1), fma2(h2z, sub2(Ey0, Ey1), Bx1));
            Ny1 = fma2(mh2z, sub2(Ex0, Ex1), fma2(h2x, sub2(Ez_xp, Ez1), By1));
            Nz1 = fma2(mh2x, sub2(Ey_xp, Ey1), fma2(h2y, sub2(qEx[PXP], Ex1), Bz1));
            if (write_col && p >= m0 && p < m1) {
                const int64_t gi = col + plane_stride * (int64_t)p;
                store(P.Bout[3], gi, Nx1);
                store(P.Bout[4], gi, Ny1);
                store(P.Bout[5], gi, Nz1);
            }
        }
        // ---- stage 2: phi^{n+3/2} and D_t phi^{n+1} on plane t-1 ----
        {
            const int p = t - 1;
            const float2 spx = add2(sub2(ph_xp, ph1), sub2(ph_xm, ph1));
            const float2 spy = add2(sub2(qph[PXP], ph1), sub2(qph[-PXP], ph1));
            const float2 spz = add2(sub2(ph0, ph1), sub2(ph2, ph1));
            float2 acc = fma2(c0, ph1, pb1);
            acc = fma2(cx, spx, acc);
            acc = fma2(cy, spy, acc);
            acc = fma2(cz, spz, acc);
            const float2 pin = acc, nw = add2(ph1, pin);
            D1 = mul2(pin, idt);
            if (write_col && p >= m0 && p < m1) {
                const int64_t gi = col + plane_stride * (int64_t)p;
                store(P.phi_out, gi, nw);
                store(P.phib_out, gi, pin);
            }
        }
        // ---- stage 3: J^{n+1} and E^{n+3/2} on plane t-2 ----
        {
            const int p = t - 2;
            if (write_col && p >= m0 && p < m1) {
                const int64_t gi = col + plane_stride * (int64_t)p;
                store(P.Eout[3], gi, fma2(h2y, sub2(Nz2, qNz[-PXP]), fma2(mh2z, sub2(Ny2, Ny3), fma2(mhgx, add2(D2, D_xp), Ex2))));
                store(P.Eout[4], gi, fma2(h2z, sub2(Nx2, Nx3), fma2(mh2x, sub2(Nz2, Nz_xm), fma2(mhgy, add2(D2, qDt[PXP]), Ey2))));
                store(P.Eout[5], gi, fma2(h2x, sub2(Ny2, Ny_xm), fma2(mh2y, sub2(Nx2, qNx[-PXP]), fma2(mhgz, add2(D2, D1), Ez2))));
            }
        }
        Ex2 = Ex1; Ex1 = Ex0; Ey2 = Ey1; Ey1 = Ey0; Ez2 = Ez1; Ez1 = Ez0;
        Bx1 = Bx0; By1 = By0; Bz1 = Bz0;
        Nx3 = Nx2; Nx2 = Nx1; Ny3 = Ny2; Ny2 = Ny1; Nz2 = Nz1;
        ph2 = ph1; ph1 = ph0; pb1 = pb0;
        D2 = D1;
        tm2d::cp_wait<NS - 2>();
        if (t < t1) take(t + 1);
    }
    tm2d::cp_wait<0>();
}

inline cudaError_t launch_x2(const fused::Params<float> &P, int nchunks, cudaStream_t stream, int *occupancy)
{
    static int occ = 0;
    const size_t dyn = x2::smem_bytes();
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_ax3d_x2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ax3d_x2<float>, x2::NT, dyn);
        if (e != cudaSuccess) return e;
    }
    if (occupancy) *occupancy = occ;
    if (nchunks <= 0) return cudaSuccess;
    dim3 grid((P.n[0] + x2::VXC - 1) / x2::VXC, (P.n[1] + x2::VYR - 1) / x2::VYR, nchunks);
    k_ax3d_x2<float><<<grid, x2::NT, dyn, stream>>>(P);
    return cudaGetLastError();
}

template <typename T, bool INCR>
cudaError_t launch(const fused::Params<T> &P, int nchunks, cudaStream_t stream, int *occupancy)
{
    static int occ = 0;
    auto kern = k_ax3d<T, INCR>;
    const size_t dyn = smem_bytes<T>();
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Geo<T>::NT, dyn);
        if (e != cudaSuccess) return e;
    }
    if (occupancy) *occupancy = occ;
    if (nchunks <= 0) return cudaSuccess;
    dim3 grid((P.n[0] + VX - 1) / VX, (P.n[1] + Geo<T>::VY - 1) / Geo<T>::VY, nchunks);
    kern<<<grid, Geo<T>::NT, dyn, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace ax3d
}  // namespace axp

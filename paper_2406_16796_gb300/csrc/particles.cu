// particles.cu -- the perturbed-particle current of arXiv 2406.16796 Sec. 2.2
// (FPS particle method) on the GPU.
//
// Each macroparticle carries an order-0 state (x0, u0) and its first-order
// perturbation (x1, u1), u = gamma v (c = 1).  Between the field half-steps of
// Sec. 2.3 one thread per particle
//   1. gathers the fields felt at x0 + x1 at t_{n+1/2}, split as Sec. 2.2 does:
//      F_nop = sum S(r - x0) F0 (+ the uniform background),
//      F_p   = sum (dS(r - x)/dx at x0 . x1) F0 + sum S(r - x0) F1;
//   2. advances u0 by the relativistic Boris scheme (half kick, rotation, half
//      kick) and u1 by the first-order part of the same operations along
//      (u1, E_p, B_p), whose continuum limit is dp1/dt = q (E_p + v0 x B_p +
//      v1 x B_nop), v1 = (gamma0^2 u1 - u0 (u0 . u1)) / gamma0^3;
//   3. drifts x^{n+1/2} -> x^{n+3/2} with v^{n+1} and deposits
//      j0 + j1 = (q w / dV) [S v0 + (dS/dx . x1) v0 + S v1] at x^{n+1} =
//      x^{n+1/2} + (dt/2) v^{n+1}, j^{n+1} centred on the E interval it enters.
// S is the quadratic B-spline (three nodes per active axis), each component
// gathered from (and each current deposited on) its own staggered nodes, j_a on
// the E_a nodes.
//
// GB300's FP64 unit (2 operations per cycle per SM) bounds this kernel, so the
// arithmetic is arranged to do each piece once:
//  - along an axis every component sits either on cell centres or on faces, so
//    one thread computes two shapes per active axis (and two more at x^{n+1}
//    for the deposit) and every component picks its pair;
//  - the spline is separable: a gather sums each row along x first (values,
//    and x-derivative values for the first-order part), then weighs the rows;
//    a deposit forms one row factor per row and one product per node;
//  - divisions become multiplications by reciprocals formed once (1/d per
//    axis, 1/gamma, 1/(1 + t.t)).
// The results therefore differ from a plain loop over nodes in rounding only.
// Deposits are FP64 atomic adds, so the current's rounding also depends on the
// order in which particles arrive.
#include "axp_internal.h"

namespace axp {
namespace {

constexpr int kThreads = 256;

struct PDev {
    int64_t count;
    double q, qm, dt, inv_dV;
    int64_t n[3];
    double d[3], inv_d[3], lo[3];
    int active[3];
    double Bext[3], Eext[3];
    const double *E0[3], *B0[3], *E1[3], *B1[3];
    double *w, *x0[3], *u0[3], *x1[3], *u1[3];
    double *j0[3], *j1[3];
    double *out_x0[3], *out_x1[3];
};

// Three nodes of the quadratic B-spline along one axis: indices, weights and
// their derivatives with respect to the particle position.
struct AxisShape {
    int64_t node[3];
    double W[3], dW[3];
};

// The two staggerings of one axis: [0] nodes at cell centres (offset 1/2 cell),
// [1] nodes on the high faces (offset 1).  ACTIVE: the axis has more than one
// cell (a template argument, so that the stencil loops unroll and the shapes
// stay in registers); along an inactive axis the one node 0 has weight 1.
template <bool ACTIVE>
__device__ __forceinline__ void axis_shapes(const PDev &P, int b, double x, AxisShape s[2])
{
    if constexpr (!ACTIVE) {
        for (int o = 0; o < 2; o++) {
            s[o].node[0] = 0;
            s[o].W[0] = 1.0;
            s[o].dW[0] = 0.0;
        }
    } else {
        const double u = (x - P.lo[b]) * P.inv_d[b];
        const int64_t n = P.n[b];
#pragma unroll
        for (int o = 0; o < 2; o++) {
            const double xi = u - (o ? 1.0 : 0.5);
            const double c = floor(xi + 0.5);
            const double del = xi - c;
            // the nearest node, bounded before the conversion (a position far
            // outside the box, or not finite, still gives nodes inside [0, n))
            const double cb = fmin(fmax(c, -4.0e15), 4.0e15);
            int64_t base = ((int64_t)cb - 1) % n;
            if (base < 0) base += n;
#pragma unroll
            for (int t = 0; t < 3; t++) {
                int64_t q = base + t;
                if (q >= n) q -= n;
                s[o].node[t] = q;
            }
            const double lo = 0.5 - del, hi = 0.5 + del;
            s[o].W[0] = 0.5 * lo * lo;
            s[o].W[1] = 0.75 - del * del;
            s[o].W[2] = 0.5 * hi * hi;
            s[o].dW[0] = -lo * P.inv_d[b];
            s[o].dW[1] = -2.0 * del * P.inv_d[b];
            s[o].dW[2] = hi * P.inv_d[b];
        }
    }
}

template <int MASK>
struct Extent {
    static constexpr int x = (MASK & 1) ? 3 : 1, y = (MASK & 2) ? 3 : 1, z = (MASK & 4) ? 3 : 1;
};

// staggering index along axis B of component A: E_A lies on the faces along A,
// B_A on the faces along the other two axes
template <int KIND, int A, int B>
struct Stag {
    static constexpr int v = KIND == 1 ? (B == A ? 1 : 0) : (B == A ? 0 : 1);
};

template <int MASK>
__device__ __forceinline__ void all_shapes(const PDev &P, const double x[3], AxisShape sh[3][2])
{
    axis_shapes<(MASK & 1) != 0>(P, 0, x[0], sh[0]);
    axis_shapes<(MASK & 2) != 0>(P, 1, x[1], sh[1]);
    axis_shapes<(MASK & 4) != 0>(P, 2, x[2], sh[2]);
}

// f0 = sum S F0 and fp = sum (dS . x1) F0 + sum S F1 of component A of KIND
// (1 = E, 2 = B): rows along x first, then the rows weighed by their y, z factors
template <int MASK, int KIND, int A>
__device__ __forceinline__ void gather_one(const PDev &P, const AxisShape sh[3][2], const double x1[3],
                                           const double *__restrict__ F0, const double *__restrict__ F1, double &f0,
                                           double &fp)
{
    const AxisShape &sx = sh[0][Stag<KIND, A, 0>::v];
    const AxisShape &sy = sh[1][Stag<KIND, A, 1>::v];
    const AxisShape &sz = sh[2][Stag<KIND, A, 2>::v];
    f0 = 0.0;
    fp = 0.0;
#pragma unroll
    for (int tk = 0; tk < Extent<MASK>::z; tk++)
#pragma unroll
        for (int tj = 0; tj < Extent<MASK>::y; tj++) {
            const int64_t row = P.n[0] * (sy.node[tj] + P.n[1] * sz.node[tk]);
            double a0 = 0.0, ad = 0.0, a1 = 0.0;
#pragma unroll
            for (int ti = 0; ti < Extent<MASK>::x; ti++) {
                const double g0 = F0[row + sx.node[ti]], g1 = F1[row + sx.node[ti]];
                a0 = a0 + sx.W[ti] * g0;
                a1 = a1 + sx.W[ti] * g1;
                if constexpr ((MASK & 1) != 0) ad = ad + sx.dW[ti] * g0;
            }
            const double wyz = sy.W[tj] * sz.W[tk];
            double dyz = 0.0;
            if constexpr ((MASK & 2) != 0) dyz = dyz + sy.dW[tj] * sz.W[tk] * x1[1];
            if constexpr ((MASK & 4) != 0) dyz = dyz + sy.W[tj] * sz.dW[tk] * x1[2];
            f0 = f0 + wyz * a0;
            fp = fp + wyz * a1 + dyz * a0;
            if constexpr ((MASK & 1) != 0) fp = fp + wyz * x1[0] * ad;
        }
}

// adds component A of the current at the E_A nodes: j0 = c0 S, j1 = c0 (dS . x1) + c1 S
// with c0 = (q w / dV) v0_A, c1 = (q w / dV) v1_A
template <int MASK, int A>
__device__ __forceinline__ void deposit_one(const PDev &P, const AxisShape sh[3][2], const double x1[3], double c0,
                                            double c1)
{
    const AxisShape &sx = sh[0][Stag<1, A, 0>::v];
    const AxisShape &sy = sh[1][Stag<1, A, 1>::v];
    const AxisShape &sz = sh[2][Stag<1, A, 2>::v];
#pragma unroll
    for (int tk = 0; tk < Extent<MASK>::z; tk++)
#pragma unroll
        for (int tj = 0; tj < Extent<MASK>::y; tj++) {
            const int64_t row = P.n[0] * (sy.node[tj] + P.n[1] * sz.node[tk]);
            const double wyz = sy.W[tj] * sz.W[tk];
            double dyz = 0.0;
            if constexpr ((MASK & 2) != 0) dyz = dyz + sy.dW[tj] * sz.W[tk] * x1[1];
            if constexpr ((MASK & 4) != 0) dyz = dyz + sy.W[tj] * sz.dW[tk] * x1[2];
            const double r0 = wyz * c0;               // S v0 per unit x weight
            const double rx = wyz * x1[0] * c0;       // dS/dx x1x v0 per unit x derivative
            const double r1 = dyz * c0 + wyz * c1;    // the y, z derivative terms and S v1
#pragma unroll
            for (int ti = 0; ti < Extent<MASK>::x; ti++) {
                double add1 = sx.W[ti] * r1;
                if constexpr ((MASK & 1) != 0) add1 = add1 + sx.dW[ti] * rx;
                atomicAdd(P.j0[A] + row + sx.node[ti], sx.W[ti] * r0);
                atomicAdd(P.j1[A] + row + sx.node[ti], add1);
            }
        }
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// v0 = u0 / gamma0 and its first-order part v1 = (gamma0^2 u1 - u0 (u0 . u1)) / gamma0^3
__device__ __forceinline__ void velocities(const double u0[3], const double u1[3], double v0[3], double v1[3])
{
    const double g0 = sqrt(1.0 + dot3(u0, u0));
    const double ig = 1.0 / g0, ig3 = ig * ig * ig;
    const double uu = dot3(u0, u1);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        v0[a] = u0[a] * ig;
        v1[a] = (g0 * g0 * u1[a] - u0[a] * uu) * ig3;
    }
}

// Boris update of u0 and its first-order part
__device__ __forceinline__ void kick(double qm, double dt, const double u0[3], const double u1[3],
                                     const double E[3], const double B[3], const double Ep[3], const double Bp[3],
                                     double o0[3], double o1[3])
{
    const double h = qm * dt * 0.5;
    double um[3], dum[3], t[3], dtv[3], up[3], dup[3], sv[3], dsv[3], c1[3], c2[3], c3[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        um[a] = u0[a] + h * E[a];
        dum[a] = u1[a] + h * Ep[a];
    }
    // t = h B / gamma(u-) and its first-order part
    const double igm = 1.0 / sqrt(1.0 + dot3(um, um));
    const double dgm_over_gm = dot3(um, dum) * igm * igm;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        t[a] = h * B[a] * igm;
        dtv[a] = h * Bp[a] * igm - t[a] * dgm_over_gm;
    }
    cross3(um, t, c1);
    cross3(dum, t, c2);
    cross3(um, dtv, c3);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        up[a] = um[a] + c1[a];
        dup[a] = dum[a] + c2[a] + c3[a];
    }
    // s = 2 t / (1 + t.t)
    const double i1 = 1.0 / (1.0 + dot3(t, t)), dtt = 2.0 * dot3(t, dtv);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        sv[a] = 2.0 * t[a] * i1;
        dsv[a] = 2.0 * dtv[a] * i1 - 2.0 * t[a] * dtt * i1 * i1;
    }
    cross3(up, sv, c1);
    cross3(dup, sv, c2);
    cross3(up, dsv, c3);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        o0[a] = (um[a] + c1[a]) + h * E[a];
        o1[a] = ((dum[a] + c2[a]) + c3[a]) + h * Ep[a];
    }
}

template <int MASK>
__device__ __forceinline__ void deposit(const PDev &P, double qw, const double x0[3], const double x1[3],
                                        const double v0[3], const double v1[3])
{
    AxisShape sh[3][2];
    all_shapes<MASK>(P, x0, sh);
    const double k = qw * P.inv_dV;
    deposit_one<MASK, 0>(P, sh, x1, k * v0[0], k * v1[0]);
    deposit_one<MASK, 1>(P, sh, x1, k * v0[1], k * v1[1]);
    deposit_one<MASK, 2>(P, sh, x1, k * v0[2], k * v1[2]);
}

__device__ __forceinline__ double wrap_pos(const PDev &P, int b, double x)
{
    if (!P.active[b]) return x;
    const double L = (double)P.n[b] * P.d[b];
    if (x >= P.lo[b] + L) return x - L;
    if (x < P.lo[b]) return x + L;
    return x;
}

__device__ __forceinline__ void load(const PDev &P, int64_t q, double x0[3], double x1[3], double u0[3],
                                     double u1[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        x0[a] = P.x0[a][q];
        x1[a] = P.x1[a][q];
        u0[a] = P.u0[a][q];
        u1[a] = P.u1[a][q];
    }
}

// j^n from the positions at t_n, then the positions moved to t_{n+1/2}
template <int MASK>
__global__ void __launch_bounds__(kThreads) k_particles_start(PDev P)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.count;
         q += (int64_t)gridDim.x * blockDim.x) {
        double x0[3], x1[3], u0[3], u1[3], v0[3], v1[3];
        load(P, q, x0, x1, u0, u1);
        velocities(u0, u1, v0, v1);
        deposit<MASK>(P, P.q * P.w[q], x0, x1, v0, v1);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            P.x0[a][q] = wrap_pos(P, a, x0[a] + (P.dt * 0.5) * v0[a]);
            P.x1[a][q] = x1[a] + (P.dt * 0.5) * v1[a];
        }
    }
}

template <int MASK>
__global__ void __launch_bounds__(kThreads) k_particles_push(PDev P)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.count;
         q += (int64_t)gridDim.x * blockDim.x) {
        double x0[3], x1[3], u0[3], u1[3];
        double E[3], B[3], Ep[3], Bp[3], o0[3], o1[3], v0[3], v1[3], xc0[3], xc1[3];
        load(P, q, x0, x1, u0, u1);
        {
            AxisShape sh[3][2];
            all_shapes<MASK>(P, x0, sh);
            gather_one<MASK, 1, 0>(P, sh, x1, P.E0[0], P.E1[0], E[0], Ep[0]);
            gather_one<MASK, 1, 1>(P, sh, x1, P.E0[1], P.E1[1], E[1], Ep[1]);
            gather_one<MASK, 1, 2>(P, sh, x1, P.E0[2], P.E1[2], E[2], Ep[2]);
            gather_one<MASK, 2, 0>(P, sh, x1, P.B0[0], P.B1[0], B[0], Bp[0]);
            gather_one<MASK, 2, 1>(P, sh, x1, P.B0[1], P.B1[1], B[1], Bp[1]);
            gather_one<MASK, 2, 2>(P, sh, x1, P.B0[2], P.B1[2], B[2], Bp[2]);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            E[a] = E[a] + P.Eext[a];
            B[a] = B[a] + P.Bext[a];
        }
        kick(P.qm, P.dt, u0, u1, E, B, Ep, Bp, o0, o1);
        velocities(o0, o1, v0, v1);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            xc0[a] = x0[a] + (P.dt * 0.5) * v0[a];
            xc1[a] = x1[a] + (P.dt * 0.5) * v1[a];
            P.x0[a][q] = wrap_pos(P, a, x0[a] + P.dt * v0[a]);
            P.x1[a][q] = x1[a] + P.dt * v1[a];
            P.u0[a][q] = o0[a];
            P.u1[a][q] = o1[a];
        }
        deposit<MASK>(P, P.q * P.w[q], xc0, xc1, v0, v1);
    }
}

__global__ void __launch_bounds__(kThreads) k_particles_now(PDev P)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.count;
         q += (int64_t)gridDim.x * blockDim.x) {
        double x0[3], x1[3], u0[3], u1[3], v0[3], v1[3];
        load(P, q, x0, x1, u0, u1);
        velocities(u0, u1, v0, v1);
        for (int a = 0; a < 3; a++) {
            P.out_x0[a][q] = wrap_pos(P, a, x0[a] - (P.dt * 0.5) * v0[a]);
            P.out_x1[a][q] = x1[a] - (P.dt * 0.5) * v1[a];
        }
    }
}

PDev make_pdev(axp_grid *g)
{
    const Particles &S = *g->parts;
    PDev P;
    P.count = S.count;
    P.q = S.q;
    P.qm = S.q / S.m;
    P.dt = g->desc.dt;
    P.inv_dV = 1.0 / (g->desc.d[0] * g->desc.d[1] * g->desc.d[2]);
    for (int a = 0; a < 3; a++) {
        P.n[a] = g->desc.n[a];
        P.d[a] = g->desc.d[a];
        P.inv_d[a] = 1.0 / g->desc.d[a];
        P.lo[a] = g->desc.lo[a];
        P.active[a] = g->desc.n[a] > 1;
        P.Bext[a] = g->B_ext[a];
        P.Eext[a] = g->E_ext[a];
        P.E0[a] = P.B0[a] = P.E1[a] = P.B1[a] = nullptr;
        P.x0[a] = S.x0[a];
        P.u0[a] = S.u0[a];
        P.x1[a] = S.x1[a];
        P.u1[a] = S.u1[a];
        P.j0[a] = S.j[0][a];
        P.j1[a] = S.j[1][a];
        P.out_x0[a] = S.scratch[a];
        P.out_x1[a] = S.scratch[3 + a];
    }
    P.w = S.w;
    return P;
}

int mask_of(const axp_grid *g)
{
    return (g->desc.n[0] > 1 ? 1 : 0) | (g->desc.n[1] > 1 ? 2 : 0) | (g->desc.n[2] > 1 ? 4 : 0);
}

// launch KERNEL<mask> for the grid's active axes
#define AXP_LAUNCH_MASKED(KERNEL, MASKV, BLOCKS, STREAM, ARG)                    \
    switch (MASKV) {                                                           \
    case 0: KERNEL<0><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 1: KERNEL<1><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 2: KERNEL<2><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 3: KERNEL<3><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 4: KERNEL<4><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 5: KERNEL<5><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    case 6: KERNEL<6><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;            \
    default: KERNEL<7><<<BLOCKS, kThreads, 0, STREAM>>>(ARG); break;           \
    }

int blocks_for(int64_t count)
{
    const int64_t b = (count + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

cudaError_t zero_currents(axp_grid *g)
{
    const size_t bytes = sizeof(double) * (size_t)(g->desc.n[0] * g->desc.n[1] * g->desc.n[2]);
    for (int o = 0; o < 2; o++)
        for (int a = 0; a < 3; a++) {
            cudaError_t e = cudaMemsetAsync(g->parts->j[o][a], 0, bytes, g->stream);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

}  // namespace

size_t particles_bytes(const axp_grid_desc &d, int64_t count)
{
    const size_t per = align_up(sizeof(double) * (size_t)std::max<int64_t>(count, 1));
    const size_t cells = align_up(sizeof(double) * (size_t)(d.n[0] * d.n[1] * d.n[2]));
    return 19 * per + 6 * cells;  // w, x0, u0, x1, u1, read-back scratch; j of both orders
}

void particles_layout(const axp_grid_desc &d, Particles *P)
{
    const size_t per = align_up(sizeof(double) * (size_t)std::max<int64_t>(P->count, 1));
    const size_t cells = align_up(sizeof(double) * (size_t)(d.n[0] * d.n[1] * d.n[2]));
    char *p = P->ws;
    auto take = [&](size_t b) {
        double *r = reinterpret_cast<double *>(p);
        p += b;
        return r;
    };
    P->w = take(per);
    for (int a = 0; a < 3; a++) P->x0[a] = take(per);
    for (int a = 0; a < 3; a++) P->u0[a] = take(per);
    for (int a = 0; a < 3; a++) P->x1[a] = take(per);
    for (int a = 0; a < 3; a++) P->u1[a] = take(per);
    for (int i = 0; i < 6; i++) P->scratch[i] = take(per);
    for (int o = 0; o < 2; o++)
        for (int a = 0; a < 3; a++) P->j[o][a] = take(cells);
}

cudaError_t particles_start(axp_grid *g)
{
    cudaError_t e = zero_currents(g);
    if (e != cudaSuccess) return e;
    if (g->parts->count == 0) return cudaSuccess;
    AXP_LAUNCH_MASKED(k_particles_start, mask_of(g), blocks_for(g->parts->count), g->stream, make_pdev(g));
    g->launches++;
    return cudaGetLastError();
}

cudaError_t particles_push(axp_grid *g, const View<double> &v)
{
    cudaError_t e = zero_currents(g);
    if (e != cudaSuccess) return e;
    if (g->parts->count == 0) return cudaSuccess;
    PDev P = make_pdev(g);
    for (int a = 0; a < 3; a++) {
        P.E0[a] = v.f[kE0 + a];
        P.B0[a] = v.f[kB0 + a];
        P.E1[a] = v.f[kE1 + a];
        P.B1[a] = v.f[kB1 + a];
    }
    AXP_LAUNCH_MASKED(k_particles_push, mask_of(g), blocks_for(P.count), g->stream, P);
    g->launches++;
    return cudaGetLastError();
}

cudaError_t particles_now(axp_grid *g)
{
    if (g->parts->count == 0) return cudaSuccess;
    k_particles_now<<<blocks_for(g->parts->count), kThreads, 0, g->stream>>>(make_pdev(g));
    g->launches++;
    return cudaGetLastError();
}

}  // namespace axp

// kernels_line1d.cuh -- time-blocked step for FP64 1D grids periodic along x
// (arXiv 2406.16796 Sec. 2.3; the 1D conversion workload).
//
// A 1D grid of a few thousand cells is far too small to fill the GPU: launched
// one step at a time its steps cost launch and synchronisation latency, not
// arithmetic.  Here one cooperative launch runs a whole run of steps.  Each
// block owns `seg` consecutive cells and holds them, with `halo` cells on each
// side, in shared memory; it advances that window `tblock` steps on its own,
// writes its owned cells to the other buffer set and meets the other blocks at
// a grid-wide wait (bounded in polls and in time) before it reads its next
// window.  A step's dependency cone is one cell wide and the axion current
// widens it by two, so the owned cells stay exact while halo >= tblock + 2
// (kept at tblock + 3); outside the window the closure is zero.
//
// The state and the update are those of the single-pass kernels: E at n+1/2,
// B at n, phi at n+1/2 and n-1/2.  Along x only the y and z components curl;
// E_x of order 1 changes through the axion current alone, B_x and E0_x not at
// all.  Per step, one barrier after each stage:
//   1. B^{n+1/2}, B^{n+1} = B^n - h curl E^{n+1/2} (twice)
//   2. S^{n+1/2} = g Ebar0 . Bbar0 (E0^{n+1/2}, B0^{n+1/2}); phi^{n+3/2};
//      2 phi^{n+1}, dt D_t phi^{n+1}; E0^{n+1} = E0^{n+1/2} + h curl B0^{n+1}
//   3. P^{n+1} = (D_t phi) Bbar0 - Ebar0 x grad_c phi at cell centres
//   4. J^{n+1} (face average of P along x); E1^{n+3/2} = E1^{n+1/2}
//      + 2h (curl B1^{n+1} - g J^{n+1}); E0^{n+3/2} = 2 E0^{n+1} - E0^{n+1/2}
// with the averages of Sec. 2.3 reduced to 1D (a 4-point mean over cells that
// coincide along y and z is the 2-point mean along x).
#pragma once

#include "kernels_fused.cuh"

namespace axp {
namespace line1d {

// Four warps: each SM sub-partition has its own FP64 unit, which takes about 64
// cycles per warp instruction, so a warp issues at most a quarter of the SM's
// FP64 rate.  The window's cells are covered by two warps and each stage's work
// on a cell is split into two halves of independent outputs: warps 0-1 take one
// half and warps 2-3 (the other two sub-partitions) the other.
constexpr int kThreads = 128;
constexpr int kLanes = 64;               // cells a pass of one half covers
constexpr int kArrays = 27;              // window arrays (listed in k_line1d)
constexpr int kMaxWindow = 1000;         // cells: kArrays x 1000 x 8 B = 216 KB of shared memory
constexpr unsigned kSpinLimit = 1u << 26;        // polls of a grid-wide wait before it gives up ...
constexpr unsigned long long kWaitNs = 1000000000ull;  // ... or one second, whichever comes first

struct Args {
    const double *E[2][6], *B[2][6];  // buffer sets: order-0 xyz, order-1 xyz (E^{n+1/2}, B^n)
    double *Ew[2][6], *Bw[2][6];      // the same arrays, written
    double *phi[2][2];                // per set: phi^{n+1/2}, phi^{n-1/2}
    int64_t n;                        // cells
    int64_t nsteps;
    int tblock, halo, seg;
    // step constants
    double cB;      // h/dx: one B or E0 half-step per difference
    double c2B;     // 2h/dx: the two half-steps of E1 (and of B1) per difference
    double h2g;     // 2hg: the current's term in E1's two half-steps
    double lap_0, lap_c, dt2g;  // phi^{n+3/2} = lap_0 phi + lap_c (phi+ + phi-) - phi^{n-1/2} + dt2g S/g
    double inv_dt, q4dx;        // 1/dt; 1/(4 dx) for the central gradient of 2 phi^{n+1}
    double Bext[3];
    unsigned *ctr;  // grid-wait arrivals (zeroed before the launch)
    int *err;       // 1 once a wait gave up
    int absent;     // failure-detection test: this block leaves before its first wait (-1: none)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide wait on an arrival counter, bounded: after kSpinLimit polls, a
// second, or once another block has given up, it records the failure and
// returns false.
__device__ __forceinline__ bool grid_wait(unsigned *ctr, unsigned target, int *err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        ok = 1;
        unsigned spins = 0;
        const unsigned long long t0 = global_ns();
        while (*(volatile unsigned *)ctr < target) {
            if (++spins > kSpinLimit || *(volatile int *)err || global_ns() - t0 > kWaitNs) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(kThreads) k_line1d(Args A)
{
    extern __shared__ __align__(16) double l1_sm[];
    const int64_t N = A.n;
    const int64_t s0 = (int64_t)blockIdx.x * A.seg;
    const int own = (int)(min(N, s0 + A.seg) - s0);
    const int H = A.halo, W = own + 2 * H, Wm = A.seg + 2 * A.halo;
    const int tid = threadIdx.x, nt = blockDim.x;
    // window arrays: E (6), B (6), phi^{n+1/2}, phi^{n-1/2}, B0^{n+1/2} y z, E0^{n+1} y z,
    // 2 phi^{n+1}, dt D_t phi^{n+1}, P (3), Bbar0^{n+1} y z (with B_ext), and two values that
    // stay fixed over a window's steps: E0x and B0x do not change in 1D (no curl along x),
    // so Bbar0_x = B0x + B_ext,x and the source's term Ebar0_x Bbar0_x are formed once
    double *E[6], *B[6];
    for (int q = 0; q < 6; q++) {
        E[q] = l1_sm + (size_t)q * Wm;
        B[q] = l1_sm + (size_t)(6 + q) * Wm;
    }
    double *cur = l1_sm + (size_t)12 * Wm, *old = l1_sm + (size_t)13 * Wm;
    double *Bhy = l1_sm + (size_t)14 * Wm, *Bhz = l1_sm + (size_t)15 * Wm;
    double *Eny = l1_sm + (size_t)16 * Wm, *Enz = l1_sm + (size_t)17 * Wm;
    double *SM = l1_sm + (size_t)18 * Wm, *DF = l1_sm + (size_t)19 * Wm;
    double *Px = l1_sm + (size_t)20 * Wm, *PY = l1_sm + (size_t)21 * Wm, *PZ = l1_sm + (size_t)22 * Wm;
    double *BY = l1_sm + (size_t)23 * Wm, *BZ = l1_sm + (size_t)24 * Wm;
    double *BXT = l1_sm + (size_t)25 * Wm, *SX = l1_sm + (size_t)26 * Wm;
    const int half = tid / kLanes, lane = tid % kLanes;  // (a warp-uniform half)
    // values beyond the window's ends: the zero closure
    auto at = [&](const double *a, int w) { return (w >= 0 && w < W) ? a[w] : 0.0; };
    const double Bx = A.Bext[0], By = A.Bext[1], Bz = A.Bext[2];

    int par = 0;
    unsigned waits = 0;
    for (int64_t done = 0; done < A.nsteps; done += A.tblock) {
        const int steps = (int)min((int64_t)A.tblock, A.nsteps - done);
        for (int w = tid; w < W; w += nt) {
            int64_t gi = (s0 - H + w) % N;
            if (gi < 0) gi += N;
#pragma unroll
            for (int q = 0; q < 6; q++) {
                E[q][w] = A.E[par][q][gi];
                B[q][w] = A.B[par][q][gi];
            }
            cur[w] = A.phi[par][0][gi];
            old[w] = A.phi[par][1][gi];
        }
        __syncthreads();
        for (int w = tid; w < W; w += nt) {
            const double ex = 0.5 * (E[0][w] + at(E[0], w - 1));
            const double bx = B[0][w] + Bx;
            BXT[w] = bx;
            SX[w] = ex * bx;
        }
        __syncthreads();
        for (int st = 0; st < steps; st++) {
            // 1. B^{n+1/2} and B^{n+1}: (curl E)_y = -D_x E_z, (curl E)_z = D_x E_y (forward)
            for (int w = lane; w < W; w += kLanes) {
                if (half == 0) {
                    const double d0z = at(E[2], w + 1) - E[2][w], d1z = at(E[5], w + 1) - E[5][w];
                    const double hy = fma(A.cB, d0z, B[1][w]);
                    Bhy[w] = hy;
                    B[1][w] = fma(A.cB, d0z, hy);
                    B[4][w] = fma(A.c2B, d1z, B[4][w]);
                } else {
                    const double d0y = at(E[1], w + 1) - E[1][w], d1y = at(E[4], w + 1) - E[4][w];
                    const double hz = fma(-A.cB, d0y, B[2][w]);
                    Bhz[w] = hz;
                    B[2][w] = fma(-A.cB, d0y, hz);
                    B[5][w] = fma(-A.c2B, d1y, B[5][w]);
                }
            }
            __syncthreads();
            // 2. source, phi^{n+3/2}, 2 phi^{n+1}, dt D_t phi^{n+1} | E0^{n+1}, Bbar0^{n+1} y z
            for (int w = lane; w < W; w += kLanes) {
                if (half == 0) {
                    const double by = fma(0.5, Bhy[w] + at(Bhy, w - 1), By);
                    const double bz = fma(0.5, Bhz[w] + at(Bhz, w - 1), Bz);
                    const double S = fma(E[2][w], bz, fma(E[1][w], by, SX[w]));  // S/g
                    const double ph = cur[w];
                    double nw = fma(A.lap_0, ph, -old[w]);
                    nw = fma(A.lap_c, at(cur, w + 1) + at(cur, w - 1), nw);
                    nw = fma(A.dt2g, S, nw);
                    old[w] = nw;  // phi^{n+3/2} over phi^{n-1/2} (read by this cell only)
                    SM[w] = nw + ph;
                    DF[w] = nw - ph;
                } else {
                    // (curl B0)_y = -D_x B0z, (curl B0)_z = D_x B0y (backward)
                    Eny[w] = fma(-A.cB, B[2][w] - at(B[2], w - 1), E[1][w]);
                    Enz[w] = fma(A.cB, B[1][w] - at(B[1], w - 1), E[2][w]);
                    BY[w] = fma(0.5, B[1][w] + at(B[1], w - 1), By);
                    BZ[w] = fma(0.5, B[2][w] + at(B[2], w - 1), Bz);
                }
            }
            __syncthreads();
            // 3. P^{n+1} at the cell centres
            for (int w = lane; w < W; w += kLanes) {
                const double Dt = DF[w] * A.inv_dt;
                const double dphi = (at(SM, w + 1) - at(SM, w - 1)) * A.q4dx;
                if (half == 0) {
                    PY[w] = fma(-Enz[w], dphi, Dt * BY[w]);
                } else {
                    Px[w] = Dt * BXT[w];
                    PZ[w] = fma(Eny[w], dphi, Dt * BZ[w]);
                }
            }
            __syncthreads();
            // 4. J^{n+1}; E1^{n+3/2}; E0^{n+3/2}
            for (int w = lane; w < W; w += kLanes) {
                if (half == 0) {
                    const double Jx = 0.5 * (Px[w] + at(Px, w + 1));
                    E[3][w] = fma(-A.h2g, Jx, E[3][w]);
                    E[4][w] = fma(-A.c2B, B[5][w] - at(B[5], w - 1), fma(-A.h2g, PY[w], E[4][w]));
                } else {
                    E[5][w] = fma(A.c2B, B[4][w] - at(B[4], w - 1), fma(-A.h2g, PZ[w], E[5][w]));
                    E[1][w] = fma(2.0, Eny[w], -E[1][w]);
                    E[2][w] = fma(2.0, Enz[w], -E[2][w]);
                }
            }
            double *t = cur;
            cur = old;
            old = t;
            __syncthreads();
        }
        for (int w = H + tid; w < H + own; w += nt) {
            const int64_t gi = s0 + (w - H);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                A.Ew[1 - par][q][gi] = E[q][w];
                A.Bw[1 - par][q][gi] = B[q][w];
            }
            A.phi[1 - par][0][gi] = cur[w];
            A.phi[1 - par][1][gi] = old[w];
        }
        par ^= 1;
        if (done + A.tblock < A.nsteps) {
            if ((int)blockIdx.x == A.absent) return;  // never arrives: the others' waits run out
            waits++;
            if (!grid_wait(A.ctr, waits * gridDim.x, A.err)) return;
        }
    }
}

}  // namespace line1d
}  // namespace axp

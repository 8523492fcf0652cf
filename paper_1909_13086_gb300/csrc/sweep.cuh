// sweep.cuh -- the fused B-TriRT collide-and-stream kernel (device code).
//
// One thread per lattice cell.  Populations are structure-of-arrays planes
// (f_0..f_8, g_0..g_8), rows padded to 128 B.  The pull scheme reads each
// post-collision population of the previous step exactly once, so the only
// DRAM traffic is 18 loads + 18 stores per cell; the +-1 x-offset planes cost
// one extra 32 B sector per warp, which L1/L2 absorb.
//
// Per cell, in one pass (paper Sec. 2 and the readings of Sec. 3):
//   1. pull streaming; half-way bounce-back on no-slip / adiabatic walls,
//      half-way anti-bounce-back g_i = -g*_opp + 2 w_i T_h on the wall held at
//      T_h (bottom strip of the cavity, left wall of the Stefan problem);
//   2. rho, j of f; H = sum g (Eq. 1) and its inversion to (T, f_l);
//   3. F = g beta (T - T_m) y, u = f_l (j + F/2)/rho;
//   4. g collision: Eq. 2 with the equilibrium of Eq. 4;
//   5. f collision: the same block operator with rates (k0f, k1f, k2f) and a
//      forcing term whose first and second moments are (1 - k1f/2) F and
//      (1 - k2f/2)(uF + Fu);
//   6. store; optionally reduce the diagnostics in FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace btrirt {

// ---- D2Q9 (c_i, w_i, opposite) as constexpr functions: fully folded once the
//      direction loops are unrolled.
__host__ __device__ constexpr int cx_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename real>
__device__ __forceinline__ real w_of(int i) {
    return i == 0 ? real(4) / real(9) : (i <= 4 ? real(1) / real(9) : real(1) / real(36));
}

// Q_i : A with Q_i = c_i c_i - I/3 and A symmetric (xx, xy, yy).
template <typename real>
__device__ __forceinline__ real q_dot(int i, real axx, real axy, real ayy) {
    const real third = real(1) / real(3);
    const int cx = cx_of(i), cy = cy_of(i);
    return (real(cx * cx) - third) * axx + real(2 * cx * cy) * axy +
           (real(cy * cy) - third) * ayy;
}

// Moments of a D2Q9 vector n: M1 = sum c n, M2 = sum c c n.
template <typename real>
__device__ __forceinline__ void moments(const real n[9], real &m1x, real &m1y, real &m2xx,
                                        real &m2xy, real &m2yy) {
    m1x = (n[1] - n[3]) + (n[5] - n[6]) + (n[8] - n[7]);
    m1y = (n[2] - n[4]) + (n[5] + n[6]) - (n[7] + n[8]);
    const real diag = (n[5] + n[6]) + (n[7] + n[8]);
    m2xx = (n[1] + n[3]) + diag;
    m2yy = (n[2] + n[4]) + diag;
    m2xy = (n[5] + n[7]) - (n[6] + n[8]);
}

// out_i = p_i - k0 n_i - w_i [ 3 c_i.A1 + 9/2 Q_i:A2 ]  (Eq. 2 with
// A1 = (k1 - k0) M1 - source_1 and A2 = (k2 - k0) M2 - source_2 folded in).
template <typename real>
__device__ __forceinline__ void block_relax(real p[9], const real n[9], real k0, real a1x,
                                            real a1y, real a2xx, real a2xy, real a2yy) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const real c1 = real(cx_of(i)) * a1x + real(cy_of(i)) * a1y;
        p[i] = p[i] - k0 * n[i] -
               w_of<real>(i) * (real(3) * c1 + real(4.5) * q_dot<real>(i, a2xx, a2xy, a2yy));
    }
}

// ---- block reductions (deterministic for a fixed block shape) ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Sums (kind 0) or maxes (kind 1) NV values across the block; result valid in
// thread 0.  `sh` holds 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const int (&kind)[NV],
                                             double *sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthreads = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = kind[k] ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = (lane < nwarps) ? sh[k * 32 + lane] : 0.0;
            v[k] = kind[k] ? warp_max(x) : warp_sum(x);
        }
    }
}

// ---- per-cell streaming ----
template <typename real, int PROB, bool FLOW>
__device__ __forceinline__ void pull_cell(const SweepArgs<real> &a, int x, int y, real f[9],
                                          real g[9], real &q) {
    const real th2 = real(2);  // 2 T_h with T_h = 1
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sx = x - cx, sy = y - cy;
        if (PROB == kStefan) sy = (sy < 0) ? sy + a.ny : ((sy >= a.ny) ? sy - a.ny : sy);
        const bool in = (unsigned)sx < (unsigned)a.nx && (unsigned)sy < (unsigned)a.ny;
        const long long cell = in ? (long long)sy * a.pitch + sx : (long long)y * a.pitch + x;
        const int pl = in ? i : opp_of(i);
        real gv = __ldg(a.src + (long long)(9 + pl) * a.pstride + cell);
        if (FLOW) f[i] = __ldg(a.src + (long long)pl * a.pstride + cell);
        if (!in) {
            bool heated;
            if (PROB == kStefan) {
                heated = sx < 0;
            } else {
                const int xc2 = 2 * x + 1 - cx;  // twice the wall-crossing abscissa
                heated = a.strip_on && sy < 0 && xc2 >= a.lo2 && xc2 <= a.hi2;
            }
            if (heated) {
                const real wt = w_of<real>(i) * th2;
                q += wt - real(2) * gv;
                gv = wt - gv;
            }
        }
        g[i] = gv;
    }
}

template <typename real, int PROB, bool FLOW, int MODE>
__global__ void __launch_bounds__(256) lattice_kernel(const SweepArgs<real> a) {
    __shared__ double sh[32 * 4];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = x < a.nx && y < a.ny;

    real q = real(0);
    real H = real(0), T = real(0), fl = real(0), rho = real(1), ux = real(0), uy = real(0);
    if (active) {
        real f[9], g[9];
        pull_cell<real, PROB, FLOW>(a, x, y, f, g, q);

        // flow moments
        real jx = real(0), jy = real(0);
        if (FLOW) {
            rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        }
        // total enthalpy and its inversion (H_s = 0, H_l = L)
        H = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
        if (H <= real(0)) {
            T = H;
            fl = real(0);
        } else if (H >= a.Lh) {
            T = H - a.Lh;
            fl = real(1);
        } else {
            T = real(0);
            fl = H / a.Lh;
        }
        // buoyancy and solid treatment
        real Fy = real(0);
        if (FLOW) {
            Fy = a.gbeta * T;
            const real inv_rho = real(1) / rho;
            ux = fl * jx * inv_rho;
            uy = fl * (jy + real(0.5) * Fy) * inv_rho;
        }

        if (MODE == kFields) {
            const long long o = (long long)y * a.nx + x;
            if (a.oH) a.oH[o] = (double)H;
            if (a.oT) a.oT[o] = (double)T;
            if (a.oFL) a.oFL[o] = (double)fl;
            if (a.oUX) a.oUX[o] = (double)ux;
            if (a.oUY) a.oUY[o] = (double)uy;
            if (a.oRHO) a.oRHO[o] = (double)rho;
        } else {
            // g collision (Eq. 2, Eq. 4)
            {
                real n[9];
                const real w0T = w_of<real>(0) * T;
                n[0] = g[0] - (H - T + w0T);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const real cu = real(cx_of(i)) * ux + real(cy_of(i)) * uy;
                    n[i] = g[i] - w_of<real>(i) * T * (real(1) + real(3) * cu);
                }
                real m1x, m1y, m2xx, m2xy, m2yy;
                moments<real>(n, m1x, m1y, m2xx, m2xy, m2yy);
                const real d1 = a.k1 - a.k0, d2 = a.k2 - a.k0;
                block_relax<real>(g, n, a.k0, d1 * m1x, d1 * m1y, d2 * m2xx, d2 * m2xy,
                                  d2 * m2yy);
            }
            // f collision with forcing
            if (FLOW) {
                real n[9];
                const real uu = ux * ux + uy * uy;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const real cu = real(cx_of(i)) * ux + real(cy_of(i)) * uy;
                    n[i] = f[i] - w_of<real>(i) * rho *
                                      (real(1) + real(3) * cu + real(4.5) * cu * cu -
                                       real(1.5) * uu);
                }
                real m1x, m1y, m2xx, m2xy, m2yy;
                moments<real>(n, m1x, m1y, m2xx, m2xy, m2yy);
                const real d1 = a.k1f - a.k0f, d2 = a.k2f - a.k0f;
                const real s1 = real(1) - real(0.5) * a.k1f, s2 = real(1) - real(0.5) * a.k2f;
                block_relax<real>(f, n, a.k0f, d1 * m1x, d1 * m1y - s1 * Fy, d2 * m2xx,
                                  d2 * m2xy - s2 * ux * Fy, d2 * m2yy - s2 * real(2) * uy * Fy);
            }
            const long long cell = (long long)y * a.pitch + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                a.dst[(long long)(9 + i) * a.pstride + cell] = g[i];
                if (FLOW) a.dst[(long long)i * a.pstride + cell] = f[i];
            }
        }
    }

    if (MODE == kFields) return;

    // ---- heated-wall inflow of this step (blocks touching the T_h wall) ----
    // Each such block writes one partial; the last block to take a ticket
    // folds them in slot order (deterministic) and resets the counter.
    // Partials are read with ld.global.cg so that L1 cannot serve stale data.
    const bool qblock = (PROB == kCavity) ? (a.strip_on && blockIdx.y == 0) : (blockIdx.x == 0);
    if (qblock) {
        double v[1] = {(double)q};
        const int kind[1] = {0};
        block_reduce<1>(v, kind, sh);
        const int tid = threadIdx.x + threadIdx.y * blockDim.x;
        if (tid == 0) {
            const int slot = (PROB == kCavity) ? blockIdx.x : blockIdx.y;
            a.qpart[slot] = v[0];
            __threadfence();
            const unsigned ticket = atomicAdd(a.qcount, 1u);
            if (ticket == (unsigned)a.nq - 1u) {
                __threadfence();
                double s = 0.0;
                for (int k = 0; k < a.nq; ++k) s += __ldcg(a.qpart + k);
                a.rec->Q_last = s;
                a.rec->Q_cum += s;
                *a.qcount = 0u;
            }
        }
        __syncthreads();
    }

    // ---- diagnostics of this step ----
    if (MODE == kSweepDiag) {
        const real um = sqrt(ux * ux + uy * uy);
        const bool bad = active && !(isfinite((double)H) && isfinite((double)rho));
        double v[4] = {active ? (double)fl : 0.0, active ? (double)H : 0.0,
                       active ? (double)um : 0.0, bad ? 1.0 : 0.0};
        const int kind[4] = {0, 0, 1, 1};
        block_reduce<4>(v, kind, sh);
        const int tid = threadIdx.x + threadIdx.y * blockDim.x;
        const unsigned nblk = gridDim.x * gridDim.y;
        const unsigned bid = blockIdx.x + blockIdx.y * gridDim.x;
        __shared__ bool last;
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.dpart[4 * (size_t)bid + k] = v[k];
            __threadfence();
            last = atomicAdd(a.dcount, 1u) == nblk - 1u;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            const int nthreads = blockDim.x * blockDim.y;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (unsigned b = tid; b < nblk; b += nthreads) {
                acc[0] += __ldcg(a.dpart + 4 * (size_t)b + 0);
                acc[1] += __ldcg(a.dpart + 4 * (size_t)b + 1);
                acc[2] = fmax(acc[2], __ldcg(a.dpart + 4 * (size_t)b + 2));
                acc[3] = fmax(acc[3], __ldcg(a.dpart + 4 * (size_t)b + 3));
            }
            __syncthreads();
            block_reduce<4>(acc, kind, sh);
            if (tid == 0) {
                a.rec->step = (double)a.step;
                a.rec->melt_sum = acc[0];
                a.rec->H_sum = acc[1];
                a.rec->max_u = acc[2];
                a.rec->nan_flag = acc[3];
                a.rec->valid = 1.0;
                *a.dcount = 0u;
            }
        }
    }
}

// SplitMix64 output function (Steele, Lea & Flood 2014; Vigna's public-domain
// reference): golden-ratio increment, two xor-shift-multiply rounds, xor-shift.
__device__ __forceinline__ uint64_t splitmix64(uint64_t v) {
    uint64_t z = v + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Step-0 state: H0 = amp (2r - 1) (solid at T_m = 0 with a seeded perturbation
// of T), f_i = w_i, g_i = g_eq(H0, T(H0), u = 0) (Eq. 4); reduces the step-0
// diagnostics.
template <typename real>
__global__ void __launch_bounds__(256) init_kernel(const SweepArgs<real> a, double amp,
                                                   uint64_t seed) {
    __shared__ double sh[32 * 4];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = x < a.nx && y < a.ny;
    real H = real(0), fl = real(0);
    if (active) {
        const uint64_t cell = (uint64_t)y * (uint64_t)a.nx + (uint64_t)x;
        const double r = (double)(splitmix64(seed ^ cell) >> 11) * 0x1.0p-53;
        H = (real)(amp * (2.0 * r - 1.0));
        real T;
        if (H <= real(0)) {
            T = H;
            fl = real(0);
        } else if (H >= a.Lh) {
            T = H - a.Lh;
            fl = real(1);
        } else {
            T = real(0);
            fl = H / a.Lh;
        }
        const long long c = (long long)y * a.pitch + x;
        a.dst[9 * a.pstride + c] = H - T + w_of<real>(0) * T;
#pragma unroll
        for (int i = 1; i < 9; ++i) a.dst[(long long)(9 + i) * a.pstride + c] = w_of<real>(i) * T;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            a.dst[(long long)i * a.pstride + c] = w_of<real>(i);
            if (a.aux) a.aux[(long long)i * a.pstride + c] = w_of<real>(i);
        }
    }
    const bool bad = active && !isfinite((double)H);
    double v[4] = {(double)fl, (double)H, 0.0, bad ? 1.0 : 0.0};
    const int kind[4] = {0, 0, 1, 1};
    block_reduce<4>(v, kind, sh);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.x + blockIdx.y * gridDim.x;
    __shared__ bool last;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a.dpart[4 * (size_t)bid + k] = v[k];
        __threadfence();
        last = atomicAdd(a.dcount, 1u) == nblk - 1u;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const int nthreads = blockDim.x * blockDim.y;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned b = tid; b < nblk; b += nthreads) {
            acc[0] += __ldcg(a.dpart + 4 * (size_t)b + 0);
            acc[1] += __ldcg(a.dpart + 4 * (size_t)b + 1);
            acc[3] = fmax(acc[3], __ldcg(a.dpart + 4 * (size_t)b + 3));
        }
        __syncthreads();
        block_reduce<4>(acc, kind, sh);
        if (tid == 0) {
            a.rec->step = 0.0;
            a.rec->melt_sum = acc[0];
            a.rec->H_sum = acc[1];
            a.rec->Q_last = 0.0;
            a.rec->Q_cum = 0.0;
            a.rec->max_u = 0.0;
            a.rec->nan_flag = acc[3];
            a.rec->valid = 1.0;
            *a.dcount = 0u;
        }
    }
}

// Fields of the step-0 state (no streaming; u = 0 by definition).
template <typename real, bool FLOW>
__global__ void __launch_bounds__(256) fields0_kernel(const SweepArgs<real> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long c = (long long)y * a.pitch + x;
    real H = real(0), rho = real(1);
#pragma unroll
    for (int i = 0; i < 9; ++i) H += a.src[(long long)(9 + i) * a.pstride + c];
    if (FLOW) {
        rho = real(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) rho += a.src[(long long)i * a.pstride + c];
    }
    real T, fl;
    if (H <= real(0)) {
        T = H;
        fl = real(0);
    } else if (H >= a.Lh) {
        T = H - a.Lh;
        fl = real(1);
    } else {
        T = real(0);
        fl = H / a.Lh;
    }
    const long long o = (long long)y * a.nx + x;
    if (a.oH) a.oH[o] = (double)H;
    if (a.oT) a.oT[o] = (double)T;
    if (a.oFL) a.oFL[o] = (double)fl;
    if (a.oUX) a.oUX[o] = 0.0;
    if (a.oUY) a.oUY[o] = 0.0;
    if (a.oRHO) a.oRHO[o] = (double)rho;
}

// ---- launch dispatch (instantiated per precision in sweep_fp32/64.cu) ----
template <typename real, int PROB, bool FLOW>
static cudaError_t launch_mode(const SweepArgs<real> &a, int mode, dim3 grid, dim3 block,
                               cudaStream_t s) {
    switch (mode) {
        case kSweep: lattice_kernel<real, PROB, FLOW, kSweep><<<grid, block, 0, s>>>(a); break;
        case kSweepDiag:
            lattice_kernel<real, PROB, FLOW, kSweepDiag><<<grid, block, 0, s>>>(a);
            break;
        case kFields: lattice_kernel<real, PROB, FLOW, kFields><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_lattice(const SweepArgs<real> &a, int problem, bool flow, int mode,
                           dim3 grid, dim3 block, cudaStream_t s) {
    if (problem == kCavity)
        return flow ? launch_mode<real, kCavity, true>(a, mode, grid, block, s)
                    : launch_mode<real, kCavity, false>(a, mode, grid, block, s);
    return flow ? launch_mode<real, kStefan, true>(a, mode, grid, block, s)
                : launch_mode<real, kStefan, false>(a, mode, grid, block, s);
}

template <typename real>
cudaError_t launch_init(const SweepArgs<real> &a, double amp, uint64_t seed, dim3 grid,
                        dim3 block, cudaStream_t s) {
    init_kernel<real><<<grid, block, 0, s>>>(a, amp, seed);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fields0(const SweepArgs<real> &a, bool flow, dim3 grid, dim3 block,
                           cudaStream_t s) {
    if (flow)
        fields0_kernel<real, true><<<grid, block, 0, s>>>(a);
    else
        fields0_kernel<real, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace btrirt

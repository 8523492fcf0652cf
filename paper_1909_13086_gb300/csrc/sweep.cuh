// sweep.cuh -- the fused B-TriRT collide-and-stream kernel (device code).
//
// Layout: tile-major structure of arrays (lbm_internal.h).  One thread per
// lattice column of a kTW-wide tile, walking `rows` rows; a warp covers 32
// consecutive cells of one row, so every load and store is a coalesced 128 B
// line (FP32).  In the interior the 18 pull loads of a cell are one base
// register plus compile-time offsets; boundary rows and the two warps of a
// row that touch a side wall take a generic path with the wall rules.
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
//   6. store; reduce the heated-wall inflow (and the diagnostics).
//
// The collisions are evaluated in moment space.  With a = 1 - k0, Eq. 2 reads
//   p*_i = a p_i + k0 p^eq_i - w_i [3 c_i.A1 + 9/2 Q_i:A2],  Q_i = c_i c_i - I/3,
// where A1 = (k1 - k0) M1 and A2 = (k2 - k0) M2 are built from the raw moments
// of p minus the equilibrium moments (Eq. 4: sum c g_eq = T u, sum cc g_eq =
// T/3 I; flow: rho u and rho (I/3 + uu)).  Folding p^eq in gives
//   p*_i = a p_i + w_i [B0 + 3 c_i.B1 + 9/2 Q_i:B2]  (+ k0 (H - T) for g_0),
// about 4 flops per population instead of re-forming every n_i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "lbm_internal.h"

namespace btrirt {

// ---- D2Q9 (c_i, w_i, opposite), folded at compile time in unrolled loops.
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

// ---- storage encodings ----
// FP32 / FP64: populations as they are.  FP16 / BF16 (arithmetic in FP32):
// f_i is stored as its deviation f_i - w_i from the rest state (rho = 1, u = 0),
// g_i as it is -- its rest state (solid at T_m = 0) is zero.  The 16-bit codecs
// round to nearest (ties to even) or, with SR, stochastically: up with
// probability equal to the discarded fraction of an ulp, so that increments
// smaller than half an ulp survive on average instead of stagnating.
template <bool SR>
struct F16 {};
template <bool SR>
struct BF16 {};

// Each codec has two faces.  Physical values, for set-up and read-back: ldf /
// stf_rn decode / encode an f plane (the stored value is f_i - w_i for the
// 16-bit codecs, see f_ofs), ldg / stg_rn a g plane.  Stored units, for the
// sweep (see ld_f): ldr reads a value as stored, str_rn / strs / st2r write
// one rounded to nearest, one stochastically, or a (g_i, f_i - w_i) pair
// stochastically.
template <typename S>
struct Store;
template <>
struct Store<float> {
    using elem = float;
    static constexpr bool kDev = false, kSR = false;
    __device__ static float ldf(const float *p) { return __ldg(p); }
    __device__ static float ldg(const float *p) { return __ldg(p); }
    __device__ static void stf_rn(float *p, float v) { *p = v; }
    __device__ static void stg_rn(float *p, float v) { *p = v; }
    // stored units (see the 16-bit codecs): the values themselves
    static constexpr float kF = 1.0f, kG = 1.0f;
    __device__ static float ldr(const float *p) { return __ldg(p); }
    __device__ static void str_rn(float *p, float v) { *p = v; }
    __device__ static void strs(float *p, float v, uint32_t) { *p = v; }
    __device__ static void st2r(float *pg, float *pf, float g, float f, uint32_t) { *pg = g; *pf = f; }
};
template <>
struct Store<double> {
    using elem = double;
    static constexpr bool kDev = false, kSR = false;
    __device__ static double ldf(const double *p) { return __ldg(p); }
    __device__ static double ldg(const double *p) { return __ldg(p); }
    __device__ static void stf_rn(double *p, double v) { *p = v; }
    __device__ static void stg_rn(double *p, double v) { *p = v; }
    static constexpr double kF = 1.0, kG = 1.0;
    __device__ static double ldr(const double *p) { return __ldg(p); }
    __device__ static void str_rn(double *p, double v) { *p = v; }
    __device__ static void strs(double *p, double v, uint32_t) { *p = v; }
    __device__ static void st2r(double *pg, double *pf, double g, double f, uint32_t) {
        *pg = g;
        *pf = f;
    }
};

// Stochastic rounding by "add random bits below the cut, then truncate": a
// float's bit pattern plus a uniform integer below the first discarded bit,
// truncated toward zero, rounds the magnitude up with probability equal to the
// discarded fraction (a carry into the exponent is the correct round-up).  r is
// 16 random bits.  Only finite values may take this path (an infinity plus
// random bits would become a NaN): the sweep uses it for single values, on
// lattices without flow, and stores a non-finite cell there with the _rn
// encoders.  The paired hardware conversion (cvt_rs_*) needs no such check: it
// keeps NaN a NaN and an infinity an infinity, and rounds an FP16 overflow to
// an infinity (checked on GB300 for NaN, +-Inf, +-7e4 and +-3e38).
__device__ __forceinline__ float sr_add(float v, uint32_t add) {
    return __uint_as_float(__float_as_uint(v) + add);
}

// Two floats to 16-bit values in one conversion with stochastic rounding (the
// sm_100-family cvt with .rs rounding: the 32-bit random operand supplies the
// bits added below each half's cut).  hi lands in the upper half, lo in the
// lower half.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}

// FP16 is stored scaled by a power of two (exact): g by 2^6, f - w by 2^10, so
// that the working values sit in FP16's normal range (g down to ~1e-6, f - w
// down to ~6e-8) while g up to 1000 (latent heat 1/Ste included) and |f - w| up
// to 64 still fit.  In the normal range 13 float mantissa bits are discarded.
template <bool SR>
struct Store<F16<SR>> {
    using elem = __half;
    static constexpr bool kDev = true, kSR = SR;
    static constexpr float kG = 64.0f, kF = 1024.0f;
    __device__ static void enc(__half *p, float v, uint32_t r) {
        *p = SR ? __float2half_rz(sr_add(v, r >> 3)) : __float2half_rn(v);
    }
    __device__ static float ldf(const __half *p) { return __half2float(__ldg(p)) * (1.0f / kF); }
    __device__ static float ldg(const __half *p) { return __half2float(__ldg(p)) * (1.0f / kG); }
    __device__ static void stf_rn(__half *p, float v) { *p = __float2half_rn(v * kF); }
    __device__ static void stg_rn(__half *p, float v) { *p = __float2half_rn(v * kG); }
    // stored units: g_i kG and (f_i - w_i) kF, converted without scaling
    __device__ static float ldr(const __half *p) { return __half2float(__ldg(p)); }
    __device__ static void str_rn(__half *p, float v) { *p = __float2half_rn(v); }
    __device__ static void strs(__half *p, float v, uint32_t r) { enc(p, v, r); }
    __device__ static void st2r(__half *pg, __half *pf, float g, float f, uint32_t rbits) {
        const uint32_t d = cvt_rs_f16x2(g, f, rbits);
        *pg = __ushort_as_half((unsigned short)(d >> 16));
        *pf = __ushort_as_half((unsigned short)(d & 0xffffu));
    }
    // a (g, f) word of the paired layout: g in the high half, f in the low one
    __device__ static float hi(uint32_t u) { return __half2float(__ushort_as_half((unsigned short)(u >> 16))); }
    __device__ static float lo(uint32_t u) { return __half2float(__ushort_as_half((unsigned short)(u & 0xffffu))); }
    __device__ static uint32_t pack_rn(float g, float f) {
        return ((uint32_t)__half_as_ushort(__float2half_rn(g)) << 16) | __half_as_ushort(__float2half_rn(f));
    }
    __device__ static uint32_t pack_sr(float g, float f, uint32_t rbits) { return cvt_rs_f16x2(g, f, rbits); }
};
// BF16 has FP32's exponent range, so no scaling; 16 bits are discarded.
template <bool SR>
struct Store<BF16<SR>> {
    using elem = __nv_bfloat16;
    static constexpr bool kDev = true, kSR = SR;
    __device__ static float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st(__nv_bfloat16 *p, float v, uint32_t r) {
        *p = SR ? __ushort_as_bfloat16((unsigned short)(__float_as_uint(sr_add(v, r)) >> 16))
                : __float2bfloat16_rn(v);
    }
    __device__ static float ldf(const __nv_bfloat16 *p) { return ld(p); }
    __device__ static float ldg(const __nv_bfloat16 *p) { return ld(p); }
    __device__ static void stf_rn(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static void stg_rn(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    // stored units: g_i and f_i - w_i (no scaling)
    static constexpr float kF = 1.0f, kG = 1.0f;
    __device__ static float ldr(const __nv_bfloat16 *p) { return ld(p); }
    __device__ static void str_rn(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static void strs(__nv_bfloat16 *p, float v, uint32_t r) { st(p, v, r); }
    __device__ static void st2r(__nv_bfloat16 *pg, __nv_bfloat16 *pf, float g, float f,
                                uint32_t rbits) {
        const uint32_t d = cvt_rs_bf16x2(g, f, rbits);
        *pg = __ushort_as_bfloat16((unsigned short)(d >> 16));
        *pf = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
    }
    // a (g, f) word of the paired layout: a BF16 value is the top half of a float
    __device__ static float hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
    __device__ static float lo(uint32_t u) { return __uint_as_float(u << 16); }
    __device__ static uint32_t pack_rn(float g, float f) {
        return ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(g)) << 16) |
               __bfloat16_as_ushort(__float2bfloat16_rn(f));
    }
    __device__ static uint32_t pack_sr(float g, float f, uint32_t rbits) { return cvt_rs_bf16x2(g, f, rbits); }
};
// Where plane p (0..8: f_0..f_8, 9..17: g_0..g_8) of the cell in column lx of
// a tile row lives, counted in elements from the row's first one.  FP32 /
// FP64: plane after plane, kTW values each (lbm_internal.h).  16-bit storage:
// f_i and g_i, which stream from the same source cell, share one 32-bit word
// -- f_i in the low half, g_i in the high half -- and the nine words of the
// directions follow one another kTW at a time, so that one 32-bit load and one
// 32-bit store move both populations of a direction.  A tile row holds the
// same 18 kTW values either way.
template <typename S>
__host__ __device__ constexpr int plane_ofs(int p, int lx) {
    return Store<S>::kDev ? 2 * ((p % 9) * kTW + lx) + (p >= 9 ? 1 : 0) : p * kTW + lx;
}
template <typename S>
__host__ __device__ inline long long cell_index(int x, int y, int p, int ny) {
    return ((long long)(x / kTW) * ny + y) * kRS + plane_ofs<S>(p, x % kTW);
}
// Elements from one column to the next within a plane (2 in the paired layout).
template <typename S>
__host__ __device__ constexpr int col_step() {
    return Store<S>::kDev ? 2 : 1;
}

// Offset added to a stored f value (plane i) to recover f_i.
template <typename real, typename S>
__device__ __forceinline__ real f_ofs(int i) {
    return Store<S>::kDev ? w_of<real>(i) : real(0);
}
// The sweep works in stored units: f as stored (f_i itself, or the scaled
// deviation (f_i - w_i) kF of the 16-bit codecs) and g_i kG, so that no
// population is rescaled or offset on its way in or out; cell_update carries
// the scales and the rest state in a few per-cell terms instead.
template <typename real, typename S>
__device__ __forceinline__ real ld_f(const typename Store<S>::elem *p, int) {
    return Store<S>::ldr(p);
}
template <typename real, typename S>
__device__ __forceinline__ real ld_g(const typename Store<S>::elem *p, int) {
    return Store<S>::ldr(p);
}

// Counter-based random bits for stochastic rounding: a 32-bit integer hash
// (Wellons' "lowbias32" finaliser) of the step seed and the cell index seeds a
// linear congruential generator (Numerical Recipes' constants).  lcg_next
// gives the top 16 bits of the next state (one value); lcg_next32 gives 32
// bits (a pair of values), the state xor its top half shifted down so that the
// low half does not carry the LCG's short-period low bits.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint32_t lcg_next(uint32_t &s) {
    s = s * 1664525u + 1013904223u;
    return s >> 16;
}
__device__ __forceinline__ uint32_t lcg_next32(uint32_t &s) {
    s = s * 1664525u + 1013904223u;
    return s ^ (s >> 16);
}

// ---- H -> (T, f_l): H_s = C_p T_m = 0, H_l = H_s + L.
template <typename real>
__device__ __forceinline__ void invert(real H, real Lh, real inv_Lh, real &T, real &fl) {
    if (H <= real(0)) {
        T = H;
        fl = real(0);
    } else if (H >= Lh) {
        T = H - Lh;
        fl = real(1);
    } else {
        T = real(0);
        fl = H * inv_Lh;
    }
}

// 1 / x: the fast reciprocal in FP32 (about 2 ulp; the FP32 path's tolerance
// is 1e-5), the exact quotient in FP64 (the parity path).
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// p_i <- a p_i + w_i [B0 + 3 c_i.B1 + 9/2 Q_i:B2]  for all nine directions.
// With X = B2xx, Y = B2yy, Z = B2xy, S = X + Y and Q_i = c_i c_i - I/3, the
// products w_i * 9/2 Q_i:B2 are -2S/3 (rest), X/3 - Y/6 (+-x), Y/3 - X/6
// (+-y), S/12 + Z/4 (diagonals 5, 7) and S/12 - Z/4 (6, 8); w_i * 3 c_i.B1 is
// +-B1x/3, +-B1y/3, +-(B1x + B1y)/12 and +-(B1y - B1x)/12.  In FP32 the
// rounded weights sum to 1 + 7.45e-9, which would add k0 B0 7.45e-9 to every
// cell's sum each step (a steady growth of the FP32 density); the rest weight's
// share is therefore taken as B0 - 4 (w1 B0 + w5 B0), so that the shares sum
// to B0 up to rounding.  FP64's weights sum to 1 within 1e-16 and keep w0 B0.
template <typename real>
__device__ __forceinline__ void emit(real p[9], real a, real B0, real B1x, real B1y, real B2xx,
                                     real B2xy, real B2yy) {
    const real third = real(1) / real(3), sixth = real(1) / real(6), twelfth = real(1) / real(12);
    const real w0 = real(4) / real(9), w1 = real(1) / real(9), w5 = real(1) / real(36);
    const real S = B2xx + B2yy;
    const real W1 = w1 * B0, W5 = w5 * B0;
    const real W0 = sizeof(real) == 4 ? B0 - real(4) * (W1 + W5) : w0 * B0;
    p[0] = a * p[0] + (W0 - (real(2) / real(3)) * S);
    const real e13 = W1 + third * B2xx - sixth * B2yy, t1 = third * B1x;
    p[1] = a * p[1] + (e13 + t1);
    p[3] = a * p[3] + (e13 - t1);
    const real e24 = W1 + third * B2yy - sixth * B2xx, t2 = third * B1y;
    p[2] = a * p[2] + (e24 + t2);
    p[4] = a * p[4] + (e24 - t2);
    const real e5 = W5 + twelfth * S, z4 = real(0.25) * B2xy;
    const real e57 = e5 + z4, t5 = twelfth * (B1x + B1y);
    p[5] = a * p[5] + (e57 + t5);
    p[7] = a * p[7] + (e57 - t5);
    const real e68 = e5 - z4, t6 = twelfth * (B1y - B1x);
    p[6] = a * p[6] + (e68 + t6);
    p[8] = a * p[8] + (e68 - t6);
}

// Raw first and second moments of nine populations (the diagonal pairs'
// sums and differences shared).
template <typename real>
__device__ __forceinline__ void raw_moments(const real p[9], real &jx, real &jy, real &pxx,
                                            real &pxy, real &pyy) {
    const real s57 = p[5] + p[7], s68 = p[6] + p[8];
    const real d57 = p[5] - p[7], d68 = p[6] - p[8];
    jx = (p[1] - p[3]) + (d57 - d68);
    jy = (p[2] - p[4]) + (d57 + d68);
    const real d = s57 + s68;
    pxx = (p[1] + p[3]) + d;
    pyy = (p[2] + p[4]) + d;
    pxy = s57 - s68;
}

template <typename real>
__device__ __forceinline__ real sum9(const real p[9]) {
    return (((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]))) + p[8];
}

template <typename real>
struct Macro {
    real H, T, fl, rho, ux, uy;
};

// Steps 2-5 on one cell: macroscopic fields, then both collisions in place
// (COLLIDE = false stops after the fields).  f and g are in stored units (see
// ld_f); the returned fields are physical.  With the 16-bit codecs f holds
// delta_i = (f_i - w_i) kF: its raw moments are kF times those of f less the
// rest state's (j; the second moments less I/3), rho = 1 + sum(delta) / kF,
// and the block collision of delta is that of f with B0 = k0 (rho - 1) kF,
// since a + k0 = 1 cancels the rest state; g holds g_i kG and collides with
// T kG and H kG in place of T and H.
template <typename real, typename S, bool FLOW, bool COLLIDE>
__device__ __forceinline__ Macro<real> cell_update(const SweepArgs<real> &a, real f[9], real g[9]) {
    constexpr bool kDev = Store<S>::kDev;
    constexpr real kF = real(Store<S>::kF), kG = real(Store<S>::kG);
    Macro<real> m;
    real fs = real(0), fjx = real(0), fjy = real(0), fxx = real(0), fxy = real(0), fyy = real(0);
    m.rho = real(1);
    if (FLOW) {
        fs = sum9(f);
        raw_moments(f, fjx, fjy, fxx, fxy, fyy);
        if constexpr (kDev) m.rho = real(1) + fs * (real(1) / kF);
        else m.rho = fs;
    }
    const real Hs = sum9(g);
    if constexpr (kG != real(1)) m.H = Hs * (real(1) / kG);
    else m.H = Hs;
    invert(m.H, a.Lh, a.inv_Lh, m.T, m.fl);
    real Fy = real(0), Fk = real(0);
    m.ux = real(0);
    m.uy = real(0);
    if (FLOW) {
        Fy = a.gbeta * m.T;
        real iu = recip(m.rho);
        Fk = Fy;
        if constexpr (kF != real(1)) {
            iu = iu * (real(1) / kF);
            Fk = Fy * kF;
        }
        m.ux = m.fl * fjx * iu;
        m.uy = m.fl * (fjy + real(0.5) * Fk) * iu;
    }
    if (!COLLIDE) return m;

    const real third = real(1) / real(3);
    // ---- g (Eq. 2 with Eq. 4)
    {
        real gjx, gjy, gxx, gxy, gyy;
        raw_moments(g, gjx, gjy, gxx, gxy, gyy);
        real T = m.T;
        if constexpr (kG != real(1)) T = m.T * kG;
        const real T3 = T * third;
        const real d1 = a.k1 - a.k0, d2 = a.k2 - a.k0;
        const real k0T = a.k0 * T;
        const real B1x = k0T * m.ux - d1 * (gjx - T * m.ux);
        const real B1y = k0T * m.uy - d1 * (gjy - T * m.uy);
        emit(g, real(1) - a.k0, k0T, B1x, B1y, -d2 * (gxx - T3), -d2 * gxy, -d2 * (gyy - T3));
        g[0] += a.k0 * (Hs - T);
    }
    // ---- f (same block operator, forcing folded into A1 and A2)
    if (FLOW) {
        const real ux = m.ux, uy = m.uy;
        real rk = m.rho, R0 = m.rho;  // rho in stored units; the density term of B0
        if constexpr (kDev) {
            R0 = fs;
            if constexpr (kF != real(1)) rk = m.rho * kF;
        }
        const real rux = rk * ux, ruy = rk * uy;
        const real rxx = rux * ux, rxy = rux * uy, ryy = ruy * uy, r3 = R0 * third;
        const real d1 = a.k1f - a.k0f, d2 = a.k2f - a.k0f;
        const real s1 = real(1) - real(0.5) * a.k1f, s2 = real(1) - real(0.5) * a.k2f;
        const real A1x = d1 * (fjx - rux);
        const real A1y = d1 * (fjy - ruy) - s1 * Fk;
        const real A2xx = d2 * (fxx - r3 - rxx);
        const real A2xy = d2 * (fxy - rxy) - s2 * ux * Fk;
        const real A2yy = d2 * (fyy - r3 - ryy) - s2 * real(2) * uy * Fk;
        const real k0 = a.k0f;
        emit(f, real(1) - k0, k0 * R0, k0 * rux - A1x, k0 * ruy - A1y, k0 * rxx - A2xx,
             k0 * rxy - A2xy, k0 * ryy - A2yy);
        // FP32 storage: the collision conserves mass, sum f*_i = sum f_i, and
        // the rest population is taken from that invariant, so that the
        // rounding of the nine emitted values leaves no drift in the density
        // (other rounding biases of the emitted values add ~4e-9 per step in
        // a convecting cavity).  16-bit storage rounds f*_i stochastically on
        // store, which is unbiased.
        if constexpr (!kDev && sizeof(real) == 4)
            f[0] = fs - (((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
    }
    return m;
}

// ---- streaming ----
// Interior cell: no wall in reach.  b points at (x, y, plane 0); bL / bR equal
// b except at the tile's first / last column, where they are shifted so that
// bL[-1] / bR[+1] land in the neighbouring tile.
template <typename real, typename S, bool FLOW>
__device__ __forceinline__ void pull_fast(const typename Store<S>::elem *__restrict__ b,
                                          const typename Store<S>::elem *__restrict__ bL,
                                          const typename Store<S>::elem *__restrict__ bR, real f[9],
                                          real g[9]) {
    if constexpr (Store<S>::kDev) {
        // paired layout: word i of a cell holds (g_i, f_i); a row is kRS / 2
        // words, a direction's words kTW apart
        constexpr int R = kRS / 2, W = kTW;
        if (FLOW) {
            const uint32_t *w = reinterpret_cast<const uint32_t *>(b);
            const uint32_t *wl = reinterpret_cast<const uint32_t *>(bL);
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(bR);
            uint32_t u[9];
            u[0] = __ldg(w + 0 * W);
            u[1] = __ldg(wl + 1 * W - 1);
            u[2] = __ldg(w + 2 * W - R);
            u[3] = __ldg(wr + 3 * W + 1);
            u[4] = __ldg(w + 4 * W + R);
            u[5] = __ldg(wl + 5 * W - R - 1);
            u[6] = __ldg(wr + 6 * W - R + 1);
            u[7] = __ldg(wr + 7 * W + R + 1);
            u[8] = __ldg(wl + 8 * W + R - 1);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = Store<S>::lo(u[i]);
                g[i] = Store<S>::hi(u[i]);
            }
        } else {  // the high halves only: element 2 * word + 1
            g[0] = Store<S>::ldr(b + 2 * (0 * W) + 1);
            g[1] = Store<S>::ldr(bL + 2 * (1 * W - 1) + 1);
            g[2] = Store<S>::ldr(b + 2 * (2 * W - R) + 1);
            g[3] = Store<S>::ldr(bR + 2 * (3 * W + 1) + 1);
            g[4] = Store<S>::ldr(b + 2 * (4 * W + R) + 1);
            g[5] = Store<S>::ldr(bL + 2 * (5 * W - R - 1) + 1);
            g[6] = Store<S>::ldr(bR + 2 * (6 * W - R + 1) + 1);
            g[7] = Store<S>::ldr(bR + 2 * (7 * W + R + 1) + 1);
            g[8] = Store<S>::ldr(bL + 2 * (8 * W + R - 1) + 1);
        }
        return;
    }
    constexpr int R = kRS, W = kTW;
#define BTRIRT_PULL(P, arr, LD)                             \
    arr[0] = LD<real, S>(b + (P + 0) * W, 0);               \
    arr[1] = LD<real, S>(bL + (P + 1) * W - 1, 1);          \
    arr[2] = LD<real, S>(b + (P + 2) * W - R, 2);           \
    arr[3] = LD<real, S>(bR + (P + 3) * W + 1, 3);          \
    arr[4] = LD<real, S>(b + (P + 4) * W + R, 4);           \
    arr[5] = LD<real, S>(bL + (P + 5) * W - R - 1, 5);      \
    arr[6] = LD<real, S>(bR + (P + 6) * W - R + 1, 6);      \
    arr[7] = LD<real, S>(bR + (P + 7) * W + R + 1, 7);      \
    arr[8] = LD<real, S>(bL + (P + 8) * W + R - 1, 8);
    BTRIRT_PULL(9, g, ld_g)
    if (FLOW) {
        BTRIRT_PULL(0, f, ld_f)
    }
#undef BTRIRT_PULL
}

// Half-way bounce-back at the cavity's adiabatic no-slip side walls for a cell
// of an interior row, after pull_fast: the directions whose source lies beyond
// x = 0 (c_x = +1: 1, 5, 8) or beyond x = nx - 1 (c_x = -1: 3, 6, 7) take the
// cell's own post-collision opposite populations, as pull_any does.
// The cell's own post-collision populations of direction o (b points at the
// cell's element of plane 0).
template <typename real, typename S, bool FLOW>
__device__ __forceinline__ void load_own(const typename Store<S>::elem *b, int o, real &f, real &g) {
    if constexpr (Store<S>::kDev) {
        if (FLOW) {
            const uint32_t u = __ldg(reinterpret_cast<const uint32_t *>(b) + o * kTW);
            f = Store<S>::lo(u);
            g = Store<S>::hi(u);
        } else {
            g = Store<S>::ldr(b + 2 * o * kTW + 1);
        }
    } else {
        g = ld_g<real, S>(b + (9 + o) * kTW, o);
        if (FLOW) f = ld_f<real, S>(b + o * kTW, o);
    }
}

template <typename real, typename S, bool FLOW>
__device__ __forceinline__ void bounce_side_walls(const typename Store<S>::elem *b, int x, int nx,
                                                  real f[9], real g[9]) {
    if (x == 0) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (cx_of(i) != 1) continue;
            load_own<real, S, FLOW>(b, opp_of(i), f[i], g[i]);
        }
    }
    if (x == nx - 1) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (cx_of(i) != -1) continue;
            load_own<real, S, FLOW>(b, opp_of(i), f[i], g[i]);
        }
    }
}

// A cavity warp that touches a side wall, on an interior row, in the push
// sweep of one-buffer streaming: pull_fast's bases and offsets, except that a
// direction whose source lies beyond the side wall reads the cell's own slot
// opp(i) (its post-collision opposite population, which the adiabatic wall
// returns as it is) instead of a clamped address -- so, unlike pull_fast plus
// bounce_side_walls, the warp reads only what its own cells write.
template <typename real, typename S, bool FLOW>
__device__ __forceinline__ void pull_sidewall(const typename Store<S>::elem *b,
                                              const typename Store<S>::elem *bL,
                                              const typename Store<S>::elem *bR, int x, int nx, real f[9],
                                              real g[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        const bool wall = (cx > 0 && x == 0) || (cx < 0 && x == nx - 1);
        const typename Store<S>::elem *from = (cx > 0 ? bL : (cx < 0 ? bR : b)) - cy * kRS - cx * col_step<S>();
        real fv = real(0), gv;
        load_own<real, S, FLOW>(wall ? b : from, wall ? opp_of(i) : i, fv, gv);
        if (FLOW) f[i] = fv;
        g[i] = gv;
    }
}

// The rule for the g population of direction i entering cell x from beyond a
// wall (source (sx, sy) outside the lattice), given gv = the cell's own
// post-collision g*_opp(i): half-way bounce-back (gv as it is) on adiabatic
// walls; anti-bounce-back 2 w_i C_p T_h - gv on the wall held at T_h (the
// Stefan problem's left wall, the cavity's heated bottom segment), whose
// inflow 2 w_i T_h - 2 gv enters q.  Values in g's stored units; q physical.
template <typename real, typename S, int PROB>
__device__ __forceinline__ real wall_rule_g(const SweepArgs<real> &a, int x, int i, int sx, int sy, real gv,
                                            double &q) {
    bool heated;
    if (PROB == kStefan) {
        heated = sx < 0;
    } else {
        const int xc2 = 2 * x + 1 - cx_of(i);  // twice the wall-crossing abscissa
        heated = a.strip_on && sy < 0 && xc2 >= a.lo2 && xc2 <= a.hi2;
    }
    if (!heated) return gv;
    const real wt = real(2) * w_of<real>(i) * real(Store<S>::kG);  // 2 w_i C_p T_h, T_h = 1
    q += (double)((wt - real(2) * gv) * (real(1) / real(Store<S>::kG)));
    return wt - gv;
}

// Any cell: explicit source test per direction and the wall rules.
template <typename real, typename S, int PROB, bool FLOW>
__device__ __forceinline__ void pull_any(const SweepArgs<real> &a, int x, int y, real f[9],
                                         real g[9], double &q) {
    const auto *src = static_cast<const typename Store<S>::elem *>(a.src);
    const long long self = cell_index<S>(x, y, 0, a.ny);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sx = x - cx, sy = y - cy;
        if (PROB == kStefan) sy = (sy < 0) ? sy + a.ny : ((sy >= a.ny) ? sy - a.ny : sy);
        const bool in = (unsigned)sx < (unsigned)a.nx && (unsigned)sy < (unsigned)a.ny;
        const long long cell = in ? cell_index<S>(sx, sy, 0, a.ny) : self;
        const int pl = in ? i : opp_of(i);
        real gv, fv = real(0);
        load_own<real, S, FLOW>(src + cell, pl, fv, gv);
        if (FLOW) f[i] = fv;
        if (!in) gv = wall_rule_g<real, S, PROB>(a, x, i, sx, sy, gv, q);
        g[i] = gv;
    }
}

// The local sweep of one-buffer streaming: f_i(x) is the cell's own slot
// opp(i) -- put there by the neighbour x - c_i's push, or, where x - c_i lies
// beyond a wall, by the cell's own push of f*_opp(i)(x) -- so a cell takes all
// its populations from its own tile row (b: its element of plane 0).
template <typename real, typename S, bool FLOW>
__device__ __forceinline__ void pull_local(const typename Store<S>::elem *b, real f[9], real g[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        real fv = real(0), gv;
        load_own<real, S, FLOW>(b, opp_of(i), fv, gv);
        if (FLOW) f[i] = fv;
        g[i] = gv;
    }
}
// Wall rules of the local sweep for a cell on the lattice's edge: the slots
// of wall-crossing directions hold the cell's own f*_opp(i)(x), the value
// pull_any reads there, and take the same rule (bounce-back as it is;
// anti-bounce-back on the wall held at T_h, whose inflow enters q).
template <typename real, typename S, int PROB, bool FLOW>
__device__ __forceinline__ void wall_rules_local(const SweepArgs<real> &a, int x, int y, real g[9],
                                                 double &q) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sx = x - cx, sy = y - cy;
        if (PROB == kStefan) sy = (sy < 0) ? sy + a.ny : ((sy >= a.ny) ? sy - a.ny : sy);
        const bool in = (unsigned)sx < (unsigned)a.nx && (unsigned)sy < (unsigned)a.ny;
        if (!in) g[i] = wall_rule_g<real, S, PROB>(a, x, i, sx, sy, g[i], q);
    }
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// launched with the programmatic-serialization attribute may start while the
// previous kernel of its stream is still running: each block first lets the
// next kernel be scheduled (that happens once every block of this grid has
// done so, i.e. when the last wave is resident), then waits until the previous
// kernel has completed and its memory is visible before it reads or writes
// anything.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- reductions ----
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Sums (kind 0) or maxes (kind 1) NV values over the block, one value per
// warp (lane 0 holds it); result valid in thread 0.  `sh` holds 32*NV 8-byte
// values.
template <int NV, typename T>
__device__ __forceinline__ void block_fold(T (&v)[NV], const int (&kind)[NV], void *shv) {
    T *sh = static_cast<T *>(shv);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T x = (lane < nwarps) ? sh[k * 32 + lane] : T(0);
            v[k] = kind[k] ? warp_max(x) : warp_sum(x);
        }
    }
    __syncthreads();
}

// ---- diagnostics accumulators ----
// FP64 path: FP64 throughout.  FP32 path: each cell's f_l and H are encoded as
// fixed point (2^-24 units, rounded to nearest once per cell) and every sum
// from there on is an exact integer sum -- independent of the order, so of
// the launch shape and of batching, and on the integer pipes: on GB300 the
// FP64 rate (~2 FMA/clock/SM) makes FP64 shuffle folds cost as much as the
// sweep itself.  In the sweeps each row of a warp is summed at once by the
// warp-reduction unit in 32-bit integers (see diag_row).  The maximum |u|
// travels as the bit pattern of a non-negative float (integer order = float
// order).  The record receives FP64 values decoded once at the end.  Range:
// |H| < 2^31 per cell, totals up to 2^39 (5.5e11) per quantity.
template <typename real>
struct DiagAcc {
    using T = double;
};
template <>
struct DiagAcc<float> {
    using T = long long;
};
constexpr float kFixScale = 16777216.0f;  // 2^24
__device__ __forceinline__ long long enc_sum(float v) { return __float2ll_rn(v * kFixScale); }
__device__ __forceinline__ double enc_sum(double v) { return v; }
__device__ __forceinline__ long long enc_max(float v) { return (long long)__float_as_int(v); }
__device__ __forceinline__ double enc_max(double v) { return v; }
__device__ __forceinline__ double dec_sum(long long q) { return (double)q * (1.0 / 16777216.0); }
__device__ __forceinline__ double dec_sum(double v) { return v; }
__device__ __forceinline__ double dec_max(long long q) { return (double)__int_as_float((int)q); }
__device__ __forceinline__ double dec_max(double v) { return v; }

// Per-block diagnostics partials.  A sweep (or the init kernel) writes one
// record of 4 accumulators per block with plain stores -- no fence, no ticket,
// so a block's lifetime does not grow -- and diag_reduce_kernel, launched
// right after on the same stream, folds them into the FP64 record.  Inputs
// here are the thread's sums of enc_sum(f_l) and enc_sum(H) over its cells
// (the init kernel, and the FP64 sweeps).
template <typename real>
__device__ __forceinline__ void diag_partial(typename DiagAcc<real>::T sfl,
                                             typename DiagAcc<real>::T sH, real umax2, bool bad,
                                             double *dpart, size_t bid, double *sh) {
    using A = typename DiagAcc<real>::T;
    const real wu = warp_max(umax2);
    const int wbad = __any_sync(0xffffffffu, bad) ? 1 : 0;
    A v[4] = {warp_sum(sfl), warp_sum(sH), enc_max(sqrt(wu)), A(wbad)};
    const int kind[4] = {0, 0, 1, 1};
    block_fold<4, A>(v, kind, sh);
    if (threadIdx.x == 0) {
        A *d = reinterpret_cast<A *>(dpart) + 4 * bid;
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = v[k];
    }
}

// Fold of the per-block partials in two levels: thread t of fold block r
// folds partials r T + t, r T + t + G T, ... (G fold blocks, T threads each;
// a fixed order), then the block folds its threads' values (fixed tree) into
// a level-2 partial; the last of the G blocks to take a ticket folds the
// level-2 partials the same way and writes the record.  The order is fixed,
// so the record is bitwise reproducible (and on the FP32 path exact in fixed
// point).  G is at most T, so the second level is one pass of one block.
constexpr int kReduceThreads = 1024;

template <typename A>
__device__ __forceinline__ void load4(A (&acc)[4], const A *part, unsigned idx, bool ok) {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = ok ? __ldcg(part + 4 * (size_t)idx + k) : A(0);
}

// acc (kinds {sum, sum, max, max}) folded with partials first, first + step, ...
// below n.
template <typename A>
__device__ __forceinline__ void fold4_strided(A (&acc)[4], const A *part, size_t first, size_t step,
                                              size_t n) {
    for (size_t i = first; i < n; i += step) {
        const A *q = part + 4 * i;
        acc[0] += __ldcg(q + 0);
        acc[1] += __ldcg(q + 1);
        acc[2] = max(acc[2], __ldcg(q + 2));
        acc[3] = max(acc[3], __ldcg(q + 3));
    }
}

// A full history entry at a diagnostic step: step, this step's heated-wall
// inflow, melt fraction.
__device__ __forceinline__ void hist_put(double *hist, long long cap, const DevRecord *rec,
                                         double ncells) {
    const long long st = (long long)rec->step;
    double *e = hist + 4 * (st % cap);
    e[0] = rec->step;
    e[1] = rec->Q_last;
    e[2] = rec->melt_sum / ncells;
}

template <typename A>
__global__ void __launch_bounds__(kReduceThreads)
    diag_reduce_kernel(const double *dpart, unsigned nblk, double *part2, unsigned *ticket,
                       DevRecord *rec, int init, double *hist, long long hist_cap, double ncells) {
    __shared__ double sh[32 * 4];
    __shared__ bool last;
    const int kind[4] = {0, 0, 1, 1};
    pdl_launch_dependents();
    pdl_wait();  // the sweep's partials
    A acc[4] = {A(0), A(0), A(0), A(0)};
    fold4_strided(acc, reinterpret_cast<const A *>(dpart), (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                  (size_t)gridDim.x * blockDim.x, nblk);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = kind[k] ? warp_max(acc[k]) : warp_sum(acc[k]);
    block_fold<4, A>(acc, kind, sh);
    if (threadIdx.x == 0) {
        A *d = reinterpret_cast<A *>(part2) + 4 * (size_t)blockIdx.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = acc[k];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    load4(acc, reinterpret_cast<const A *>(part2), threadIdx.x, threadIdx.x < gridDim.x);  // G <= T
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = kind[k] ? warp_max(acc[k]) : warp_sum(acc[k]);
    block_fold<4, A>(acc, kind, sh);
    if (threadIdx.x == 0) {
        rec->step = init ? 0.0 : (double)rec->counter;
        rec->melt_sum = dec_sum(acc[0]);
        rec->H_sum = dec_sum(acc[1]);
        rec->max_u = dec_max(acc[2]);
        rec->nan_flag = acc[3] != A(0) ? 1.0 : 0.0;
        rec->valid = 1.0;
        if (init) {
            rec->Q_last = 0.0;
            rec->Q_cum = 0.0;
            rec->counter = 0ull;
        }
        *ticket = 0u;
        if (hist && !init) hist_put(hist, hist_cap, rec, ncells);
    }
}

// Bulk prefetch of one contiguous tile row (all 18 planes, kRS values) into
// L2: a single TMA-unit request, no registers or shared memory involved.  The
// address is 16 B aligned (tile rows are kRS * sizeof(E) bytes apart from a
// 256 B aligned base) and the size a multiple of 16.
template <typename E>
__device__ __forceinline__ void prefetch_tile_row_l2(const E *p) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p),
                 "r"((unsigned)(kRS * sizeof(E)))
                 : "memory");
}

// ---- the sweep ----
// Per-step bookkeeping at a block's start: the device-side step counter
// (advanced by block (0, 0); read by the diagnostics fold after this launch)
// and the stochastic-rounding seed of this step, read from the word of the
// source buffer's parity -- block (0, 0) hands the next value to the other
// word, which only the next step reads: no race, and graph replays see a new
// seed every step.
template <typename real, typename S, int MODE>
__device__ __forceinline__ uint32_t step_prologue(const SweepArgs<real> &a, int bx, int by) {
    if (MODE != kFields && threadIdx.x == 0 && bx == 0 && by == 0) a.rec->counter += 1ull;
    uint32_t step_seed = 0;
    if (Store<S>::kSR && MODE != kFields) {
        const unsigned long long sd = a.rec->rng[a.parity];
        if (threadIdx.x == 0 && bx == 0 && by == 0) a.rec->rng[a.parity ^ 1] = sd + 1ull;
        step_seed = hash32((uint32_t)sd ^ 0x5bd1e995u);
    }
    return step_seed;
}

// Diagnostics accumulators of one thread.
// The heated-wall inflow is summed in FP64 from the first crossing on: a sum
// of a band's working-precision terms is then exact, so the flux does not
// depend on how many rows a block covers.  sfl and sH: the thread's sums
// (FP64 sweeps), or the warp's sums over its rows so far, held by every lane
// (FP32 sweeps, see diag_row).
template <typename real>
struct CellSums {
    double q = 0.0;
    real umax2 = real(0);
    typename DiagAcc<real>::T sfl = 0, sH = 0;
    bool bad = false;
};

// The diagnostics of one cell; zero for a lane without a cell.
template <typename real>
struct CellDiag {
    real fl = real(0), H = real(0), u2 = real(0);
    bool bad = false;
};

// One row of a warp into the accumulators; every lane of the warp calls it.
// FP32: f_l (at most 2^24 in fixed point) and H -- split into its integer part
// and its fraction, both exact in a float, so that each partial fits in 32
// bits -- are summed over the row's 32 cells by the warp-reduction unit, and
// the totals widened to 64 bits: the same exact sum of the cells' rounded
// values that encoding every cell in 64 bits gives (trunc(H) is an integer, so
// rounding H 2^24 to nearest equals trunc(H) 2^24 + rounding its fraction),
// for a handful of instructions per cell instead of a 64-bit conversion on
// the FP64 pipe and a 64-bit shuffle tree per block.
__device__ __forceinline__ void diag_row(CellSums<float> &acc, const CellDiag<float> &c) {
    const unsigned full = 0xffffffffu;
    const int fl = __float2int_rn(c.fl * kFixScale);
    const float hi = truncf(c.H);
    const int h_hi = (int)hi;
    const int h_lo = __float2int_rn((c.H - hi) * kFixScale);
    acc.sfl += (long long)__reduce_add_sync(full, fl);
    acc.sH += ((long long)__reduce_add_sync(full, h_hi) << 24) + (long long)__reduce_add_sync(full, h_lo);
    acc.umax2 = fmaxf(acc.umax2, c.u2);
    acc.bad |= c.bad;
}
__device__ __forceinline__ void diag_row(CellSums<double> &acc, const CellDiag<double> &c) {
    acc.sfl += c.fl;
    acc.sH += c.H;
    acc.umax2 = max(acc.umax2, c.u2);
    acc.bad |= c.bad;
}

// The block's partial from the accumulators of diag_row.  FP32: lane 0 of
// each warp holds the warp's sums; the warps meet in shared memory and thread
// 0 adds them in warp order.  FP64: the thread sums go through diag_partial.
__device__ __forceinline__ void diag_partial_rows(const CellSums<float> &acc, double *dpart, size_t bid,
                                                  double *shv) {
    const unsigned full = 0xffffffffu;
    // non-negative floats compare as their bit patterns
    const unsigned um = __reduce_max_sync(full, __float_as_uint(acc.umax2));
    const int wbad = __any_sync(full, acc.bad) ? 1 : 0;
    long long *sh = reinterpret_cast<long long *>(shv);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[4 * warp + 0] = acc.sfl;
        sh[4 * warp + 1] = acc.sH;
        sh[4 * warp + 2] = (long long)um;
        sh[4 * warp + 3] = wbad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long v[4] = {0, 0, 0, 0};
        const int nwarps = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nwarps; ++w) {
            v[0] += sh[4 * w + 0];
            v[1] += sh[4 * w + 1];
            v[2] = max(v[2], sh[4 * w + 2]);
            v[3] = max(v[3], sh[4 * w + 3]);
        }
        long long *d = reinterpret_cast<long long *>(dpart) + 4 * bid;
        d[0] = v[0];
        d[1] = v[1];
        d[2] = enc_max(sqrtf(__uint_as_float((unsigned)v[2])));
        d[3] = v[3];
    }
}
__device__ __forceinline__ void diag_partial_rows(const CellSums<double> &acc, double *dpart, size_t bid,
                                                  double *sh) {
    diag_partial<double>(acc.sfl, acc.sH, acc.umax2, acc.bad, dpart, bid, sh);
}

// Where a cell's post-collision population of direction i goes: cell(i) is
// the target cell's element of plane 0, slot(i) the direction slot written
// there.  OwnDst: the cell's own slot i (the pull sweeps, and the local sweep
// of one-buffer streaming).  PushFast / PushAny: the push sweep of one-buffer
// streaming (Streaming in lbm_internal.h), slot opp(i) of cell x + c_i, or the
// cell's own slot i where x + c_i lies beyond a wall.  PushFast serves cells
// whose eight neighbours all lie inside the lattice: its targets are the
// base pointers of pull_fast (b, and bL / bR shifted into the neighbouring
// tile at the tile's first / last column) plus compile-time offsets.
template <typename S>
struct OwnDst {
    typename Store<S>::elem *d;
    __device__ __forceinline__ typename Store<S>::elem *cell(int) const { return d; }
    __device__ __forceinline__ int slot(int i) const { return i; }
};
template <typename S>
struct PushFast {
    typename Store<S>::elem *b, *bL, *bR;
    __device__ __forceinline__ typename Store<S>::elem *cell(int i) const {
        const int cx = cx_of(i), cy = cy_of(i);
        return (cx > 0 ? bR : (cx < 0 ? bL : b)) + cy * kRS + cx * col_step<S>();
    }
    __device__ __forceinline__ int slot(int i) const { return opp_of(i); }
};
// A cavity side-wall warp on an interior row (see pull_sidewall): PushFast's
// targets, except that a direction leaving through the side wall goes to the
// cell's own slot i.
template <typename S>
struct PushSide {
    typename Store<S>::elem *b, *bL, *bR;
    int x, nx;
    __device__ __forceinline__ bool wall(int i) const {
        const int cx = cx_of(i);
        return (cx > 0 && x == nx - 1) || (cx < 0 && x == 0);
    }
    __device__ __forceinline__ typename Store<S>::elem *cell(int i) const {
        const int cx = cx_of(i), cy = cy_of(i);
        return wall(i) ? b : (cx > 0 ? bR : (cx < 0 ? bL : b)) + cy * kRS + cx * col_step<S>();
    }
    __device__ __forceinline__ int slot(int i) const { return wall(i) ? i : opp_of(i); }
};
template <typename S, int PROB>
struct PushAny {
    typename Store<S>::elem *buf;  // the buffer's first element
    int x, y, nx, ny;
    __device__ __forceinline__ bool inside(int i, int &tx, int &ty) const {
        tx = x + cx_of(i);
        ty = y + cy_of(i);
        if (PROB == kStefan) ty = (ty < 0) ? ty + ny : ((ty >= ny) ? ty - ny : ty);  // periodic in y
        return (unsigned)tx < (unsigned)nx && (unsigned)ty < (unsigned)ny;
    }
    __device__ __forceinline__ typename Store<S>::elem *cell(int i) const {
        int tx, ty;
        return buf + (inside(i, tx, ty) ? cell_index<S>(tx, ty, 0, ny) : cell_index<S>(x, y, 0, ny));
    }
    __device__ __forceinline__ int slot(int i) const {
        int tx, ty;
        return inside(i, tx, ty) ? opp_of(i) : i;
    }
};

// Collide the streamed populations of cell (x, y) and store them where dst
// says (MODE == kFields: write the fields instead).
template <typename real, typename S, bool FLOW, int MODE, typename Dst>
__device__ __forceinline__ void finish_cell(const SweepArgs<real> &a, int x, int y, const Dst &dst, real f[9],
                                            real g[9], uint32_t step_seed, CellDiag<real> &cd) {
    using E = typename Store<S>::elem;
    if (MODE == kFields) {
        const Macro<real> m = cell_update<real, S, FLOW, false>(a, f, g);
        const long long o = (long long)y * a.nx + x;
        if (a.oH) a.oH[o] = (double)m.H;
        if (a.oT) a.oT[o] = (double)m.T;
        if (a.oFL) a.oFL[o] = (double)m.fl;
        if (a.oUX) a.oUX[o] = (double)m.ux;
        if (a.oUY) a.oUY[o] = (double)m.uy;
        if (a.oRHO) a.oRHO[o] = (double)m.rho;
        return;
    }
    const Macro<real> m = cell_update<real, S, FLOW, true>(a, f, g);
    if constexpr (Store<S>::kDev) {
        // paired layout: one 32-bit (g_i, f_i) word per direction; without
        // flow only the g halves are written
        if (!Store<S>::kSR || (!FLOW && !(isfinite(m.H) && isfinite(m.rho)))) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                E *d = dst.cell(i);
                const int s = dst.slot(i);
                if (FLOW) reinterpret_cast<uint32_t *>(d)[s * kTW] = Store<S>::pack_rn(g[i], f[i]);
                else Store<S>::str_rn(d + 2 * s * kTW + 1, g[i]);
            }
        } else {
            uint32_t rs = hash32(step_seed ^ (uint32_t)((long long)y * a.nx + x));
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                E *d = dst.cell(i);
                const int s = dst.slot(i);
                if (FLOW) reinterpret_cast<uint32_t *>(d)[s * kTW] = Store<S>::pack_sr(g[i], f[i], lcg_next32(rs));
                else Store<S>::strs(d + 2 * s * kTW + 1, g[i], lcg_next(rs));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            E *d = dst.cell(i);
            const int s = dst.slot(i);
            Store<S>::str_rn(d + (9 + s) * kTW, g[i]);
            if (FLOW) Store<S>::str_rn(d + s * kTW, f[i]);
        }
    }
    if (MODE == kSweepDiag) {
        cd.fl = m.fl;
        cd.H = m.H;
        cd.u2 = m.ux * m.ux + m.uy * m.uy;
        cd.bad = !(isfinite(m.H) && isfinite(m.rho));
    }
}

// A block's end: the heated-wall inflow of this step (blocks touching the T_h
// wall: the cavity's bottom row band, the Stefan problem's first tile column),
// folded by the last such block to take a ticket, and the diagnostics
// partials.  bx, by: the block's tile column and row band; gx: tile columns.
template <typename real, int PROB, int MODE>
__device__ __forceinline__ void block_epilogue(const SweepArgs<real> &a, int bx, int by, int gx,
                                               const CellSums<real> &acc, double *sh) {
    if (MODE == kFields) return;
    const bool qblock = (PROB == kCavity) ? (a.strip_on && by == 0) : (bx == 0);
    if (qblock) {
        const int kind[1] = {0};
        double v[1] = {warp_sum(acc.q)};
        block_fold<1>(v, kind, sh);
        __shared__ bool qlast;
        if (threadIdx.x == 0) {
            const int slot = (PROB == kCavity) ? bx : by;
            a.qpart[slot] = v[0];
            __threadfence();
            qlast = atomicAdd(a.qcount, 1u) == (unsigned)a.nq - 1u;
        }
        __syncthreads();
        if (qlast) {
            __threadfence();
            double s = 0.0;
            for (int k = threadIdx.x; k < a.nq; k += blockDim.x) s += __ldcg(a.qpart + k);
            v[0] = warp_sum(s);
            block_fold<1>(v, kind, sh);
            if (threadIdx.x == 0) {
                a.rec->Q_last = v[0];
                a.rec->Q_cum += v[0];
                *a.qcount = 0u;
                if (a.hist) {  // this step's inflow; the melt fraction comes with diagnostics
                    const long long st = (long long)__ldcg(&a.rec->counter);  // integer load
                    double *e = a.hist + 4 * (st % a.hist_cap);
                    e[0] = (double)st;
                    e[1] = v[0];
                    e[2] = __longlong_as_double(0x7ff8000000000000ll);
                }
            }
        }
    }
    // ---- diagnostics: sums within the warp in the working precision (32
    // threads x their cells), then FP64 across warps and blocks ----
    if (MODE == kSweepDiag) diag_partial_rows(acc, a.dpart, (size_t)bx + (size_t)by * gx, sh);
}

// Row-block order of a sweep: the row band a block of launch position k (of
// gy bands) works on.  Successive steps visit the interior bands in opposite
// directions (rev = 1: descending; the source buffer's parity alternates with
// the step), so that a step starts on the rows the previous step wrote last,
// which are still in L2: the populations of a large lattice exceed L2, and a
// sweep in a fixed direction would start on rows long evicted.  The
// two wall bands (boundary pulls; the bottom one also folds the heated-wall
// inflow in the cavity) go first in both directions, so that they do not form
// the launch's tail.  A permutation of 0 .. gy - 1 for either direction.
__device__ __forceinline__ int row_band(const int k, const int gy, const int rev) {
    if (k == 0 || gy < 3) return k;
    if (k == 1) return gy - 1;
    return rev ? gy - k : k - 1;
}

// One block's work: the tile column bx (kTW cells) and the row band by
// (a.rows rows) of the lattice described by a; gx is the number of tile
// columns (for the block's partial-sum slot).  Called by lattice_kernel (one
// lattice, bx = blockIdx.x) and batch_kernel (a block of a batch of lattices).
// SM: kPull, or one of the two sweeps of one-buffer streaming (kAAPush,
// kAALocal; a.src == a.dst).
template <typename real, typename S, int PROB, bool FLOW, int MODE, int SM = kPull>
__device__ __forceinline__ void sweep_block(const SweepArgs<real> &a, const int bx, const int by,
                                            const int gx, double *sh) {
    using E = typename Store<S>::elem;
    const E *src = static_cast<const E *>(a.src);
    const int lx = threadIdx.x;
    const int x = bx * kTW + lx;
    const int y0 = by * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    // Blocks are scheduled roughly in launch order, so the rows `prefetch`
    // rows ahead in the sweep's direction (row_band) belong to a block that
    // starts a little later: fetching them into L2 now shortens that block's
    // load latency.  One bulk prefetch per row of the block, each from its own
    // thread.
    if (a.prefetch > 0 && (int)threadIdx.x < y1 - y0) {
        const int yp = (a.parity ? y0 - a.prefetch : y0 + a.prefetch) + (int)threadIdx.x;
        if (yp >= 0 && yp < a.ny) prefetch_tile_row_l2(src + cell_index<S>(bx * kTW, yp, 0, a.ny));
    }
    const uint32_t step_seed = step_prologue<real, S, MODE>(a, bx, by);
    const bool active = x < a.nx;
    // the warp's 32 columns are clear of both side walls (warp-uniform)
    const int xw = bx * kTW + (lx & ~31);
    const bool fastcol = xw >= 1 && xw + 31 <= a.nx - 2;
    // A cavity warp that touches a side wall also takes the fast loads on the
    // interior rows: the wall lane's out-of-lattice neighbour pointer is
    // clamped to its own cell (the loads then stay inside its tile row) and
    // its wall directions are replaced by bounce-back afterwards.
    const bool sidewall = PROB == kCavity && !fastcol;

    long long i0 = cell_index<S>(x, y0, 0, a.ny), iL = i0, iR = i0;
    if (fastcol || sidewall) {
        constexpr int cs = col_step<S>();
        iL = (lx == 0 && x > 0) ? cell_index<S>(x - 1, y0, 0, a.ny) + cs : i0;
        iR = (lx == kTW - 1 && x < a.nx - 1) ? cell_index<S>(x + 1, y0, 0, a.ny) - cs : i0;
    }

    E *const dst = static_cast<E *>(a.dst);
    CellSums<real> acc;
    for (int y = y0; y < y1; ++y, i0 += kRS, iL += kRS, iR += kRS) {
        CellDiag<real> cd;
        if (active) {
            real f[9], g[9];
            const bool inner = y >= 1 && y <= a.ny - 2;
            if (SM == kAALocal) {
                pull_local<real, S, FLOW>(src + i0, f, g);
                if (x == 0 || x == a.nx - 1 || (PROB == kCavity && (y == 0 || y == a.ny - 1)))
                    wall_rules_local<real, S, PROB, FLOW>(a, x, y, g, acc.q);
            } else if ((fastcol || (SM == kPull && sidewall)) && inner) {
                // (a side-wall warp's clamped loads read other cells' slots,
                // which the push sweep may be rewriting: it pulls those warps
                // with pull_sidewall, which reads only what its cells write)
                pull_fast<real, S, FLOW>(src + i0, src + iL, src + iR, f, g);
                if (SM == kPull && sidewall) bounce_side_walls<real, S, FLOW>(src + i0, x, a.nx, f, g);
            } else if (SM == kAAPush && sidewall && inner) {
                pull_sidewall<real, S, FLOW>(src + i0, src + iL, src + iR, x, a.nx, f, g);
            } else {
                pull_any<real, S, PROB, FLOW>(a, x, y, f, g, acc.q);
            }
            if (SM == kAAPush) {
                if (fastcol && inner)
                    finish_cell<real, S, FLOW, MODE>(a, x, y, PushFast<S>{dst + i0, dst + iL, dst + iR}, f, g,
                                                     step_seed, cd);
                else if (sidewall && inner)
                    finish_cell<real, S, FLOW, MODE>(a, x, y, PushSide<S>{dst + i0, dst + iL, dst + iR, x, a.nx},
                                                     f, g, step_seed, cd);
                else
                    finish_cell<real, S, FLOW, MODE>(a, x, y, PushAny<S, PROB>{dst, x, y, a.nx, a.ny}, f, g,
                                                     step_seed, cd);
            } else {
                finish_cell<real, S, FLOW, MODE>(a, x, y, OwnDst<S>{dst + i0}, f, g, step_seed, cd);
            }
        }
        if (MODE == kSweepDiag) diag_row(acc, cd);  // the whole warp, active or not
    }
    block_epilogue<real, PROB, MODE>(a, bx, by, gx, acc, sh);
}

// FP32 arithmetic: at least 8 blocks of 128 threads per SM (registers capped at
// 64, the occupancy the memory pipeline needs); FP64 is ALU-bound and keeps its
// registers.
template <typename real, typename S, int PROB, bool FLOW, int MODE, int SM = kPull>
__global__ void __launch_bounds__(kTW, sizeof(real) == 4 ? 1024 / kTW : 1)
    lattice_kernel(const SweepArgs<real> a) {
    __shared__ double sh[32 * 4];
    pdl_launch_dependents();
    pdl_wait();  // the previous sweep's populations, tickets and record
    sweep_block<real, S, PROB, FLOW, MODE, SM>(a, blockIdx.x,
                                               row_band((int)blockIdx.y, (int)gridDim.y, a.parity), gridDim.x,
                                               sh);
}

// ---- the staged sweep (16-bit storage) ----
// A block owns a band of consecutive rows of one tile column and streams the
// tile rows it needs through a ring of kStSlots shared-memory slots, filled by
// TMA bulk copies (cp.async.bulk, completion counted on one mbarrier per
// slot) two rows ahead of the row being computed, so that the loads are in
// flight while the block collides -- without holding registers.  A staged row
// keeps, per direction, 4 words of the left neighbour tile, the tile's 128
// words and 4 words of the right neighbour tile (each piece a 16-byte-aligned
// bulk copy), so every lane reads its pull sources from shared memory at
// uniform offsets.  Bands alternate direction (even bands top-down in y, odd
// bottom-up), so that two bands reach the rows they share at the same time
// and the second read of a halo row comes from L2.  Every wait is bounded:
// when one runs out, the block records a timeout in the diagnostics record,
// waits (bounded) for its copies still in flight and returns.
constexpr int kStW = kTW + 8;        // words per direction in a staged row
constexpr int kStRow = 9 * kStW;     // words per staged row
constexpr int kStSlots = 5;          // ring depth: rows p, p + 1, p + 2 in use, 2 in flight
constexpr size_t kStSmem = (size_t)kStSlots * kStRow * 4 + (kStSlots + 1) * 8;
constexpr long long kStDrainLimit = 1ll << 22;  // tries per in-flight copy after a timeout

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity, trying at most limit + 1 times.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit) {
    for (long long it = 0; it <= limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Global -> shared bulk copy; bytes and both addresses multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Staged row s of a band (y = ys0 + s dir) into slot s % kStSlots, issued by
// warp 0.  Rows outside the cavity are not loaded (walls); their slot's phase
// is completed by a plain arrival, so that every slot's phases keep counting
// one per staged row.
template <typename S, int PROB>
__device__ __forceinline__ void stage_row(const void *srcv, int nx, int ny, int ntx, int bx, int ys0, int dir,
                                          int s, uint32_t *rows, uint64_t *bar) {
    const int lane = threadIdx.x & 31;
    const int slot = s % kStSlots;
    int y = ys0 + s * dir;
    if (PROB == kStefan) y = (y % ny + ny) % ny;
    if ((unsigned)y >= (unsigned)ny) {
        if (lane == 0) mbar_arrive(bar + slot);
        return;
    }
    const bool left = bx > 0, right = bx < ntx - 1;
    if (lane == 0) {
        // the slot was last read before the block barrier that preceded this
        // call; order those reads before the asynchronous writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar + slot, 9u * 512u + (left ? 9u * 16u : 0u) + (right ? 9u * 16u : 0u));
    }
    __syncwarp();
    const uint32_t *src = static_cast<const uint32_t *>(srcv);
    constexpr long long kRowWords = kRS / 2;
    uint32_t *dst = rows + (size_t)slot * kStRow;
    (void)nx;
    if (lane < 9) {
        bulk_g2s(dst + lane * kStW + 4, src + ((long long)bx * ny + y) * kRowWords + lane * kTW, 512u, bar + slot);
    } else if (lane < 18) {
        const int i = lane - 9;
        if (left)
            bulk_g2s(dst + i * kStW, src + ((long long)(bx - 1) * ny + y) * kRowWords + i * kTW + (kTW - 4), 16u,
                     bar + slot);
    } else if (lane < 27) {
        const int i = lane - 18;
        if (right)
            bulk_g2s(dst + i * kStW + 4 + kTW, src + ((long long)(bx + 1) * ny + y) * kRowWords + i * kTW, 16u,
                     bar + slot);
    }
}

// Pull of cell (x, y) from three staged rows (lattice rows y - 1, y, y + 1),
// column c = 4 + lx within each direction's words; wall rules as pull_any.
template <typename real, typename S, int PROB, bool FLOW>
__device__ __forceinline__ void pull_staged(const SweepArgs<real> &a, const uint32_t *rm, const uint32_t *rc,
                                            const uint32_t *rp, int c, int x, int y, bool interior,
                                            real f[9], real g[9], double &q) {
    uint32_t u[9];
    if (interior) {  // no wall in reach (side-wall lanes are bounced afterwards)
        u[0] = rc[0 * kStW + c];
        u[1] = rc[1 * kStW + c - 1];
        u[2] = rm[2 * kStW + c];
        u[3] = rc[3 * kStW + c + 1];
        u[4] = rp[4 * kStW + c];
        u[5] = rm[5 * kStW + c - 1];
        u[6] = rm[6 * kStW + c + 1];
        u[7] = rp[7 * kStW + c + 1];
        u[8] = rp[8 * kStW + c - 1];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (FLOW) f[i] = Store<S>::lo(u[i]);
            g[i] = Store<S>::hi(u[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        const int sx = x - cx;
        int sy = y - cy;
        if (PROB == kStefan) sy = (sy < 0) ? sy + a.ny : ((sy >= a.ny) ? sy - a.ny : sy);
        const bool in = (unsigned)sx < (unsigned)a.nx && (unsigned)sy < (unsigned)a.ny;
        const uint32_t *r = cy > 0 ? rm : (cy < 0 ? rp : rc);
        const uint32_t w = in ? r[i * kStW + c - cx] : rc[opp_of(i) * kStW + c];
        if (FLOW) f[i] = Store<S>::lo(w);
        real gv = Store<S>::hi(w);
        if (!in) {
            bool heated;
            if (PROB == kStefan) {
                heated = sx < 0;
            } else {
                const int xc2 = 2 * x + 1 - cx;
                heated = a.strip_on && sy < 0 && xc2 >= a.lo2 && xc2 <= a.hi2;
            }
            if (heated) {
                const real wt = real(2) * w_of<real>(i) * real(Store<S>::kG);
                q += (double)((wt - real(2) * gv) * (real(1) / real(Store<S>::kG)));
                gv = wt - gv;
            }
        }
        g[i] = gv;
    }
}

template <typename real, typename S, int PROB, bool FLOW, int MODE>
__global__ void __launch_bounds__(kTW, sizeof(real) == 4 ? 1024 / kTW : 1)
    staged_kernel(const SweepArgs<real> a) {
    static_assert(Store<S>::kDev, "the staged sweep reads the paired 16-bit layout");
    extern __shared__ __align__(16) unsigned char st_smem[];
    __shared__ double sh[32 * 4];
    __shared__ int ok_sh;
    uint32_t *rows = reinterpret_cast<uint32_t *>(st_smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(st_smem + (size_t)kStSlots * kStRow * 4);  // + 1 spare
    pdl_launch_dependents();
    const int lx = threadIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = blockIdx.x, band = blockIdx.y, nbands = gridDim.y;
    const int y0 = (int)((long long)band * a.ny / nbands);
    const int y1 = (int)((long long)(band + 1) * a.ny / nbands);
    const int nb = y1 - y0;
    const int dir = (band & 1) ? -1 : 1;
    const int ys0 = (dir > 0 ? y0 : y1 - 1) - dir;  // staged row s: y = ys0 + s dir
    if (threadIdx.x == 0) {
        for (int k = 0; k <= kStSlots; ++k) mbar_init(bar + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();  // the previous step's populations
    const uint32_t step_seed = step_prologue<real, S, MODE>(a, bx, band);
    const int x = bx * kTW + lx;
    const bool active = x < a.nx;
    const int xw = bx * kTW + (lx & ~31);
    const bool fastcol = xw >= 1 && xw + 31 <= a.nx - 2;
    const int c = 4 + lx;

    int issued = -1;  // last staged row issued (warp 0 keeps it)
    if (warp == 0) {
        const int n0 = min(kStSlots, nb + 2);
        for (int s = 0; s < n0; ++s) stage_row<S, PROB>(a.src, a.nx, a.ny, a.ntx, bx, ys0, dir, s, rows, bar);
        issued = n0 - 1;
    }
    CellSums<real> acc;
    for (int p = 0; p < nb; ++p) {
        if (p > 0) __syncthreads();  // every thread is done with staged row p - 1
        if (warp == 0) {
            const int s_new = p - 1 + kStSlots;
            if (p > 0 && s_new <= nb + 1) {
                stage_row<S, PROB>(a.src, a.nx, a.ny, a.ntx, bx, ys0, dir, s_new, rows, bar);
                issued = s_new;
            }
            if (lane == 0) {
                bool ok = true;
                if (a.force_timeout && p == 0) ok = mbar_wait_bounded(bar + kStSlots, 0, a.wait_limit);
                for (int s = (p == 0 ? 0 : p + 2); s <= p + 2 && ok; ++s)
                    ok = mbar_wait_bounded(bar + s % kStSlots, (unsigned)(s / kStSlots) & 1u, a.wait_limit);
                ok_sh = ok ? 1 : 0;
            }
        }
        __syncthreads();
        if (!ok_sh) {
            // a wait ran out: record it, let the copies in flight land, return
            if (threadIdx.x == 0) {
                a.rec->timeout = 1.0;
                for (int s = (p == 0 ? 0 : p + 2); s <= issued; ++s)
                    mbar_wait_bounded(bar + s % kStSlots, (unsigned)(s / kStSlots) & 1u, kStDrainLimit);
            }
            __syncthreads();
            return;
        }
        // every thread observes the completed phases (immediate: thread 0 saw them)
        for (int s = (p == 0 ? 0 : p + 2); s <= p + 2; ++s)
            mbar_wait_bounded(bar + s % kStSlots, (unsigned)(s / kStSlots) & 1u, a.wait_limit);
        CellDiag<real> cd;
        if (!active) {
            if (MODE == kSweepDiag) diag_row(acc, cd);
            continue;
        }
        const int y = ys0 + (p + 1) * dir;
        // staged rows of lattice rows y - 1 and y + 1 (s = p + 1 -+ dir)
        const uint32_t *rc = rows + (size_t)((p + 1) % kStSlots) * kStRow;
        const uint32_t *rlo = rows + (size_t)((dir > 0 ? p : p + 2) % kStSlots) * kStRow;
        const uint32_t *rhi = rows + (size_t)((dir > 0 ? p + 2 : p) % kStSlots) * kStRow;
        const bool rowok = PROB == kStefan || (y >= 1 && y <= a.ny - 2);
        const bool wallfree = PROB == kCavity ? true : fastcol;  // Stefan: the left wall is heated
        real f[9], g[9];
        pull_staged<real, S, PROB, FLOW>(a, rlo, rc, rhi, c, x, y, rowok && wallfree, f, g, acc.q);
        if (PROB == kCavity && rowok && !fastcol) {
            // side-wall lanes: their wall directions bounce back (own cell)
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if ((cx_of(i) == 1 && x == 0) || (cx_of(i) == -1 && x == a.nx - 1)) {
                    const uint32_t w = rc[opp_of(i) * kStW + c];
                    if (FLOW) f[i] = Store<S>::lo(w);
                    g[i] = Store<S>::hi(w);
                }
            }
        }
        finish_cell<real, S, FLOW, MODE>(
            a, x, y, OwnDst<S>{static_cast<typename Store<S>::elem *>(a.dst) + cell_index<S>(x, y, 0, a.ny)}, f, g,
            step_seed, cd);
        if (MODE == kSweepDiag) diag_row(acc, cd);
    }
    block_epilogue<real, PROB, MODE>(a, bx, band, gridDim.x, acc, sh);
}

// ---- batches: many lattices of one precision and problem kind per launch ----
// Block b of a batch launch belongs to the entry r with starts[r] <= b <
// starts[r + 1]; within it, local block l = b - starts[r] is tile column
// l % gx, row band l / gx.  Each entry holds the lattice's arguments for both
// buffer parities; the launch for step j of a chunk uses parity
// parity[r] ^ (j & 1).  The block's start-up is two dependent reads: the
// search over the compact starts array (its first lines stay in L1 for the
// blocks an SM runs), then the whole entry, copied into shared memory 16 bytes
// per thread, alongside the parity word.  When every entry has the same number
// of blocks (`uniform`; a serving group's lattices share one size) the entry
// is blockIdx.x / uniform and the search and its barrier are skipped; with
// `interleave` set (uniform batches only) consecutive blocks belong to
// consecutive entries instead -- entry b mod n, local block b / n -- so that
// the blocks resident at one time spread over all the lattices.
__device__ __forceinline__ int batch_find(const int *starts, int n, int b) {
    int lo = 0, hi = n - 1;  // last entry with starts[r] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(starts + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// SM: kPull, or a sweep of one-buffer streaming (kAAPush at even j, kAALocal
// at odd j): the member's arguments for its buffer parity[r] are then used
// with the destination set to the source and the parity word to
// parity[r] ^ (j & 1), patched in the 16-byte pieces of the shared-memory
// copy that hold them, as they are copied.
template <typename real>
struct EntryLayout {
    static constexpr unsigned kArgs = sizeof(SweepArgs<real>);
    static constexpr unsigned kSrc = offsetof(SweepArgs<real>, src);
    static constexpr unsigned kDst = offsetof(SweepArgs<real>, dst);
    static constexpr unsigned kPar = offsetof(SweepArgs<real>, parity);
    static_assert(kArgs % 16 == 0 && kSrc % 16 == 0 && kDst == kSrc + 8,
                  "src and dst of each argument set share one 16-byte piece");
    static_assert(offsetof(BatchEntry<real>, a) == 0, "the argument sets open the entry");
};
template <typename real, typename S, int PROB, bool FLOW, int MODE, int SM = kPull>
__global__ void __launch_bounds__(kTW, sizeof(real) == 4 ? 1024 / kTW : 1)
    batch_kernel(const BatchEntry<real> *entries, const int *starts, const int *parity, int n,
                 int uniform, int interleave, int j) {
    static_assert(sizeof(BatchEntry<real>) % 16 == 0, "entries are copied in 16-byte pieces");
    using L = EntryLayout<real>;
    __shared__ double sh[32 * 4];
    __shared__ __align__(16) unsigned char entry_sh[sizeof(BatchEntry<real>)];
    __shared__ int meta[2];
    pdl_launch_dependents();
    // The table and the parity words are written only by copies the host
    // orders before the batch's launches, never by a kernel: the block reads
    // its entry while the previous step may still be running, and waits for
    // that step only before touching the populations.
    int r;
    if (uniform > 0) {
        r = interleave ? (int)(blockIdx.x % (unsigned)n) : (int)(blockIdx.x / (unsigned)uniform);
    } else {
        if (threadIdx.x == 0) meta[0] = batch_find(starts, n, blockIdx.x);
        __syncthreads();
        r = meta[0];
    }
    // every thread reads the parity word (one broadcast load, issued with the
    // copy's loads), so the pieces are patched on the way and one barrier
    // publishes the copy
    const int p = __ldg(parity + r) ^ (SM == kPull ? (j & 1) : 0);
    const int4 *s4 = reinterpret_cast<const int4 *>(entries + r);
    int4 *d4 = reinterpret_cast<int4 *>(entry_sh);
    for (unsigned k = threadIdx.x; k < sizeof(BatchEntry<real>) / 16; k += blockDim.x) {
        int4 v = __ldg(s4 + k);
        if constexpr (SM != kPull) {
            const unsigned base = (unsigned)p * L::kArgs;  // a[p] within the entry
            if (k == (base + L::kSrc) / 16) {
                v.z = v.x;  // dst = src (the same 8 bytes)
                v.w = v.y;
            }
            if (k == (base + L::kPar) / 16) {
                const int par = p ^ (j & 1);
                switch ((L::kPar % 16) / 4) {
                    case 0: v.x = par; break;
                    case 1: v.y = par; break;
                    case 2: v.z = par; break;
                    default: v.w = par; break;
                }
            }
        }
        d4[k] = v;
    }
    if (threadIdx.x == 0) meta[1] = p;  // read back after the barrier: no register held across it
    __syncthreads();
    pdl_wait();
    const BatchEntry<real> &e = *reinterpret_cast<const BatchEntry<real> *>(entry_sh);
    const SweepArgs<real> &a = e.a[meta[1]];
    const int l = (uniform > 0 && interleave) ? (int)(blockIdx.x / (unsigned)n) : (int)blockIdx.x - e.start;
    sweep_block<real, S, PROB, FLOW, MODE, SM>(a, l % e.gx, row_band(l / e.gx, e.gy, a.parity), e.gx, sh);
}

// Per-entry diagnostics fold after a diagnostic batch step: block r folds the
// gx * gy partials of entry r (thread t: partials t, t + T, ... in order, then
// a fixed tree) into that lattice's record.
template <typename real, typename A>
__global__ void __launch_bounds__(kReduceThreads)
    batch_diag_reduce_kernel(const BatchEntry<real> *entries) {
    __shared__ double sh[32 * 4];
    const int kind[4] = {0, 0, 1, 1};
    pdl_launch_dependents();
    pdl_wait();  // the batch step's partials
    const BatchEntry<real> &e = entries[blockIdx.x];
    const SweepArgs<real> &a = e.a[0];
    const unsigned nblk = (unsigned)e.gx * (unsigned)e.gy;
    A acc[4] = {A(0), A(0), A(0), A(0)};
    const A *part = reinterpret_cast<const A *>(a.dpart);
    for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x) {
        acc[0] += part[4 * (size_t)b + 0];
        acc[1] += part[4 * (size_t)b + 1];
        acc[2] = max(acc[2], part[4 * (size_t)b + 2]);
        acc[3] = max(acc[3], part[4 * (size_t)b + 3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = kind[k] ? warp_max(acc[k]) : warp_sum(acc[k]);
    block_fold<4, A>(acc, kind, sh);
    if (threadIdx.x == 0) {
        DevRecord *rec = a.rec;
        rec->step = (double)rec->counter;
        rec->melt_sum = dec_sum(acc[0]);
        rec->H_sum = dec_sum(acc[1]);
        rec->max_u = dec_max(acc[2]);
        rec->nan_flag = acc[3] != A(0) ? 1.0 : 0.0;
        rec->valid = 1.0;
        if (a.hist) hist_put(a.hist, a.hist_cap, rec, (double)a.nx * (double)a.ny);
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
template <typename real, typename S>
__global__ void __launch_bounds__(kTW) init_kernel(const SweepArgs<real> a, double amp,
                                                   uint64_t seed) {
    using E = typename Store<S>::elem;
    E *dst = static_cast<E *>(a.dst);
    E *aux = static_cast<E *>(a.aux);
    __shared__ double sh[32 * 4];
    const int x = blockIdx.x * kTW + threadIdx.x;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    typename DiagAcc<real>::T sfl = 0, sH = 0;
    bool bad = false;
    if (x < a.nx) {
        for (int y = y0; y < y1; ++y) {
            const uint64_t cell = (uint64_t)y * (uint64_t)a.nx + (uint64_t)x;
            const double r = (double)(splitmix64(seed ^ cell) >> 11) * 0x1.0p-53;
            const real H = (real)(amp * (2.0 * r - 1.0));
            real T, fl;
            invert(H, a.Lh, a.inv_Lh, T, fl);
            // initial state: rounded to nearest
            Store<S>::stg_rn(dst + cell_index<S>(x, y, 9, a.ny), H - T + w_of<real>(0) * T);
#pragma unroll
            for (int i = 1; i < 9; ++i) Store<S>::stg_rn(dst + cell_index<S>(x, y, 9 + i, a.ny), w_of<real>(i) * T);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const real fi = w_of<real>(i) - f_ofs<real, S>(i);
                const long long c = cell_index<S>(x, y, i, a.ny);
                Store<S>::stf_rn(dst + c, fi);
                if (aux) Store<S>::stf_rn(aux + c, fi);
            }
            sfl += enc_sum(fl);
            sH += enc_sum(H);
            bad |= !isfinite(H);
        }
    }
    diag_partial<real>(sfl, sH, real(0), bad, a.dpart, blockIdx.x + (size_t)blockIdx.y * gridDim.x, sh);
}

// Fields of the step-0 state (no streaming; u = 0 by definition).
template <typename real, typename S, bool FLOW>
__global__ void __launch_bounds__(kTW) fields0_kernel(const SweepArgs<real> a) {
    const auto *src = static_cast<const typename Store<S>::elem *>(a.src);
    const int x = blockIdx.x * kTW + threadIdx.x;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    if (x >= a.nx) return;
    for (int y = y0; y < y1; ++y) {
        real g[9], H, rho = real(1);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Store<S>::ldg(src + cell_index<S>(x, y, 9 + i, a.ny));
        H = sum9(g);
        if (FLOW) {
            real f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = Store<S>::ldf(src + cell_index<S>(x, y, i, a.ny)) + f_ofs<real, S>(i);
            rho = sum9(f);
        }
        real T, fl;
        invert(H, a.Lh, a.inv_Lh, T, fl);
        const long long o = (long long)y * a.nx + x;
        if (a.oH) a.oH[o] = (double)H;
        if (a.oT) a.oT[o] = (double)T;
        if (a.oFL) a.oFL[o] = (double)fl;
        if (a.oUX) a.oUX[o] = 0.0;
        if (a.oUY) a.oUY[o] = 0.0;
        if (a.oRHO) a.oRHO[o] = (double)rho;
    }
}

// Tile-major <-> plane-major FP64 staging, one thread per cell.
template <typename S>
__global__ void repack_kernel(void *bufv, void *buf2v, double *stage, int nx, int ny,
                              bool to_staging) {
    using E = typename Store<S>::elem;
    using real = typename std::conditional<sizeof(E) == 8, double, float>::type;
    E *buf = static_cast<E *>(bufv), *buf2 = static_cast<E *>(buf2v);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const long long P = (long long)nx * ny, o = (long long)y * nx + x;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const bool isf = p < 9;
        const real ofs = isf ? f_ofs<real, S>(p) : real(0);
        const long long c = cell_index<S>(x, y, p, ny);
        E *q = buf + c;
        if (to_staging) {
            stage[p * P + o] = (double)((isf ? Store<S>::ldf(q) : Store<S>::ldg(q)) + ofs);
        } else {
            const real v = (real)stage[p * P + o] - ofs;
            // caller data: stochastic codecs round it to nearest as well
            if (isf) {
                Store<S>::stf_rn(q, v);
                if (buf2) Store<S>::stf_rn(buf2 + c, v);
            } else {
                Store<S>::stg_rn(q, v);
            }
        }
    }
}

// ---- launch dispatch (instantiated per storage type in sweep_*.cu) ----
// A launch, with the programmatic-serialization attribute when pdl is set.
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                            bool pdl, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename real, typename S, int PROB, bool FLOW>
static cudaError_t launch_mode(const SweepArgs<real> &a, int mode, dim3 grid, dim3 block,
                               cudaStream_t s, bool pdl, int streaming) {
    if (streaming == kAAPush || streaming == kAALocal) {  // one-buffer streaming: sweeps only
        if (a.src != a.dst || a.staged) return cudaErrorInvalidValue;
        const bool push = streaming == kAAPush;
        switch (mode) {
            case kSweep:
                return push ? launch_k(lattice_kernel<real, S, PROB, FLOW, kSweep, kAAPush>, grid, block, s, pdl, a)
                            : launch_k(lattice_kernel<real, S, PROB, FLOW, kSweep, kAALocal>, grid, block, s, pdl, a);
            case kSweepDiag:
                return push ? launch_k(lattice_kernel<real, S, PROB, FLOW, kSweepDiag, kAAPush>, grid, block, s, pdl,
                                       a)
                            : launch_k(lattice_kernel<real, S, PROB, FLOW, kSweepDiag, kAALocal>, grid, block, s,
                                       pdl, a);
            default: return cudaErrorInvalidValue;
        }
    }
    if (streaming != kPull) return cudaErrorInvalidValue;
    if constexpr (Store<S>::kDev) {
        if (a.staged && (mode == kSweep || mode == kSweepDiag)) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = block;
            cfg.dynamicSmemBytes = kStSmem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = pdl ? 1 : 0;
            return mode == kSweep ? cudaLaunchKernelEx(&cfg, staged_kernel<real, S, PROB, FLOW, kSweep>, a)
                                  : cudaLaunchKernelEx(&cfg, staged_kernel<real, S, PROB, FLOW, kSweepDiag>, a);
        }
    }
    switch (mode) {
        case kSweep: return launch_k(lattice_kernel<real, S, PROB, FLOW, kSweep>, grid, block, s, pdl, a);
        case kSweepDiag:
            return launch_k(lattice_kernel<real, S, PROB, FLOW, kSweepDiag>, grid, block, s, pdl, a);
        case kFields: lattice_kernel<real, S, PROB, FLOW, kFields><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The fold after a diagnostic sweep (or the init kernel); pdl as for the sweep.
template <typename real>
static cudaError_t launch_diag_reduce(const SweepArgs<real> &a, dim3 grid, bool init, cudaStream_t s,
                                      bool pdl) {
    const unsigned nblk = grid.x * grid.y;
    unsigned nred = (nblk + kReduceThreads - 1) / kReduceThreads;
    if (nred > (unsigned)kReduceThreads) nred = kReduceThreads;  // level 2 is one block's pass
    return launch_k(diag_reduce_kernel<typename DiagAcc<real>::T>, dim3(nred), dim3(kReduceThreads), s,
                    pdl, (const double *)a.dpart, nblk, a.dpart2, a.dticket, a.rec, init ? 1 : 0,
                    a.hist, a.hist_cap, (double)a.nx * (double)a.ny);
}

template <typename real, typename S>
cudaError_t launch_lattice(const SweepArgs<real> &a, int problem, bool flow, int mode,
                           dim3 grid, dim3 block, cudaStream_t s, bool pdl, int streaming) {
    cudaError_t e;
    if (problem == kCavity)
        e = flow ? launch_mode<real, S, kCavity, true>(a, mode, grid, block, s, pdl, streaming)
                 : launch_mode<real, S, kCavity, false>(a, mode, grid, block, s, pdl, streaming);
    else
        e = flow ? launch_mode<real, S, kStefan, true>(a, mode, grid, block, s, pdl, streaming)
                 : launch_mode<real, S, kStefan, false>(a, mode, grid, block, s, pdl, streaming);
    if (e == cudaSuccess && mode == kSweepDiag) e = launch_diag_reduce(a, grid, false, s, pdl);
    return e;
}

template <typename real, typename S>
cudaError_t launch_batch(const void *entries, const int *starts, const int *parity, int n,
                         int uniform, int interleave, int nblocks, int problem, bool flow, bool diag,
                         int j, cudaStream_t s, bool pdl, int streaming) {
    const BatchEntry<real> *e = static_cast<const BatchEntry<real> *>(entries);
    const dim3 grid(nblocks), block(kTW);
    cudaError_t err;
    if (streaming != kPull && streaming != kAAPush && streaming != kAALocal) return cudaErrorInvalidValue;
#define BTRIRT_BATCH_SM(PROB, FLOW, SM)                                                                \
    err = diag ? launch_k(batch_kernel<real, S, PROB, FLOW, kSweepDiag, SM>, grid, block, s, pdl, e, starts, \
                          parity, n, uniform, interleave, j)                                           \
               : launch_k(batch_kernel<real, S, PROB, FLOW, kSweep, SM>, grid, block, s, pdl, e, starts,  \
                          parity, n, uniform, interleave, j);
#define BTRIRT_BATCH(PROB, FLOW)                                                                   \
    if (streaming == kAAPush) {                                                                    \
        BTRIRT_BATCH_SM(PROB, FLOW, kAAPush)                                                       \
    } else if (streaming == kAALocal) {                                                            \
        BTRIRT_BATCH_SM(PROB, FLOW, kAALocal)                                                      \
    } else {                                                                                       \
        BTRIRT_BATCH_SM(PROB, FLOW, kPull)                                                         \
    }
    if (problem == kCavity) {
        if (flow) { BTRIRT_BATCH(kCavity, true) } else { BTRIRT_BATCH(kCavity, false) }
    } else {
        if (flow) { BTRIRT_BATCH(kStefan, true) } else { BTRIRT_BATCH(kStefan, false) }
    }
#undef BTRIRT_BATCH
#undef BTRIRT_BATCH_SM
    if (err == cudaSuccess && diag)
        err = launch_k(batch_diag_reduce_kernel<real, typename DiagAcc<real>::T>, dim3(n),
                       dim3(kReduceThreads), s, pdl, e);
    return err;
}

template <typename real, typename S>
cudaError_t launch_init(const SweepArgs<real> &a, double amp, uint64_t seed, dim3 grid,
                        dim3 block, cudaStream_t s) {
    init_kernel<real, S><<<grid, block, 0, s>>>(a, amp, seed);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_diag_reduce(a, grid, true, s, false);
    return e;
}

template <typename real, typename S>
cudaError_t launch_fields0(const SweepArgs<real> &a, bool flow, dim3 grid, dim3 block,
                           cudaStream_t s) {
    if (flow)
        fields0_kernel<real, S, true><<<grid, block, 0, s>>>(a);
    else
        fields0_kernel<real, S, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_repack(void *buf, void *buf2, double *stage, int nx, int ny, bool to_staging,
                          cudaStream_t s) {
    dim3 block(256), grid((nx + 255) / 256, ny);
    repack_kernel<S><<<grid, block, 0, s>>>(buf, buf2, stage, nx, ny, to_staging);
    return cudaGetLastError();
}

// Explicit instantiation of every launcher for one (compute, storage) pair.
#define BTRIRT_INSTANTIATE(REAL, S)                                                             \
    template cudaError_t launch_lattice<REAL, S>(const SweepArgs<REAL> &, int, bool, int, dim3,  \
                                                 dim3, cudaStream_t, bool, int);                 \
    template cudaError_t launch_init<REAL, S>(const SweepArgs<REAL> &, double, uint64_t, dim3,   \
                                              dim3, cudaStream_t);                               \
    template cudaError_t launch_fields0<REAL, S>(const SweepArgs<REAL> &, bool, dim3, dim3,      \
                                                 cudaStream_t);                                  \
    template cudaError_t launch_repack<S>(void *, void *, double *, int, int, bool, cudaStream_t); \
    template cudaError_t launch_batch<REAL, S>(const void *, const int *, const int *, int, int,  \
                                               int, int, int, bool, bool, int, cudaStream_t, bool, int);

}  // namespace btrirt

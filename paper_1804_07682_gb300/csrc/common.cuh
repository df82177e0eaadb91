// common.cuh -- device-side building blocks of the oscillation chain.
//
// Notation follows the paper's Sec. 4.1 formula for alpha = beta = e:
//   P = 1 - A21 sin^2 D21 - A31 sin^2 D31 - A32 sin^2 D32,
//   A_ij = 4 |U_ei|^2 |U_ej|^2,  D_ij = K dm2_ij L / E,  D31 = D21 + D32,
// with K = 1266.932679419849 rad MeV / (eV^2 km).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ff_consts.h"

#define GNA_NLMAX 16
#define GNA_MAX_ORDER 65536
// K = 10^3 / (4 hbar c), hbar c = 0.1973269804 GeV fm: dm2[eV^2] L[km] / (4 E) -> rad for E in MeV
#define GNA_K_PHASE 1266.932679419849

// Number of reduced values per (point, bin): combined prediction M, four
// tangents, then per-baseline integrals when requested.
#define GNA_NV_BASE 5

// Per-point constants prepared on the device from the gna_osc "variables"
// (step a0): oscillation amplitudes, their derivatives with respect to
// sin^2 theta12 and sin^2 theta13, and the phase constants K dm2 L_r both in
// double and split into a pair of floats (hi + lo).
struct PointConst {
    double c21[GNA_NLMAX];
    double c32[GNA_NLMAX];
    float c21h[GNA_NLMAX], c21l[GNA_NLMAX];
    float c32h[GNA_NLMAX], c32l[GNA_NLMAX];
    double A[3];     // A21, A31, A32
    double dA12[3];  // d A_ij / d sin^2 theta12
    double dA13[3];  // d A_ij / d sin^2 theta13
    float Af[3], dA12f[3], dA13f[3];
    float Alo[3];    // A - (double)Af: the amplitudes enter P as hi + lo
};

// Plan-wide constants passed by value.
struct BaseConst {
    float om[GNA_NLMAX];    // omega_r rounded to FP32
    float omlo[GNA_NLMAX];  // omega_r - om_r (FP32)
    float wkl[GNA_NLMAX];   // 2 omega_r K L_r: d sin^2 D / d dm2 = sin 2D K L / E
    double omd[GNA_NLMAX];  // omega_r (FP64)
    double kld[GNA_NLMAX];  // K L_r (FP64)
    float wsum;             // sum_r om_r rounded to FP32
    double wsum_lo;         // sum_r om_r - wsum (exact sum of the FP32 weights)
    int nL;
};

// ---------------------------------------------------------------- Kahan --
struct KahanF {
    float s, c;  // value = s - c
};

__device__ __forceinline__ void kzero(KahanF& k) {
    k.s = 0.f;
    k.c = 0.f;
}

// k += a * b with Kahan compensation (the product is fused into the first step).
__device__ __forceinline__ void kadd_prod(KahanF& k, float a, float b) {
    float y = __fmaf_rn(a, b, -k.c);
    float t = __fadd_rn(k.s, y);
    k.c = __fsub_rn(__fsub_rn(t, k.s), y);
    k.s = t;
}

// ---------------------------------------------------- double-float sums --
// Unevaluated sum hi + lo; error-free transformation of two floats (TwoSum).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float s = __fadd_rn(a.x, b.x);
    float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    float lo = __fadd_rn(__fadd_rn(a.y, b.y), e);
    float hi = __fadd_rn(s, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return make_float2(hi, lo);
}

__device__ __forceinline__ float2 kahan_to_ff(const KahanF& k) { return make_float2(k.s, -k.c); }

__device__ __forceinline__ float2 shfl_xor_f2(float2 v, int o) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    return v;
}

// Transposed warp reduction of NVP (power of two, <= 32) double-float values:
// at each level a lane keeps half of its values and adds the partner's copy of
// that half, so the work halves with every level.  Afterwards lane l holds the
// warp-wide sum of value index (l >> (5 - log2 NVP)) in v[0].
template <int NVP>
__device__ __forceinline__ void warp_transpose_reduce(float2 (&v)[NVP], int lane) {
    constexpr int LOG = (NVP >= 32) ? 5 : (NVP >= 16) ? 4 : (NVP >= 8) ? 3 : (NVP >= 4) ? 2 : (NVP >= 2) ? 1 : 0;
    static_assert((1 << LOG) == NVP, "NVP must be a power of two <= 32");
#pragma unroll
    for (int lvl = 0; lvl < 5; lvl++) {
        const int o = 16 >> lvl;
        const int cnt = NVP >> lvl;  // values still held (>= 1 after LOG levels)
        if (cnt > 1) {
            const int half = cnt / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < half; j++) {
                float2 send = upper ? v[j] : v[j + half];
                float2 keep = upper ? v[j + half] : v[j];
                v[j] = ff_add(keep, shfl_xor_f2(send, o));
            }
        } else {
            v[0] = ff_add(v[0], shfl_xor_f2(v[0], o));
        }
    }
}

// ----------------------------------------- phase reduction and sin / cos --
// sin r and cos r on |r| <= pi/2 (+ margin), FP32 polynomials (ff_consts.h).
// Horner tails S1 + u (S2 + ...) and C1 + u (C2 + ...); the generated
// header defines four or five coefficients of each.
__device__ __forceinline__ float sin_tail(float u) {
#if defined(GNA_SIN_C5)
    float ps = fmaf(GNA_SIN_C5, u, GNA_SIN_C4);
#else
    float ps = GNA_SIN_C4;
#endif
    ps = fmaf(ps, u, GNA_SIN_C3);
    ps = fmaf(ps, u, GNA_SIN_C2);
    return fmaf(ps, u, GNA_SIN_C1);
}

__device__ __forceinline__ float cos_tail(float u) {
#if defined(GNA_COS_C5)
    float pc = fmaf(GNA_COS_C5, u, GNA_COS_C4);
#else
    float pc = GNA_COS_C4;
#endif
    pc = fmaf(pc, u, GNA_COS_C3);
    pc = fmaf(pc, u, GNA_COS_C2);
    return fmaf(pc, u, GNA_COS_C1);
}

__device__ __forceinline__ void sincos_poly(float r, float& s, float& c) {
    float u = __fmul_rn(r, r);
    s = fmaf(__fmul_rn(r, u), sin_tail(u), r);
    c = fmaf(u, cos_tail(u), 1.0f);
}

__device__ __forceinline__ float sin_poly(float r) {
    float u = __fmul_rn(r, r);
    return fmaf(__fmul_rn(r, u), sin_tail(u), r);
}

// 1.5 * 2^23: adding it rounds a float of magnitude < 2^22 to an integer.
#define GNA_ROUND_MAGIC 12582912.0f

// Phase c * e with c = ch + cl and e = eh + el (double-float), reduced modulo
// pi: returns r with phase = q pi + r, |r| <= pi/2 (+ rounding), valid for
// phase < 2^12 pi.  The product hi part is exact through the FMA residual;
// q PI_A is exact (12-bit PI_A, integer q < 2^12) and the FMA with PI_B2
// rounds once; PI_A + PI_B2 misses pi by GNA_PI_E2 (5e-12), so the reduction
// adds at most q * 5e-12 (2e-8 rad at the largest phase) to the float
// rounding of r.
__device__ __forceinline__ float reduce_pi_ff(float ch, float cl, float eh, float el) {
    float p = __fmul_rn(ch, eh);
    float e = __fmaf_rn(ch, eh, -p);
    float lo = __fmaf_rn(ch, el, __fmaf_rn(cl, eh, e));
    float q = __fsub_rn(__fmaf_rn(p, GNA_INV_PI_F, GNA_ROUND_MAGIC), GNA_ROUND_MAGIC);
    float r = __fmaf_rn(-q, GNA_PI_A, p);
    r = __fmaf_rn(-q, GNA_PI_B2, r);
    return __fadd_rn(r, lo);
}

// The same reduction with the phase formed and reduced in double.
__device__ __forceinline__ float reduce_pi_f64(double c, double e) {
    double p = c * e;
    double q = rint(p * GNA_INV_PI_D);
    double r = fma(-q, GNA_PI_DA, p);
    r = fma(-q, GNA_PI_DB, r);
    r = fma(-q, GNA_PI_DC, r);
    return (float)r;
}

// Double reduction modulo pi returning a double remainder (FP64 mode).
__device__ __forceinline__ double reduce_pi_d(double p) {
    double q = rint(p * GNA_INV_PI_D);
    double r = fma(-q, GNA_PI_DA, p);
    r = fma(-q, GNA_PI_DB, r);
    return fma(-q, GNA_PI_DC, r);
}

// Split a double into hi + lo floats.
__host__ __device__ __forceinline__ void split_ff(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// 1 / E as a float pair without an FP64 division (FP64 runs at 1/64 of the
// FP32 rate here): r = rcp(E_hi), then one Newton-Raphson step carried in
// double-float, 1/E = r / (1 - e) = r (1 + e + e^2 ...), e = 1 - E r, whose
// leading part 1 - E_hi r the FMA forms exactly.  Relative error ~e^2 < 2^-44.
__device__ __forceinline__ void ff_recip(double E, float& rh, float& rl) {
    float eh, el;
    split_ff(E, eh, el);
    const float r = __frcp_rn(eh);
    const float e = fmaf(-el, r, fmaf(-eh, r, 1.0f));
    const float lo = r * e;
    rh = r + lo;
    rl = lo - (rh - r);
}

// lbm_device.cuh -- sm_103a kernels of the STG wall-modelled MRT-LES lattice
// Boltzmann channel step (Xue, Yao & Davidson, arXiv 2304.04214).
//
// Bandwidth-bound stencil: one thread per cell, pull streaming from the
// structure-of-arrays lattice f[q][k][j][i] (i fastest, warps along i so every
// load and store of a direction plane is coalesced), the 19x19 moment
// transform factorized into opposite-pair sums and differences and kept in
// registers.  No tensor cores: there is no dense contraction on this path.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace lbmk {

// ---------------------------------------------------------------------------
// D3Q19 in the velocity order of Sec. 2.1 (eq:vel-set).  q and 18-q are
// opposite; 9 is the rest velocity.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int CX(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 13 || q == 17) ? 1
         : (q == 1 || q == 5 || q == 8 || q == 11 || q == 15) ? -1 : 0;
}
__host__ __device__ constexpr int CY(int q) {
    return (q == 4 || q == 11 || q == 12 || q == 13 || q == 18) ? 1
         : (q == 0 || q == 5 || q == 6 || q == 7 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int CZ(int q) {
    return (q >= 14) ? 1 : (q <= 4) ? -1 : 0;
}
// weights (Sec. 2.1): 1/3 rest, 1/18 axis, 1/36 diagonal
__host__ __device__ constexpr float WQ(int q) {
    return q == 9 ? (1.0f / 3.0f)
         : (CX(q) * CX(q) + CY(q) * CY(q) + CZ(q) * CZ(q) == 1) ? (1.0f / 18.0f) : (1.0f / 36.0f);
}
// Relaxation rates that do not follow the viscosity (App. A.1 eq:freeparams):
constexpr float S_E = 1.19f;     // energy e (moment 1)
constexpr float S_EPS = 1.6f;    // energy square (moment 2)
constexpr float S_Q = 1.2f;      // heat fluxes (moments 4, 6, 8)
constexpr float S_PI = 1.6f;     // moments 10, 12
constexpr float S_M = 1.98f;     // moments 16, 17, 18

// ---------------------------------------------------------------------------
// Storage of one population.  FP32 storage holds f itself; FP16 holds the
// deviation f - w_q; BF16 (ROWBASE) holds the deviation from the equilibrium
// of its row's creation-time mean flow, f - f^eq_q(1, (U0(j), 0, 0)), which in
// a channel is about ten times smaller than f - w_q, so that BF16's 8
// significant bits round it ten times less coarsely in absolute terms.
// SHIFTED tells the collision that its registers hold f - w (the loads add
// the row base back, the stores take it off); the arithmetic is FP32 always.
// ---------------------------------------------------------------------------
// ld2 / st2 move two adjacent populations (even offset) in one access, ld4 /
// st4 four (offset a multiple of four).
struct StoreF32 {
    using T = float;
    static constexpr bool SHIFTED = false;
    static constexpr bool ROWBASE = false;
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
    static __device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    static __device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
};
struct StoreF16 {
    using T = __half;
    static constexpr bool SHIFTED = true;
    static constexpr bool ROWBASE = false;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float2 ld2(const __half *p) {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ void st2(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
    }
    static __device__ __forceinline__ float4 ld4(const __half *p) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        __half2 lo, hi;
        memcpy(&lo, &u.x, 4); memcpy(&hi, &u.y, 4);
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void st4(__half *p, float4 v) {
        const __half2 lo = __float22half2_rn(make_float2(v.x, v.y)), hi = __float22half2_rn(make_float2(v.z, v.w));
        uint2 u;
        memcpy(&u.x, &lo, 4); memcpy(&u.y, &hi, 4);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr bool SHIFTED = true;
    static constexpr bool ROWBASE = true;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
    }
    static __device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        __nv_bfloat162 lo, hi;
        memcpy(&lo, &u.x, 4); memcpy(&hi, &u.y, 4);
        const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void st4(__nv_bfloat16 *p, float4 v) {
        const __nv_bfloat162 lo = __float22bfloat162_rn(make_float2(v.x, v.y));
        const __nv_bfloat162 hi = __float22bfloat162_rn(make_float2(v.z, v.w));
        uint2 u;
        memcpy(&u.x, &lo, 4); memcpy(&u.y, &hi, 4);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

// FP16 words holding the row-base deviation (as StoreBF16 does in BF16).
struct StoreF16R : StoreF16 {
    static constexpr bool ROWBASE = true;
};

// Approximate reciprocal and square root (PTX rcp/sqrt.approx, about one ulp);
// the collision uses them where a rounding error of that size is harmless.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// Reichardt law, Sec. 2.3 eq:reichard with the textbook coefficients
// (1/kappa, kappa, B), and its derivative in y+.
// ---------------------------------------------------------------------------
// The law and its derivative together, with the fast exponential and
// logarithm (MUFU-based intrinsics): at the y+ of a first cell their relative
// errors (~1e-6 in e^{-y+/3}) enter u+ below 1e-7, under FP32 rounding of the
// Newton residual.  The two exponentials are shared by the law and its slope.
__device__ __forceinline__ void reichardt_fast(float yp, float kap, float B, float &up, float &dup) {
    const float e11 = __expf(yp * (-1.0f / 11.0f)), e3 = __expf(yp * (-1.0f / 3.0f));
    const float ky = fmaf(kap, yp, 1.0f);
    const float ik = rcp_approx(kap);
    up = __logf(ky) * ik + B * (1.0f - e11 - yp * (1.0f / 11.0f) * e3);
    dup = rcp_approx(ky) + B * ((e11 - e3) * (1.0f / 11.0f) + yp * (1.0f / 33.0f) * e3);
}
__device__ __forceinline__ double reichardt_d(double yp, double kap, double B) {
    return log1p(kap * yp) / kap + B * (1.0 - exp(-yp / 11.0) - yp / 11.0 * exp(-yp / 3.0));
}
__device__ __forceinline__ double reichardt_dy_d(double yp, double kap, double B) {
    const double e3 = exp(-yp / 3.0);
    return 1.0 / (1.0 + kap * yp) + B * (exp(-yp / 11.0) / 11.0 - e3 / 11.0 + yp / 33.0 * e3);
}

// Newton solve of eq:u_tau_implicit, u u+(y1 u / nu) = uhat, uhat > 0, warm
// started; FP32 first, FP64 if FP32 did not settle.  *ok = false if neither did.
// FP32 stops after a step |du| <= 2e-4 u: the error after a Newton step is
// about (u R''/2R') (du/u)^2 u, and u R''/2R' of this law lies between 0.06
// (log layer) and 0.5 (viscous sublayer), so the returned value is within
// 2e-8 u of the root -- below FP32 rounding.  From the previous step's u_tau
// that is usually one step.
__device__ __forceinline__ float solve_utau_dev(float uhat, float y1_nu, float kap, float B, float guess,
                                             bool *ok) {
    float u = guess > 0.0f ? guess : 1e-3f;
    for (int it = 0; it < 12; ++it) {
        const float yp = y1_nu * u;
        float up, dup;
        reichardt_fast(yp, kap, B, up, dup);
        const float r = u * up - uhat;
        const float dr = up + yp * dup;
        const float du = r * rcp_approx(dr);
        float un = u - du;
        if (!(un > 0.0f)) un = 0.5f * u;
        if (fabsf(du) <= 2e-4f * un) { *ok = true; return un; }
        u = un;
    }
    double ud = u;
    for (int it = 0; it < 40; ++it) {
        const double yp = (double)y1_nu * ud;
        const double up = reichardt_d(yp, kap, B);
        const double du = (ud * up - uhat) / (up + yp * reichardt_dy_d(yp, kap, B));
        double un = ud - du;
        if (!(un > 0.0)) un = 0.5 * ud;
        ud = un;
        if (fabs(du) <= 1e-12 * ud) { *ok = true; return (float)ud; }
    }
    *ok = false;
    return (float)ud;
}


// ---------------------------------------------------------------------------
// MRT collision with the Guo force in moment space (eq:lbe_mrt,
// eq:bodyforce; reading: F_force = M^-1 (I - S/2) M F~), Smagorinsky tau_eff
// (eq:tau_eff) on the viscous moments 9, 11, 13, 14, 15.
//
// f[] holds f (SHIFTED = false) or f - w (SHIFTED = true).  In: drho =
// rho - 1, momentum jx..jz (= sum f c), force density F (HAS_FORCE).  The
// update is f* = f - M^T g with g_k = (s_k (m_k - m_k^eq) - (1 - s_k/2)
// (M F~)_k) / |row_k|^2, evaluated with sums s_p = f_p + f_{18-p} and
// differences d_p = f_p - f_{18-p} of the nine opposite pairs; the rows of M
// are the d'Humieres moments.  M w = (1, -11, 3, 0, ..., 0) supplies the
// constant terms that differ between f and f - w.
// ---------------------------------------------------------------------------
struct Pairs {
    float s[9], d[9];      // s_p = f_p + f_{18-p}, d_p = f_p - f_{18-p}, p = 0..8
    float drho, jx, jy, jz;
};

// Pair sums and differences, density deviation and momentum (eq:density,
// eq:momentum without the force) from f (SHIFTED = false) or f - w.
template <bool SHIFTED>
__device__ __forceinline__ void make_pairs(const float (&f)[19], Pairs &P) {
#pragma unroll
    for (int p = 0; p < 9; ++p) { P.s[p] = f[p] + f[18 - p]; P.d[p] = f[p] - f[18 - p]; }
    const float *s = P.s, *d = P.d;
    P.drho = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + (s[8] + f[9])
           - (SHIFTED ? 0.0f : 1.0f);
    P.jx = (d[3] - d[1]) + (d[7] - d[5]) - d[8];
    P.jy = (d[4] - d[0]) - (d[5] + d[7]) - d[6];
    P.jz = -(d[0] + d[4]) - (d[1] + d[3]) - d[2];
}

template <bool SHIFTED, bool HAS_FORCE>
__device__ __forceinline__ void collide_mrt(float (&f)[19], const Pairs &P, float Fx, float Fy, float Fz,
                                            float tau0, float csm18, float &ux_o, float &uy_o, float &uz_o) {
    const float s0 = P.s[0], d0 = P.d[0], s1 = P.s[1], d1 = P.d[1], s2 = P.s[2], d2 = P.d[2];
    const float s3 = P.s[3], d3 = P.d[3], s4 = P.s[4], d4 = P.d[4], s5 = P.s[5], d5 = P.d[5];
    const float s6 = P.s[6], d6 = P.d[6], s7 = P.s[7], d7 = P.d[7], s8 = P.s[8], d8 = P.d[8];
    const float f9 = f[9];
    const float drho = P.drho, jx = P.jx, jy = P.jy, jz = P.jz;

    const float rho = 1.0f + drho;
    const float irho = rcp_approx(rho);
    // eq:momentum: rho u = sum f c + F/2
    const float rux = HAS_FORCE ? jx + 0.5f * Fx : jx;
    const float ruy = HAS_FORCE ? jy + 0.5f * Fy : jy;
    const float ruz = HAS_FORCE ? jz + 0.5f * Fz : jz;
    const float ux = rux * irho, uy = ruy * irho, uz = ruz * irho;
    ux_o = ux; uy_o = uy; uz_o = uz;
    const float uxx = rux * ux, uyy = ruy * uy, uzz = ruz * uz;       // rho u_a u_a
    const float uxy = rux * uy, uyz = ruy * uz, uxz = rux * uz;
    const float usq = uxx + uyy + uzz;

    // non-equilibrium moments n_k = m_k - m_k^eq
    const float Sax = s2 + s6 + s8;
    const float Sdg = (s0 + s4) + (s1 + s3) + (s5 + s7);
    const float e1 = -30.0f * f9 - 11.0f * Sax + 8.0f * Sdg;    // M_1 f
    const float e2 = 12.0f * f9 - 4.0f * Sax + Sdg;             // M_2 f
    // m1^eq = -11 rho + 19 rho u^2, m2^eq = 3 rho - 11/2 rho u^2 (= M f^eq)
    const float n1 = SHIFTED ? e1 + 11.0f * drho - 19.0f * usq : e1 + 11.0f * rho - 19.0f * usq;
    const float n2 = SHIFTED ? e2 - 3.0f * drho + 5.5f * usq : e2 - 3.0f * rho + 5.5f * usq;
    // q_a = j_a + 5 d_axis: q_x + 2/3 rho u_x etc.
    const float n4 = jx + 5.0f * d8 + (2.0f / 3.0f) * rux;
    const float n6 = jy + 5.0f * d6 + (2.0f / 3.0f) * ruy;
    const float n8 = jz + 5.0f * d2 + (2.0f / 3.0f) * ruz;
    const float s04 = s0 + s4, s13 = s1 + s3, s57 = s5 + s7;
    const float pxx_eq = 2.0f * uxx - uyy - uzz;                   // m9^eq
    const float pww_eq = uyy - uzz;                                // m11^eq
    const float n9 = 2.0f * s8 - (s2 + s6) - 2.0f * s04 + (s13 + s57) - pxx_eq;
    const float n10 = -4.0f * s8 + 2.0f * (s2 + s6) - 2.0f * s04 + (s13 + s57) + 0.5f * pxx_eq;
    const float n11 = (s6 - s2) + (s57 - s13) - pww_eq;
    const float n12 = 2.0f * (s2 - s6) + (s57 - s13) + 0.5f * pww_eq;
    const float n13 = (s5 - s7) - uxy;
    const float n14 = (s0 - s4) - uyz;
    const float n15 = (s1 - s3) - uxz;
    const float n16 = (d1 - d3) + (d7 - d5);
    const float n17 = (d4 - d0) + (d5 + d7);
    const float n18 = (d0 + d4) - (d1 + d3);

    // Pi_neq from the second-order non-equilibrium moments, Q^(1/2) = |Pi_neq|_F
    const float c2 = n1 * (1.0f / 19.0f);
    const float pxx = (c2 + n9) * (1.0f / 3.0f);
    const float pyy = (c2 - 0.5f * n9 + 1.5f * n11) * (1.0f / 3.0f);
    const float pzz = (c2 - 0.5f * n9 - 1.5f * n11) * (1.0f / 3.0f);
    const float qq = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (n13 * n13 + n14 * n14 + n15 * n15);
    // eq:tau_eff: s_nu = 1 / tau_eff = 2 / (tau0 + sqrt(tau0^2 + 18 sqrt2 C Q^(1/2) / rho))
    const float sv = 2.0f * rcp_approx(tau0 + sqrt_approx(fmaf(csm18 * sqrt_approx(qq), irho, tau0 * tau0)));

    float G1, G2 = S_EPS * n2 * (1.0f / 252.0f);
    float G3 = 0.0f, G5 = 0.0f, G7 = 0.0f;
    float G4 = S_Q * n4 * (1.0f / 40.0f), G6 = S_Q * n6 * (1.0f / 40.0f), G8 = S_Q * n8 * (1.0f / 40.0f);
    float G9 = sv * n9 * (1.0f / 36.0f), G10 = S_PI * n10 * (1.0f / 72.0f);
    float G11 = sv * n11 * (1.0f / 12.0f), G12 = S_PI * n12 * (1.0f / 24.0f);
    float G13 = sv * n13 * 0.25f, G14 = sv * n14 * 0.25f, G15 = sv * n15 * 0.25f;
    if (HAS_FORCE) {
        // moments of the Guo source M F~ (second-order Hermite form)
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const float F9 = 4.0f * ux * Fx - 2.0f * (uy * Fy + uz * Fz);
        const float F11 = 2.0f * (uy * Fy - uz * Fz);
        const float F13 = ux * Fy + uy * Fx, F14 = uy * Fz + uz * Fy, F15 = ux * Fz + uz * Fx;
        const float hv = 1.0f - 0.5f * sv;
        const float cq = (1.0f - 0.5f * S_Q) * (2.0f / 3.0f);
        G1 = (S_E * n1 - (1.0f - 0.5f * S_E) * 38.0f * uF) * (1.0f / 2394.0f);
        G2 += (1.0f - 0.5f * S_EPS) * 11.0f * uF * (1.0f / 252.0f);
        G3 = -0.1f * Fx; G5 = -0.1f * Fy; G7 = -0.1f * Fz;
        G4 += cq * Fx * (1.0f / 40.0f); G6 += cq * Fy * (1.0f / 40.0f); G8 += cq * Fz * (1.0f / 40.0f);
        G9 -= hv * F9 * (1.0f / 36.0f);
        G10 += (1.0f - 0.5f * S_PI) * 0.5f * F9 * (1.0f / 72.0f);
        G11 -= hv * F11 * (1.0f / 12.0f);
        G12 += (1.0f - 0.5f * S_PI) * 0.5f * F11 * (1.0f / 24.0f);
        G13 -= hv * F13 * 0.25f; G14 -= hv * F14 * 0.25f; G15 -= hv * F15 * 0.25f;
    } else {
        G1 = S_E * n1 * (1.0f / 2394.0f);
    }
    const float G16 = S_M * n16 * 0.125f, G17 = S_M * n17 * 0.125f, G18 = S_M * n18 * 0.125f;

    // f* = f - M^T g, by opposite pairs: even part E (same for p and 18-p),
    // odd part O (sign flips).
    const float Aax = -11.0f * G1 - 4.0f * G2;
    const float Ddg = 8.0f * G1 + G2;
    const float Jx = G3 + G4, Jy = G5 + G6, Jz = G7 + G8;
    const float g9_10 = G9 + G10, g11_12 = G11 + G12;
    float E, O;
    E = Ddg - 2.0f * g9_10 + G14;              O = -Jy - Jz - G17 + G18;      // pair 0/18
    f[0] -= E + O; f[18] -= E - O;
    E = Ddg + g9_10 - g11_12 + G15;            O = -Jx - Jz + G16 - G18;      // pair 1/17
    f[1] -= E + O; f[17] -= E - O;
    E = Aax - G9 + 2.0f * G10 - G11 + 2.0f * G12; O = -G7 + 4.0f * G8;        // pair 2/16
    f[2] -= E + O; f[16] -= E - O;
    E = Ddg + g9_10 - g11_12 - G15;            O = Jx - Jz - G16 - G18;       // pair 3/15
    f[3] -= E + O; f[15] -= E - O;
    E = Ddg - 2.0f * g9_10 - G14;              O = Jy - Jz + G17 + G18;       // pair 4/14
    f[4] -= E + O; f[14] -= E - O;
    E = Ddg + g9_10 + g11_12 + G13;            O = -Jx - Jy - G16 + G17;      // pair 5/13
    f[5] -= E + O; f[13] -= E - O;
    E = Aax - G9 + 2.0f * G10 + G11 - 2.0f * G12; O = -G5 + 4.0f * G6;        // pair 6/12
    f[6] -= E + O; f[12] -= E - O;
    E = Ddg + g9_10 + g11_12 - G13;            O = Jx - Jy + G16 + G17;       // pair 7/11
    f[7] -= E + O; f[11] -= E - O;
    E = Aax + 2.0f * G9 - 4.0f * G10;          O = -G3 + 4.0f * G4;           // pair 8/10
    f[8] -= E + O; f[10] -= E - O;
    f[9] += 30.0f * G1 - 12.0f * G2;
}

// ---------------------------------------------------------------------------
// Two cells per thread: packed FP32x2 arithmetic (sm_100 family) so that one
// instruction updates both cells.  V2 holds (cell i, cell i+1).
// ---------------------------------------------------------------------------
typedef float2 V2;
__device__ __forceinline__ V2 vdup(float s) { return make_float2(s, s); }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return __fadd2_rn(a, b); }
// a - b as a packed add of the negated operand: the negation folds into the
// add, where a multiply-add with a (-1, -1) pair needs that pair in registers
// (measured: 1-2% off the 16-bit step kernels, which are bound by instruction
// issue)
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ V2 operator-(V2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ V2 operator*(float s, V2 b) { return __fmul2_rn(vdup(s), b); }
__device__ __forceinline__ V2 operator*(V2 b, float s) { return __fmul2_rn(b, vdup(s)); }
__device__ __forceinline__ V2 vfma(V2 a, V2 b, V2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ V2 vfma(float a, V2 b, V2 c) { return __ffma2_rn(vdup(a), b, c); }
__device__ __forceinline__ V2 vrcp(V2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ V2 vsqrt(V2 a) { return make_float2(sqrt_approx(a.x), sqrt_approx(a.y)); }

// Pair sums / differences, density and momentum of two cells (eq:density,
// eq:momentum without the force).
struct Pairs2 {
    V2 s[9], d[9], f9;
    V2 s04, s13, s57, s26, Sdg, Sax;
    V2 rho, jx, jy, jz;
};
template <bool SHIFTED>
__device__ __forceinline__ void make_pairs2(const V2 (&f)[19], Pairs2 &P) {
#pragma unroll
    for (int p = 0; p < 9; ++p) { P.s[p] = f[p] + f[18 - p]; P.d[p] = f[p] - f[18 - p]; }
    const V2 *s = P.s, *d = P.d;
    P.f9 = f[9];
    P.s04 = s[0] + s[4]; P.s13 = s[1] + s[3]; P.s57 = s[5] + s[7]; P.s26 = s[2] + s[6];
    P.Sdg = (P.s04 + P.s13) + P.s57;
    P.Sax = P.s26 + s[8];
    P.rho = SHIFTED ? (P.Sdg + P.Sax) + P.f9 + vdup(1.0f) : (P.Sdg + P.Sax) + P.f9;
    const V2 Dx = (d[3] - d[1]) + (d[7] - d[5]);
    const V2 Dy = (d[4] - d[0]) - (d[5] + d[7]);
    const V2 Dz = -(d[0] + d[4]) - (d[1] + d[3]);
    P.jx = Dx - d[8]; P.jy = Dy - d[6]; P.jz = Dz - d[2];
}

// MRT-LES collision of two cells: the algebra of collide_mrt written with
// fused packed operations.  HAS_FORCE adds the moment-space Guo source of a
// wall force (Fx, 0, Fz) per cell -- the wall-model force is tangential, so
// its y component is zero by construction (eq:force_wm, the wall normal is y).
template <bool SHIFTED, bool HAS_FORCE>
__device__ __forceinline__ void collide_pairs2(const Pairs2 &P, V2 (&f)[19], V2 Fx, V2 Fz, V2 tau0,
                                               float csm18, V2 &ux_o, V2 &uy_o, V2 &uz_o) {
    const V2 *s = P.s, *d = P.d;
    const V2 f9 = P.f9, s04 = P.s04, s13 = P.s13, s57 = P.s57, s26 = P.s26;
    const V2 Sdg = P.Sdg, Sax = P.Sax, rho = P.rho, jx = P.jx, jy = P.jy, jz = P.jz;
    const V2 irho = vrcp(rho);
    // eq:momentum: rho u = sum f c + F/2
    const V2 rux = HAS_FORCE ? vfma(0.5f, Fx, jx) : jx;
    const V2 ruz = HAS_FORCE ? vfma(0.5f, Fz, jz) : jz;
    const V2 ux = rux * irho, uy = jy * irho, uz = ruz * irho;
    ux_o = ux; uy_o = uy; uz_o = uz;
    const V2 uxx = rux * ux, uyy = jy * uy, uzz = ruz * uz;
    const V2 uxy = rux * uy, uyz = jy * uz, uxz = rux * uz;
    const V2 usq = (uxx + uyy) + uzz;
    // non-equilibrium moments; M w = (1, -11, 3, 0, ...) sets the constants
    const V2 e1 = vfma(-30.0f, f9, vfma(8.0f, Sdg, -11.0f * Sax));
    const V2 e2 = vfma(12.0f, f9, vfma(-4.0f, Sax, Sdg));
    const V2 r11 = SHIFTED ? 11.0f * (rho - vdup(1.0f)) : 11.0f * rho;
    const V2 r3 = SHIFTED ? -3.0f * (rho - vdup(1.0f)) : -3.0f * rho;
    const V2 n1 = vfma(-19.0f, usq, e1 + r11);
    const V2 n2 = vfma(5.5f, usq, e2 + r3);
    const V2 n4 = vfma(5.0f, d[8], vfma(2.0f / 3.0f, rux, jx));
    const V2 n6 = vfma(5.0f, d[6], vfma(2.0f / 3.0f, jy, jy));
    const V2 n8 = vfma(5.0f, d[2], vfma(2.0f / 3.0f, ruz, jz));
    const V2 pxx_eq = vfma(2.0f, uxx, -(uyy + uzz));
    const V2 pww_eq = uyy - uzz;
    const V2 t1357 = s13 + s57;
    const V2 n9 = vfma(2.0f, s[8] - s04, t1357 - s26) - pxx_eq;
    const V2 n10 = vfma(-4.0f, s[8], vfma(2.0f, s26 - s04, t1357)) + 0.5f * pxx_eq;
    const V2 d57m13 = s57 - s13;
    const V2 n11 = (s[6] - s[2]) + d57m13 - pww_eq;
    const V2 n12 = vfma(2.0f, s[2] - s[6], d57m13) + 0.5f * pww_eq;
    const V2 n13 = (s[5] - s[7]) - uxy;
    const V2 n14 = (s[0] - s[4]) - uyz;
    const V2 n15 = (s[1] - s[3]) - uxz;
    const V2 n16 = (d[1] - d[3]) + (d[7] - d[5]);
    const V2 n17 = (d[4] - d[0]) + (d[5] + d[7]);
    const V2 n18 = (d[0] + d[4]) - (d[1] + d[3]);
    // Pi_neq and the Smagorinsky rate (eq:tau_eff)
    const V2 c2 = n1 * (1.0f / 57.0f);                 // (n1 / 19) / 3
    const V2 pxx = vfma(1.0f / 3.0f, n9, c2);
    const V2 pyz_common = vfma(-1.0f / 6.0f, n9, c2);
    const V2 pyy = vfma(0.5f, n11, pyz_common);
    const V2 pzz = vfma(-0.5f, n11, pyz_common);
    V2 qq = vfma(pxx, pxx, vfma(pyy, pyy, pzz * pzz));
    qq = vfma(2.0f * n13, n13, vfma(2.0f * n14, n14, vfma(2.0f * n15, n15, qq)));
    const V2 tt = tau0;
    const V2 sv = 2.0f * vrcp(tt + vsqrt(vfma(csm18 * vsqrt(qq), irho, tt * tt)));
    // relaxation: G_k = s_k n_k / |row_k|^2
    V2 G1 = n1 * (S_E / 2394.0f), G2 = n2 * (S_EPS / 252.0f);
    V2 G4 = n4 * (S_Q / 40.0f), G6 = n6 * (S_Q / 40.0f), G8 = n8 * (S_Q / 40.0f);
    const V2 sv36 = sv * (1.0f / 36.0f), sv12 = sv * (1.0f / 12.0f), sv4 = sv * 0.25f;
    V2 G9 = sv36 * n9, G10 = n10 * (S_PI / 72.0f);
    V2 G11 = sv12 * n11, G12 = n12 * (S_PI / 24.0f);
    V2 G13 = sv4 * n13, G14 = sv4 * n14, G15 = sv4 * n15;
    const V2 G16 = n16 * (S_M * 0.125f), G17 = n17 * (S_M * 0.125f), G18 = n18 * (S_M * 0.125f);
    // odd parts of the conserved-momentum rows (G3, G5, G7) and the heat fluxes
    V2 Jx = G4, Jz = G8, Ox = 4.0f * G4, Oz = 4.0f * G8;
    const V2 Jy = G6, Oy = 4.0f * G6;
    if (HAS_FORCE) {
        // moments of the Guo source M F~ (second-order Hermite form), F_y = 0
        const V2 uF = vfma(ux, Fx, uz * Fz);
        const V2 hv = vfma(-0.5f, sv, vdup(1.0f));
        const float cq = (1.0f - 0.5f * S_Q) * (2.0f / 3.0f) * (1.0f / 40.0f);
        const V2 F9 = vfma(4.0f, ux * Fx, -2.0f * (uz * Fz));
        const V2 F11 = -2.0f * (uz * Fz);
        G1 = vfma(-(1.0f - 0.5f * S_E) * 38.0f / 2394.0f, uF, G1);
        G2 = vfma((1.0f - 0.5f * S_EPS) * 11.0f / 252.0f, uF, G2);
        G4 = vfma(cq, Fx, G4); G8 = vfma(cq, Fz, G8);
        G9 = G9 - hv * F9 * (1.0f / 36.0f);
        G10 = vfma((1.0f - 0.5f * S_PI) * 0.5f / 72.0f, F9, G10);
        G11 = G11 - hv * F11 * (1.0f / 12.0f);
        G12 = vfma((1.0f - 0.5f * S_PI) * 0.5f / 24.0f, F11, G12);
        G13 = G13 - hv * (uy * Fx) * 0.25f;
        G14 = G14 - hv * (uy * Fz) * 0.25f;
        G15 = G15 - hv * vfma(ux, Fz, uz * Fx) * 0.25f;
        const V2 G3 = -0.1f * Fx, G7 = -0.1f * Fz;
        Jx = G3 + G4; Jz = G7 + G8;
        Ox = vfma(4.0f, G4, -G3); Oz = vfma(4.0f, G8, -G7);
    }
    // f* = f - M^T g by opposite pairs, rebuilt from the pair sums:
    // f*_p = (s_p/2 - E) + (d_p/2 - O), f*_{18-p} = (s_p/2 - E) - (d_p/2 - O)
    const V2 Aax = vfma(-11.0f, G1, -4.0f * G2);
    const V2 Ddg = vfma(8.0f, G1, G2);
    const V2 g9_10 = G9 + G10, g11_12 = G11 + G12;
    const V2 Xa = vfma(-2.0f, g9_10, Ddg);            // pairs 0, 4
    const V2 Xb = (Ddg + g9_10) - g11_12;             // pairs 1, 3
    const V2 Xc = (Ddg + g9_10) + g11_12;             // pairs 5, 7
    auto put = [&](int p, V2 E, V2 O) {
        const V2 hs = vfma(0.5f, s[p], -E), hd = vfma(0.5f, d[p], -O);
        f[p] = hs + hd;
        f[18 - p] = hs - hd;
    };
    put(0, Xa + G14, (G18 - G17) - (Jy + Jz));
    put(1, Xb + G15, (G16 - G18) - (Jx + Jz));
    put(2, vfma(2.0f, G10 + G12, Aax - (G9 + G11)), Oz);
    put(3, Xb - G15, (Jx - Jz) - (G16 + G18));
    put(4, Xa - G14, (Jy - Jz) + (G17 + G18));
    put(5, Xc + G13, (G17 - G16) - (Jx + Jy));
    put(6, vfma(2.0f, G10 - G12, (Aax - G9) + G11), Oy);
    put(7, Xc - G13, (Jx - Jy) + (G16 + G17));
    put(8, vfma(2.0f, G9, vfma(-4.0f, G10, Aax)), Ox);
    f[9] = vfma(30.0f, G1, vfma(-12.0f, G2, f9));
}

// Force-free collision of two cells (interior rows).
template <bool SHIFTED>
__device__ __forceinline__ void collide_mrt2(V2 (&f)[19], V2 tau0, float csm18, V2 &ux_o, V2 &uy_o,
                                             V2 &uz_o) {
    Pairs2 P;
    make_pairs2<SHIFTED>(f, P);
    collide_pairs2<SHIFTED, false>(P, f, vdup(0.0f), vdup(0.0f), tau0, csm18, ux_o, uy_o, uz_o);
}

// ---------------------------------------------------------------------------
// Pull source of population q for cell (i, j, k) under the boundary rules:
// z periodic; x clamped (inlet on: the inlet rebuilds c_x > 0, the outlet
// copy is the clamp at nx-1) or periodic; specular slip walls mirror c_y and
// read from the same row.  Returns the source plane and the cell offset.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int mirror_y(int q) {
    // pairs (0,4), (5,11), (6,12), (7,13), (14,18)
    return (q == 0) ? 4 : (q == 4) ? 0 : (q == 14) ? 18 : (q == 18) ? 14
         : (q == 5 || q == 6 || q == 7) ? q + 6 : (q == 11 || q == 12 || q == 13) ? q - 6 : q;
}
__device__ __forceinline__ void pull_source(int q, int i, int j, int k, int nx, int ny, int nz, int inlet,
                                            int &plane, int &off) {
    int sx = i - CX(q), sy = j - CY(q), sz = k - CZ(q);
    sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
    if (inlet) sx = min(max(sx, 0), nx - 1);
    else sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    plane = q;
    if (sy < 0 || sy >= ny) { sy = j; plane = mirror_y(q); }
    off = (sz * ny + sy) * nx + sx;
}

// ---------------------------------------------------------------------------
// Arguments of the fused step kernel.  Every population plane has its own
// base pointer (offsets stay 32-bit).
// ---------------------------------------------------------------------------
template <class S>
struct StepArgs {
    const typename S::T *in[19];             // post-collision state, read by pull
    typename S::T *out[19];                  // new post-collision state
    const float *__restrict__ vprime;        // [nz][ny][3] STG field v' of this step (eq:aux_vec)
    const float *__restrict__ UR;            // [ny] inlet mean profile (eq:u_couple)
    const float *__restrict__ amat;          // [ny][6] amp * Cholesky factor (eq:v_fluc)
    const float *utau_in;                    // [2][nz][nx] u_tau warm start (previous step)
    float *utau;                             // [2][nz][nx] u_tau of this step (may alias utau_in)
    float *__restrict__ fw;                  // [2][nz][nx][3] wall force of this step
    float *__restrict__ ubuf;                // [3][ncell] velocity (statistics steps)
    unsigned *__restrict__ flags;            // [0] Newton failures, [1] divergence
    const float *__restrict__ rowbase;       // [ny][RB_W] row base of ROWBASE storage (else unused)
    int nx, ny, nz;
    int inlet, wall_model;
    int check;                               // test |u| < 0.3 and finiteness this step
    int reverse;                             // traverse the lattice backwards this step
    int wall_planes;                         // z planes each wall-kernel block walks
    float tau0, csm18;                       // tau0, 18 sqrt2 C_smag
    float sp_x0, sp_inv, sp_3nu;             // outlet sponge: start x, 1 / length, 3 nu_s (0: none)
    float y1_nu, kappa, B;                   // y1 / nu, Reichardt constants
    // objective accumulators (null: none): [0] sum of tau_w over the wall cells
    // with obj_i0 <= i < obj_i1; [1 + 3j ..] sums over z of u, v, u v at i = obj_iR
    double *obj;
    int obj_i0, obj_i1, obj_iR;
};

// tau0 of a cell at x = i + 1/2 with the outlet sponge (reading A24): the
// viscosity rises by nu_s r^2 over the zone, r the position in it.
__device__ __forceinline__ float sponge_tau0(float tau0, float x0, float inv, float s3nu, int i) {
    if (s3nu == 0.0f) return tau0;
    const float r = fminf(fmaxf(((float)i + 0.5f - x0) * inv, 0.0f), 1.0f);
    return fmaf(s3nu, r * r, tau0);
}
template <class S>
__device__ __forceinline__ float cell_tau0(const StepArgs<S> &a, int i) {
    return sponge_tau0(a.tau0, a.sp_x0, a.sp_inv, a.sp_3nu, i);
}
template <class S>
__device__ __forceinline__ V2 pair_tau0(const StepArgs<S> &a, int i0) {
    return make_float2(cell_tau0(a, i0), cell_tau0(a, i0 + 1));
}

// ---------------------------------------------------------------------------
// Row base of ROWBASE storage: rb[j * RB_W + q] = f^eq_q(1, (U0(j), 0, 0)) -
// w_q, the stored word of plane q in row j being f - w_q - rb.  A pulled
// population q of a cell in row j comes from row j - c_y(q) of plane q, except
// through a slip wall, where it comes from plane mirror_y(q) of row j.
// ---------------------------------------------------------------------------
constexpr int RB_W = 20;
template <class S>
__device__ __forceinline__ float rowbase(const StepArgs<S> &a, int row, int plane) {
    return S::ROWBASE ? __ldg(a.rowbase + row * RB_W + plane) : 0.0f;
}
// pulled populations of interior cells (rows 1 .. ny-2) in row j: add the base back
template <class S>
__device__ __forceinline__ void rowbase_decode(const StepArgs<S> &a, V2 (&f)[19], int j) {
    if constexpr (S::ROWBASE) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] = f[q] + vdup(rowbase(a, j - CY(q), q));
    }
}
template <class S>
__device__ __forceinline__ void rowbase_decode(const StepArgs<S> &a, float (&f)[19], int j) {
    if constexpr (S::ROWBASE) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] += rowbase(a, j - CY(q), q);
    }
}
// post-collision populations of cells in row j: take the base off before the store
template <class S>
__device__ __forceinline__ void rowbase_encode(const StepArgs<S> &a, V2 (&f)[19], int j) {
    if constexpr (S::ROWBASE) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] = f[q] - vdup(rowbase(a, j, q));
    }
}
template <class S>
__device__ __forceinline__ void rowbase_encode(const StepArgs<S> &a, float (&f)[19], int j) {
    if constexpr (S::ROWBASE) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] -= rowbase(a, j, q);
    }
}

constexpr int BY = 2;  // rows per block: (0,1) and (ny-2,ny-1) share a block
constexpr int WALL_THREADS = 128;   // threads (x-cells) per block of the wall-row kernel
#ifndef LBM_STEP_THREADS
#define LBM_STEP_THREADS 128   // threads per block of the step kernel (BX x BY)
#endif
#ifndef LBM_STEP_MINB
#define LBM_STEP_MINB 8        // resident blocks per SM the register budget aims for
#endif
constexpr int STEP_THREADS = LBM_STEP_THREADS;

// Load the 19 pulled populations.  WALL: the row touches a slip wall, so the
// populations that would come through it are read mirrored from this row.
template <class S, bool WALL>
__device__ __forceinline__ void load_pulled(const StepArgs<S> &a, float (&f)[19], int o00, int ozm, int ozp,
                                            int oym, int oyp, int ic, int xm, int xp, bool bot, bool top) {
    // source offsets: row shift -c_y, plane shift -c_z (ozm: source for c_z=+1)
    const int rm = o00 + oym, rp = o00 + oyp;      // rows for c_y = +1 / -1
#define LDQ(q, plane, off) f[q] = S::ld(a.in[plane] + (off))
    LDQ(1, 1, o00 + ozp + xp);  LDQ(2, 2, o00 + ozp + ic);  LDQ(3, 3, o00 + ozp + xm);
    LDQ(8, 8, o00 + xp);        LDQ(9, 9, o00 + ic);        LDQ(10, 10, o00 + xm);
    LDQ(15, 15, o00 + ozm + xp); LDQ(16, 16, o00 + ozm + ic); LDQ(17, 17, o00 + ozm + xm);
    if (!WALL) {
        LDQ(0, 0, rp + ozp + ic);   LDQ(4, 4, rm + ozp + ic);
        LDQ(5, 5, rp + xp);         LDQ(6, 6, rp + ic);         LDQ(7, 7, rp + xm);
        LDQ(11, 11, rm + xp);       LDQ(12, 12, rm + ic);       LDQ(13, 13, rm + xm);
        LDQ(14, 14, rp + ozm + ic); LDQ(18, 18, rm + ozm + ic);
    } else {
        // c_y = -1 populations (0, 5, 6, 7, 14) come from row j+1, or at the top
        // wall from this row with c_y mirrored (4, 11, 12, 13, 18); and the other way
        // round for c_y = +1 at the bottom wall.
        LDQ(0, top ? 4 : 0, rp + ozp + ic);      LDQ(4, bot ? 0 : 4, rm + ozp + ic);
        LDQ(5, top ? 11 : 5, rp + xp);           LDQ(6, top ? 12 : 6, rp + ic);
        LDQ(7, top ? 13 : 7, rp + xm);           LDQ(11, bot ? 5 : 11, rm + xp);
        LDQ(12, bot ? 6 : 12, rm + ic);          LDQ(13, bot ? 7 : 13, rm + xm);
        LDQ(14, top ? 18 : 14, rp + ozm + ic);   LDQ(18, bot ? 14 : 18, rm + ozm + ic);
    }
#undef LDQ
}

// Regularized velocity inlet (Sec. 3.1, Algorithm 1 steps 6-7) for the cell at
// x = 0: rebuild all 19 populations from the known ones (c_x <= 0) and
// u_in = (U_R, 0, 0) + a v' (eq:u_couple, eq:v_fluc).
template <class S>
__device__ __forceinline__ void inlet_rebuild(const StepArgs<S> &a, float (&f)[19], int j, int k) {
    const int ny = a.ny;
    const float *vp = a.vprime + ((size_t)k * ny + j) * 3;
    const float *m = a.amat + 6 * j;
    const float vx = a.UR[j] + m[0] * vp[0];
    const float vy = m[1] * vp[0] + m[2] * vp[1];
    const float vz = m[3] * vp[0] + m[4] * vp[1] + m[5] * vp[2];
    if (!S::SHIFTED) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] -= WQ(q);
    }
    // Zou-He density from the known populations; with f - w the weights
    // contribute exactly 1
    const float sk = (f[0] + f[2] + f[4] + f[6] + f[9] + f[12] + f[14] + f[16] + f[18])
                   + 2.0f * (f[1] + f[5] + f[8] + f[11] + f[15]);
    const float rin = (1.0f + sk) / (1.0f - vx);
    const float drin = rin - 1.0f;
    const float vv = vx * vx + vy * vy + vz * vz;
    // f^eq_q - w_q of eq:bc_eq at (rho_in, u_in)
    auto feq = [&](int q) {
        const float cu = CX(q) * vx + CY(q) * vy + CZ(q) * vz;
        return WQ(q) * (drin + rin * (3.0f * cu + 4.5f * cu * cu - 1.5f * vv));
    };
    // f^neq in place: known populations (c_x <= 0) first, then the unknown
    // ones (c_x > 0) take f^neq of the opposite direction
#pragma unroll
    for (int q = 0; q < 19; ++q) if (CX(q) <= 0) f[q] -= feq(q);
#pragma unroll
    for (int q = 0; q < 19; ++q) if (CX(q) > 0) f[q] = f[18 - q];
    float pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0, tr = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        pxx += CX(q) * CX(q) * f[q]; pyy += CY(q) * CY(q) * f[q]; pzz += CZ(q) * CZ(q) * f[q];
        pxy += CX(q) * CY(q) * f[q]; pyz += CY(q) * CZ(q) * f[q]; pxz += CX(q) * CZ(q) * f[q];
        tr += f[q];
    }
    // Pi_neq = sum_q Q_q f^neq_q with Q_q = c c - I/3
    pxx -= tr * (1.0f / 3.0f); pyy -= tr * (1.0f / 3.0f); pzz -= tr * (1.0f / 3.0f);
    const float trp = (pxx + pyy + pzz) * (1.0f / 3.0f);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float qp = CX(q) * CX(q) * pxx + CY(q) * CY(q) * pyy + CZ(q) * CZ(q) * pzz
                       + 2.0f * (CX(q) * CY(q) * pxy + CY(q) * CZ(q) * pyz + CX(q) * CZ(q) * pxz) - trp;
        f[q] = feq(q) + 4.5f * WQ(q) * qp + (S::SHIFTED ? 0.0f : WQ(q));   // w / (2 cs^4) = 9 w / 2
    }
}

// Store the post-collision populations and the statistics / divergence checks.
template <class S, bool STATS>
__device__ __forceinline__ void finish_cell(const StepArgs<S> &a, const float (&f)[19], int c, float ux, float uy,
                                            float uz) {
#pragma unroll
    for (int q = 0; q < 19; ++q) S::st(a.out[q] + c, f[q]);
    if (STATS) {
        const long long N = (long long)a.nx * a.ny * a.nz;
        a.ubuf[c] = ux; a.ubuf[N + c] = uy; a.ubuf[2 * N + c] = uz;
    }
    if (a.check) {
        const float uu = ux * ux + uy * uy + uz * uz;
        if (!(uu < 0.09f)) atomicAdd(a.flags + 1, 1u);    // also catches NaN
    }
}

// The first and last block rows: the cells next to the slip walls (mirrored
// pulls) and the wall model (Sec. 2.3, Algorithm 1 steps 9-14) on the first
// off-wall cells, whose second cell sits in the same block.  Kept out of line
// so that the interior path gets its own register allocation.  The nthr
// threads that call it (a multiple of 32) meet at named barrier 1.
template <class S, bool STATS>
__device__ __noinline__ void wall_rows(const StepArgs<S> &a, int i, int j, int k, int tx, int o00, int ozm,
                                       int ozp, int ic, int xm, int xp, int nthr) {
    __shared__ float su2[2 * STEP_THREADS / BY][3];   // slot tx (one or two per thread)
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool bot = j == 0, top = j == ny - 1;
    const bool valid = i < nx;
    const int oym = bot ? 0 : -nx, oyp = top ? 0 : nx;
    float f[19];
    if (bot || top) load_pulled<S, true>(a, f, o00, ozm, ozp, oym, oyp, ic, xm, xp, bot, top);
    else load_pulled<S, false>(a, f, o00, ozm, ozp, oym, oyp, ic, xm, xp, bot, top);
    if constexpr (S::ROWBASE) {
        // through a slip wall the population comes mirrored from this row
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const bool mir = (bot && CY(q) > 0) || (top && CY(q) < 0);
            f[q] += mir ? rowbase(a, j, mirror_y(q)) : rowbase(a, j - CY(q), q);
        }
    }
    if (a.inlet && i == 0) inlet_rebuild<S>(a, f, j, k);
    Pairs P;
    make_pairs<S::SHIFTED>(f, P);
    float ux, uy, uz;
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    const bool is_wall = bot || top;
    if (a.wall_model) {                                   // block-uniform
        const float irho = 1.0f / (1.0f + P.drho);
        if (!is_wall) { su2[tx][0] = P.jx * irho; su2[tx][1] = P.jy * irho; su2[tx][2] = P.jz * irho; }
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
        if (is_wall && valid) {
            const int w = bot ? 0 : 1;
            const float u2x = su2[tx][0], u2z = su2[tx][2];
            // eq:base: tangential part of u_2 (the wall normal is along y), normalized
            const float tn = sqrtf(u2x * u2x + u2z * u2z);
            const size_t iu = ((size_t)w * nz + k) * nx + i;
            float ut_new = a.utau_in[iu];
            if (tn >= 1e-12f) {
                const float ex = u2x / tn, ez = u2z / tn;
                // eq:uhat with the first-cell velocity (no half-force term)
                const float uhat = (P.jx * ex + P.jz * ez) * irho;
                const float sg = uhat < 0.0f ? -1.0f : 1.0f;
                const float ua = fabsf(uhat);
                float ut = 0.0f;
                if (ua > 0.0f) {
                    bool ok;
                    ut = solve_utau_dev(ua, a.y1_nu, a.kappa, a.B, a.utau_in[iu], &ok);
                    if (!ok) atomicAdd(a.flags, 1u);
                }
                ut_new = ut;
                // tau_w = rho u_tau^2, eq:force_wm with A = 1
                const float tw = (1.0f + P.drho) * ut * ut * sg;
                Fx = -tw * ex; Fz = -tw * ez;
            }
            a.utau[iu] = ut_new;
            float *fwp = a.fw + (((size_t)w * nz + k) * nx + i) * 3;
            fwp[0] = Fx; fwp[1] = Fy; fwp[2] = Fz;
        }
    }
    if (a.wall_model && is_wall) collide_mrt<S::SHIFTED, true>(f, P, Fx, Fy, Fz, cell_tau0(a, i), a.csm18, ux, uy, uz);
    else collide_mrt<S::SHIFTED, false>(f, P, 0.f, 0.f, 0.f, cell_tau0(a, i), a.csm18, ux, uy, uz);
    rowbase_encode<S>(a, f, j);
    if (valid) finish_cell<S, STATS>(a, f, o00 + i, ux, uy, uz);
}

// One time step of Algorithm 1 for every cell: pull streaming with the
// boundary rules, the regularized inlet at x = 0 (steps 6-8), the Reichardt
// wall force on j = 0 and j = ny-1 (steps 9-14), the MRT-LES collision (step 15).
template <class S, bool STATS>
__global__ void __launch_bounds__(LBM_STEP_THREADS, LBM_STEP_MINB) step_kernel(const __grid_constant__ StepArgs<S> a) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // every other step runs the blocks in reverse order, so that a step starts
    // on the planes the previous step wrote last (still resident in L2)
    const int bxi = a.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int byi = a.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int i = bxi * blockDim.x + tx;
    const int j = byi * BY + ty;
    const int k = a.reverse ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    const int ic = i < nx ? i : nx - 1;

    int xm = ic - 1, xp = ic + 1;                    // sources for c_x = +1 / -1
    if (a.inlet) { xm = max(xm, 0); xp = min(xp, nx - 1); }
    else { xm = xm < 0 ? nx - 1 : xm; xp = xp >= nx ? 0 : xp; }
    const int plane = nx * ny;
    const int ozm = k == 0 ? (nz - 1) * plane : -plane;     // source plane for c_z = +1
    const int ozp = k == nz - 1 ? -(nz - 1) * plane : plane;  // source plane for c_z = -1
    const int o00 = (k * ny + j) * nx;

    if (byi == 0 || byi == gridDim.y - 1) {               // block-uniform
        wall_rows<S, STATS>(a, i, j, k, tx, o00, ozm, ozp, ic, xm, xp, blockDim.x * blockDim.y);
        return;
    }
    float f[19];
    load_pulled<S, false>(a, f, o00, ozm, ozp, -nx, nx, ic, xm, xp, false, false);
    rowbase_decode<S>(a, f, j);
    if (a.inlet && i == 0) inlet_rebuild<S>(a, f, j, k);
    Pairs P;
    make_pairs<S::SHIFTED>(f, P);
    float ux, uy, uz;
    collide_mrt<S::SHIFTED, false>(f, P, 0.f, 0.f, 0.f, cell_tau0(a, i), a.csm18, ux, uy, uz);
    rowbase_encode<S>(a, f, j);
    if (i < nx) finish_cell<S, STATS>(a, f, o00 + i, ux, uy, uz);
}

// Load the pulled populations of two x-adjacent cells (i0, i0 + 1) of the
// interior row whose offset is o00 (row start in its plane): vector loads where
// c_x = 0, two scalar loads where c_x != 0.  ozm / ozp: plane shifts of the
// c_z = +1 / -1 sources (periodic z); the rows of the c_y = +1 / -1 sources are
// o00 -/+ nx.  xm0 / xp1: the sources of the lo cell's c_x = +1 and the hi
// cell's c_x = -1 populations.
template <class S>
__device__ __forceinline__ void load_pair(const StepArgs<S> &a, V2 (&f)[19], int o00, int ozm, int ozp, int ic,
                                          int xm0, int xp1) {
    const int rm = o00 - a.nx, rp = o00 + a.nx;      // rows for c_y = +1 / -1
#define LD_C0(q, row) f[q] = S::ld2(a.in[q] + (row) + ic)
#define LD_CP(q, row) f[q] = make_float2(S::ld(a.in[q] + (row) + xm0), S::ld(a.in[q] + (row) + ic))
#define LD_CM(q, row) f[q] = make_float2(S::ld(a.in[q] + (row) + ic + 1), S::ld(a.in[q] + (row) + xp1))
    LD_C0(0, rp + ozp); LD_CM(1, o00 + ozp); LD_C0(2, o00 + ozp); LD_CP(3, o00 + ozp); LD_C0(4, rm + ozp);
    LD_CM(5, rp);       LD_C0(6, rp);        LD_CP(7, rp);        LD_CM(8, o00);       LD_C0(9, o00);
    LD_CP(10, o00);     LD_CM(11, rm);       LD_C0(12, rm);       LD_CP(13, rm);       LD_C0(14, rp + ozm);
    LD_CM(15, o00 + ozm); LD_C0(16, o00 + ozm); LD_CP(17, o00 + ozm); LD_C0(18, rm + ozm);
#undef LD_C0
#undef LD_CP
#undef LD_CM
}

// Inlet velocity u_in = (U_R, 0, 0) + a v' of row j, plane k (eq:u_couple, eq:v_fluc).
template <class S>
__device__ __forceinline__ void inlet_velocity(const StepArgs<S> &a, int j, int k, float &vx, float &vy,
                                               float &vz) {
    const float *vp = a.vprime + ((size_t)k * a.ny + j) * 3;
    const float *m = a.amat + 6 * j;
    vx = a.UR[j] + m[0] * vp[0];
    vy = m[1] * vp[0] + m[2] * vp[1];
    vz = m[3] * vp[0] + m[4] * vp[1] + m[5] * vp[2];
}

// The wall rows j = 0 and j = ny - 1 of the step: one thread per (x, z) takes
// the bottom and the top wall cell as the two lanes of the packed collision
// (.x bottom, .y top).  Launched beside the interior kernel (the rows are
// disjoint).  Per lane: the pulled populations, mirrored at the wall; u_2 of
// the second cell (row 1 / ny - 2) summed from its pulled populations; the
// regularized inlet at x = 0; the wall model (Sec. 2.3, Algorithm 1 steps
// 9-14) with a scalar Newton solve; then the packed collision with the force.
// Each block walks a.wall_planes consecutive z planes: the kernel is a long
// dependent chain per cell with few warps, so fewer, longer-lived blocks hold
// fewer of the registers the interior kernel beside it could use, as long as
// the walk still ends inside the interior kernel's time.
template <class S, bool STATS>
__global__ void __launch_bounds__(WALL_THREADS, 4) wall_kernel(const __grid_constant__ StepArgs<S> a) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
    for (int kk = 0; kk < a.wall_planes; ++kk) {
    const int k = blockIdx.y * a.wall_planes + kk;
    if (k >= nz) return;
    const bool valid = i < nx;
    const int ic = valid ? i : nx - 1;
    int xm = ic - 1, xp = ic + 1;                    // sources for c_x = +1 / -1
    if (a.inlet) { xm = max(xm, 0); xp = min(xp, nx - 1); }
    else { xm = xm < 0 ? nx - 1 : xm; xp = xp >= nx ? 0 : xp; }
    const int plane = nx * ny;
    const int ozm = k == 0 ? (nz - 1) * plane : -plane;       // source plane for c_z = +1
    const int ozp = k == nz - 1 ? -(nz - 1) * plane : plane;  // source plane for c_z = -1
    const int ob = k * plane, ot = ob + (ny - 1) * nx;        // rows 0 and ny - 1
    V2 f[19];
    V2 r2 = vdup(0.0f), jx2 = vdup(0.0f), jz2 = vdup(0.0f);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int oz = CZ(q) > 0 ? ozm : (CZ(q) < 0 ? ozp : 0);
        const int x = CX(q) > 0 ? xm : (CX(q) < 0 ? xp : ic);
        // bottom: c_y = +1 comes through the wall (mirrored, same row); top: c_y = -1
        const int pb = CY(q) > 0 ? mirror_y(q) : q, pt = CY(q) < 0 ? mirror_y(q) : q;
        const int rb = CY(q) < 0 ? nx : 0, rt = CY(q) > 0 ? -nx : 0;
        f[q] = make_float2(S::ld(a.in[pb] + ob + rb + oz + x), S::ld(a.in[pt] + ot + rt + oz + x));
        if constexpr (S::ROWBASE)                    // source rows: 0 or 1, ny - 1 or ny - 2
            f[q] = f[q] + make_float2(rowbase(a, CY(q) < 0 ? 1 : 0, pb), rowbase(a, CY(q) > 0 ? ny - 2 : ny - 1, pt));
        if (a.wall_model) {                          // second cells: rows 1 and ny - 2
            const int ry = -CY(q) * nx;
            V2 g = make_float2(S::ld(a.in[q] + ob + nx + ry + oz + x),
                               S::ld(a.in[q] + ot - nx + ry + oz + x));
            if constexpr (S::ROWBASE)
                g = g + make_float2(rowbase(a, 1 - CY(q), q), rowbase(a, ny - 2 - CY(q), q));
            r2 = r2 + g;
            if (CX(q) > 0) jx2 = jx2 + g;
            if (CX(q) < 0) jx2 = jx2 - g;
            if (CZ(q) > 0) jz2 = jz2 + g;
            if (CZ(q) < 0) jz2 = jz2 - g;
        }
    }
    const bool inlet_cell = a.inlet && i == 0;
    if (inlet_cell) {
        float fl[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) fl[q] = f[q].x;
        inlet_rebuild<S>(a, fl, 0, k);
#pragma unroll
        for (int q = 0; q < 19; ++q) { f[q].x = fl[q]; fl[q] = f[q].y; }
        inlet_rebuild<S>(a, fl, ny - 1, k);
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q].y = fl[q];
    }
    Pairs2 P;
    make_pairs2<S::SHIFTED>(f, P);
    V2 Fx = vdup(0.0f), Fz = vdup(0.0f);
    if (a.wall_model) {
        // u_2 of the second cells: tangential momentum over density (at the
        // inlet: u_in, the velocity their regularized rebuild gives)
        if (S::SHIFTED) r2 = r2 + vdup(1.0f);
        const V2 ir2 = vrcp(r2);
        float u2[2][2] = {{jx2.x * ir2.x, jz2.x * ir2.x}, {jx2.y * ir2.y, jz2.y * ir2.y}};
        if (inlet_cell) {
            float vy;
            inlet_velocity<S>(a, 1, k, u2[0][0], vy, u2[0][1]);
            inlet_velocity<S>(a, ny - 2, k, u2[1][0], vy, u2[1][1]);
        }
        const float rw[2] = {P.rho.x, P.rho.y}, jxw[2] = {P.jx.x, P.jx.y}, jzw[2] = {P.jz.x, P.jz.y};
        float Fo[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            // eq:base: e_x from the tangential part of u_2 (the wall normal is y);
            // eq:uhat with the first-cell velocity; Newton for u_tau; tau_w = rho u_tau^2
            const float u2x = u2[w][0], u2z = u2[w][1];
            const float tn = sqrtf(u2x * u2x + u2z * u2z);
            const size_t iu = ((size_t)w * nz + k) * nx + ic;
            float ut_new = a.utau_in[iu];
            if (tn >= 1e-12f) {
                const float itn = rcp_approx(tn);
                const float ex = u2x * itn, ez = u2z * itn;
                const float uhat = (jxw[w] * ex + jzw[w] * ez) * rcp_approx(rw[w]);
                const float sg = uhat < 0.0f ? -1.0f : 1.0f;
                const float ua = fabsf(uhat);
                float ut = 0.0f;
                if (ua > 0.0f && valid) {
                    bool ok;
                    ut = solve_utau_dev(ua, a.y1_nu, a.kappa, a.B, ut_new, &ok);
                    if (!ok) atomicAdd(a.flags, 1u);
                }
                ut_new = ut;
                const float tw = rw[w] * ut * ut * sg;       // eq:force_wm with A = 1
                Fo[w][0] = -tw * ex; Fo[w][1] = -tw * ez;
            }
            if (valid) {
                a.utau[iu] = ut_new;
                float *fwp = a.fw + iu * 3;
                fwp[0] = Fo[w][0]; fwp[1] = 0.0f; fwp[2] = Fo[w][1];
            }
        }
        Fx = make_float2(Fo[0][0], Fo[1][0]);
        Fz = make_float2(Fo[0][1], Fo[1][1]);
    }
    V2 ux, uy, uz;
    const V2 t0w = vdup(cell_tau0(a, ic));           // bottom and top cells share x
    if (a.wall_model) collide_pairs2<S::SHIFTED, true>(P, f, Fx, Fz, t0w, a.csm18, ux, uy, uz);
    else collide_pairs2<S::SHIFTED, false>(P, f, Fx, Fz, t0w, a.csm18, ux, uy, uz);
    if (a.obj) {                                     // objective sums (launch-uniform branch)
        float tw = 0.0f;
        if (valid && i >= a.obj_i0 && i < a.obj_i1)
            tw = sqrtf(Fx.x * Fx.x + Fz.x * Fz.x) + sqrtf(Fx.y * Fx.y + Fz.y * Fz.y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tw += __shfl_xor_sync(0xffffffffu, tw, o);
        if ((threadIdx.x & 31) == 0 && tw != 0.0f) atomicAdd(a.obj, (double)tw);
        if (valid && i == a.obj_iR) {
            atomicAdd(a.obj + 1, (double)ux.x);
            atomicAdd(a.obj + 2, (double)uy.x);
            atomicAdd(a.obj + 3, (double)(ux.x * uy.x));
            atomicAdd(a.obj + 1 + 3 * (ny - 1), (double)ux.y);
            atomicAdd(a.obj + 2 + 3 * (ny - 1), (double)uy.y);
            atomicAdd(a.obj + 3 + 3 * (ny - 1), (double)(ux.y * uy.y));
        }
    }
    if (!valid) continue;
    if constexpr (S::ROWBASE) {
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] = f[q] - make_float2(rowbase(a, 0, q), rowbase(a, ny - 1, q));
    }
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        S::st(a.out[q] + ob + i, f[q].x);
        S::st(a.out[q] + ot + i, f[q].y);
    }
    if (STATS) {
        const long long N = (long long)plane * nz;
        a.ubuf[ob + i] = ux.x; a.ubuf[N + ob + i] = uy.x; a.ubuf[2 * N + ob + i] = uz.x;
        a.ubuf[ot + i] = ux.y; a.ubuf[N + ot + i] = uy.y; a.ubuf[2 * N + ot + i] = uz.y;
    }
    if (a.check) {
        const V2 uu = vfma(ux, ux, vfma(uy, uy, uz * uz));
        if (!(uu.x < 0.09f) || !(uu.y < 0.09f)) atomicAdd(a.flags + 1, 1u);   // also catches NaN
    }
    }
}

// Interior rows 1 .. ny - 2, two x-adjacent cells (i, i+1), i even, per
// thread: vector loads for the populations with c_x = 0, two scalar loads for
// the shifted ones, packed FP32x2 arithmetic, vector stores.  nx must be even.
// Grid (x range, row pair, plane).
// Resident blocks per SM the register budget aims for: FP32 storage is bound
// by memory latency at five, the 16-bit formats move half the bytes and gain
// from the sixth block's extra warps.
#ifndef LBM_STEP2_MINB32
#define LBM_STEP2_MINB32 5
#endif
#ifndef LBM_STEP2_MINB16
#define LBM_STEP2_MINB16 6
#endif
template <class S> struct Step2Blocks { static constexpr int value = LBM_STEP2_MINB16; };
template <> struct Step2Blocks<StoreF32> { static constexpr int value = LBM_STEP2_MINB32; };

template <class S, bool STATS>
__global__ void __launch_bounds__(LBM_STEP_THREADS, Step2Blocks<S>::value) step2_kernel(const __grid_constant__ StepArgs<S> a) {
    const int nx = a.nx, ny = a.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // every other step walks the blocks backwards, so that a step starts on
    // the planes the previous step wrote last (still in L2)
    const int bxi = a.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int byi = a.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int k = a.reverse ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    const int i0 = 2 * (bxi * blockDim.x + tx);
    const int j = 1 + byi * BY + ty;
    const bool valid = i0 < nx;
    const int ic = valid ? i0 : nx - 2;
    int xm0 = ic - 1, xp1 = ic + 2;                  // lo cell's c_x=+1 source, hi cell's c_x=-1 source
    if (a.inlet) { xm0 = max(xm0, 0); xp1 = min(xp1, nx - 1); }
    else { xm0 = xm0 < 0 ? nx - 1 : xm0; xp1 = xp1 >= nx ? 0 : xp1; }
    const int plane = nx * ny;
    const int ozm = k == 0 ? (a.nz - 1) * plane : -plane;      // source plane for c_z = +1
    const int ozp = k == a.nz - 1 ? -(a.nz - 1) * plane : plane;  // source plane for c_z = -1
    V2 f[19];
    load_pair<S>(a, f, (k * ny + j) * nx, ozm, ozp, ic, xm0, xp1);
    rowbase_decode<S>(a, f, j);
    if (a.inlet && i0 == 0) {                        // the lo cell is an inlet cell
        float fl[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) fl[q] = f[q].x;
        inlet_rebuild<S>(a, fl, j, k);
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q].x = fl[q];
    }
    V2 ux, uy, uz;
    collide_mrt2<S::SHIFTED>(f, pair_tau0(a, i0), a.csm18, ux, uy, uz);
    if (!valid) return;
    if (a.obj && (i0 == a.obj_iR || i0 + 1 == a.obj_iR)) {     // J_R sums at x = i_R
        const float u = i0 == a.obj_iR ? ux.x : ux.y, v = i0 == a.obj_iR ? uy.x : uy.y;
        atomicAdd(a.obj + 1 + 3 * j, (double)u);
        atomicAdd(a.obj + 2 + 3 * j, (double)v);
        atomicAdd(a.obj + 3 + 3 * j, (double)(u * v));
    }
    const int c = (k * ny + j) * nx + ic;
    rowbase_encode<S>(a, f, j);
#pragma unroll
    for (int q = 0; q < 19; ++q) S::st2(a.out[q] + c, f[q]);
    if (STATS) {
        const long long N = (long long)nx * ny * a.nz;
        *reinterpret_cast<float2 *>(a.ubuf + c) = ux;
        *reinterpret_cast<float2 *>(a.ubuf + N + c) = uy;
        *reinterpret_cast<float2 *>(a.ubuf + 2 * N + c) = uz;
    }
    if (a.check) {
        const V2 uu = vfma(ux, ux, vfma(uy, uy, uz * uz));
        if (!(uu.x < 0.09f) || !(uu.y < 0.09f)) atomicAdd(a.flags + 1, 1u);   // also catches NaN
    }
}

// Interior rows, four x-adjacent cells (x0 .. x0 + 3, x0 a multiple of four)
// per thread: one vector load per direction, the x halo (x0 - 1 for c_x = +1,
// x0 + 4 for c_x = -1) from the neighbouring lane by a warp shuffle -- lanes 0
// and 31 and the lattice ends load theirs -- two packed collisions, one vector
// store per direction.  Per cell this halves the address arithmetic, loads
// and stores of step2_kernel, which is what bounds the 16-bit storages.
// nx must be a multiple of four.  Block (32, 2): a warp is 128 cells of a row.
#ifndef LBM_STEP4_MINB
#define LBM_STEP4_MINB 4
#endif
template <class S, bool STATS>
__global__ void __launch_bounds__(64, 2 * LBM_STEP4_MINB) step4_kernel(const __grid_constant__ StepArgs<S> a) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int bxi = a.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int byi = a.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int k = a.reverse ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    const int x0 = 4 * (bxi * 32 + lane);
    const int j = 1 + byi * BY + ty;
    const bool valid = x0 < nx;
    const int xc = valid ? x0 : nx - 4;
    // halo sources: x0 - 1 and x0 + 4 with the x boundary rule
    int xm = xc - 1, xp = xc + 4;
    if (a.inlet) { xm = max(xm, 0); xp = min(xp, nx - 1); }
    else { xm = xm < 0 ? nx - 1 : xm; xp = xp >= nx ? 0 : xp; }
    const bool own_left = lane == 0 || x0 == 0;       // cannot take x0 - 1 from lane - 1
    const bool own_right = lane == 31 || x0 + 4 >= nx;  // nor x0 + 4 from lane + 1
    const int plane = nx * ny;
    const int ozm = k == 0 ? (nz - 1) * plane : -plane;       // source plane for c_z = +1
    const int ozp = k == nz - 1 ? -(nz - 1) * plane : plane;  // source plane for c_z = -1
    const int o00 = (k * ny + j) * nx, rm = o00 - nx, rp = o00 + nx;
    V2 fa[19], fb[19];                                // cells (x0, x0+1), (x0+2, x0+3)
    auto quad = [&](int q, int row) {
        const typename S::T *r = a.in[q] + row;
        const float4 v = S::ld4(r + xc);
        if (CX(q) == 0) {
            fa[q] = make_float2(v.x, v.y); fb[q] = make_float2(v.z, v.w);
        } else if (CX(q) > 0) {                       // source x - 1
            float left = __shfl_up_sync(0xffffffffu, v.w, 1);
            if (own_left) left = S::ld(r + xm);
            fa[q] = make_float2(left, v.x); fb[q] = make_float2(v.y, v.z);
        } else {                                      // source x + 1
            float right = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (own_right) right = S::ld(r + xp);
            fa[q] = make_float2(v.y, v.z); fb[q] = make_float2(v.w, right);
        }
    };
    quad(0, rp + ozp); quad(1, o00 + ozp); quad(2, o00 + ozp); quad(3, o00 + ozp); quad(4, rm + ozp);
    quad(5, rp);       quad(6, rp);        quad(7, rp);        quad(8, o00);       quad(9, o00);
    quad(10, o00);     quad(11, rm);       quad(12, rm);       quad(13, rm);       quad(14, rp + ozm);
    quad(15, o00 + ozm); quad(16, o00 + ozm); quad(17, o00 + ozm); quad(18, rm + ozm);
    rowbase_decode<S>(a, fa, j);
    rowbase_decode<S>(a, fb, j);
    if (a.inlet && x0 == 0) {                        // cell x0 is an inlet cell
        float fl[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) fl[q] = fa[q].x;
        inlet_rebuild<S>(a, fl, j, k);
#pragma unroll
        for (int q = 0; q < 19; ++q) fa[q].x = fl[q];
    }
    V2 uxa, uya, uza, uxb, uyb, uzb;
    collide_mrt2<S::SHIFTED>(fa, pair_tau0(a, x0), a.csm18, uxa, uya, uza);
    collide_mrt2<S::SHIFTED>(fb, pair_tau0(a, x0 + 2), a.csm18, uxb, uyb, uzb);
    if (!valid) return;
    const int c = o00 + x0;
    rowbase_encode<S>(a, fa, j);
    rowbase_encode<S>(a, fb, j);
#pragma unroll
    for (int q = 0; q < 19; ++q) S::st4(a.out[q] + c, make_float4(fa[q].x, fa[q].y, fb[q].x, fb[q].y));
    if (STATS) {
        const long long N = (long long)plane * nz;
        *reinterpret_cast<float4 *>(a.ubuf + c) = make_float4(uxa.x, uxa.y, uxb.x, uxb.y);
        *reinterpret_cast<float4 *>(a.ubuf + N + c) = make_float4(uya.x, uya.y, uyb.x, uyb.y);
        *reinterpret_cast<float4 *>(a.ubuf + 2 * N + c) = make_float4(uza.x, uza.y, uzb.x, uzb.y);
    }
    if (a.check) {
        const V2 ua = vfma(uxa, uxa, vfma(uya, uya, uza * uza));
        const V2 ub = vfma(uxb, uxb, vfma(uyb, uyb, uzb * uzb));
        if (!(ua.x < 0.09f) || !(ua.y < 0.09f) || !(ub.x < 0.09f) || !(ub.y < 0.09f))
            atomicAdd(a.flags + 1, 1u);                  // also catches NaN
    }
}

// ---------------------------------------------------------------------------
// Halo of an x-slab (one column, the five populations of one c_x sign):
// buf[p][k][j] <-> lattice plane qs[p], column `col`.  One thread per (p, j, k).
// ---------------------------------------------------------------------------
struct HaloArgs {
    int qs[5];
    int col, nx, ny, nz;
    long long ncell;
};
template <class T>
__global__ void halo_pack_kernel(const T *__restrict__ lat, T *__restrict__ buf, const HaloArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long plane = (long long)a.ny * a.nz;
    if (e >= 5 * plane) return;
    const int p = (int)(e / plane);
    const long long r = e % plane;                       // k * ny + j
    buf[e] = lat[(long long)a.qs[p] * a.ncell + r * a.nx + a.col];
}
template <class T>
__global__ void halo_unpack_kernel(T *__restrict__ lat, const T *__restrict__ buf, const HaloArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long plane = (long long)a.ny * a.nz;
    if (e >= 5 * plane) return;
    const int p = (int)(e / plane);
    const long long r = e % plane;
    lat[(long long)a.qs[p] * a.ncell + r * a.nx + a.col] = buf[e];
}

// ---------------------------------------------------------------------------
// STG field v' for a batch of steps (Sec. 3.1 eq:aux_vec, Algorithm 1 step 4).
// It depends neither on the flow nor on the inlet profile, so one launch fills
// a ring of nsteps time levels; the step kernel applies u_in = U_R + a v'.  Block = one row j, 32 spanwise
// cells x 8 time levels; the mode tables of the row sit in shared memory.
// The phase k_n d_n . x' + phi_n is carried in 32-bit fixed-point turns:
//   alpha[j][n] = k_n d_ny y_j / 2pi, beta[k][n] = k_n d_nz z_k / 2pi,
//   phi32[n] = phi_n / 2pi, and the time part -nu_n t (nu_n = d_nx U_b / max l_e)
// in 64-bit fixed point, so the argument stays exact for any t.
// ---------------------------------------------------------------------------
struct StgArgs {
    const uint32_t *__restrict__ alpha;   // [ny][N]
    const uint32_t *__restrict__ betaT;   // [N][nz]
    const uint32_t *__restrict__ phi32;   // [N]
    const uint64_t *__restrict__ rate64;  // [N]  (-nu_n) in 2^-64 turns per step
    const float4 *__restrict__ sqsig;     // [ny][N] (sqrt(6 q_n(y)), sigma_n)
    const float *__restrict__ amat;       // [ny][6] amp * Cholesky factor
    const float *__restrict__ UR;         // [ny] mean profile
    float *__restrict__ out;              // [nsteps][nz][ny][3]: v', or u_in if apply_profile
    long long t0;                         // time of slot 0
    const long long *t0_dev;              // if set, the time of slot 0 is read here (graph replays)
    int nsteps, ny, nz, n_modes;
    int apply_profile;
};

// The one value a graph replay needs that differs between its launches.
__global__ void set_time_kernel(long long *dst, long long v) { *dst = v; }

constexpr int STG_KZ = 32, STG_KT = 8, STG_MCHUNK = 256;

// Block = STG_KZ planes k x STG_KT thread rows, each row TT consecutive time
// levels, for one row j; the modes are taken in chunks whose phases (per time
// level) and amplitude/direction entries are staged in shared memory.  A
// thread loads the mode's beta_n(k) once for its TT levels.
template <int TT>
__global__ void __launch_bounds__(STG_KZ * STG_KT) stg_kernel(const __grid_constant__ StgArgs a) {
    constexpr int NT = STG_KT * TT;                  // time levels per block
    __shared__ __align__(16) uint32_t s_ph[STG_MCHUNK][NT];   // alpha + phi + time part
    __shared__ float4 s_sq[STG_MCHUNK];
    const int j = blockIdx.y;
    const int lz = threadIdx.x % STG_KZ, lt0 = (threadIdx.x / STG_KZ) * TT;
    const int k = blockIdx.x * STG_KZ + lz;
    const int N = a.n_modes;
    const long long t0 = a.t0_dev ? *a.t0_dev : a.t0;
    float vx[TT], vy[TT], vz[TT];
#pragma unroll
    for (int tt = 0; tt < TT; ++tt) vx[tt] = vy[tt] = vz[tt] = 0.0f;
    for (int n0 = 0; n0 < N; n0 += STG_MCHUNK) {
        const int nc = min(STG_MCHUNK, N - n0);
        __syncthreads();
        for (int e = threadIdx.x; e < NT * nc; e += blockDim.x) {
            const int m = e / NT, tl = e % NT, n = n0 + m;
            const uint64_t t = (uint64_t)(t0 + (long long)blockIdx.z * NT + tl);
            s_ph[m][tl] = a.alpha[(size_t)j * N + n] + a.phi32[n] + (uint32_t)((a.rate64[n] * t) >> 32);
        }
        for (int e = threadIdx.x; e < nc; e += blockDim.x) s_sq[e] = a.sqsig[(size_t)j * N + n0 + e];
        __syncthreads();
        if (k < a.nz) {
            const uint32_t *be = a.betaT + (size_t)n0 * a.nz + k;
#pragma unroll 2
            for (int m = 0; m < nc; ++m) {
                const uint32_t b = be[(size_t)m * a.nz];
                const float4 qs = s_sq[m];
                uint32_t ph[TT];
                if constexpr (TT == 4) {
                    const uint4 p4 = *reinterpret_cast<const uint4 *>(&s_ph[m][lt0]);
                    ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                } else {
#pragma unroll
                    for (int tt = 0; tt < TT; ++tt) ph[tt] = s_ph[m][lt0 + tt];
                }
#pragma unroll
                for (int tt = 0; tt < TT; ++tt) {
                    const float x = (float)(int32_t)(ph[tt] + b) * 1.4629180792671596e-09f;   // 2 pi / 2^32
                    const float cw = qs.x * __cosf(x);
                    vx[tt] = fmaf(cw, qs.y, vx[tt]);
                    vy[tt] = fmaf(cw, qs.z, vy[tt]);
                    vz[tt] = fmaf(cw, qs.w, vz[tt]);
                }
            }
        }
    }
    if (k >= a.nz) return;
#pragma unroll
    for (int tt = 0; tt < TT; ++tt) {
        const int ts = blockIdx.z * NT + lt0 + tt;
        if (ts >= a.nsteps) break;
        float *o = a.out + (((size_t)ts * a.nz + k) * a.ny + j) * 3;
        if (a.apply_profile) {
            const float *m = a.amat + 6 * j;
            o[0] = a.UR[j] + m[0] * vx[tt];
            o[1] = m[1] * vx[tt] + m[2] * vy[tt];
            o[2] = m[3] * vx[tt] + m[4] * vy[tt] + m[5] * vz[tt];
        } else {
            o[0] = vx[tt]; o[1] = vy[tt]; o[2] = vz[tt];
        }
    }
}

// ---------------------------------------------------------------------------
// Initial state f^eq(1, (U_R(y), 0, 0)) and the diagnostics kernels.
// ---------------------------------------------------------------------------
template <class S>
__global__ void init_kernel(typename S::T *f, const float *UR, const float *rowbase, int nx, int ny,
                            long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int j = (int)((c / nx) % ny);
    const float u = UR[j];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float cu = CX(q) * u;
        const float dev = WQ(q) * (3.0f * cu + 4.5f * cu * cu - 1.5f * u * u);
        const float base = S::ROWBASE ? rowbase[j * RB_W + q] : 0.0f;
        S::st(f + q * ncell + c, S::SHIFTED ? dev - base : dev + WQ(q));
    }
}

// rho = sum f*, rho u = sum f* c - F/2 of the stored post-collision state
template <class S>
__global__ void fields_kernel(const typename S::T *f, const float *rowbase, const float *fw, float *rho,
                              float *u, int nx, int ny, int nz, long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int jr = (int)((c / nx) % ny);
    float v[19];
#pragma unroll
    for (int q = 0; q < 19; ++q)
        v[q] = S::ld(f + q * ncell + c) + (S::ROWBASE ? rowbase[jr * RB_W + q] : 0.0f) - (S::SHIFTED ? 0.0f : WQ(q));
    float dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) { dr += v[q]; jx += CX(q) * v[q]; jy += CY(q) * v[q]; jz += CZ(q) * v[q]; }
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    if (j == 0 || j == ny - 1) {
        const float *F = fw + (((size_t)(j == 0 ? 0 : 1) * nz + k) * nx + i) * 3;
        jx -= 0.5f * F[0]; jy -= 0.5f * F[1]; jz -= 0.5f * F[2];
    }
    const float r = 1.0f + dr;
    rho[c] = r;
    u[3 * c] = jx / r; u[3 * c + 1] = jy / r; u[3 * c + 2] = jz / r;
}

// z-sums of the velocity moments added to the FP64 accumulators.  Block =
// 32 consecutive (i, j) columns x 8 chunks of z; each thread sums its chunk in
// FP32, the chunks are combined in shared memory and one thread per column adds
// the sample to the FP64 sums.  The blocks past the columns do the u_tau sums
// the same way, over 32 consecutive (wall, i) entries each.
constexpr int ST_COLS = 32, ST_CHUNKS = 8;
__global__ void __launch_bounds__(ST_COLS * ST_CHUNKS) stats_kernel(
        const float *__restrict__ ubuf, const float *__restrict__ utau, double *st, double *st_utau, int nx,
        int ny, int nz, long long ncell, int wall) {
    __shared__ float part[ST_CHUNKS][7][ST_COLS];
    const int col = threadIdx.x % ST_COLS, ch = threadIdx.x / ST_COLS;
    const int nxy = nx * ny;
    const int nblk_cols = (nxy + ST_COLS - 1) / ST_COLS;
    if ((int)blockIdx.x < nblk_cols) {
        const int t = blockIdx.x * ST_COLS + col;
        float s[7] = {0, 0, 0, 0, 0, 0, 0};
        if (t < nxy) {
#pragma unroll 4
            for (int k = ch; k < nz; k += ST_CHUNKS) {
                const long long c = (long long)k * nxy + t;
                const float u = ubuf[c], v = ubuf[ncell + c], w = ubuf[2 * ncell + c];
                s[0] += u; s[1] += v; s[2] += w;
                s[3] = fmaf(u, u, s[3]); s[4] = fmaf(v, v, s[4]); s[5] = fmaf(w, w, s[5]); s[6] = fmaf(u, v, s[6]);
            }
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) part[ch][q][col] = s[q];
        __syncthreads();
        if (ch == 0 && t < nxy) {
            double *o = st + (size_t)t * 7;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                float a = 0.0f;
#pragma unroll
                for (int c = 0; c < ST_CHUNKS; ++c) a += part[c][q][col];
                o[q] += (double)a;
            }
        }
    } else if (wall) {
        const int r = ((int)blockIdx.x - nblk_cols) * ST_COLS + col;   // entry w * nx + i
        float s = 0.0f;
        if (r < 2 * nx) {
            const int w = r / nx, i = r % nx;
#pragma unroll 4
            for (int k = ch; k < nz; k += ST_CHUNKS) s += utau[((size_t)w * nz + k) * nx + i];
        }
        part[ch][0][col] = s;
        __syncthreads();
        if (ch == 0 && r < 2 * nx) {
            float a = 0.0f;
#pragma unroll
            for (int c = 0; c < ST_CHUNKS; ++c) a += part[c][0][col];
            st_utau[r] += (double)a;
        }
    }
}

// tau_w = |F_w| (= rho u_tau^2) averaged over z, per wall and x
// z-average of |F_w| (= tau_w) per wall and x: a block takes 32 x-columns
// of one wall, its 16 thread rows split z, and their FP32 partial sums are
// added in shared memory.
constexpr int WS_X = 32, WS_Z = 16;
__global__ void __launch_bounds__(WS_X * WS_Z) wall_shear_kernel(const float *fw, double *out, int nx, int nz) {
    __shared__ float part[WS_Z][WS_X];
    const int i = blockIdx.x * WS_X + threadIdx.x, w = blockIdx.y;
    float s = 0.0f;
    if (i < nx) {
#pragma unroll 8
        for (int k = threadIdx.y; k < nz; k += WS_Z) {
            const float *F = fw + (((size_t)w * nz + k) * nx + i) * 3;
            s += sqrtf(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
        }
    }
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && i < nx) {
        float t = 0.0f;
#pragma unroll
        for (int g = 0; g < WS_Z; ++g) t += part[g][threadIdx.x];
        out[(size_t)w * nx + i] = (double)t / nz;
    }
}

}  // namespace lbmk

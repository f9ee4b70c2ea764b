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
// Storage of one population: registers always hold the shifted value
// ft = f - w_q in FP32.
// ---------------------------------------------------------------------------
struct StoreF32 {
    using T = float;
    static __device__ __forceinline__ float ld(const float *p, float w) { return *p - w; }
    static __device__ __forceinline__ void st(float *p, float v, float w) { *p = v + w; }
};
struct StoreF16 {
    using T = __half;
    static __device__ __forceinline__ float ld(const __half *p, float) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v, float) { *p = __float2half_rn(v); }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// Reichardt law, Sec. 2.3 eq:reichard with the textbook coefficients
// (1/kappa, kappa, B), and its derivative in y+.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float reichardt_f(float yp, float kap, float B) {
    return log1pf(kap * yp) / kap + B * (1.0f - expf(-yp * (1.0f / 11.0f))
                                         - yp * (1.0f / 11.0f) * expf(-yp * (1.0f / 3.0f)));
}
__device__ __forceinline__ float reichardt_dy_f(float yp, float kap, float B) {
    const float e3 = expf(-yp * (1.0f / 3.0f));
    return 1.0f / (1.0f + kap * yp)
         + B * (expf(-yp * (1.0f / 11.0f)) * (1.0f / 11.0f) - e3 * (1.0f / 11.0f) + yp * (1.0f / 33.0f) * e3);
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
__device__ __noinline__ float solve_utau_dev(float uhat, float y1_nu, float kap, float B, float guess,
                                             bool *ok) {
    float u = guess > 0.0f ? guess : 1e-3f;
    for (int it = 0; it < 12; ++it) {
        const float yp = y1_nu * u;
        const float up = reichardt_f(yp, kap, B);
        const float r = u * up - uhat;
        const float dr = up + yp * reichardt_dy_f(yp, kap, B);
        const float du = r / dr;
        float un = u - du;
        if (!(un > 0.0f)) un = 0.5f * u;
        if (fabsf(du) <= 4e-7f * un) { *ok = true; return un; }
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
// f[] holds shifted populations f - w.  In: drho = rho - 1, momentum jx..jz
// (= sum f c), force density F.  The update is f* = f - M^T g with
// g_k = (s_k (m_k - m_k^eq) - (1 - s_k/2) (M F~)_k) / |row_k|^2, evaluated with
// sums s_p = f_p + f_{18-p} and differences d_p = f_p - f_{18-p} of the nine
// opposite pairs; the rows of M are the d'Humieres moments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void collide_mrt(float (&f)[19], float drho, float jx, float jy, float jz,
                                            float Fx, float Fy, float Fz, float tau0, float csm18,
                                            float &ux_o, float &uy_o, float &uz_o) {
    const float s0 = f[0] + f[18], d0 = f[0] - f[18];
    const float s1 = f[1] + f[17], d1 = f[1] - f[17];
    const float s2 = f[2] + f[16], d2 = f[2] - f[16];
    const float s3 = f[3] + f[15], d3 = f[3] - f[15];
    const float s4 = f[4] + f[14], d4 = f[4] - f[14];
    const float s5 = f[5] + f[13], d5 = f[5] - f[13];
    const float s6 = f[6] + f[12], d6 = f[6] - f[12];
    const float s7 = f[7] + f[11], d7 = f[7] - f[11];
    const float s8 = f[8] + f[10], d8 = f[8] - f[10];
    const float f9 = f[9];

    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    // eq:momentum: rho u = sum f c + F/2
    const float rux = jx + 0.5f * Fx, ruy = jy + 0.5f * Fy, ruz = jz + 0.5f * Fz;
    const float ux = rux * irho, uy = ruy * irho, uz = ruz * irho;
    ux_o = ux; uy_o = uy; uz_o = uz;
    const float uxx = rux * ux, uyy = ruy * uy, uzz = ruz * uz;       // rho u_a u_a
    const float uxy = rux * uy, uyz = ruy * uz, uxz = rux * uz;
    const float usq = uxx + uyy + uzz;

    // non-equilibrium moments n_k = m_k - m_k^eq (m of f, shifted: M w = (1,-11,3,0...))
    const float Sax = s2 + s6 + s8;
    const float Sdg = (s0 + s4) + (s1 + s3) + (s5 + s7);
    const float n1 = -30.0f * f9 - 11.0f * Sax + 8.0f * Sdg + 11.0f * drho - 19.0f * usq;
    const float n2 = 12.0f * f9 - 4.0f * Sax + Sdg - 3.0f * drho + 5.5f * usq;
    const float Dx = (d3 - d1) + (d7 - d5);
    const float Dy = (d4 - d0) - (d5 + d7);
    const float Dz = -(d0 + d4) - (d1 + d3);
    const float n4 = Dx + 4.0f * d8 + (2.0f / 3.0f) * rux;   // q_x + 2/3 rho u_x
    const float n6 = Dy + 4.0f * d6 + (2.0f / 3.0f) * ruy;
    const float n8 = Dz + 4.0f * d2 + (2.0f / 3.0f) * ruz;
    const float s04 = s0 + s4, s13 = s1 + s3, s57 = s5 + s7;
    const float pxx_eq = 2.0f * uxx - uyy - uzz;                   // m9^eq
    const float pww_eq = uyy - uzz;                                // m11^eq
    const float n9 = 2.0f * s8 - s2 - s6 - 2.0f * s04 + s13 + s57 - pxx_eq;
    const float n10 = -4.0f * s8 + 2.0f * (s2 + s6) - 2.0f * s04 + s13 + s57 + 0.5f * pxx_eq;
    const float n11 = (s6 - s2) + s57 - s13 - pww_eq;
    const float n12 = 2.0f * (s2 - s6) + s57 - s13 + 0.5f * pww_eq;
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
    // eq:tau_eff: tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt2 C Q^(1/2) / rho)) / 2
    const float te = 0.5f * (tau0 + sqrtf(tau0 * tau0 + csm18 * sqrtf(qq) * irho));
    const float sv = 1.0f / te;

    // moments of the Guo source M F~ (second-order Hermite form)
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float F9 = 4.0f * ux * Fx - 2.0f * (uy * Fy + uz * Fz);
    const float F11 = 2.0f * (uy * Fy - uz * Fz);
    const float F13 = ux * Fy + uy * Fx, F14 = uy * Fz + uz * Fy, F15 = ux * Fz + uz * Fx;

    const float g1 = (S_E * n1 - (1.0f - 0.5f * S_E) * 38.0f * uF) * (1.0f / 2394.0f);
    const float g2 = (S_EPS * n2 + (1.0f - 0.5f * S_EPS) * 11.0f * uF) * (1.0f / 252.0f);
    const float g3 = -0.1f * Fx, g5 = -0.1f * Fy, g7 = -0.1f * Fz;
    const float cq = (1.0f - 0.5f * S_Q) * (2.0f / 3.0f);
    const float g4 = (S_Q * n4 + cq * Fx) * (1.0f / 40.0f);
    const float g6 = (S_Q * n6 + cq * Fy) * (1.0f / 40.0f);
    const float g8 = (S_Q * n8 + cq * Fz) * (1.0f / 40.0f);
    const float hv = 1.0f - 0.5f * sv;
    const float g9 = (sv * n9 - hv * F9) * (1.0f / 36.0f);
    const float g10 = (S_PI * n10 + (1.0f - 0.5f * S_PI) * 0.5f * F9) * (1.0f / 72.0f);
    const float g11 = (sv * n11 - hv * F11) * (1.0f / 12.0f);
    const float g12 = (S_PI * n12 + (1.0f - 0.5f * S_PI) * 0.5f * F11) * (1.0f / 24.0f);
    const float g13 = (sv * n13 - hv * F13) * 0.25f;
    const float g14 = (sv * n14 - hv * F14) * 0.25f;
    const float g15 = (sv * n15 - hv * F15) * 0.25f;
    const float g16 = S_M * n16 * 0.125f, g17 = S_M * n17 * 0.125f, g18 = S_M * n18 * 0.125f;

    // f* = f - M^T g, by opposite pairs: even part E (same for p and 18-p),
    // odd part O (sign flips).
    const float Aax = -11.0f * g1 - 4.0f * g2;
    const float Ddg = 8.0f * g1 + g2;
    const float Jx = g3 + g4, Jy = g5 + g6, Jz = g7 + g8;
    const float g9_10 = g9 + g10, g11_12 = g11 + g12;
    float E, O;
    E = Ddg - 2.0f * g9_10 + g14;              O = -Jy - Jz - g17 + g18;      // pair 0/18
    f[0] -= E + O; f[18] -= E - O;
    E = Ddg + g9_10 - g11_12 + g15;            O = -Jx - Jz + g16 - g18;      // pair 1/17
    f[1] -= E + O; f[17] -= E - O;
    E = Aax - g9 + 2.0f * g10 - g11 + 2.0f * g12; O = -g7 + 4.0f * g8;        // pair 2/16
    f[2] -= E + O; f[16] -= E - O;
    E = Ddg + g9_10 - g11_12 - g15;            O = Jx - Jz - g16 - g18;       // pair 3/15
    f[3] -= E + O; f[15] -= E - O;
    E = Ddg - 2.0f * g9_10 - g14;              O = Jy - Jz + g17 + g18;       // pair 4/14
    f[4] -= E + O; f[14] -= E - O;
    E = Ddg + g9_10 + g11_12 + g13;            O = -Jx - Jy - g16 + g17;      // pair 5/13
    f[5] -= E + O; f[13] -= E - O;
    E = Aax - g9 + 2.0f * g10 + g11 - 2.0f * g12; O = -g5 + 4.0f * g6;        // pair 6/12
    f[6] -= E + O; f[12] -= E - O;
    E = Ddg + g9_10 + g11_12 - g13;            O = Jx - Jy + g16 + g17;       // pair 7/11
    f[7] -= E + O; f[11] -= E - O;
    E = Aax + 2.0f * g9 - 4.0f * g10;          O = -g3 + 4.0f * g4;           // pair 8/10
    f[8] -= E + O; f[10] -= E - O;
    f[9] += 30.0f * g1 - 12.0f * g2;
}

// ---------------------------------------------------------------------------
// Arguments of the fused step kernel.
// ---------------------------------------------------------------------------
template <class S>
struct StepArgs {
    const typename S::T *__restrict__ fin;   // post-collision state, read by pull
    typename S::T *__restrict__ fout;        // new post-collision state
    const float *__restrict__ uin;           // [nz][ny][3] inlet velocity of this step
    float *__restrict__ utau;                // [2][nz][nx] wall friction velocity
    float *__restrict__ fw;                  // [2][nz][nx][3] wall force of this step
    float *__restrict__ ubuf;                // [3][ncell] velocity (statistics steps)
    unsigned *__restrict__ flags;            // [0] Newton failures, [1] divergence
    long long *__restrict__ t_dev;           // STG time, advanced once per step
    long long ncell;
    int nx, ny, nz;
    int inlet, wall_model;
    float tau0, csm18;                       // tau0, 18 sqrt2 C_smag
    float y1_nu, kappa, B;                   // y1 / nu, Reichardt constants
};

constexpr int BY = 2;  // rows per block: (0,1) and (ny-2,ny-1) share a block

// One time step of Algorithm 1 for every cell: pull streaming with the
// boundary rules, regularized STG inlet at x = 0 (steps 6-8), Reichardt wall
// force on j = 0 and j = ny-1 (steps 9-14), MRT-LES collision (step 15).
template <class S, bool STATS>
__global__ void __launch_bounds__(128) step_kernel(const StepArgs<S> a) {
    using T = typename S::T;
    __shared__ float su2[128 / BY][3];

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * blockDim.x + tx;
    const int j = blockIdx.y * BY + ty;
    const int k = blockIdx.z;
    const bool valid = i < nx;
    const int ic = valid ? i : nx - 1;
    const long long N = a.ncell;

    // pull sources: x - c_x with a clamp (inlet / zero-gradient outlet) or wrap
    int xm = ic - 1, xp = ic + 1;
    if (a.inlet) { xm = max(xm, 0); xp = min(xp, nx - 1); }
    else { xm = xm < 0 ? nx - 1 : xm; xp = xp >= nx ? 0 : xp; }
    const int km = k == 0 ? nz - 1 : k - 1;          // source plane for c_z = +1
    const int kp = k == nz - 1 ? 0 : k + 1;          // source plane for c_z = -1
    const bool bot = j == 0, top = j == ny - 1;
    const int jm = bot ? 0 : j - 1;                  // for c_y = +1 (mirror at the bottom wall)
    const int jp = top ? j : j + 1;                  // for c_y = -1 (mirror at the top wall)
    const int rk = k * ny, rkm = km * ny, rkp = kp * ny;
    // row starts
    const int r00 = (rk + j) * nx, r0m = (rkm + j) * nx, r0p = (rkp + j) * nx;
    const int rm0 = (rk + jm) * nx, rmm = (rkm + jm) * nx, rmp = (rkp + jm) * nx;
    const int rp0 = (rk + jp) * nx, rpm = (rkm + jp) * nx, rpp = (rkp + jp) * nx;
    // specular slip walls: a population leaving through the wall comes back
    // with c_y mirrored from the same cell row (mirror pairs 0-4, 5-11, 6-12,
    // 7-13, 14-18).
    const long long mt4 = top ? 4 * N : 0, mt6 = top ? 6 * N : 0;
    const long long mb4 = bot ? -4 * N : 0, mb6 = bot ? -6 * N : 0;
    const T *fi = a.fin;

    float f[19];
    f[0] = S::ld(fi + 0 * N + mt4 + rpp + ic, WQ(0));
    f[1] = S::ld(fi + 1 * N + r0p + xp, WQ(1));
    f[2] = S::ld(fi + 2 * N + r0p + ic, WQ(2));
    f[3] = S::ld(fi + 3 * N + r0p + xm, WQ(3));
    f[4] = S::ld(fi + 4 * N + mb4 + rmp + ic, WQ(4));
    f[5] = S::ld(fi + 5 * N + mt6 + rp0 + xp, WQ(5));
    f[6] = S::ld(fi + 6 * N + mt6 + rp0 + ic, WQ(6));
    f[7] = S::ld(fi + 7 * N + mt6 + rp0 + xm, WQ(7));
    f[8] = S::ld(fi + 8 * N + r00 + xp, WQ(8));
    f[9] = S::ld(fi + 9 * N + r00 + ic, WQ(9));
    f[10] = S::ld(fi + 10 * N + r00 + xm, WQ(10));
    f[11] = S::ld(fi + 11 * N + mb6 + rm0 + xp, WQ(11));
    f[12] = S::ld(fi + 12 * N + mb6 + rm0 + ic, WQ(12));
    f[13] = S::ld(fi + 13 * N + mb6 + rm0 + xm, WQ(13));
    f[14] = S::ld(fi + 14 * N + mt4 + rpm + ic, WQ(14));
    f[15] = S::ld(fi + 15 * N + r0m + xp, WQ(15));
    f[16] = S::ld(fi + 16 * N + r0m + ic, WQ(16));
    f[17] = S::ld(fi + 17 * N + r0m + xm, WQ(17));
    f[18] = S::ld(fi + 18 * N + mb4 + rmm + ic, WQ(18));

    // ---- regularized velocity inlet (Sec. 3.1), lane with i = 0 only ----
    if (a.inlet && i == 0) {
        const float *up = a.uin + ((size_t)k * ny + j) * 3;
        const float vx = up[0], vy = up[1], vz = up[2];
        // Zou-He density from the known populations (c_x <= 0)
        const float sk = (f[0] + f[2] + f[4] + f[6] + f[9] + f[12] + f[14] + f[16] + f[18])
                       + 2.0f * (f[1] + f[5] + f[8] + f[11] + f[15]);
        const float rin = (1.0f + sk) / (1.0f - vx);
        const float drin = rin - 1.0f;
        const float vv = vx * vx + vy * vy + vz * vz;
        float feq[19], fneq[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const float cu = CX(q) * vx + CY(q) * vy + CZ(q) * vz;
            feq[q] = WQ(q) * (drin + rin * (3.0f * cu + 4.5f * cu * cu - 1.5f * vv));
        }
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            // unknown populations (c_x > 0) take f^neq of the opposite direction
            fneq[q] = CX(q) > 0 ? (f[18 - q] - feq[18 - q]) : (f[q] - feq[q]);
        }
        float pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pxz = 0, tr = 0;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            pxx += CX(q) * CX(q) * fneq[q]; pyy += CY(q) * CY(q) * fneq[q]; pzz += CZ(q) * CZ(q) * fneq[q];
            pxy += CX(q) * CY(q) * fneq[q]; pyz += CY(q) * CZ(q) * fneq[q]; pxz += CX(q) * CZ(q) * fneq[q];
            tr += fneq[q];
        }
        // Pi_neq = sum_q Q_q f^neq_q, Q_q = c c - I/3
        pxx -= tr * (1.0f / 3.0f); pyy -= tr * (1.0f / 3.0f); pzz -= tr * (1.0f / 3.0f);
        const float trp = (pxx + pyy + pzz) * (1.0f / 3.0f);
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const float qp = CX(q) * CX(q) * pxx + CY(q) * CY(q) * pyy + CZ(q) * CZ(q) * pzz
                           + 2.0f * (CX(q) * CY(q) * pxy + CY(q) * CZ(q) * pyz + CX(q) * CZ(q) * pxz) - trp;
            f[q] = feq[q] + 4.5f * WQ(q) * qp;   // w / (2 cs^4) = 9 w / 2
        }
    }

    // ---- macroscopic moments (eq:density, eq:momentum without the force) ----
    float drho = 0.0f;
#pragma unroll
    for (int q = 0; q < 19; ++q) drho += f[q];
    const float jx = (f[3] + f[7] + f[10] + f[13] + f[17]) - (f[1] + f[5] + f[8] + f[11] + f[15]);
    const float jy = (f[4] + f[11] + f[12] + f[13] + f[18]) - (f[0] + f[5] + f[6] + f[7] + f[14]);
    const float jz = (f[14] + f[15] + f[16] + f[17] + f[18]) - (f[0] + f[1] + f[2] + f[3] + f[4]);

    // ---- wall model (Sec. 2.3) on the first off-wall cells ----
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    const bool wall_block = a.wall_model && (blockIdx.y == 0 || blockIdx.y == gridDim.y - 1);
    if (wall_block) {                                   // block-uniform
        const bool is_wall = bot || top;
        const float irho = 1.0f / (1.0f + drho);
        if (!is_wall) { su2[tx][0] = jx * irho; su2[tx][1] = jy * irho; su2[tx][2] = jz * irho; }
        __syncthreads();
        if (is_wall && valid) {
            const int w = bot ? 0 : 1;
            const float ny_ = bot ? 1.0f : -1.0f;      // wall normal into the fluid
            const float u2x = su2[tx][0], u2y = su2[tx][1], u2z = su2[tx][2];
            // eq:base: tangential part of u_2, normalized
            const float un = u2y * ny_;
            const float tx_ = u2x, ty_ = u2y - un * ny_, tz_ = u2z;
            const float tn = sqrtf(tx_ * tx_ + ty_ * ty_ + tz_ * tz_);
            float *utp = a.utau + ((size_t)w * nz + k) * nx + i;
            if (tn >= 1e-12f) {
                const float ex = tx_ / tn, ey = ty_ / tn, ez = tz_ / tn;
                // eq:uhat with the first-cell velocity (no half-force term)
                const float uhat = (jx * ex + jy * ey + jz * ez) * irho;
                const float sg = uhat < 0.0f ? -1.0f : 1.0f;
                const float ua = fabsf(uhat);
                float ut = 0.0f;
                if (ua > 0.0f) {
                    bool ok;
                    ut = solve_utau_dev(ua, a.y1_nu, a.kappa, a.B, *utp, &ok);
                    if (!ok) atomicAdd(a.flags, 1u);
                }
                *utp = ut;
                // tau_w = rho u_tau^2, eq:force_wm with A = 1
                const float tw = (1.0f + drho) * ut * ut * sg;
                Fx = -tw * ex; Fy = -tw * ey; Fz = -tw * ez;
            }
            float *fwp = a.fw + (((size_t)w * nz + k) * nx + i) * 3;
            fwp[0] = Fx; fwp[1] = Fy; fwp[2] = Fz;
        }
    }

    float ux, uy, uz;
    collide_mrt(f, drho, jx, jy, jz, Fx, Fy, Fz, a.tau0, a.csm18, ux, uy, uz);

    if (!valid) return;
    const long long c = r00 + i;
    T *fo = a.fout;
#pragma unroll
    for (int q = 0; q < 19; ++q) S::st(fo + q * N + c, f[q], WQ(q));

    if (STATS) {
        a.ubuf[c] = ux; a.ubuf[N + c] = uy; a.ubuf[2 * N + c] = uz;
    }
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(uu < 0.09f)) atomicAdd(a.flags + 1, 1u);        // also catches NaN
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tx == 0 && ty == 0) *a.t_dev += 1;
}

// ---------------------------------------------------------------------------
// STG inlet velocity (Sec. 3.1 eq:u_couple, eq:v_fluc, eq:aux_vec).  One warp
// per inlet cell; lanes split the N modes and reduce by warp shuffles.  The
// phase k_n d_n . x' + phi_n is carried in 32-bit fixed-point turns:
//   alpha[j][n] = k_n d_ny y_j / 2pi,  beta[k][n] = k_n d_nz z_k / 2pi,
//   phi32[n] = phi_n / 2pi,  time part -nu_n t with nu_n = d_nx U_b / max l_e
// in 64-bit fixed point, so the argument stays exact for any t.
// ---------------------------------------------------------------------------
struct StgArgs {
    const uint32_t *__restrict__ alpha;   // [ny][N]
    const uint32_t *__restrict__ beta;    // [nz][N]
    const uint32_t *__restrict__ phi32;   // [N]
    const uint64_t *__restrict__ rate64;  // [N]  (-nu_n) in 2^-64 turns per step
    const float *__restrict__ sq;         // [ny][N] sqrt(6 q_n(y))
    const float *__restrict__ sig;        // [3][N] sigma_n
    const float *__restrict__ amat;       // [ny][6] amp * Cholesky factor
    const float *__restrict__ UR;         // [ny] mean profile
    float *__restrict__ uin;              // [nz][ny][3]
    const long long *__restrict__ t_dev;  // time (if not null) ...
    long long t_val;                      // ... else this time
    int ny, nz, n_modes;
};

__global__ void __launch_bounds__(256) stg_kernel(const StgArgs a) {
    const int lane = threadIdx.x & 31;
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= a.ny * a.nz) return;                  // whole warp
    const int j = cell % a.ny, k = cell / a.ny;
    const int N = a.n_modes;
    const uint64_t t = (uint64_t)(a.t_dev ? *a.t_dev : a.t_val);
    const uint32_t *al = a.alpha + (size_t)j * N;
    const uint32_t *be = a.beta + (size_t)k * N;
    const float *sq = a.sq + (size_t)j * N;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f;
    for (int n = lane; n < N; n += 32) {
        const uint32_t tt = (uint32_t)((a.rate64[n] * t) >> 32);
        const uint32_t ph = al[n] + be[n] + a.phi32[n] + tt;
        const float x = (float)(int32_t)ph * 1.4629180792671596e-09f;   // 2 pi / 2^32
        const float cw = sq[n] * __cosf(x);
        vx = fmaf(cw, a.sig[n], vx);
        vy = fmaf(cw, a.sig[N + n], vy);
        vz = fmaf(cw, a.sig[2 * N + n], vz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vx += __shfl_xor_sync(0xffffffffu, vx, o);
        vy += __shfl_xor_sync(0xffffffffu, vy, o);
        vz += __shfl_xor_sync(0xffffffffu, vz, o);
    }
    if (lane == 0) {
        const float *m = a.amat + 6 * j;
        float *o = a.uin + ((size_t)k * a.ny + j) * 3;
        o[0] = a.UR[j] + m[0] * vx;
        o[1] = m[1] * vx + m[2] * vy;
        o[2] = m[3] * vx + m[4] * vy + m[5] * vz;
    }
}

// ---------------------------------------------------------------------------
// Initial state f^eq(1, (U_R(y), 0, 0)) and the diagnostics kernels.
// ---------------------------------------------------------------------------
template <class S>
__global__ void init_kernel(typename S::T *f, const float *UR, int nx, int ny, long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int j = (int)((c / nx) % ny);
    const float u = UR[j];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float cu = CX(q) * u;
        S::st(f + q * ncell + c, WQ(q) * (3.0f * cu + 4.5f * cu * cu - 1.5f * u * u), WQ(q));
    }
}

// rho = sum f*, rho u = sum f* c - F/2 of the stored post-collision state
template <class S>
__global__ void fields_kernel(const typename S::T *f, const float *fw, float *rho, float *u, int nx,
                              int ny, int nz, long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    float v[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) v[q] = S::ld(f + q * ncell + c, WQ(q));
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

// z-sums of the velocity moments and of u_tau, accumulated in FP64
__global__ void stats_kernel(const float *ubuf, const float *utau, double *st, double *st_utau, int nx,
                             int ny, int nz, long long ncell, int wall) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nx * ny) {
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < nz; ++k) {
            const long long c = (long long)k * nx * ny + t;
            const double u = ubuf[c], v = ubuf[ncell + c], w = ubuf[2 * ncell + c];
            s[0] += u; s[1] += v; s[2] += w; s[3] += u * u; s[4] += v * v; s[5] += w * w; s[6] += u * v;
        }
        double *o = st + (size_t)t * 7;
#pragma unroll
        for (int q = 0; q < 7; ++q) o[q] += s[q];
    } else if (wall && t < nx * ny + 2 * nx) {
        const int r = t - nx * ny, w = r / nx, i = r % nx;
        double s = 0;
        for (int k = 0; k < nz; ++k) s += utau[((size_t)w * nz + k) * nx + i];
        st_utau[w * nx + i] += s;
    }
}

// tau_w = |F_w| (= rho u_tau^2) averaged over z, per wall and x
__global__ void wall_shear_kernel(const float *fw, double *out, int nx, int nz) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * nx) return;
    const int w = t / nx, i = t % nx;
    double s = 0;
    for (int k = 0; k < nz; ++k) {
        const float *F = fw + (((size_t)w * nz + k) * nx + i) * 3;
        s += sqrt((double)F[0] * F[0] + (double)F[1] * F[1] + (double)F[2] * F[2]);
    }
    out[t] = s / nz;
}

}  // namespace lbmk

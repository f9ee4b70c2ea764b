// lbm_adjoint.cuh -- hand-written adjoint (vector-Jacobian product) of one
// fused time step, for gradients of a downstream objective with respect to the
// state and to theta = (ell_e, amp, kappa, B).
//
// Forward step (state = post-collision populations, FP32):
//   p = Pull(s_n) -> [x = 0: p = Rebuild(p_known, u_in)] -> wall force F(p, p_2)
//     -> s_{n+1} = C(p, F).
// Reverse: given lambda = dJ/ds_{n+1} at every cell, recompute the forward
// values of the cell, run the chain backwards (collision, SGS closure,
// equilibrium, Guo force, Reichardt wall model through the implicit function
// theorem, regularized inlet) and push the adjoint of every pulled population
// back to the cell and plane it was pulled from.  The pull is a permutation
// except at the x faces: the inlet's unknown populations are not read (their
// adjoint is zero), the outlet's clamped reads land on cells that the regular
// pull also reads (their adjoint goes to a side buffer added afterwards), and
// the two planes nobody reads get zeros.
#pragma once
#include "lbm_device.cuh"

namespace lbmk {

// adjoint of the collision inputs
struct AdjIn {
    float ls[9], ld[9];     // of the pair sums / differences
    float lf9;              // of f_9
    float lrho, ljx, ljy, ljz;   // of rho and of the momentum sum f c (before the force)
    float lFx, lFy, lFz;    // of the force density
};

// Forward recompute and reverse of collide_mrt<false, HAS_FORCE> (FP32, f not
// shifted).  lam: dJ/df* of the cell.  (lux, luy, luz): direct dJ/du of the
// physical velocity (objective seeds).  Output: A (adjoint of the inputs; the
// identity part lam itself is added by the caller).
template <bool HAS_FORCE>
__device__ __forceinline__ void collide_adjoint(const float (&lam)[19], const Pairs &P, float f9, float Fx,
                                                float Fy, float Fz, float tau0, float csm18, float lux, float luy,
                                                float luz, AdjIn &A) {
    const float *s = P.s;
    // ---------------- forward values ----------------
    const float rho = 1.0f + P.drho, irho = rcp_approx(rho);
    const float rux = P.jx + 0.5f * Fx, ruy = P.jy + 0.5f * Fy, ruz = P.jz + 0.5f * Fz;
    const float ux = rux * irho, uy = ruy * irho, uz = ruz * irho;
    const float uxx = rux * ux, uyy = ruy * uy, uzz = ruz * uz;
    const float usq = uxx + uyy + uzz;
    const float Sax = s[2] + s[6] + s[8];
    const float Sdg = (s[0] + s[4]) + (s[1] + s[3]) + (s[5] + s[7]);
    const float n1 = -30.0f * f9 - 11.0f * Sax + 8.0f * Sdg + 11.0f * rho - 19.0f * usq;
    const float s04 = s[0] + s[4], s13 = s[1] + s[3], s57 = s[5] + s[7];
    const float pxx_eq = 2.0f * uxx - uyy - uzz, pww_eq = uyy - uzz;
    const float n9 = 2.0f * s[8] - (s[2] + s[6]) - 2.0f * s04 + (s13 + s57) - pxx_eq;
    const float n11 = (s[6] - s[2]) + (s57 - s13) - pww_eq;
    const float n13 = (s[5] - s[7]) - rux * uy;
    const float n14 = (s[0] - s[4]) - ruy * uz;
    const float n15 = (s[1] - s[3]) - rux * uz;
    const float c2 = n1 * (1.0f / 19.0f);
    const float pxx = (c2 + n9) * (1.0f / 3.0f);
    const float pyy = (c2 - 0.5f * n9 + 1.5f * n11) * (1.0f / 3.0f);
    const float pzz = (c2 - 0.5f * n9 - 1.5f * n11) * (1.0f / 3.0f);
    const float qq = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (n13 * n13 + n14 * n14 + n15 * n15);
    const float Qh = sqrt_approx(qq);
    const float Rr = sqrt_approx(tau0 * tau0 + csm18 * Qh * irho);
    const float sv = 2.0f * rcp_approx(tau0 + Rr);
    const float hv = 1.0f - 0.5f * sv;
    float F9 = 0.f, F11 = 0.f, F13 = 0.f, F14 = 0.f, F15 = 0.f;
    if (HAS_FORCE) {
        F9 = 4.0f * ux * Fx - 2.0f * (uy * Fy + uz * Fz);
        F11 = 2.0f * (uy * Fy - uz * Fz);
        F13 = ux * Fy + uy * Fx; F14 = uy * Fz + uz * Fy; F15 = ux * Fz + uz * Fx;
    }
    // ---------------- mu = M lambda ----------------
    float ls[9], ld[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) { ls[p] = lam[p] + lam[18 - p]; ld[p] = lam[p] - lam[18 - p]; }
    const float l9 = lam[9];
    const float LSax = ls[2] + ls[6] + ls[8];
    const float LSdg = (ls[0] + ls[4]) + (ls[1] + ls[3]) + (ls[5] + ls[7]);
    const float m1 = -30.0f * l9 - 11.0f * LSax + 8.0f * LSdg;
    const float m2 = 12.0f * l9 - 4.0f * LSax + LSdg;
    const float DX = (ld[3] - ld[1]) + (ld[7] - ld[5]);
    const float DY = (ld[4] - ld[0]) - (ld[5] + ld[7]);
    const float DZ = -(ld[0] + ld[4]) - (ld[1] + ld[3]);
    const float m3 = DX - ld[8], m4 = DX + 4.0f * ld[8];
    const float m5 = DY - ld[6], m6 = DY + 4.0f * ld[6];
    const float m7 = DZ - ld[2], m8 = DZ + 4.0f * ld[2];
    const float L04 = ls[0] + ls[4], L13 = ls[1] + ls[3], L57 = ls[5] + ls[7];
    const float m9 = 2.0f * ls[8] - (ls[2] + ls[6]) - 2.0f * L04 + (L13 + L57);
    const float m10 = -4.0f * ls[8] + 2.0f * (ls[2] + ls[6]) - 2.0f * L04 + (L13 + L57);
    const float m11 = (ls[6] - ls[2]) + (L57 - L13);
    const float m12 = 2.0f * (ls[2] - ls[6]) + (L57 - L13);
    const float m13 = ls[5] - ls[7], m14 = ls[0] - ls[4], m15 = ls[1] - ls[3];
    const float m16 = (ld[1] - ld[3]) + (ld[7] - ld[5]);
    const float m17 = (ld[4] - ld[0]) + (ld[5] + ld[7]);
    const float m18 = (ld[0] + ld[4]) - (ld[1] + ld[3]);
    // L = lambda . f* = lambda . f - sum_k mu_k G_k  ->  a_k = dL/dG_k = -mu_k
    // ---------------- reverse through G ----------------
    float bn1 = -m1 * (S_E / 2394.0f);
    float bn2 = -m2 * (S_EPS / 252.0f);
    const float bn4 = -m4 * (S_Q / 40.0f), bn6 = -m6 * (S_Q / 40.0f), bn8 = -m8 * (S_Q / 40.0f);
    float bn9 = -m9 * sv * (1.0f / 36.0f);
    const float bn10 = -m10 * (S_PI / 72.0f);
    float bn11 = -m11 * sv * (1.0f / 12.0f);
    const float bn12 = -m12 * (S_PI / 24.0f);
    float bn13 = -m13 * sv * 0.25f, bn14 = -m14 * sv * 0.25f, bn15 = -m15 * sv * 0.25f;
    const float bn16 = -m16 * S_M * 0.125f, bn17 = -m17 * S_M * 0.125f, bn18 = -m18 * S_M * 0.125f;
    // d/dsv of (sv n - (1 - sv/2) F) = n + F/2
    float bsv = -m9 * (n9 + 0.5f * F9) * (1.0f / 36.0f) - m11 * (n11 + 0.5f * F11) * (1.0f / 12.0f)
              - (m13 * (n13 + 0.5f * F13) + m14 * (n14 + 0.5f * F14) + m15 * (n15 + 0.5f * F15)) * 0.25f;
    float lFx = 0.f, lFy = 0.f, lFz = 0.f;
    float lux_ = lux, luy_ = luy, luz_ = luz;
    if (HAS_FORCE) {
        const float cq = (1.0f - 0.5f * S_Q) * (2.0f / 3.0f);
        const float buF = m1 * ((1.0f - 0.5f * S_E) * 38.0f / 2394.0f) - m2 * ((1.0f - 0.5f * S_EPS) * 11.0f / 252.0f);
        lFx += 0.1f * m3 - m4 * (cq * (1.0f / 40.0f));
        lFy += 0.1f * m5 - m6 * (cq * (1.0f / 40.0f));
        lFz += 0.1f * m7 - m8 * (cq * (1.0f / 40.0f));
        const float bF9 = m9 * hv * (1.0f / 36.0f) - m10 * ((1.0f - 0.5f * S_PI) * 0.5f / 72.0f);
        const float bF11 = m11 * hv * (1.0f / 12.0f) - m12 * ((1.0f - 0.5f * S_PI) * 0.5f / 24.0f);
        const float bF13 = m13 * hv * 0.25f, bF14 = m14 * hv * 0.25f, bF15 = m15 * hv * 0.25f;
        // uF = u . F
        lux_ += buF * Fx; luy_ += buF * Fy; luz_ += buF * Fz;
        lFx += buF * ux; lFy += buF * uy; lFz += buF * uz;
        // F9 = 4 ux Fx - 2 uy Fy - 2 uz Fz
        lux_ += 4.0f * Fx * bF9; lFx += 4.0f * ux * bF9;
        luy_ -= 2.0f * Fy * bF9; lFy -= 2.0f * uy * bF9;
        luz_ -= 2.0f * Fz * bF9; lFz -= 2.0f * uz * bF9;
        // F11 = 2 uy Fy - 2 uz Fz
        luy_ += 2.0f * Fy * bF11; lFy += 2.0f * uy * bF11;
        luz_ -= 2.0f * Fz * bF11; lFz -= 2.0f * uz * bF11;
        // F13 = ux Fy + uy Fx, F14 = uy Fz + uz Fy, F15 = ux Fz + uz Fx
        lux_ += Fy * bF13; lFy += ux * bF13; luy_ += Fx * bF13; lFx += uy * bF13;
        luy_ += Fz * bF14; lFz += uy * bF14; luz_ += Fy * bF14; lFy += uz * bF14;
        lux_ += Fz * bF15; lFz += ux * bF15; luz_ += Fx * bF15; lFx += uz * bF15;
    }
    // ---------------- SGS: sv = 2 / (tau0 + sqrt(tau0^2 + c Qh / rho)) ----------------
    float lirho = 0.f;
    {
        const float lR = bsv * (-0.5f * sv * sv);
        const float lX = lR * 0.5f * rcp_approx(Rr);
        const float lQh = lX * csm18 * irho;
        lirho += lX * csm18 * Qh;
        const float lqq = Qh > 1e-30f ? lQh * 0.5f * rcp_approx(Qh) : 0.0f;
        const float lpxx = 2.0f * pxx * lqq, lpyy = 2.0f * pyy * lqq, lpzz = 2.0f * pzz * lqq;
        bn13 += 4.0f * n13 * lqq; bn14 += 4.0f * n14 * lqq; bn15 += 4.0f * n15 * lqq;
        const float lc2 = (lpxx + lpyy + lpzz) * (1.0f / 3.0f);
        bn9 += (lpxx - 0.5f * lpyy - 0.5f * lpzz) * (1.0f / 3.0f);
        bn11 += (1.5f * lpyy - 1.5f * lpzz) * (1.0f / 3.0f);
        bn1 += lc2 * (1.0f / 19.0f);
    }
    // ---------------- n_k -> pair moments, rho, rho u ----------------
    float las[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, lad[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    float lf9 = 0.f, lrho = 0.f, lusq = 0.f;
    float lrux = 0.f, lruy = 0.f, lruz = 0.f, ljx = 0.f, ljy = 0.f, ljz = 0.f;
    // n1 = e1 + 11 rho - 19 usq, n2 = e2 - 3 rho + 5.5 usq
    lrho += 11.0f * bn1 - 3.0f * bn2;
    lusq += -19.0f * bn1 + 5.5f * bn2;
    lf9 += -30.0f * bn1 + 12.0f * bn2;
    const float lSax = -11.0f * bn1 - 4.0f * bn2, lSdg = 8.0f * bn1 + bn2;
    las[2] += lSax; las[6] += lSax; las[8] += lSax;
    las[0] += lSdg; las[4] += lSdg; las[1] += lSdg; las[3] += lSdg; las[5] += lSdg; las[7] += lSdg;
    // n4 = jx + 5 d8 + 2/3 rux (and y, z)
    ljx += bn4; lad[8] += 5.0f * bn4; lrux += (2.0f / 3.0f) * bn4;
    ljy += bn6; lad[6] += 5.0f * bn6; lruy += (2.0f / 3.0f) * bn6;
    ljz += bn8; lad[2] += 5.0f * bn8; lruz += (2.0f / 3.0f) * bn8;
    // n9, n10 and the equilibrium part pxx_eq
    las[8] += 2.0f * bn9 - 4.0f * bn10;
    las[2] += -bn9 + 2.0f * bn10; las[6] += -bn9 + 2.0f * bn10;
    las[0] += -2.0f * bn9 - 2.0f * bn10; las[4] += -2.0f * bn9 - 2.0f * bn10;
    las[1] += bn9 + bn10; las[3] += bn9 + bn10; las[5] += bn9 + bn10; las[7] += bn9 + bn10;
    const float lpxxeq = -bn9 + 0.5f * bn10;
    // n11, n12 and pww_eq
    las[6] += bn11 - 2.0f * bn12; las[2] += -bn11 + 2.0f * bn12;
    las[5] += bn11 + bn12; las[7] += bn11 + bn12; las[1] -= bn11 + bn12; las[3] -= bn11 + bn12;
    const float lpwweq = -bn11 + 0.5f * bn12;
    // n13..n15
    las[5] += bn13; las[7] -= bn13; las[0] += bn14; las[4] -= bn14; las[1] += bn15; las[3] -= bn15;
    const float luxy = -bn13, luyz = -bn14, luxz = -bn15;
    // n16..n18
    lad[1] += bn16 - bn18; lad[3] += -bn16 - bn18; lad[7] += bn16 + bn17; lad[5] += -bn16 + bn17;
    lad[4] += bn17 + bn18; lad[0] += -bn17 + bn18;
    // quadratic equilibrium terms: uxx = rux ux etc., uxy = rux uy, uyz = ruy uz, uxz = rux uz
    const float luxx = lusq + 2.0f * lpxxeq, luyy = lusq - lpxxeq + lpwweq, luzz = lusq - lpxxeq - lpwweq;
    lrux += ux * luxx + uy * luxy + uz * luxz; lux_ += rux * luxx;
    lruy += uy * luyy + uz * luyz;             luy_ += ruy * luyy + rux * luxy;
    lruz += uz * luzz;                         luz_ += ruz * luzz + ruy * luyz + rux * luxz;
    // u = ru / rho
    lrux += irho * lux_; lruy += irho * luy_; lruz += irho * luz_;
    lirho += rux * lux_ + ruy * luy_ + ruz * luz_;
    lrho += -irho * irho * lirho;
    // ru = j + F/2
    ljx += lrux; ljy += lruy; ljz += lruz;
    if (HAS_FORCE) { lFx += 0.5f * lrux; lFy += 0.5f * lruy; lFz += 0.5f * lruz; }
#pragma unroll
    for (int p = 0; p < 9; ++p) { A.ls[p] = las[p]; A.ld[p] = lad[p]; }
    A.lf9 = lf9; A.lrho = lrho; A.ljx = ljx; A.ljy = ljy; A.ljz = ljz;
    A.lFx = lFx; A.lFy = lFy; A.lFz = lFz;
}

// lambda of the pulled populations from the adjoint of (pairs, f9, rho, j):
// rho = 1 + sum s + f9 - 1, j from d, s_p = f_p + f_{18-p}, d_p = f_p - f_{18-p}.
__device__ __forceinline__ void adjoint_to_pops(const float (&lam)[19], AdjIn &A, float (&lp)[19]) {
    float ls[9], ld[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) { ls[p] = A.ls[p] + A.lrho; ld[p] = A.ld[p]; }
    const float lf9 = A.lf9 + A.lrho;
    // jx = (d3 - d1) + (d7 - d5) - d8 ; jy = (d4 - d0) - (d5 + d7) - d6 ; jz = -(d0 + d4) - (d1 + d3) - d2
    ld[3] += A.ljx; ld[1] -= A.ljx; ld[7] += A.ljx; ld[5] -= A.ljx; ld[8] -= A.ljx;
    ld[4] += A.ljy; ld[0] -= A.ljy; ld[5] -= A.ljy; ld[7] -= A.ljy; ld[6] -= A.ljy;
    ld[0] -= A.ljz; ld[4] -= A.ljz; ld[1] -= A.ljz; ld[3] -= A.ljz; ld[2] -= A.ljz;
#pragma unroll
    for (int p = 0; p < 9; ++p) { lp[p] = lam[p] + ls[p] + ld[p]; lp[18 - p] = lam[18 - p] + ls[p] - ld[p]; }
    lp[9] = lam[9] + lf9;
}

// Reichardt law derivatives for the implicit-function theorem:
// R(u) = u u+(y1 u / nu) - uhat; dR/du = u+ + y+ u+'; dR/dkappa = u du+/dkappa; dR/dB = u du+/dB.
__device__ __forceinline__ void reichardt_partials(float yp, float kap, float B, float &up, float &dup, float &dk,
                                                   float &dB) {
    // fast exponential / logarithm (kappa y+ >= ~1 at a first cell, where
    // log(1 + x) loses nothing): errors of a few ulp, far below the 1e-3 of
    // the gradients
    const float e11 = __expf(-yp * (1.0f / 11.0f)), e3 = __expf(-yp * (1.0f / 3.0f));
    const float l1 = __logf(1.0f + kap * yp);
    up = l1 * (1.0f / kap) + B * (1.0f - e11 - yp * (1.0f / 11.0f) * e3);
    dup = rcp_approx(1.0f + kap * yp) + B * (e11 * (1.0f / 11.0f) - e3 * (1.0f / 11.0f) + yp * (1.0f / 33.0f) * e3);
    dk = (-l1 + kap * yp * rcp_approx(1.0f + kap * yp)) * rcp_approx(kap * kap);
    dB = 1.0f - e11 - yp * (1.0f / 11.0f) * e3;
}

// ---------------------------------------------------------------------------
struct AdjArgs {
    const float *in[19];            // s_n (FP32 f), read by pull
    float *lam;                     // [19][ncell] dJ/ds_{n+1} (its outlet c_x < 0 entries are zeroed
                                    // once read: the buffer receives atomics in the next adjoint step)
    float *lout;                    // [19][ncell] dJ/ds_n (written by push; its outlet c_x < 0 entries
                                    // must be zero on entry)
    const float *__restrict__ utau;  // [2][nz][nx] u_tau of this step (the forward step's solution)
    const float *__restrict__ vprime;  // [nz][ny][3] STG field of this step
    const float *__restrict__ UR;
    const float *__restrict__ amat;
    float *__restrict__ luin;       // [nz][ny][3] dJ/du_in of this step (null: not needed)
    double *__restrict__ gtheta;    // [4] accumulated dJ/dtheta (wall-model part: kappa, B)
    // objective seeds (null: none)
    const float *__restrict__ jr_coef;  // [ny] 2 r_j / (u_tau^2 T nz) of J_R
    const float *__restrict__ jr_mean;  // [2][ny] <u>_j, <v>_j
    float jtau_w;                   // dJ/dtau_w of one wall cell (J_tau weight), 0 if none
    int i_tau0, i_tau1, i_R;
    int nx, ny, nz;
    int inlet, wall_model;
    float tau0, csm18, y1_nu, kappa, B;
    float sp_x0, sp_inv, sp_3nu;    // outlet sponge as in StepArgs
};

// Pull source of population q (compile-time after unrolling) from the
// per-cell row offsets of the forward kernel: plane (mirrored at a slip wall)
// and cell offset.
struct PullGeom {
    int o00, ozm, ozp, oym, oyp, ic, xm, xp;
    bool bot, top;
};
__device__ __forceinline__ int src_plane(int q, const PullGeom &g) {
    return ((CY(q) < 0 && g.top) || (CY(q) > 0 && g.bot)) ? mirror_y(q) : q;
}
__device__ __forceinline__ int src_off(int q, const PullGeom &g) {
    const int oz = CZ(q) < 0 ? g.ozp : (CZ(q) > 0 ? g.ozm : 0);
    const int oy = CY(q) < 0 ? g.oyp : (CY(q) > 0 ? g.oym : 0);
    const int x = CX(q) < 0 ? g.xp : (CX(q) > 0 ? g.xm : g.ic);
    return g.o00 + oy + oz + x;
}

// Forward recomputation of the regularized inlet of the cell at x = 0 (as
// inlet_rebuild, with f holding f itself): u_in and rho_in are returned for
// the reverse.
__device__ __forceinline__ void adjoint_inlet_forward(const AdjArgs &a, float (&f)[19], int j, int k, float &vx,
                                                      float &vy, float &vz, float &rin) {
    const int ny = a.ny;
    const float *vp = a.vprime + ((size_t)k * ny + j) * 3;
    const float *m = a.amat + 6 * j;
    vx = a.UR[j] + m[0] * vp[0];
    vy = m[1] * vp[0] + m[2] * vp[1];
    vz = m[3] * vp[0] + m[4] * vp[1] + m[5] * vp[2];
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] -= WQ(q);
    const float sk = (f[0] + f[2] + f[4] + f[6] + f[9] + f[12] + f[14] + f[16] + f[18])
                   + 2.0f * (f[1] + f[5] + f[8] + f[11] + f[15]);
    rin = (1.0f + sk) * rcp_approx(1.0f - vx);
    const float drin = rin - 1.0f, vv = vx * vx + vy * vy + vz * vz;
    auto feq = [&](int q) {
        const float cu = CX(q) * vx + CY(q) * vy + CZ(q) * vz;
        return WQ(q) * (drin + rin * (3.0f * cu + 4.5f * cu * cu - 1.5f * vv));
    };
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
    pxx -= tr * (1.0f / 3.0f); pyy -= tr * (1.0f / 3.0f); pzz -= tr * (1.0f / 3.0f);
    const float trp = (pxx + pyy + pzz) * (1.0f / 3.0f);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float qp = CX(q) * CX(q) * pxx + CY(q) * CY(q) * pyy + CZ(q) * CZ(q) * pzz
                       + 2.0f * (CX(q) * CY(q) * pxy + CY(q) * CZ(q) * pyz + CX(q) * CZ(q) * pxz) - trp;
        f[q] = feq(q) + 4.5f * WQ(q) * qp + WQ(q);
    }
}

// Reverse of the regularized inlet: lp (adjoint of the rebuilt populations)
// becomes the adjoint of the pulled ones; dJ/du_in goes to a.luin.  f is
// scratch.
__device__ __forceinline__ void adjoint_inlet_reverse(const AdjArgs &a, float (&f)[19], float (&lp)[19], int j,
                                                      int k, float vx, float vy, float vz, float rin) {
    const int ny = a.ny;
    const float vv = vx * vx + vy * vy + vz * vz;
    // out_q = fe_q + 4.5 w_q (c c : Pi - tr Pi / 3) + w_q
    float lPxx = 0, lPyy = 0, lPzz = 0, lPxy = 0, lPyz = 0, lPxz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float lq = 4.5f * WQ(q) * lp[q];
        lPxx += (CX(q) * CX(q) - 1.0f / 3.0f) * lq; lPyy += (CY(q) * CY(q) - 1.0f / 3.0f) * lq;
        lPzz += (CZ(q) * CZ(q) - 1.0f / 3.0f) * lq;
        lPxy += 2.0f * CX(q) * CY(q) * lq; lPyz += 2.0f * CY(q) * CZ(q) * lq; lPxz += 2.0f * CX(q) * CZ(q) * lq;
    }
    // Pi = sum c c fn - I tr/3: adjoint of fn_q (kept in f[])
    const float ltr = -(lPxx + lPyy + lPzz) * (1.0f / 3.0f);
#pragma unroll
    for (int q = 0; q < 19; ++q)
        f[q] = CX(q) * CX(q) * lPxx + CY(q) * CY(q) * lPyy + CZ(q) * CZ(q) * lPzz
             + CX(q) * CY(q) * lPxy + CY(q) * CZ(q) * lPyz + CX(q) * CZ(q) * lPxz + ltr;
    // unknown populations copied f^neq of the opposite one
#pragma unroll
    for (int q = 0; q < 19; ++q) if (CX(q) > 0) { f[18 - q] += f[q]; f[q] = 0.0f; }
    // fn = fin - fe for the known ones; fe also enters out directly:
    // lfe = lp - lfn, lfin = lfn
    float lrin = 0.f, lvx = 0.f, lvy = 0.f, lvz = 0.f, lvv = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float lfe = lp[q] - f[q];
        const float cu = CX(q) * vx + CY(q) * vy + CZ(q) * vz;
        lrin += WQ(q) * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * vv) * lfe;
        const float lcu = WQ(q) * rin * (3.0f + 9.0f * cu) * lfe;
        lvx += CX(q) * lcu; lvy += CY(q) * lcu; lvz += CZ(q) * lcu;
        lvv += -1.5f * WQ(q) * rin * lfe;
    }
    lvx += 2.0f * vx * lvv; lvy += 2.0f * vy * lvv; lvz += 2.0f * vz * lvv;
    // rin = (1 + sk) / (1 - vx), sk = sum_{c_x=0} fin + 2 sum_{c_x<0} fin
    const float ivx = rcp_approx(1.0f - vx);
    const float lsk = lrin * ivx;
    lvx += lrin * rin * ivx;
#pragma unroll
    for (int q = 0; q < 19; ++q)
        lp[q] = CX(q) > 0 ? 0.0f : f[q] + (CX(q) == 0 ? lsk : 2.0f * lsk);
    if (a.luin) {
        float *o = a.luin + ((size_t)k * ny + j) * 3;
        o[0] = lvx; o[1] = lvy; o[2] = lvz;
    }
}

template <bool WALLBLOCK, bool SPONGE>
__device__ __forceinline__ void adjoint_cell(const AdjArgs &a, int i, int j, int k, int tx, float (*sh)[4]) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool valid = i < nx;
    const long long N = (long long)nx * ny * nz;
    PullGeom G;
    G.ic = valid ? i : nx - 1;
    G.xm = G.ic - 1; G.xp = G.ic + 1;
    if (a.inlet) { G.xm = max(G.xm, 0); G.xp = min(G.xp, nx - 1); }
    else { G.xm = G.xm < 0 ? nx - 1 : G.xm; G.xp = G.xp >= nx ? 0 : G.xp; }
    const int plane = nx * ny;
    G.ozm = k == 0 ? (nz - 1) * plane : -plane;
    G.ozp = k == nz - 1 ? -(nz - 1) * plane : plane;
    G.bot = j == 0; G.top = j == ny - 1;
    G.oym = G.bot ? 0 : -nx; G.oyp = G.top ? 0 : nx;
    G.o00 = (k * ny + j) * nx;
    // ---- forward recompute: pull; the cell's lambda is loaded with it, so
    // that its latency overlaps the recomputation ----
    float f[19], lam[19];
    const int c = G.o00 + G.ic;
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] = a.in[WALLBLOCK ? src_plane(q, G) : q][src_off(q, G)];
#pragma unroll
    for (int q = 0; q < 19; ++q) lam[q] = valid ? a.lam[q * N + c] : 0.0f;
    // ---- inlet rebuild (eq:f_i, eq:bc_eq, eq:f_i_neq, eq:density_bc) ----
    const bool is_inlet = a.inlet && i == 0;
    float vx = 0.f, vy = 0.f, vz = 0.f, rin = 1.f;
    if (is_inlet) adjoint_inlet_forward(a, f, j, k, vx, vy, vz, rin);
    Pairs P;
    make_pairs<false>(f, P);
    const float f9 = f[9];
    // ---- wall model forward ----
    const bool bot = G.bot, top = G.top, is_wall = WALLBLOCK && a.wall_model && (bot || top);
    float Fx = 0.f, Fz = 0.f;
    float ex = 0.f, ez = 0.f, tn = 0.f, ut = 0.f, sg = 1.f, irho_w = 0.f;
    float irho2 = 0.f, j2x = 0.f, j2z = 0.f;
    if (WALLBLOCK && a.wall_model) {
        if (!(bot || top)) { sh[tx][0] = P.jx; sh[tx][1] = P.jz; sh[tx][2] = rcp_approx(1.0f + P.drho); }
        __syncthreads();
        if (is_wall) {
            j2x = sh[tx][0]; j2z = sh[tx][1]; irho2 = sh[tx][2];
            const float u2x = j2x * irho2, u2z = j2z * irho2;
            irho_w = rcp_approx(1.0f + P.drho);
            tn = sqrt_approx(u2x * u2x + u2z * u2z);
            if (tn >= 1e-12f) {
                const float itn = rcp_approx(tn);
                ex = u2x * itn; ez = u2z * itn;
                const float uhat = (P.jx * ex + P.jz * ez) * irho_w;
                sg = uhat < 0.0f ? -1.0f : 1.0f;
                const float ua = fabsf(uhat);
                // the forward step stored this step's solution of eq:u_tau_implicit
                if (ua > 0.0f && valid) ut = a.utau[((size_t)(bot ? 0 : 1) * nz + k) * nx + i];
                const float tw = (1.0f + P.drho) * ut * ut * sg;
                Fx = -tw * ex; Fz = -tw * ez;
            }
        }
        __syncthreads();   // the shared slots are reused for the reverse below
    }
    // ---- reverse of the collision (with the objective seeds) ----
    if (a.inlet && valid && i == nx - 1) {
        // these entries get the atomics of the next (earlier) adjoint step
#pragma unroll
        for (int q = 0; q < 19; ++q) if (CX(q) < 0) a.lam[q * N + c] = 0.0f;
    }
    float lux = 0.f, luy = 0.f;
    if (a.jr_coef && i == a.i_R && valid) {
        // J_R: d/du of the <u'v'> terms, u and v of this collision
        const float rho = 1.0f + P.drho;
        const float ir = rcp_approx(rho);
        const float uu = (P.jx + 0.5f * Fx) * ir, vv = P.jy * ir;
        const float cj = a.jr_coef[j];
        lux = cj * (vv - a.jr_mean[ny + j]);
        luy = cj * (uu - a.jr_mean[j]);
    }
    AdjIn A;
    const float t0c = SPONGE ? sponge_tau0(a.tau0, a.sp_x0, a.sp_inv, a.sp_3nu, G.ic) : a.tau0;
    if (is_wall) collide_adjoint<true>(lam, P, f9, Fx, 0.f, Fz, t0c, a.csm18, lux, luy, 0.f, A);
    else collide_adjoint<false>(lam, P, f9, 0.f, 0.f, 0.f, t0c, a.csm18, lux, luy, 0.f, A);

    // ---- reverse of the wall model (implicit function theorem for u_tau) ----
    if (WALLBLOCK && a.wall_model) {
        float lj2x = 0.f, lj2z = 0.f, lirho2 = 0.f, gk = 0.f, gB = 0.f;
        if (is_wall && tn >= 1e-12f && valid) {
            const float tw = (1.0f + P.drho) * ut * ut * sg;
            const float ltw = -(A.lFx * ex + A.lFz * ez);
            float lex = -tw * A.lFx, lez = -tw * A.lFz;
            // tau = rho ut^2 (unsigned), tw = tau sg; J_tau weight on tau
            float ltau = sg * ltw;
            if (i >= a.i_tau0 && i < a.i_tau1) ltau += a.jtau_w;
            A.lrho += ut * ut * ltau;
            const float lut = 2.0f * (1.0f + P.drho) * ut * ltau;
            if (ut > 0.0f) {
                float up, dup, dk, dB;
                const float yp = a.y1_nu * ut;
                reichardt_partials(yp, a.kappa, a.B, up, dup, dk, dB);
                const float Ru = up + yp * dup;
                const float iRu = rcp_approx(Ru);
                const float lua = lut * iRu;
                gk = -lut * ut * dk * iRu;
                gB = -lut * ut * dB * iRu;
                const float luh = sg * lua;
                // uhat = (jx ex + jz ez) irho_w
                A.ljx += ex * irho_w * luh; A.ljz += ez * irho_w * luh;
                lex += P.jx * irho_w * luh; lez += P.jz * irho_w * luh;
                const float lirw = (P.jx * ex + P.jz * ez) * luh;
                A.lrho += -irho_w * irho_w * lirw;
            }
            // e = t / |t|, t = (u2x, u2z)
            const float dot = lex * ex + lez * ez;
            const float itn = rcp_approx(tn);
            const float lu2x = (lex - dot * ex) * itn, lu2z = (lez - dot * ez) * itn;
            // u2 = j2 irho2
            lj2x = irho2 * lu2x; lj2z = irho2 * lu2z;
            lirho2 = j2x * lu2x + j2z * lu2z;
        }
        if (is_wall) { sh[tx][0] = lj2x; sh[tx][1] = lj2z; sh[tx][2] = lirho2; }
        __syncthreads();
        if (!(bot || top)) {
            const float li2 = sh[tx][2];
            const float ir = rcp_approx(1.0f + P.drho);
            A.ljx += sh[tx][0]; A.ljz += sh[tx][1];
            A.lrho += -ir * ir * li2;
        }
        // theta gradient of the wall model: warp reduction, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gk += __shfl_xor_sync(0xffffffffu, gk, o);
            gB += __shfl_xor_sync(0xffffffffu, gB, o);
        }
        if ((threadIdx.x & 31) == 0 && (gk != 0.f || gB != 0.f)) {
            atomicAdd(a.gtheta + 2, (double)gk);
            atomicAdd(a.gtheta + 3, (double)gB);
        }
    }
    if (!valid) return;
    float lp[19];
    adjoint_to_pops(lam, A, lp);

    // ---- reverse of the inlet rebuild ----
    if (is_inlet) adjoint_inlet_reverse(a, f, lp, j, k, vx, vy, vz, rin);

    // ---- push the adjoint back to the pull sources ----
    // The outlet column's c_x < 0 entries are read twice in the forward step
    // (by x = nx-2 and, clamped, by x = nx-1): both contributions are added
    // atomically into entries that start at zero.  Unknown inlet populations
    // were not read.  The planes nobody reads (c_x = -1 at x = 0, c_x = +1 at
    // x = nx-1) get zeros.
    auto dst = [&](int q) { return a.lout + (size_t)(WALLBLOCK ? src_plane(q, G) : q) * N + src_off(q, G); };
    const bool is_outlet = a.inlet && i == nx - 1;
    const bool shares_outlet = a.inlet && i >= nx - 2;
    if (!is_inlet && !shares_outlet) {
#pragma unroll
        for (int q = 0; q < 19; ++q) *dst(q) = lp[q];
    } else if (is_inlet) {
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            if (CX(q) > 0) continue;
            if (CX(q) < 0 && shares_outlet) atomicAdd(dst(q), lp[q]);
            else *dst(q) = lp[q];
        }
#pragma unroll
        for (int q = 0; q < 19; ++q) if (CX(q) < 0) a.lout[(size_t)q * N + c] = 0.0f;
    } else {
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            if (CX(q) < 0) atomicAdd(dst(q), lp[q]);
            else *dst(q) = lp[q];
        }
    }
    if (is_outlet) {
#pragma unroll
        for (int q = 0; q < 19; ++q) if (CX(q) > 0) a.lout[(size_t)q * N + c] = 0.0f;
    }
}

// Rows 0, 1 (blockIdx.y = 0) and ny-2, ny-1 (blockIdx.y = 1): the wall cells
// and their second cells, which exchange u_2 and its adjoint through shared
// memory.  Launched beside the interior kernel: every pushed entry has one
// writer (the outlet entries take atomics), so the two never write the same
// word.
template <bool SPONGE>
__global__ void __launch_bounds__(128, 4) adjoint_wall_kernel(const __grid_constant__ AdjArgs a) {
    __shared__ float sh[128 / BY][4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y == 0 ? threadIdx.y : a.ny - 2 + threadIdx.y;
    adjoint_cell<true, SPONGE>(a, i, j, blockIdx.z, threadIdx.x, sh);
}

// Rows 2 .. ny-3.  Latency-bound: five resident blocks per SM (a register
// budget of 102) beat four without spills.  SPONGE: the outlet sponge is on
// (a separate instantiation keeps the per-cell tau0 out of the plain kernel).
#ifndef LBM_ADJ_MINB
#define LBM_ADJ_MINB 5
#endif
template <bool SPONGE>
__global__ void __launch_bounds__(128, LBM_ADJ_MINB) adjoint_kernel(const __grid_constant__ AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 2 + blockIdx.y * BY + threadIdx.y;
    adjoint_cell<false, SPONGE>(a, i, j, blockIdx.z, threadIdx.x, nullptr);
}

// ---------------------------------------------------------------------------
// Interior rows, two x-adjacent cells (i0, i0 + 1) per thread with packed FP32x2
// arithmetic -- the reverse of collide_pairs2<false, false> and of the pull,
// the same chain as adjoint_cell written for two cells at once.  Only regular
// pairs take this path: a pair holding the inlet cell, or a cell whose
// populations the outlet's clamped pull reads twice, goes through
// adjoint_cell one cell at a time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ V2 vsel(bool a, bool b, V2 v) {   // per-lane keep or zero
    return make_float2(a ? v.x : 0.0f, b ? v.y : 0.0f);
}

// Adjoint of the collision inputs of two cells (the packed AdjIn).
struct AdjIn2 {
    V2 ls[9], ld[9];        // of the pair sums / differences
    V2 lf9, lrho;           // of f_9 and rho
    V2 ljx, ljy, ljz;       // of the momentum sum f c (before the force)
    V2 lFx, lFz;            // of the wall force (F_y = 0: the force is wall-parallel)
};

// Reverse of collide_pairs2<false, HAS_FORCE> for two cells: lam = dJ/df*;
// (lux, luy) direct dJ/du seeds; (Fx, 0, Fz) the wall force when HAS_FORCE.
// A receives the adjoint of the collision's inputs (the identity part lam is
// added by adjoint_to_pops2).
template <bool HAS_FORCE>
__device__ __forceinline__ void collide_adjoint2(const V2 (&lam)[19], const Pairs2 &P, V2 Fx, V2 Fz, V2 tau0,
                                                 float csm18, V2 lux, V2 luy, AdjIn2 &A) {
    const V2 *s = P.s;
    // ---- forward values ----
    const V2 rho = P.rho, irho = vrcp(rho);
    const V2 rux = HAS_FORCE ? vfma(0.5f, Fx, P.jx) : P.jx, ruy = P.jy;
    const V2 ruz = HAS_FORCE ? vfma(0.5f, Fz, P.jz) : P.jz;
    const V2 ux = rux * irho, uy = ruy * irho, uz = ruz * irho;
    const V2 uxx = rux * ux, uyy = ruy * uy, uzz = ruz * uz;
    const V2 usq = (uxx + uyy) + uzz;
    const V2 n1 = vfma(-19.0f, usq, vfma(11.0f, rho, vfma(-30.0f, P.f9, vfma(8.0f, P.Sdg, -11.0f * P.Sax))));
    const V2 pxx_eq = vfma(2.0f, uxx, -(uyy + uzz)), pww_eq = uyy - uzz;
    const V2 t1357 = P.s13 + P.s57;
    const V2 n9 = vfma(2.0f, s[8] - P.s04, t1357 - P.s26) - pxx_eq;
    const V2 n11 = (s[6] - s[2]) + (P.s57 - P.s13) - pww_eq;
    const V2 n13 = (s[5] - s[7]) - rux * uy;
    const V2 n14 = (s[0] - s[4]) - ruy * uz;
    const V2 n15 = (s[1] - s[3]) - rux * uz;
    const V2 c2 = n1 * (1.0f / 57.0f);
    const V2 pxx = vfma(1.0f / 3.0f, n9, c2);
    const V2 pyz = vfma(-1.0f / 6.0f, n9, c2);
    const V2 pyy = vfma(0.5f, n11, pyz), pzz = vfma(-0.5f, n11, pyz);
    V2 qq = vfma(pxx, pxx, vfma(pyy, pyy, pzz * pzz));
    qq = vfma(2.0f * n13, n13, vfma(2.0f * n14, n14, vfma(2.0f * n15, n15, qq)));
    const V2 Qh = vsqrt(qq);
    const V2 Rr = vsqrt(vfma(csm18 * Qh, irho, tau0 * tau0));
    const V2 sv = 2.0f * vrcp(tau0 + Rr);
    // Guo source moments with F_y = 0 (collide_pairs2)
    V2 F9 = vdup(0.0f), F11 = vdup(0.0f), F13 = vdup(0.0f), F14 = vdup(0.0f), F15 = vdup(0.0f);
    if (HAS_FORCE) {
        F9 = vfma(4.0f, ux * Fx, -2.0f * (uz * Fz));
        F11 = -2.0f * (uz * Fz);
        F13 = uy * Fx; F14 = uy * Fz; F15 = vfma(ux, Fz, uz * Fx);
    }
    // ---- mu = M lambda ----
    V2 ls[9], ld[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) { ls[p] = lam[p] + lam[18 - p]; ld[p] = lam[p] - lam[18 - p]; }
    const V2 l9 = lam[9];
    const V2 L04 = ls[0] + ls[4], L13 = ls[1] + ls[3], L57 = ls[5] + ls[7], L26 = ls[2] + ls[6];
    const V2 LSax = L26 + ls[8], LSdg = (L04 + L13) + L57;
    const V2 m1 = vfma(-30.0f, l9, vfma(8.0f, LSdg, -11.0f * LSax));
    const V2 m2 = vfma(12.0f, l9, vfma(-4.0f, LSax, LSdg));
    const V2 DX = (ld[3] - ld[1]) + (ld[7] - ld[5]);
    const V2 DY = (ld[4] - ld[0]) - (ld[5] + ld[7]);
    const V2 DZ = -(ld[0] + ld[4]) - (ld[1] + ld[3]);
    const V2 m4 = vfma(4.0f, ld[8], DX), m6 = vfma(4.0f, ld[6], DY), m8 = vfma(4.0f, ld[2], DZ);
    const V2 m9 = vfma(2.0f, ls[8] - L04, (L13 + L57) - L26);
    const V2 m10 = vfma(-4.0f, ls[8], vfma(2.0f, L26 - L04, L13 + L57));
    const V2 m11 = (ls[6] - ls[2]) + (L57 - L13);
    const V2 m12 = vfma(2.0f, ls[2] - ls[6], L57 - L13);
    const V2 m13 = ls[5] - ls[7], m14 = ls[0] - ls[4], m15 = ls[1] - ls[3];
    const V2 m16 = (ld[1] - ld[3]) + (ld[7] - ld[5]);
    const V2 m17 = (ld[4] - ld[0]) + (ld[5] + ld[7]);
    const V2 m18 = (ld[0] + ld[4]) - (ld[1] + ld[3]);
    // ---- reverse through G_k = s_k n_k / |row_k|^2: a_k = -mu_k ----
    V2 bn1 = m1 * (-S_E / 2394.0f);
    const V2 bn2 = m2 * (-S_EPS / 252.0f);
    const V2 bn4 = m4 * (-S_Q / 40.0f), bn6 = m6 * (-S_Q / 40.0f), bn8 = m8 * (-S_Q / 40.0f);
    const V2 msv = -sv;
    V2 bn9 = m9 * msv * (1.0f / 36.0f);
    const V2 bn10 = m10 * (-S_PI / 72.0f);
    V2 bn11 = m11 * msv * (1.0f / 12.0f);
    const V2 bn12 = m12 * (-S_PI / 24.0f);
    const V2 sv4 = msv * 0.25f;
    V2 bn13 = m13 * sv4, bn14 = m14 * sv4, bn15 = m15 * sv4;
    const V2 bn16 = m16 * (-S_M * 0.125f), bn17 = m17 * (-S_M * 0.125f), bn18 = m18 * (-S_M * 0.125f);
    // d/dsv of (sv n - (1 - sv/2) F) = n + F/2
    const V2 bsv = HAS_FORCE
        ? vfma(m9 * vfma(0.5f, F9, n9), vdup(-1.0f / 36.0f),
               vfma(m11 * vfma(0.5f, F11, n11), vdup(-1.0f / 12.0f),
                    (vfma(m13, vfma(0.5f, F13, n13), vfma(m14, vfma(0.5f, F14, n14), m15 * vfma(0.5f, F15, n15)))) *
                        -0.25f))
        : vfma(m9 * n9, vdup(-1.0f / 36.0f),
               vfma(m11 * n11, vdup(-1.0f / 12.0f), (vfma(m13, n13, vfma(m14, n14, m15 * n15))) * -0.25f));
    V2 lux_ = lux, luy_ = luy, luz_ = vdup(0.0f), lFx = vdup(0.0f), lFz = vdup(0.0f);
    if (HAS_FORCE) {
        const V2 m3 = DX - ld[8], m7 = DZ - ld[2];
        const V2 hv = vfma(-0.5f, sv, vdup(1.0f));
        const float cq = (1.0f - 0.5f * S_Q) * (2.0f / 3.0f) * (1.0f / 40.0f);
        const V2 buF = vfma(-(1.0f - 0.5f * S_EPS) * 11.0f / 252.0f, m2, m1 * ((1.0f - 0.5f * S_E) * 38.0f / 2394.0f));
        lFx = vfma(0.1f, m3, m4 * -cq);
        lFz = vfma(0.1f, m7, m8 * -cq);
        const V2 bF9 = vfma(m9 * (1.0f / 36.0f), hv, m10 * (-(1.0f - 0.5f * S_PI) * 0.5f / 72.0f));
        const V2 bF11 = vfma(m11 * (1.0f / 12.0f), hv, m12 * (-(1.0f - 0.5f * S_PI) * 0.5f / 24.0f));
        const V2 bF13 = m13 * hv * 0.25f, bF14 = m14 * hv * 0.25f, bF15 = m15 * hv * 0.25f;
        // uF = ux Fx + uz Fz; F9 = 4 ux Fx - 2 uz Fz; F11 = -2 uz Fz;
        // F13 = uy Fx; F14 = uy Fz; F15 = ux Fz + uz Fx
        lux_ = vfma(Fx, buF + 4.0f * bF9, vfma(Fz, bF15, lux_));
        luy_ = vfma(Fx, bF13, vfma(Fz, bF14, luy_));
        luz_ = vfma(Fz, buF - 2.0f * (bF9 + bF11), Fx * bF15);
        lFx = vfma(ux, buF + 4.0f * bF9, vfma(uy, bF13, vfma(uz, bF15, lFx)));
        lFz = vfma(uz, buF - 2.0f * (bF9 + bF11), vfma(uy, bF14, vfma(ux, bF15, lFz)));
    }
    // ---- SGS: sv = 2 / (tau0 + sqrt(tau0^2 + c Qh / rho)) ----
    const V2 lX = bsv * (-0.25f) * sv * sv * vrcp(Rr);
    const V2 lQh = lX * irho * csm18;
    V2 lirho = lX * Qh * csm18;
    const V2 iQh = vrcp(Qh);
    const V2 lqq = vsel(Qh.x > 1e-30f, Qh.y > 1e-30f, 0.5f * lQh * iQh);
    const V2 lpxx = 2.0f * pxx * lqq, lpyy = 2.0f * pyy * lqq, lpzz = 2.0f * pzz * lqq;
    const V2 lqq4 = 4.0f * lqq;
    bn13 = vfma(n13, lqq4, bn13); bn14 = vfma(n14, lqq4, bn14); bn15 = vfma(n15, lqq4, bn15);
    const V2 lc2 = ((lpxx + lpyy) + lpzz) * (1.0f / 3.0f);
    bn9 = bn9 + (lpxx - 0.5f * (lpyy + lpzz)) * (1.0f / 3.0f);
    bn11 = bn11 + (lpyy - lpzz) * 0.5f;
    bn1 = vfma(1.0f / 19.0f, lc2, bn1);
    // ---- n_k -> pair sums / differences, rho, rho u ----
    V2 lrho = vfma(11.0f, bn1, -3.0f * bn2);
    const V2 lusq = vfma(-19.0f, bn1, 5.5f * bn2);
    A.lf9 = vfma(-30.0f, bn1, 12.0f * bn2);
    const V2 lSax = vfma(-11.0f, bn1, -4.0f * bn2), lSdg = vfma(8.0f, bn1, bn2);
    const V2 b910 = bn9 + bn10, b1112 = bn11 + bn12;
    A.ls[0] = (lSdg - 2.0f * b910) + bn14;
    A.ls[4] = (lSdg - 2.0f * b910) - bn14;
    A.ls[1] = ((lSdg + b910) - b1112) + bn15;
    A.ls[3] = ((lSdg + b910) - b1112) - bn15;
    A.ls[5] = ((lSdg + b910) + b1112) + bn13;
    A.ls[7] = ((lSdg + b910) + b1112) - bn13;
    A.ls[2] = vfma(2.0f, bn10 + bn12, lSax - (bn9 + bn11));
    A.ls[6] = vfma(2.0f, bn10 - bn12, (lSax - bn9) + bn11);
    A.ls[8] = vfma(2.0f, bn9, vfma(-4.0f, bn10, lSax));
    A.ld[1] = bn16 - bn18; A.ld[3] = -(bn16 + bn18);
    A.ld[7] = bn16 + bn17; A.ld[5] = bn17 - bn16;
    A.ld[4] = bn17 + bn18; A.ld[0] = bn18 - bn17;
    A.ld[8] = 5.0f * bn4; A.ld[6] = 5.0f * bn6; A.ld[2] = 5.0f * bn8;
    const V2 lpxxeq = vfma(0.5f, bn10, -bn9), lpwweq = vfma(0.5f, bn12, -bn11);
    const V2 luxx = vfma(2.0f, lpxxeq, lusq), luyy = (lusq - lpxxeq) + lpwweq, luzz = (lusq - lpxxeq) - lpwweq;
    // uxx = rux ux, uyy = ruy uy, uzz = ruz uz, uxy = rux uy, uyz = ruy uz, uxz = rux uz
    // with a_uxy = -bn13, a_uyz = -bn14, a_uxz = -bn15; u = ru / rho
    lux_ = vfma(rux, luxx, lux_);
    luy_ = vfma(ruy, luyy, luy_) - rux * bn13;
    luz_ = vfma(ruz, luzz, luz_) - (ruy * bn14 + rux * bn15);
    V2 lrux = vfma(2.0f / 3.0f, bn4, vfma(ux, luxx, -(uy * bn13 + uz * bn15)));
    V2 lruy = vfma(2.0f / 3.0f, bn6, vfma(uy, luyy, -(uz * bn14)));
    V2 lruz = vfma(2.0f / 3.0f, bn8, uz * luzz);
    lrux = vfma(irho, lux_, lrux); lruy = vfma(irho, luy_, lruy); lruz = vfma(irho, luz_, lruz);
    lirho = lirho + vfma(rux, lux_, vfma(ruy, luy_, ruz * luz_));
    A.lrho = lrho - irho * irho * lirho;
    // n4 = jx + 5 d8 + 2/3 rux and ru = j + F/2
    A.ljx = bn4 + lrux; A.ljy = bn6 + lruy; A.ljz = bn8 + lruz;
    A.lFx = HAS_FORCE ? vfma(0.5f, lrux, lFx) : lFx;
    A.lFz = HAS_FORCE ? vfma(0.5f, lruz, lFz) : lFz;
}

// The adjoint of the pulled populations of two cells from that of the
// collision inputs: rho = sum f, j from the differences, s / d the pairs.
__device__ __forceinline__ void adjoint_to_pops2(const V2 (&lam)[19], const AdjIn2 &A, V2 (&lp)[19]) {
    V2 ld[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) ld[p] = A.ld[p];
    ld[3] = ld[3] + A.ljx - A.ljz; ld[1] = ld[1] - A.ljx - A.ljz; ld[7] = ld[7] + A.ljx - A.ljy;
    ld[5] = ld[5] - A.ljx - A.ljy; ld[8] = ld[8] - A.ljx;
    ld[4] = ld[4] + A.ljy - A.ljz; ld[0] = ld[0] - A.ljy - A.ljz; ld[6] = ld[6] - A.ljy;
    ld[2] = ld[2] - A.ljz;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const V2 a = A.ls[p] + A.lrho;
        lp[p] = (lam[p] + a) + ld[p];
        lp[18 - p] = (lam[18 - p] + a) - ld[p];
    }
    lp[9] = (lam[9] + A.lf9) + A.lrho;
}

// Pull geometry of two x-adjacent cells (i0, i0 + 1) of row j, plane k: the
// source plane of population q (mirrored through a slip wall) and the row /
// plane offset of its source; x sources xm0 (the lo cell's c_x = +1) and xp1
// (the hi cell's c_x = -1), wrapped when the inlet is off.
struct PairGeom {
    int o00, ozm, ozp, xm0, xp1, nx;
    bool bot, top;
    __device__ __forceinline__ int plane(int q) const {
        return ((CY(q) > 0 && bot) || (CY(q) < 0 && top)) ? mirror_y(q) : q;
    }
    __device__ __forceinline__ int row(int q) const {
        const bool mir = (CY(q) > 0 && bot) || (CY(q) < 0 && top);
        return o00 + (mir ? 0 : (CY(q) < 0 ? nx : (CY(q) > 0 ? -nx : 0))) +
               (CZ(q) < 0 ? ozp : (CZ(q) > 0 ? ozm : 0));
    }
};
__device__ __forceinline__ PairGeom pair_geom(const AdjArgs &a, int i0, int j, int k) {
    PairGeom g;
    g.nx = a.nx;
    g.xm0 = i0 - 1; g.xp1 = i0 + 2;
    if (!a.inlet) { g.xm0 = g.xm0 < 0 ? a.nx - 1 : g.xm0; g.xp1 = g.xp1 >= a.nx ? 0 : g.xp1; }
    const int plane = a.nx * a.ny;
    g.ozm = k == 0 ? (a.nz - 1) * plane : -plane;
    g.ozp = k == a.nz - 1 ? -(a.nz - 1) * plane : plane;
    g.o00 = (k * a.ny + j) * a.nx;
    g.bot = j == 0; g.top = j == a.ny - 1;
    return g;
}
__device__ __forceinline__ void pull_pair(const AdjArgs &a, const PairGeom &g, int i0, V2 (&f)[19]) {
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float *r = a.in[g.plane(q)] + g.row(q);
        if (CX(q) == 0) f[q] = *reinterpret_cast<const float2 *>(r + i0);
        else if (CX(q) > 0) f[q] = make_float2(r[g.xm0], r[i0]);
        else f[q] = make_float2(r[i0 + 1], r[g.xp1]);
    }
}
__device__ __forceinline__ void push_pair(const AdjArgs &a, const PairGeom &g, int i0, const V2 (&lp)[19]) {
    const long long N = (long long)a.nx * a.ny * a.nz;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        float *r = a.lout + g.plane(q) * N + g.row(q);
        if (CX(q) == 0) *reinterpret_cast<float2 *>(r + i0) = lp[q];
        else if (CX(q) > 0) { r[g.xm0] = lp[q].x; r[i0] = lp[q].y; }
        else { r[i0 + 1] = lp[q].x; r[g.xp1] = lp[q].y; }
    }
}
// J_R seeds (dJ_R/du, dJ_R/dv) of the two cells when one of them sits at x = i_R
__device__ __forceinline__ void jr_seeds2(const AdjArgs &a, const Pairs2 &P, V2 Fx, int i0, int j, V2 &lux,
                                          V2 &luy) {
    lux = luy = vdup(0.0f);
    if (a.jr_coef && (i0 == a.i_R || i0 + 1 == a.i_R)) {
        const V2 ir = vrcp(P.rho);
        const V2 uu = vfma(0.5f, Fx, P.jx) * ir, vv = P.jy * ir;
        const float cj = a.jr_coef[j];
        const bool lo = i0 == a.i_R;
        lux = vsel(lo, !lo, cj * (vv - vdup(a.jr_mean[a.ny + j])));
        luy = vsel(lo, !lo, cj * (uu - vdup(a.jr_mean[j])));
    }
}
template <bool SPONGE>
__device__ __forceinline__ V2 pair_tau0_adj(const AdjArgs &a, int i0) {
    return SPONGE ? make_float2(sponge_tau0(a.tau0, a.sp_x0, a.sp_inv, a.sp_3nu, i0),
                                sponge_tau0(a.tau0, a.sp_x0, a.sp_inv, a.sp_3nu, i0 + 1))
                  : vdup(a.tau0);
}

// Interior rows 2 .. ny-3, two cells per thread (neither the inlet cell nor
// one whose populations the outlet's clamped pull shares).
template <bool SPONGE>
__device__ __forceinline__ void adjoint_pair(const AdjArgs &a, int i0, int j, int k) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    const PairGeom g = pair_geom(a, i0, j, k);
    V2 f[19], lam[19];
    pull_pair(a, g, i0, f);
    const int c = g.o00 + i0;
#pragma unroll
    for (int q = 0; q < 19; ++q) lam[q] = *reinterpret_cast<const float2 *>(a.lam + q * N + c);
    Pairs2 P;
    make_pairs2<false>(f, P);
    V2 lux, luy;
    jr_seeds2(a, P, vdup(0.0f), i0, j, lux, luy);
    AdjIn2 A;
    collide_adjoint2<false>(lam, P, vdup(0.0f), vdup(0.0f), pair_tau0_adj<SPONGE>(a, i0), a.csm18, lux, luy, A);
    V2 lp[19];
    adjoint_to_pops2(lam, A, lp);
    push_pair(a, g, i0, lp);
}

// A wall row and its second row, two x-adjacent cells per thread: the
// threads of row ty = 0 and ty = 1 of the block hold the wall row and the
// second row (bottom: 0 and 1; top: ny-2 and ny-1) at the same x, and trade
// u_2 (forward) and its adjoint through sh[slot], slot = the cell's x within
// the block.  `active`: a pair away from the inlet and the outlet's shared
// reads (the others take the one-cell path); every thread reaches the two
// barriers, inactive ones on in-bounds placeholder cells whose results are
// dropped.  The reverse of the wall model (Sec. 2.3) runs per lane as in
// adjoint_cell: u_tau through the implicit function theorem, then e_x and u_2.
template <bool SPONGE>
__device__ __forceinline__ void adjoint_wall_pair(const AdjArgs &a, int i0, int j, int k, bool active, int slot,
                                                  float (*sh)[4]) {
    const int nx = a.nx, nz = a.nz;
    const long long N = (long long)nx * a.ny * nz;
    const int ic = active ? i0 : 2;
    const PairGeom g = pair_geom(a, ic, j, k);
    const bool is_wall = g.bot || g.top;                  // warp-uniform (one row per warp)
    V2 f[19], lam[19];
    pull_pair(a, g, ic, f);
    const int c = g.o00 + ic;
#pragma unroll
    for (int q = 0; q < 19; ++q) lam[q] = *reinterpret_cast<const float2 *>(a.lam + q * N + c);
    Pairs2 P;
    make_pairs2<false>(f, P);
    // ---- wall model forward (eq:base, eq:uhat, this step's u_tau, eq:force_wm) ----
    // Per lane from u_2 (in sh), the cell's momentum and density and this
    // step's u_tau; evaluated for the force here and again in the reverse
    // below, so that no per-lane state lives across the collision's reverse.
    const int w = g.bot ? 0 : 1;
    struct WallLane { float ex, ez, tn, ut, sg, j2x, j2z, ir2; };
    auto wall_lane = [&](int l) {
        WallLane v{0.f, 0.f, 0.f, 0.f, 1.f, sh[slot + l][0], sh[slot + l][1], sh[slot + l][2]};
        const float u2x = v.j2x * v.ir2, u2z = v.j2z * v.ir2;
        v.tn = sqrt_approx(u2x * u2x + u2z * u2z);
        if (v.tn >= 1e-12f) {
            const float itn = rcp_approx(v.tn);
            v.ex = u2x * itn; v.ez = u2z * itn;
            const float jx = l ? P.jx.y : P.jx.x, jz = l ? P.jz.y : P.jz.x, rw = l ? P.rho.y : P.rho.x;
            const float uhat = (jx * v.ex + jz * v.ez) * rcp_approx(rw);
            v.sg = uhat < 0.0f ? -1.0f : 1.0f;
            // the forward step stored this step's solution of eq:u_tau_implicit
            if (fabsf(uhat) > 0.0f && active) v.ut = a.utau[((size_t)w * nz + k) * nx + ic + l];
        }
        return v;
    };
    V2 Fx = vdup(0.0f), Fz = vdup(0.0f);
    if (a.wall_model) {
        if (!is_wall) {
            const V2 ir = vrcp(P.rho);
            sh[slot][0] = P.jx.x; sh[slot][1] = P.jz.x; sh[slot][2] = ir.x;
            sh[slot + 1][0] = P.jx.y; sh[slot + 1][1] = P.jz.y; sh[slot + 1][2] = ir.y;
        }
        __syncthreads();
        if (is_wall) {
            const WallLane v0 = wall_lane(0), v1 = wall_lane(1);
            const float tw0 = P.rho.x * v0.ut * v0.ut * v0.sg, tw1 = P.rho.y * v1.ut * v1.ut * v1.sg;
            Fx = make_float2(-tw0 * v0.ex, -tw1 * v1.ex);
            Fz = make_float2(-tw0 * v0.ez, -tw1 * v1.ez);
        }
        __syncthreads();                          // the second rows' slots stay as they are until
                                                  // the wall rows' reverse below has read them
    }
    // ---- reverse of the collision (with the objective seeds) ----
    V2 lux, luy;
    jr_seeds2(a, P, Fx, ic, j, lux, luy);
    AdjIn2 A;
    const V2 t0c = pair_tau0_adj<SPONGE>(a, ic);
    if (is_wall && a.wall_model) collide_adjoint2<true>(lam, P, Fx, Fz, t0c, a.csm18, lux, luy, A);
    else collide_adjoint2<false>(lam, P, Fx, Fz, t0c, a.csm18, lux, luy, A);
    // ---- reverse of the wall model ----
    if (a.wall_model) {
        float gk = 0.f, gB = 0.f;
        if (is_wall) {
            const float lFx[2] = {A.lFx.x, A.lFx.y}, lFz[2] = {A.lFz.x, A.lFz.y};
            const float rw[2] = {P.rho.x, P.rho.y}, jxw[2] = {P.jx.x, P.jx.y}, jzw[2] = {P.jz.x, P.jz.y};
            const WallLane vl[2] = {wall_lane(0), wall_lane(1)};
            float dljx[2] = {0.f, 0.f}, dljz[2] = {0.f, 0.f}, dlrho[2] = {0.f, 0.f};
            float lj2x[2] = {0.f, 0.f}, lj2z[2] = {0.f, 0.f}, li2[2] = {0.f, 0.f};
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const WallLane &v = vl[l];
                if (!(v.tn >= 1e-12f && active)) continue;
                const float tw = rw[l] * v.ut * v.ut * v.sg;
                const float ltw = -(lFx[l] * v.ex + lFz[l] * v.ez);
                float lex = -tw * lFx[l], lez = -tw * lFz[l];
                // tau = rho ut^2 (unsigned), tw = tau sg; J_tau weight on tau
                float ltau = v.sg * ltw;
                if (ic + l >= a.i_tau0 && ic + l < a.i_tau1) ltau += a.jtau_w;
                dlrho[l] += v.ut * v.ut * ltau;
                const float lut = 2.0f * rw[l] * v.ut * ltau;
                if (v.ut > 0.0f) {
                    float up, dup, dk, dB;
                    const float yp = a.y1_nu * v.ut;
                    reichardt_partials(yp, a.kappa, a.B, up, dup, dk, dB);
                    const float iRu = rcp_approx(up + yp * dup);
                    gk -= lut * v.ut * dk * iRu;
                    gB -= lut * v.ut * dB * iRu;
                    const float luh = v.sg * lut * iRu;
                    const float irw = rcp_approx(rw[l]);
                    // uhat = (jx ex + jz ez) / rho_w
                    dljx[l] += v.ex * irw * luh; dljz[l] += v.ez * irw * luh;
                    lex += jxw[l] * irw * luh; lez += jzw[l] * irw * luh;
                    dlrho[l] -= irw * irw * (jxw[l] * v.ex + jzw[l] * v.ez) * luh;
                }
                // e = t / |t|, t = (u2x, u2z); u2 = j2 / rho2
                const float dot = lex * v.ex + lez * v.ez;
                const float itn = rcp_approx(v.tn);
                const float lu2x = (lex - dot * v.ex) * itn, lu2z = (lez - dot * v.ez) * itn;
                lj2x[l] = v.ir2 * lu2x; lj2z[l] = v.ir2 * lu2z;
                li2[l] = v.j2x * lu2x + v.j2z * lu2z;
            }
            A.ljx = A.ljx + make_float2(dljx[0], dljx[1]);
            A.ljz = A.ljz + make_float2(dljz[0], dljz[1]);
            A.lrho = A.lrho + make_float2(dlrho[0], dlrho[1]);
#pragma unroll
            for (int l = 0; l < 2; ++l) { sh[slot + l][0] = lj2x[l]; sh[slot + l][1] = lj2z[l]; sh[slot + l][2] = li2[l]; }
        }
        __syncthreads();
        if (!is_wall) {
            const V2 ir = vrcp(P.rho);
            A.ljx = A.ljx + make_float2(sh[slot][0], sh[slot + 1][0]);
            A.ljz = A.ljz + make_float2(sh[slot][1], sh[slot + 1][1]);
            A.lrho = A.lrho - ir * ir * make_float2(sh[slot][2], sh[slot + 1][2]);
        }
        // theta gradient of the wall model: warp reduction, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gk += __shfl_xor_sync(0xffffffffu, gk, o);
            gB += __shfl_xor_sync(0xffffffffu, gB, o);
        }
        if ((threadIdx.x & 31) == 0 && (gk != 0.f || gB != 0.f)) {
            atomicAdd(a.gtheta + 2, (double)gk);
            atomicAdd(a.gtheta + 3, (double)gB);
        }
    }
    if (!active) return;
    V2 lp[19];
    adjoint_to_pops2(lam, A, lp);
    push_pair(a, g, ic, lp);
}

#ifndef LBM_ADJ2_MINB
#define LBM_ADJ2_MINB 4
#endif

// One reverse step in one launch (nx even, block (64, BY)), in this order of
// blocks: [0, nwp) the wall rows and their second rows two cells per thread
// (adjoint_wall_pair; ty = 0, 1 the two rows, 128 x cells per block); with the
// inlet on, [nwp, nwp + nwe) the same rows at x = 0, 1, nx-2, nx-1 one cell per
// thread (adjoint_cell, tx = column + 4 x plane within 16 planes), and
// [.., + ne) those columns of rows 2..ny-3; the rest the other cells of rows
// 2..ny-3 two per thread.  Blocks start in index order, so the longer chains of
// the first parts run beside the interior pairs.  The parts write disjoint
// entries (the outlet's shared entries take atomics).
template <bool SPONGE>
__global__ void __launch_bounds__(128, LBM_ADJ2_MINB)
    adjoint_fused_kernel(const __grid_constant__ AdjArgs a, int nwp, int nwe, int ne) {
    __shared__ float sh[128][4];
    const int b = blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = a.nx;
    if (b < nwp) {                                   // wall rows, two cells per thread
        const int nbx = (nx + 127) / 128;
        const int bx = b % nbx, r = b / nbx;
        const int j = (r % 2) == 0 ? ty : a.ny - 2 + ty;
        const int i0 = 2 * (bx * 64 + tx);
        const bool active = i0 < nx && (!a.inlet || (i0 >= 2 && i0 + 2 < nx));
        adjoint_wall_pair<SPONGE>(a, i0, j, r / 2, active, 2 * tx, sh);
        return;
    }
    if (b < nwp + nwe) {                             // wall rows at the inlet / outlet columns
        const int r = b - nwp, side = r % 2, kg = r / 2;
        const int col = tx % 4, k = kg * 16 + tx / 4;
        const int i = k < a.nz ? (col < 2 ? col : nx - 4 + col) : nx;   // i = nx: a placeholder
        const int j = side == 0 ? ty : a.ny - 2 + ty;
        adjoint_cell<true, SPONGE>(a, i, j, min(k, a.nz - 1), tx, sh);
        return;
    }
    if (b < nwp + nwe + ne) {                        // x = 0, 1, nx-2, nx-1 of rows 2..ny-3
        const int e = (b - nwp - nwe) * 128 + ty * 64 + tx;
        const int rows = a.ny - 4;
        if (e >= 4 * rows * a.nz) return;
        const int c = e % 4, rr = e / 4;
        adjoint_cell<false, SPONGE>(a, c < 2 ? c : nx - 4 + c, 2 + rr % rows, rr / rows, 0, nullptr);
        return;
    }
    const int nb2 = (nx / 2 + 63) / 64, rows2 = (a.ny - 4) / BY;
    const int bi = b - nwp - nwe - ne;
    const int bx = bi % nb2, r = bi / nb2;
    const int i0 = 2 * (bx * 64 + tx);
    const int j = 2 + (r % rows2) * BY + ty;
    if (i0 >= nx || (a.inlet && (i0 == 0 || i0 + 2 >= nx))) return;
    adjoint_pair<SPONGE>(a, i0, j, r / rows2);
}

// ---------------------------------------------------------------------------
// theta gradient through the inlet velocity, u_in = U_R(j; kappa, B) +
// amp a(j) v'(j, k, t; ell_e) (eq:u_couple, eq:v_fluc, eq:aux_vec):
//   dJ/d amp   += luin . (a v'),            dJ/d ell_e += luin . (amp a dv'/d ell_e),
//   dJ/d kappa += luin_x dU_R/d kappa,      dJ/d B     += luin_x dU_R/d B.
// k_n and the time phase scale with 1/max l_e, so d(arg_n)/d ell_e =
// -(d max l_e / d ell_e) / max l_e * Theta_n with Theta_n = k_n (d_y y + d_z z) -
// 2 pi nu_n t the unreduced phase; d sqrt(6 q_n)/d ell_e comes from the host.
// Same blocking as stg_kernel (row j, 32 z x 8 time levels).
// ---------------------------------------------------------------------------
struct StgAdjArgs {
    const uint32_t *__restrict__ alpha;   // [ny][N]
    const uint32_t *__restrict__ betaT;   // [N][nz]
    const uint32_t *__restrict__ phi32;   // [N]
    const uint64_t *__restrict__ rate64;  // [N]
    const float4 *__restrict__ sqsig;     // [ny][N]
    const float *__restrict__ dsq;        // [ny][N] d sqrt(6 q_n) / d ell_e
    const float4 *__restrict__ kphase;    // [N] (k_n d_ny, k_n d_nz, 2 pi nu_n, 0)
    const float *__restrict__ aunit;      // [ny][6] Cholesky factor without amp
    const float *__restrict__ dUR;        // [2][ny] dU_R/dkappa, dU_R/dB
    const float *__restrict__ luin;       // [T][nz][ny][3]
    double *__restrict__ gtheta;          // [4]
    float amp, cell_scale;                // amp, (d max l_e / d ell_e) / max l_e
    long long t0;
    int nsteps, ny, nz, n_modes;
};

__global__ void __launch_bounds__(STG_KZ * STG_KT) stg_adjoint_kernel(const __grid_constant__ StgAdjArgs a) {
    __shared__ uint32_t s_ph[STG_KT][STG_MCHUNK];
    __shared__ float4 s_sq[STG_MCHUNK];
    __shared__ float s_dsq[STG_MCHUNK];
    __shared__ float4 s_kp[STG_MCHUNK];
    __shared__ float s_red[4][STG_KZ * STG_KT / 32];
    const int j = blockIdx.y;
    const int lz = threadIdx.x % STG_KZ, lt = threadIdx.x / STG_KZ;
    const int k = blockIdx.x * STG_KZ + lz;
    const int ts = blockIdx.z * STG_KT + lt;
    const int N = a.n_modes;
    const float t = (float)(a.t0 + ts);
    const float y = j + 0.5f, z = k + 0.5f;
    float vx = 0.f, vy = 0.f, vz = 0.f, wx = 0.f, wy = 0.f, wz = 0.f;
    for (int n0 = 0; n0 < N; n0 += STG_MCHUNK) {
        const int nc = min(STG_MCHUNK, N - n0);
        __syncthreads();
        for (int e = threadIdx.x; e < STG_KT * nc; e += blockDim.x) {
            const int tl = e / nc, n = n0 + e % nc;
            const uint64_t tt = (uint64_t)(a.t0 + (long long)blockIdx.z * STG_KT + tl);
            s_ph[tl][e % nc] = a.alpha[(size_t)j * N + n] + a.phi32[n] + (uint32_t)((a.rate64[n] * tt) >> 32);
        }
        for (int e = threadIdx.x; e < nc; e += blockDim.x) {
            s_sq[e] = a.sqsig[(size_t)j * N + n0 + e];
            s_dsq[e] = a.dsq[(size_t)j * N + n0 + e];
            s_kp[e] = a.kphase[n0 + e];
        }
        __syncthreads();
        if (k < a.nz) {
            const uint32_t *be = a.betaT + (size_t)n0 * a.nz + k;
            for (int m = 0; m < nc; ++m) {
                const uint32_t ph = s_ph[lt][m] + be[(size_t)m * a.nz];
                const float x = (float)(int32_t)ph * 1.4629180792671596e-09f;
                float sn, cs;
                __sincosf(x, &sn, &cs);
                const float4 qs = s_sq[m];
                const float4 kp = s_kp[m];
                const float Th = kp.x * y + kp.y * z - kp.z * t;
                const float cw = qs.x * cs;
                const float dw = s_dsq[m] * cs + qs.x * a.cell_scale * Th * sn;
                vx = fmaf(cw, qs.y, vx); vy = fmaf(cw, qs.z, vy); vz = fmaf(cw, qs.w, vz);
                wx = fmaf(dw, qs.y, wx); wy = fmaf(dw, qs.z, wy); wz = fmaf(dw, qs.w, wz);
            }
        }
    }
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    if (k < a.nz && ts < a.nsteps) {
        const float *L = a.luin + (((size_t)ts * a.nz + k) * a.ny + j) * 3;
        const float *m = a.aunit + 6 * j;
        const float ax = m[0] * vx, ay = m[1] * vx + m[2] * vy, az = m[3] * vx + m[4] * vy + m[5] * vz;
        const float bx = m[0] * wx, by = m[1] * wx + m[2] * wy, bz = m[3] * wx + m[4] * wy + m[5] * wz;
        g[0] = a.amp * (L[0] * bx + L[1] * by + L[2] * bz);
        g[1] = L[0] * ax + L[1] * ay + L[2] * az;
        g[2] = L[0] * a.dUR[j];
        g[3] = L[0] * a.dUR[a.ny + j];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[c] += __shfl_xor_sync(0xffffffffu, g[c], o);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) s_red[c][warp] = g[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < STG_KZ * STG_KT / 32; ++w) acc += s_red[threadIdx.x][w];
        atomicAdd(a.gtheta + threadIdx.x, acc);
    }
}

// ---------------------------------------------------------------------------
// Objective sums of one step, from the new post-collision state: the wall shear
// |F_w| = rho u_tau^2 of the wall cells with i0 <= i < i1, and at x = iR the
// z-sums of u, v and u v with rho u = sum f* c - F/2.  acc[0] = tau sum,
// acc[1 + 3 j + (0,1,2)] = (u, v, uv) sums.  Blocks 0 .. ny-1: one row j each,
// threads over z; the remaining blocks: the wall cells, one atomic per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) objective_kernel(const float *__restrict__ f, const float *__restrict__ fw,
                                                        double *acc, int nx, int ny, int nz, int i0, int i1,
                                                        int iR) {
    __shared__ double red[3][128];
    const long long N = (long long)nx * ny * nz;
    const int tid = threadIdx.x;
    if ((int)blockIdx.x < ny) {
        const int j = blockIdx.x;
        float su = 0, sv = 0, suv = 0;
        for (int k = tid; k < nz; k += blockDim.x) {
            const long long c = ((long long)k * ny + j) * nx + iR;
            float r = 0, jx = 0, jy = 0;
#pragma unroll
            for (int q = 0; q < 19; ++q) { const float v = f[q * N + c]; r += v; jx += CX(q) * v; jy += CY(q) * v; }
            if (j == 0 || j == ny - 1) {
                const float *F = fw + (((size_t)(j == 0 ? 0 : 1) * nz + k) * nx + iR) * 3;
                jx -= 0.5f * F[0]; jy -= 0.5f * F[1];
            }
            const float ir = rcp_approx(r);
            const float u = jx * ir, v = jy * ir;
            su += u; sv += v; suv += u * v;
        }
        red[0][tid] = su; red[1][tid] = sv; red[2][tid] = suv;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (tid < o) { red[0][tid] += red[0][tid + o]; red[1][tid] += red[1][tid + o]; red[2][tid] += red[2][tid + o]; }
            __syncthreads();
        }
        if (tid == 0) { acc[1 + 3 * j] += red[0][0]; acc[2 + 3 * j] += red[1][0]; acc[3 + 3 * j] += red[2][0]; }
        return;
    }
    const int w_i = i1 - i0;
    const int e = ((int)blockIdx.x - ny) * blockDim.x + tid;
    float s = 0.0f;
    if (w_i > 0 && e < 2 * nz * w_i) {
        const int ii = i0 + e % w_i, r = e / w_i, k = r % nz, w = r / nz;
        const float *F = fw + (((size_t)w * nz + k) * nx + ii) * 3;
        s = sqrtf(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    }
    red[0][tid] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[0][tid] += red[0][tid + o];
        __syncthreads();
    }
    if (tid == 0 && red[0][0] != 0.0) atomicAdd(acc, red[0][0]);
}

// J_R seeds from the window sums of objective_kernel / the step kernels, one
// thread per row j: with <.> the mean over z and the window (cnt samples),
// r_j = (<uv> - <u><v>) / u_ref^2 - R12(j) / u_ref^2 and J_R = sum_j r_j^2, so
// dJ_R/du = 2 r_j (v - <v>) / (u_ref^2 cnt) and likewise for v:
// coef[j] = 2 r_j / (u_ref^2 cnt), mean[j] = <u>, mean[ny + j] = <v>.
__global__ void objective_seed_kernel(const double *__restrict__ acc, const double *__restrict__ R12,
                                      float *__restrict__ coef, float *__restrict__ mean, int ny, double cnt,
                                      double ur2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    const double mu = acc[1 + 3 * j] / cnt, mv = acc[2 + 3 * j] / cnt, muv = acc[3 + 3 * j] / cnt;
    const double r = (muv - mu * mv) / ur2 - R12[j] / ur2;
    coef[j] = (float)(2.0 * r / (ur2 * cnt));
    mean[j] = (float)mu;
    mean[ny + j] = (float)mv;
}

}  // namespace lbmk

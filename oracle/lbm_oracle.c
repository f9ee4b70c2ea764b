/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the STG wall-modelled MRT-LES
 * lattice Boltzmann channel step of Xue, Yao & Davidson, "Synthetic turbulence
 * generator for the wall-modeled LES lattice Boltzmann method" (arXiv 2304.04214).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline / reference leg load this library.  The CUDA
 * library shares no code, header, table or constant with it.
 *
 * Everything is written to be checked against the paper by eye, not for speed:
 *   - the velocity set, weights and the 19x19 matrix M are typed from Sec. 2.1
 *     (eq:vel-set) and Appendix A.1;
 *   - m = M f and f* = M^{-1} m* are dense matrix products, M^{-1} = M^T D^{-1}
 *     with D = diag(|row_k|^2) (the rows of M are orthogonal);
 *   - the equilibrium moments are M f^eq with f^eq of eq:bc_eq (reading of the
 *     garbled rows 2, 4, 6, 8 of eq:mom_eq), the Guo force moments are M F~;
 *   - streaming is a literal pull over all cells, the boundary fix-ups are
 *     separate passes in the order stream -> outlet copy -> inlet -> wall -> collide.
 *
 * The file is compiled twice: with `real` = double (exported symbols orc_*) and
 * with `real` = double complex (symbols orcz_*).  The complex build gives
 * complex-step derivatives (Squire & Trapp 1998): with theta_k = x + i h,
 * dJ/dtheta_k = Im J / h to machine precision, because every operation below is
 * analytic in the perturbed inputs (comparisons and branches look at real parts).
 *
 * Readings of silent or garbled passages (each is listed in the design notes):
 *   A1/A2  m^eq = M f^eq          A3  conserved rates 1.0, omega_1 = 1.19
 *   A4     moment-space Guo force F = M^{-1}(I - S/2) M F~
 *   A5     g is a force density;  rho u = sum f c + F/2
 *   A6     tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt2 C Q^{1/2}/rho))/2
 *   A7     Reichardt law with textbook coefficients (1/kappa, kappa, B)
 *   A8     halfway walls: first cell centre at y = 1/2
 *   A10    u_tau Newton to 1e-13 relative, force sign follows u_hat
 *   A12    specular slip walls;  A13 Zou-He density with the 1-u form
 *   A14    f^neq = w/(2 cs^4) Q:Pi;  A15 unknown f^neq from the opposite
 *   A16    STG spectrum / modes / length scale (see stg_tables)
 *   A18    zero-gradient outlet copy;  A19 order of the boundary passes
 *   A24    outlet sponge (Sec. 4.1 names one; its form is not given): over
 *          the last L cells the viscosity rises by nu_s r^2, r = (x - (nx -
 *          L)) / L at the cell centre x = i + 1/2, so tau0(x) = tau0 + 3 nu_s r^2
 */
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef ORC_COMPLEX
#include <complex.h>
typedef double complex real;
#define RE(x) creal(x)
#define IMAG(x) cimag(x)
#define API(name) orcz_##name
#else
typedef double real;
#define RE(x) (x)
#define IMAG(x) 0.0
#define API(name) orc_##name
#endif
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define PI_D 3.14159265358979323846

/* ---- Sec. 2.1, eq:vel-set: the D3Q19 velocities in the paper's order ---- */
static const int C[Q][3] = {
    { 0,-1,-1}, {-1, 0,-1}, { 0, 0,-1}, { 1, 0,-1}, { 0, 1,-1},
    {-1,-1, 0}, { 0,-1, 0}, { 1,-1, 0}, {-1, 0, 0}, { 0, 0, 0},
    { 1, 0, 0}, {-1, 1, 0}, { 0, 1, 0}, { 1, 1, 0}, { 0,-1, 1},
    {-1, 0, 1}, { 0, 0, 1}, { 1, 0, 1}, { 0, 1, 1}};

/* ---- Sec. 2.1: weights w_9 = 1/3, axis directions 1/18, diagonals 1/36 ---- */
static const double W[Q] = {
    1./36, 1./36, 1./18, 1./36, 1./36, 1./36, 1./18, 1./36, 1./18, 1./3,
    1./18, 1./36, 1./18, 1./36, 1./36, 1./36, 1./18, 1./36, 1./36};

/* ---- Appendix A.1: the Gram-Schmidt moment matrix M, row by row ---- */
static const double M[Q][Q] = {
 { 1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1},
 { 8,  8,-11,  8,  8,  8,-11,  8,-11,-30,-11,  8,-11,  8,  8,  8,-11,  8,  8},
 { 1,  1, -4,  1,  1,  1, -4,  1, -4, 12, -4,  1, -4,  1,  1,  1, -4,  1,  1},
 { 0, -1,  0,  1,  0, -1,  0,  1, -1,  0,  1, -1,  0,  1,  0, -1,  0,  1,  0},
 { 0, -1,  0,  1,  0, -1,  0,  1,  4,  0, -4, -1,  0,  1,  0, -1,  0,  1,  0},
 {-1,  0,  0,  0,  1, -1, -1, -1,  0,  0,  0,  1,  1,  1, -1,  0,  0,  0,  1},
 {-1,  0,  0,  0,  1, -1,  4, -1,  0,  0,  0,  1, -4,  1, -1,  0,  0,  0,  1},
 {-1, -1, -1, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1,  1,  1,  1},
 {-1, -1,  4, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1, -4,  1,  1},
 {-2,  1, -1,  1, -2,  1, -1,  1,  2,  0,  2,  1, -1,  1, -2,  1, -1,  1, -2},
 {-2,  1,  2,  1, -2,  1,  2,  1, -4,  0, -4,  1,  2,  1, -2,  1,  2,  1, -2},
 { 0, -1, -1, -1,  0,  1,  1,  1,  0,  0,  0,  1,  1,  1,  0, -1, -1, -1,  0},
 { 0, -1,  2, -1,  0,  1, -2,  1,  0,  0,  0,  1, -2,  1,  0, -1,  2, -1,  0},
 { 0,  0,  0,  0,  0,  1,  0, -1,  0,  0,  0, -1,  0,  1,  0,  0,  0,  0,  0},
 { 1,  0,  0,  0, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0, -1,  0,  0,  0,  1},
 { 0,  1,  0, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0, -1,  0,  1,  0},
 { 0,  1,  0, -1,  0, -1,  0,  1,  0,  0,  0, -1,  0,  1,  0,  1,  0, -1,  0},
 {-1,  0,  0,  0,  1,  1,  0,  1,  0,  0,  0, -1,  0, -1, -1,  0,  0,  0,  1},
 { 1, -1,  0, -1,  1,  0,  0,  0,  0,  0,  0,  0,  0,  0, -1,  1,  0,  1, -1}};

/* Viscous moments relax with 1/tau_eff (Sec. 2.1 below eq:collision):
 * k = 9, 11, 13, 14, 15.  Appendix A.1 eq:freeparams, reading A3: conserved
 * moments 0, 3, 5, 7 at 1.0; omega_1 = 1.19; omega_2,10,12 = 1.6;
 * omega_4,6,8 = 1.2; omega_16,17,18 = 1.98. */
static const double S_FREE[Q] = {
    1.0, 1.19, 1.6, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 0.0,
    1.6, 0.0, 1.6, 0.0, 0.0, 0.0, 1.98, 1.98, 1.98};
static const int VISCOUS[Q] = {0,0,0,0,0,0,0,0,0,1,0,1,0,1,1,1,0,0,0};

static const double CS2 = 1.0 / 3.0;

static real rabs(real x) { return RE(x) < 0 ? -x : x; }

/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    int n_modes;
    int inlet;       /* 1: STG inlet at x = 0 and zero-gradient outlet; 0: periodic x */
    int walls;       /* 0: specular slip (the method); 1: halfway bounce-back; 2: periodic y (tests) */
    int wall_model;  /* 1: Reichardt force on the first off-wall cells (Sec. 2.3) */
    int mrt;         /* 1: rates of Appendix A.1; 0: every rate 1/tau_eff (BGK, test only) */
    int stats;       /* 1: accumulate z-averaged statistics every step */
    int threads;     /* OpenMP threads, 0 = library default */
    double re_tau;   /* friction Reynolds number u_tau delta / nu */
    double u_bulk;   /* bulk velocity U_b in lattice units */
    double c_smag;   /* C_smag Delta^2 of eq:smogrinsky_model */
    double kappa0, B0;      /* wall-law constants that fix u_tau,ref and nu at creation */
    double k_ratio;  /* geometric ratio of the STG wavenumbers */
    double beta_kmin;/* k_min = beta 2 pi / max l_e */
    double tau0;     /* > 0 overrides tau0 = 3 nu + 1/2 */
    double body_force[3];   /* uniform force density (tests only) */
    int sponge_cells;       /* outlet sponge thickness in cells (0: none), reading A24 */
    double sponge_nu;       /* viscosity added at the outlet end of the sponge */
} orc_config;

typedef struct orc {
    orc_config c;
    long ncell;
    real theta[4];          /* (l_e, A, kappa, B) */
    double delta, utau_ref, nu, tau0, ubp;  /* flow constants, real */
    /* inlet tables */
    real *UR;               /* ny: Reichardt mean profile */
    double *Rp;             /* ny*6: prescribed R+ (11,22,33,12,13,23) */
    real *a;                /* ny*6: A * Cholesky factor (a11,a21,a22,a31,a32,a33) */
    real *ell;              /* ny: l_e(y) */
    real maxl;
    real *kn;               /* N */
    double *dn, *sn, *phin; /* N*3, N*3, N */
    real *sqrtq;            /* ny*N */
    /* lattice */
    real *f, *p;            /* 19*ncell: post-collision state, post-stream work */
    real *F;                /* 3*ncell: force density of the last collision */
    real *rho, *u;          /* ncell, 3*ncell: fields of the last collision */
    real *utau;             /* 2*nz*nx */
    long t;
    /* statistics (sums over z and steps) */
    double *st;             /* nx*ny*7 */
    double *st_utau;        /* 2*nx */
    long st_n;
    /* objective */
    int obj_on, obj_i0, obj_i1, obj_iR;
    long obj_T;
    real obj_tau;           /* sum tau_w / u_tau,ref^2 */
    real *obj_u, *obj_v, *obj_uv;  /* ny sums at x = iR */
} orc;

#define IDX(h, i, j, k) (((long)(k) * (h)->c.ny + (j)) * (h)->c.nx + (i))

/* ---- Sec. 2.3 eq:reichard, reading A7: textbook coefficients ----
 * u+ = (1/kappa) ln(1 + kappa y+) + B (1 - e^{-y+/11} - (y+/11) e^{-y+/3}) */
static real reichardt(real yp, real kappa, real B) {
    return log(1.0 + kappa * yp) / kappa
         + B * (1.0 - exp(-yp / 11.0) - (yp / 11.0) * exp(-yp / 3.0));
}
static real reichardt_dy(real yp, real kappa, real B) {
    return 1.0 / (1.0 + kappa * yp)
         + B * (exp(-yp / 11.0) / 11.0 - exp(-yp / 3.0) / 11.0 + (yp / 33.0) * exp(-yp / 3.0));
}

/* ---- Sec. 2.3 eq:u_tau_implicit: solve u_tau u+(y u_tau / nu) = u_hat by
 * Newton's method (reading A10: to 1e-13 relative, at most 50 iterations,
 * two extra iterations so a complex-step perturbation converges as well). */
static real solve_utau(real uhat, double y, double nu, real kappa, real B, real guess) {
    if (RE(uhat) <= 0) return 0.0 * uhat;
    real u = RE(guess) > 0 ? guess : 0.0 * uhat + 1e-3;
    int extra = 0;
    for (int it = 0; it < 60; ++it) {
        real yp = y * u / nu;
        real r = u * reichardt(yp, kappa, B) - uhat;
        real dr = reichardt(yp, kappa, B) + yp * reichardt_dy(yp, kappa, B);
        real du = r / dr;
        u = u - du;
        if (RE(u) <= 0) u = 0.5 * (u + du);   /* stay positive */
        if (fabs(RE(du)) < 1e-13 * fabs(RE(u))) { if (++extra >= 2) break; }
    }
    return u;
}

/* ---- eq:bc_eq: second-order equilibrium f^eq_i(rho, u) ---- */
static void feq(real rho, const real u[3], real out[Q]) {
    real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        real cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        out[i] = W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2));
    }
}

/* ---- eq:mom_f: m = M f (dense) ---- */
static void moments(const real f[Q], real m[Q]) {
    for (int k = 0; k < Q; ++k) {
        real s = 0;
        for (int i = 0; i < Q; ++i) s += M[k][i] * f[i];
        m[k] = s;
    }
}

/* ---- M^{-1} m = M^T D^{-1} m with D_kk = sum_i M_ki^2 ---- */
static void inverse_moments(const real m[Q], real f[Q]) {
    double D[Q];
    for (int k = 0; k < Q; ++k) {
        double s = 0;
        for (int i = 0; i < Q; ++i) s += M[k][i] * M[k][i];
        D[k] = s;
    }
    for (int i = 0; i < Q; ++i) {
        real s = 0;
        for (int k = 0; k < Q; ++k) s += M[k][i] * m[k] / D[k];
        f[i] = s;
    }
}

/* ---- eq:tau_eff, reading A6 ---- */
static real tau_eff(double tau0, double c_smag, real rho, const real pineq[3][3]) {
    real q = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q += pineq[a][b] * pineq[a][b];
    real q12 = sqrt(q);
    return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * sqrt(2.0) * c_smag * q12 / rho));
}

/* ---- One cell: macroscopic moments (eq:density, eq:momentum, eq:tensor),
 * SGS closure (Sec. 2.2), MRT collision with the Guo force (eq:lbe_mrt,
 * eq:bodyforce in moment space, reading A4).  p are post-stream populations,
 * F the force density acting on the cell, out the post-collision populations. */
static void collide_cell(const real p[Q], const real F[3], double tau0, double c_smag,
                         int mrt, real out[Q], real *rho_out, real u_out[3]) {
    real rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        rho += p[i];
        for (int a = 0; a < 3; ++a) j[a] += p[i] * C[i][a];
    }
    real u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;

    real fe[Q];
    feq(rho, u, fe);
    real pineq[3][3] = {{0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) pineq[a][b] += C[i][a] * C[i][b] * (p[i] - fe[i]);
    real te = tau_eff(tau0, c_smag, rho, pineq);

    real s[Q];
    for (int k = 0; k < Q; ++k) {
        if (!mrt) s[k] = 1.0 / te;
        else s[k] = VISCOUS[k] ? 1.0 / te : S_FREE[k] + 0.0 * te;
    }

    /* Guo source in population space, eq:bodyforce without the (1 - omega/2) factor */
    real Ft[Q];
    for (int i = 0; i < Q; ++i) {
        real cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        real acc = 0;
        for (int a = 0; a < 3; ++a) acc += ((C[i][a] - u[a]) / CS2 + cu * C[i][a] / (CS2 * CS2)) * F[a];
        Ft[i] = W[i] * acc;
    }
    real m[Q], me[Q], mF[Q], ms[Q];
    moments(p, m);
    moments(fe, me);
    moments(Ft, mF);
    for (int k = 0; k < Q; ++k) ms[k] = m[k] - s[k] * (m[k] - me[k]) + (1.0 - 0.5 * s[k]) * mF[k];
    inverse_moments(ms, out);
    if (rho_out) *rho_out = rho;
    if (u_out) for (int a = 0; a < 3; ++a) u_out[a] = u[a];
}

/* ---- Sec. 3.1, eq:f_i, eq:bc_eq, eq:f_i_neq, eq:pi_neq, eq:density_bc:
 * regularized velocity inlet on a face with inward normal +x.  Known
 * populations after streaming are those with c_x <= 0 (readings A13-A15). */
static void inlet_reconstruct(const real p[Q], const real uin[3], real out[Q], real *rho_in) {
    real s0 = 0, sm = 0;
    for (int i = 0; i < Q; ++i) {
        if (C[i][0] == 0) s0 += p[i];
        if (C[i][0] < 0) sm += p[i];
    }
    real rho = (s0 + 2.0 * sm) / (1.0 - uin[0]);
    real fe[Q], fneq[Q];
    feq(rho, uin, fe);
    for (int i = 0; i < Q; ++i) fneq[i] = p[i] - fe[i];
    for (int i = 0; i < Q; ++i) {
        if (C[i][0] > 0) {
            int inv = -1;
            for (int k = 0; k < Q; ++k)
                if (C[k][0] == -C[i][0] && C[k][1] == -C[i][1] && C[k][2] == -C[i][2]) inv = k;
            fneq[i] = p[inv] - fe[inv];
        }
    }
    real Pi[3][3] = {{0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Pi[a][b] += (C[i][a] * C[i][b] - (a == b ? CS2 : 0.0)) * fneq[i];
    for (int i = 0; i < Q; ++i) {
        real qp = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) qp += (C[i][a] * C[i][b] - (a == b ? CS2 : 0.0)) * Pi[a][b];
        out[i] = fe[i] + W[i] / (2.0 * CS2 * CS2) * qp;
    }
    if (rho_in) *rho_in = rho;
}

/* ------------------------------------------------------------------------ */
static double wall_distance(int j, int ny) {     /* reading A8 */
    double y = j + 0.5;
    return y < ny - y ? y : ny - y;
}

/* Prescribed Reynolds stress in wall units (reading A16 vi):
 * -R12+ = s = (1 - d/delta)(1 - exp(-d+/26))^2, R11+ = 3s + 0.1,
 * R22+ = s + 0.1, R33+ = 2s + 0.1, R13 = R23 = 0; R12 changes sign in the upper half. */
static void reynolds_stress_plus(int j, int ny, double re_tau, double out[6]) {
    double delta = 0.5 * ny, d = wall_distance(j, ny), dp = d * re_tau / delta;
    double e = 1.0 - exp(-dp / 26.0);
    double s = (1.0 - d / delta) * e * e;
    out[0] = 3 * s + 0.1; out[1] = s + 0.1; out[2] = 2 * s + 0.1;
    out[3] = (j + 0.5 < 0.5 * ny) ? -s : s;
    out[4] = 0; out[5] = 0;
}

/* STG tables, reading A16 (Sec. 3.1 eq:aux_vec and the cited STG method). */
static void stg_tables(orc *h, const double *uniforms) {
    int ny = h->c.ny, N = h->c.n_modes;
    real le = h->theta[0], A = h->theta[1], kap = h->theta[2], B = h->theta[3];
    double delta = h->delta;
    /* mean profile U_R(y) = u_tau,ref u+(d u_tau,ref / nu) */
    for (int j = 0; j < ny; ++j) {
        double d = wall_distance(j, ny);
        h->UR[j] = h->utau_ref * reichardt(d * h->utau_ref / h->nu + 0.0 * kap, kap, B);
    }
    /* eq:cholesky applied to R = R+ u_tau,ref^2, times the amplitude A */
    for (int j = 0; j < ny; ++j) {
        double *Rp = h->Rp + 6 * j;
        reynolds_stress_plus(j, ny, h->c.re_tau, Rp);
        double u2 = h->utau_ref * h->utau_ref;
        double R11 = Rp[0] * u2, R22 = Rp[1] * u2, R33 = Rp[2] * u2;
        double R21 = Rp[3] * u2, R31 = Rp[4] * u2, R32 = Rp[5] * u2;
        double a11 = sqrt(R11);
        double a21 = R21 / a11;
        double a22 = sqrt(R22 - a21 * a21);
        double a31 = R31 / a11;
        double a32 = (R32 - a21 * a31) / a22;
        double a33 = sqrt(R33 - a31 * a31 - a32 * a32);
        real *a = h->a + 6 * j;
        a[0] = A * a11; a[1] = A * a21; a[2] = A * a22; a[3] = A * a31; a[4] = A * a32; a[5] = A * a33;
    }
    /* length scale l_e(y) = l_e delta tanh(2 d / (l_e delta)) */
    real maxl = 0;
    for (int j = 0; j < ny; ++j) {
        double d = wall_distance(j, ny);
        h->ell[j] = le * delta * tanh(2.0 * d / (le * delta));
        if (j == 0 || RE(h->ell[j]) > RE(maxl)) maxl = h->ell[j];
    }
    h->maxl = maxl;
    /* wavenumbers k_n = k_min r^(n-1), k_min = beta 2 pi / max l_e */
    real kmin = h->c.beta_kmin * 2.0 * PI_D / maxl;
    for (int n = 0; n < N; ++n) h->kn[n] = kmin * pow(h->c.k_ratio, (double)n);
    /* random modes: d uniform on the sphere, sigma uniform in the plane normal
     * to d, phase uniform in [0, 2 pi) -- four uniforms per mode */
    for (int n = 0; n < N; ++n) {
        const double *U = uniforms + 4 * n;
        double ct = 1.0 - 2.0 * U[0], st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 2.0 * PI_D * U[1], al = 2.0 * PI_D * U[2];
        double d[3] = {st * cos(ph), st * sin(ph), ct};
        double et[3] = {ct * cos(ph), ct * sin(ph), -st};
        double ep[3] = {-sin(ph), cos(ph), 0.0};
        for (int a = 0; a < 3; ++a) {
            h->dn[3 * n + a] = d[a];
            h->sn[3 * n + a] = cos(al) * et[a] + sin(al) * ep[a];
        }
        h->phin[n] = 2.0 * PI_D * U[3];
    }
    /* q_n(y) = E(k_n) dk_n / sum_m E(k_m) dk_m, modified von Karman spectrum */
    double kcut = 2.0 * PI_D / 2.0;
    for (int j = 0; j < ny; ++j) {
        double d = wall_distance(j, ny);
        real ke = 2.0 * PI_D / h->ell[j];
        double eps = h->utau_ref * h->utau_ref * h->utau_ref / (h->c.kappa0 * d);
        double keta = 2.0 * PI_D * pow(eps / (h->nu * h->nu * h->nu), 0.25);
        real tot = 0;
        real *E = (real *)malloc(sizeof(real) * N);
        for (int n = 0; n < N; ++n) {
            real k = h->kn[n];
            real dk = k * (1.0 - 1.0 / h->c.k_ratio);
            real r = k / ke;
            real fe = exp(-(12.0 * k / keta) * (12.0 * k / keta));
            real over = RE(k) > 0.9 * kcut ? k - 0.9 * kcut : 0.0 * k;
            real xc = 4.0 * over / kcut;
            real fc = exp(-(xc * xc * xc));
            E[n] = (r * r) * (r * r) / pow(1.0 + 2.4 * r * r, 17.0 / 6.0) * fe * fc * dk;
            tot += E[n];
        }
        for (int n = 0; n < N; ++n) h->sqrtq[(long)j * N + n] = sqrt(E[n] / tot);
        free(E);
    }
}

/* eq:u_couple, eq:v_fluc, eq:aux_vec at time t (reading A16 iv, A17):
 * u_in = (U_R, 0, 0) + a v',  v' = sqrt6 sum_n sqrt(q_n) sigma_n cos(k_n d_n . x' + phi_n),
 * x' = ((x - U_b t) 2 pi / (k_n max l_e), y, z), inlet plane at x = 0. */
static void inlet_velocity(const orc *h, int j, int k, long t, real out[3]) {
    int N = h->c.n_modes;
    double y = j + 0.5, z = k + 0.5, x = 0.0;
    real v[3] = {0, 0, 0};
    for (int n = 0; n < N; ++n) {
        real kn = h->kn[n];
        const double *d = h->dn + 3 * n, *s = h->sn + 3 * n;
        real xp = (x - h->c.u_bulk * (double)t) * 2.0 * PI_D / (kn * h->maxl);
        real arg = kn * (d[0] * xp + d[1] * y + d[2] * z) + h->phin[n];
        real c = h->sqrtq[(long)j * N + n] * cos(arg);
        for (int a = 0; a < 3; ++a) v[a] += s[a] * c;
    }
    for (int a = 0; a < 3; ++a) v[a] *= sqrt(6.0);
    const real *a = h->a + 6 * j;
    out[0] = h->UR[j] + a[0] * v[0];
    out[1] = a[1] * v[0] + a[2] * v[1];
    out[2] = a[3] * v[0] + a[4] * v[1] + a[5] * v[2];
}

/* ------------------------------------------------------------------------ */
orc *API(create)(const orc_config *cfg, const double *theta_re, const double *theta_im,
                 const double *uniforms) {
    orc *h = (orc *)calloc(1, sizeof(orc));
    h->c = *cfg;
    int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz, N = cfg->n_modes;
    h->ncell = (long)nx * ny * nz;
    for (int k = 0; k < 4; ++k) {
        h->theta[k] = theta_re[k];
#ifdef ORC_COMPLEX
        if (theta_im) h->theta[k] += I * theta_im[k];
#else
        (void)theta_im;
#endif
    }
    /* flow constants (reading A20): delta = ny/2, U_b+ = mean of u+ over the
     * cell centres with the creation constants, u_tau,ref = U_b / U_b+,
     * nu = u_tau,ref delta / Re_tau, tau0 = 3 nu + 1/2 (eq:nu). */
    h->delta = 0.5 * ny;
    double ubp = 0;
    for (int j = 0; j < ny; ++j)
        ubp += RE(reichardt(wall_distance(j, ny) * cfg->re_tau / h->delta, cfg->kappa0, cfg->B0));
    ubp /= ny;
    h->ubp = ubp;
    h->utau_ref = cfg->u_bulk / ubp;
    h->nu = h->utau_ref * h->delta / cfg->re_tau;
    h->tau0 = cfg->tau0 > 0 ? cfg->tau0 : 3.0 * h->nu + 0.5;

    h->UR = (real *)calloc(ny, sizeof(real));
    h->Rp = (double *)calloc((size_t)6 * ny, sizeof(double));
    h->a = (real *)calloc((size_t)6 * ny, sizeof(real));
    h->ell = (real *)calloc(ny, sizeof(real));
    h->kn = (real *)calloc(N > 0 ? N : 1, sizeof(real));
    h->dn = (double *)calloc((size_t)3 * (N > 0 ? N : 1), sizeof(double));
    h->sn = (double *)calloc((size_t)3 * (N > 0 ? N : 1), sizeof(double));
    h->phin = (double *)calloc(N > 0 ? N : 1, sizeof(double));
    h->sqrtq = (real *)calloc((size_t)ny * (N > 0 ? N : 1), sizeof(real));
    h->f = (real *)calloc((size_t)Q * h->ncell, sizeof(real));
    h->p = (real *)calloc((size_t)Q * h->ncell, sizeof(real));
    h->F = (real *)calloc((size_t)3 * h->ncell, sizeof(real));
    h->rho = (real *)calloc(h->ncell, sizeof(real));
    h->u = (real *)calloc((size_t)3 * h->ncell, sizeof(real));
    h->utau = (real *)calloc((size_t)2 * nz * nx, sizeof(real));
    h->st = (double *)calloc((size_t)7 * nx * ny, sizeof(double));
    h->st_utau = (double *)calloc((size_t)2 * nx, sizeof(double));
    h->obj_u = (real *)calloc(ny, sizeof(real));
    h->obj_v = (real *)calloc(ny, sizeof(real));
    h->obj_uv = (real *)calloc(ny, sizeof(real));
    if (N > 0) stg_tables(h, uniforms);
    else for (int j = 0; j < ny; ++j)
        h->UR[j] = h->utau_ref * reichardt(wall_distance(j, ny) * h->utau_ref / h->nu, h->theta[2], h->theta[3]);

    /* initial state (reading A20): f = f^eq(1, (U_R(y), 0, 0)) everywhere */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long c = IDX(h, i, j, k);
                real u[3] = {h->UR[j], 0, 0}, fe[Q];
                feq(1.0 + 0.0 * h->UR[j], u, fe);
                for (int q = 0; q < Q; ++q) h->f[(long)q * h->ncell + c] = fe[q];
                h->rho[c] = 1.0;
                h->u[3 * c] = h->UR[j];
            }
    for (long c = 0; c < 2L * nz * nx; ++c) h->utau[c] = h->utau_ref;
    return h;
}

void API(destroy)(orc *h) {
    if (!h) return;
    free(h->UR); free(h->Rp); free(h->a); free(h->ell); free(h->kn); free(h->dn); free(h->sn);
    free(h->phin); free(h->sqrtq); free(h->f); free(h->p); free(h->F); free(h->rho); free(h->u);
    free(h->utau); free(h->st); free(h->st_utau); free(h->obj_u); free(h->obj_v); free(h->obj_uv);
    free(h);
}

/* Streaming, eq:lbe left-hand side, as a pull: p_q(x) = f*_q(x - c_q).
 * z periodic; x periodic or (inlet on) marked unknown beyond the faces;
 * y: specular slip (A12), halfway bounce-back, or periodic. */
static void stream(orc *h) {
    int nx = h->c.nx, ny = h->c.ny, nz = h->c.nz;
    long n = h->ncell;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                for (int q = 0; q < Q; ++q) {
                    int sx = i - C[q][0], sy = j - C[q][1], sz = k - C[q][2], sq = q;
                    sz = (sz + nz) % nz;
                    if (sy < 0 || sy >= ny) {
                        if (h->c.walls == 2) {
                            sy = (sy + ny) % ny;
                        } else if (h->c.walls == 1) {      /* halfway bounce-back */
                            sx = i; sy = j; sz = k;
                            for (int r = 0; r < Q; ++r)
                                if (C[r][0] == -C[q][0] && C[r][1] == -C[q][1] && C[r][2] == -C[q][2]) sq = r;
                        } else {                            /* specular: mirror c_y */
                            sy = j;
                            for (int r = 0; r < Q; ++r)
                                if (C[r][0] == C[q][0] && C[r][1] == -C[q][1] && C[r][2] == C[q][2]) sq = r;
                        }
                    }
                    real v;
                    if (sx < 0 || sx >= nx) {
                        if (h->c.inlet) v = 0.0;           /* unknown; rebuilt below */
                        else { sx = (sx + nx) % nx; v = h->f[(long)sq * n + IDX(h, sx, sy, sz)]; }
                    } else {
                        v = h->f[(long)sq * n + IDX(h, sx, sy, sz)];
                    }
                    h->p[(long)q * n + IDX(h, i, j, k)] = v;
                }
    if (h->c.inlet) {
        /* reading A18: zero-gradient outlet, unknown populations at x = nx-1
         * copied from x = nx-2 after streaming */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int q = 0; q < Q; ++q)
                    if (C[q][0] < 0)
                        h->p[(long)q * n + IDX(h, nx - 1, j, k)] = h->p[(long)q * n + IDX(h, nx - 2, j, k)];
    }
}

static void cell_pops(const orc *h, long c, real out[Q]) {
    for (int q = 0; q < Q; ++q) out[q] = h->p[(long)q * h->ncell + c];
}

/* Algorithm 1 steps 4-8 on every inlet cell (x = 0). */
static void inlet_pass(orc *h) {
    int ny = h->c.ny, nz = h->c.nz;
    long n = h->ncell;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            long c = IDX(h, 0, j, k);
            real pc[Q], out[Q], uin[3];
            cell_pops(h, c, pc);
            inlet_velocity(h, j, k, h->t, uin);
            inlet_reconstruct(pc, uin, out, NULL);
            for (int q = 0; q < Q; ++q) h->p[(long)q * n + c] = out[q];
        }
}

static void macro_u0(const real p[Q], real *rho, real u0[3]) {
    real r = 0, j[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        r += p[q];
        for (int a = 0; a < 3; ++a) j[a] += p[q] * C[q][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u0[a] = j[a] / r;
}

/* Algorithm 1 steps 9-14 on the first off-wall cells (Sec. 2.3). */
static void wall_pass(orc *h) {
    int nx = h->c.nx, ny = h->c.ny, nz = h->c.nz;
    real kap = h->theta[2], B = h->theta[3];
#pragma omp parallel for collapse(2) schedule(static)
    for (int w = 0; w < 2; ++w)
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                int jw = w == 0 ? 0 : ny - 1, j2 = w == 0 ? 1 : ny - 2;
                double nrm[3] = {0, w == 0 ? 1.0 : -1.0, 0};
                long cw = IDX(h, i, jw, k), c2 = IDX(h, i, j2, k);
                real pw[Q], p2[Q], rw, r2, uw[3], u2[3];
                cell_pops(h, cw, pw);
                cell_pops(h, c2, p2);
                macro_u0(pw, &rw, uw);
                macro_u0(p2, &r2, u2);
                /* eq:base */
                real un = u2[0] * nrm[0] + u2[1] * nrm[1] + u2[2] * nrm[2];
                real tv[3], tn = 0;
                for (int a = 0; a < 3; ++a) { tv[a] = u2[a] - un * nrm[a]; tn += tv[a] * tv[a]; }
                tn = sqrt(tn);
                real *Fc = h->F + 3 * cw;
                long iu = ((long)w * nz + k) * nx + i;
                if (RE(tn) < 1e-12) { Fc[0] = Fc[1] = Fc[2] = 0.0 * tn; continue; }
                real ex[3];
                for (int a = 0; a < 3; ++a) ex[a] = tv[a] / tn;
                /* eq:uhat */
                real uhat = uw[0] * ex[0] + uw[1] * ex[1] + uw[2] * ex[2];
                double sg = RE(uhat) < 0 ? -1.0 : 1.0;
                /* eq:u_tau_implicit with the first cell centre at y = 1/2 */
                real ut = solve_utau(rabs(uhat), 0.5, h->nu, kap, B, h->utau[iu]);
                h->utau[iu] = ut;
                /* tau_w = rho u_tau^2, eq:force_wm with A = 1 (reading A11) */
                real tw = rw * ut * ut;
                for (int a = 0; a < 3; ++a) Fc[a] = Fc[a] - tw * ex[a] * sg;
            }
}

static void accumulate(orc *h) {
    int nx = h->c.nx, ny = h->c.ny, nz = h->c.nz;
    if (h->c.stats) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s[7] = {0};
                for (int k = 0; k < nz; ++k) {
                    long c = IDX(h, i, j, k);
                    double u = RE(h->u[3 * c]), v = RE(h->u[3 * c + 1]), w = RE(h->u[3 * c + 2]);
                    s[0] += u; s[1] += v; s[2] += w;
                    s[3] += u * u; s[4] += v * v; s[5] += w * w; s[6] += u * v;
                }
                for (int a = 0; a < 7; ++a) h->st[((long)j * nx + i) * 7 + a] += s[a];
            }
        if (h->c.wall_model)
            for (int w = 0; w < 2; ++w)
                for (int i = 0; i < nx; ++i) {
                    double s = 0;
                    for (int k = 0; k < nz; ++k) s += RE(h->utau[((long)w * nz + k) * nx + i]);
                    h->st_utau[w * nx + i] += s;
                }
        h->st_n += 1;
    }
    if (h->obj_on) {
        real ur2 = h->utau_ref * h->utau_ref + 0.0 * h->theta[0];
        for (int w = 0; w < 2; ++w) {
            int jw = w == 0 ? 0 : ny - 1;
            for (int k = 0; k < nz; ++k)
                for (int i = h->obj_i0; i < h->obj_i1; ++i) {
                    real ut = h->utau[((long)w * nz + k) * nx + i];
                    h->obj_tau += h->rho[IDX(h, i, jw, k)] * ut * ut / ur2;
                }
        }
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                long c = IDX(h, h->obj_iR, j, k);
                h->obj_u[j] += h->u[3 * c];
                h->obj_v[j] += h->u[3 * c + 1];
                h->obj_uv[j] += h->u[3 * c] * h->u[3 * c + 1];
            }
        h->obj_T += 1;
    }
}

/* One time step of Algorithm 1 with the state held post-collision:
 * stream (+ outlet copy) -> inlet steps 4-8 -> wall steps 9-14 -> step 15 collide. */
static void one_step(orc *h) {
    int nx = h->c.nx, ny = h->c.ny, nz = h->c.nz;
    long n = h->ncell;
    stream(h);
    if (h->c.inlet) inlet_pass(h);
    for (long c = 0; c < 3 * n; ++c) h->F[c] = 0.0;
    if (h->c.wall_model && h->c.walls == 0) wall_pass(h);
    double tau0 = h->tau0, cs = h->c.c_smag;
    int mrt = h->c.mrt;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long c = IDX(h, i, j, k);
                real pc[Q], out[Q], Fc[3], r, u[3];
                cell_pops(h, c, pc);
                for (int a = 0; a < 3; ++a) {
                    h->F[3 * c + a] += h->c.body_force[a];
                    Fc[a] = h->F[3 * c + a];
                }
                double t0c = tau0;
                if (h->c.sponge_cells > 0) {           /* A24 */
                    const double L = h->c.sponge_cells;
                    double ramp = (i + 0.5 - (nx - L)) / L;
                    ramp = ramp < 0.0 ? 0.0 : (ramp > 1.0 ? 1.0 : ramp);
                    t0c = tau0 + 3.0 * h->c.sponge_nu * ramp * ramp;
                }
                collide_cell(pc, Fc, t0c, cs, mrt, out, &r, u);
                for (int q = 0; q < Q; ++q) h->f[(long)q * n + c] = out[q];
                h->rho[c] = r;
                for (int a = 0; a < 3; ++a) h->u[3 * c + a] = u[a];
            }
    accumulate(h);
    h->t += 1;
}

void API(step)(orc *h, int nsteps) {
#ifdef _OPENMP
    if (h->c.threads > 0) omp_set_num_threads(h->c.threads);
#endif
    for (int s = 0; s < nsteps; ++s) one_step(h);
}

/* ---- state and field access (real parts) ---- */
void API(get_state)(const orc *h, double *f) {
    for (long c = 0; c < Q * h->ncell; ++c) f[c] = RE(h->f[c]);
}
void API(get_state_imag)(const orc *h, double *f) {
    for (long c = 0; c < Q * h->ncell; ++c) f[c] = IMAG(h->f[c]);
}
void API(set_state)(orc *h, const double *f_re, const double *f_im) {
    for (long c = 0; c < Q * h->ncell; ++c) {
        h->f[c] = f_re[c];
#ifdef ORC_COMPLEX
        if (f_im) h->f[c] += I * f_im[c];
#else
        (void)f_im;
#endif
    }
}
void API(get_fields)(const orc *h, double *rho, double *u) {
    for (long c = 0; c < h->ncell; ++c) {
        rho[c] = RE(h->rho[c]);
        for (int a = 0; a < 3; ++a) u[3 * c + a] = RE(h->u[3 * c + a]);
    }
}
void API(get_force)(const orc *h, double *F) {
    for (long c = 0; c < 3 * h->ncell; ++c) F[c] = RE(h->F[c]);
}
void API(get_utau)(const orc *h, double *ut) {
    for (long c = 0; c < 2L * h->c.nz * h->c.nx; ++c) ut[c] = RE(h->utau[c]);
}
void API(set_utau)(orc *h, const double *ut) {
    for (long c = 0; c < 2L * h->c.nz * h->c.nx; ++c) h->utau[c] = ut[c];
}
long API(get_time)(const orc *h) { return h->t; }
void API(set_time)(orc *h, long t) { h->t = t; }

/* constants: delta, u_tau,ref, nu, tau0, U_b+, max l_e */
void API(get_constants)(const orc *h, double out[6]) {
    out[0] = h->delta; out[1] = h->utau_ref; out[2] = h->nu; out[3] = h->tau0; out[4] = h->ubp;
    out[5] = RE(h->maxl);
}
/* tables: UR[ny], a[ny*6], Rp[ny*6], ell[ny], kn[N], dn[3N], sn[3N], phin[N], sqrtq[ny*N] */
void API(get_tables)(const orc *h, double *UR, double *a, double *Rp, double *ell, double *kn,
                     double *dn, double *sn, double *phin, double *sqrtq) {
    int ny = h->c.ny, N = h->c.n_modes;
    for (int j = 0; j < ny; ++j) {
        UR[j] = RE(h->UR[j]); ell[j] = RE(h->ell[j]);
        for (int a6 = 0; a6 < 6; ++a6) { a[6 * j + a6] = RE(h->a[6 * j + a6]); Rp[6 * j + a6] = h->Rp[6 * j + a6]; }
    }
    for (int n = 0; n < N; ++n) {
        kn[n] = RE(h->kn[n]); phin[n] = h->phin[n];
        for (int a3 = 0; a3 < 3; ++a3) { dn[3 * n + a3] = h->dn[3 * n + a3]; sn[3 * n + a3] = h->sn[3 * n + a3]; }
    }
    for (long c = 0; c < (long)ny * N; ++c) sqrtq[c] = RE(h->sqrtq[c]);
}
/* inlet velocity u_in(j, k, t) for all inlet cells: out[(k*ny + j)*3 + a] */
void API(inlet_velocity)(const orc *h, long t, double *out) {
    for (int k = 0; k < h->c.nz; ++k)
        for (int j = 0; j < h->c.ny; ++j) {
            real u[3];
            inlet_velocity(h, j, k, t, u);
            for (int a = 0; a < 3; ++a) out[((long)k * h->c.ny + j) * 3 + a] = RE(u[a]);
        }
}

/* ---- statistics ---- */
void API(stats_reset)(orc *h) {
    memset(h->st, 0, sizeof(double) * 7 * h->c.nx * h->c.ny);
    memset(h->st_utau, 0, sizeof(double) * 2 * h->c.nx);
    h->st_n = 0;
}
long API(stats_get)(const orc *h, double *sums, double *utau_sums) {
    memcpy(sums, h->st, sizeof(double) * 7 * h->c.nx * h->c.ny);
    memcpy(utau_sums, h->st_utau, sizeof(double) * 2 * h->c.nx);
    return h->st_n;
}

/* ---- objective J = J_tau + J_R over the steps after objective_begin ----
 * J_tau = mean over steps and over wall cells with i0 <= i < i1 (both walls)
 *         of tau_w / u_tau,ref^2
 * J_R   = sum_j ( <u'v'>(iR, j) / u_tau,ref^2 - R12+(j) )^2, with <.> the mean
 *         over z and steps, <u'v'> = <uv> - <u><v>. */
void API(objective_begin)(orc *h, int i0, int i1, int iR) {
    h->obj_on = 1; h->obj_i0 = i0; h->obj_i1 = i1; h->obj_iR = iR; h->obj_T = 0;
    h->obj_tau = 0;
    for (int j = 0; j < h->c.ny; ++j) h->obj_u[j] = h->obj_v[j] = h->obj_uv[j] = 0;
}
void API(objective_value)(const orc *h, double *J_re, double *J_im, double *parts) {
    int ny = h->c.ny, nz = h->c.nz;
    double T = (double)h->obj_T;
    real ur2 = h->utau_ref * h->utau_ref;
    /* an empty wall range contributes nothing */
    real Jt = h->obj_i1 > h->obj_i0 ? h->obj_tau / (T * 2.0 * (h->obj_i1 - h->obj_i0) * nz) : 0.0 * h->obj_tau;
    real JR = 0;
    for (int j = 0; j < ny; ++j) {
        double cnt = T * nz;
        real mu = h->obj_u[j] / cnt, mv = h->obj_v[j] / cnt, muv = h->obj_uv[j] / cnt;
        real r = (muv - mu * mv) / ur2 - h->Rp[6 * j + 3];
        JR += r * r;
    }
    real J = Jt + JR;
    *J_re = RE(J);
    *J_im = IMAG(J);
    if (parts) { parts[0] = RE(Jt); parts[1] = RE(JR); parts[2] = IMAG(Jt); parts[3] = IMAG(JR); }
}

/* ---- single-cell building blocks exposed for the closed-form checks ---- */
void API(matrix)(double *Mout, double *wout, int *cout) {
    for (int k = 0; k < Q; ++k)
        for (int i = 0; i < Q; ++i) Mout[k * Q + i] = M[k][i];
    for (int i = 0; i < Q; ++i) {
        wout[i] = W[i];
        for (int a = 0; a < 3; ++a) cout[3 * i + a] = C[i][a];
    }
}
void API(cell_feq)(double rho, const double u[3], double out[Q]) {
    real uu[3] = {u[0], u[1], u[2]}, o[Q];
    feq(rho, uu, o);
    for (int i = 0; i < Q; ++i) out[i] = RE(o[i]);
}
void API(cell_moments)(const double f[Q], double m[Q]) {
    real ff[Q], mm[Q];
    for (int i = 0; i < Q; ++i) ff[i] = f[i];
    moments(ff, mm);
    for (int i = 0; i < Q; ++i) m[i] = RE(mm[i]);
}
void API(cell_collide)(const double p[Q], const double F[3], double tau0, double c_smag, int mrt,
                       double out[Q], double *rho, double u[3]) {
    real pp[Q], FF[3] = {F[0], F[1], F[2]}, o[Q], r, uu[3];
    for (int i = 0; i < Q; ++i) pp[i] = p[i];
    collide_cell(pp, FF, tau0, c_smag, mrt, o, &r, uu);
    for (int i = 0; i < Q; ++i) out[i] = RE(o[i]);
    *rho = RE(r);
    for (int a = 0; a < 3; ++a) u[a] = RE(uu[a]);
}
double API(cell_tau_eff)(double tau0, double c_smag, double rho, const double pi6[6]) {
    /* pi6 = (xx, yy, zz, xy, yz, xz) */
    real P[3][3] = {{pi6[0], pi6[3], pi6[5]}, {pi6[3], pi6[1], pi6[4]}, {pi6[5], pi6[4], pi6[2]}};
    return RE(tau_eff(tau0, c_smag, rho, P));
}
void API(cell_inlet)(const double p[Q], const double uin[3], double out[Q], double *rho_in) {
    real pp[Q], uu[3] = {uin[0], uin[1], uin[2]}, o[Q], r;
    for (int i = 0; i < Q; ++i) pp[i] = p[i];
    inlet_reconstruct(pp, uu, o, &r);
    for (int i = 0; i < Q; ++i) out[i] = RE(o[i]);
    *rho_in = RE(r);
}
double API(reichardt)(double yp, double kappa, double B) { return RE(reichardt(yp, kappa, B)); }
double API(solve_utau)(double uhat, double y, double nu, double kappa, double B, double guess) {
    return RE(solve_utau(uhat, y, nu, kappa, B, guess));
}

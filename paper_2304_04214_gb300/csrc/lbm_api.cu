// lbm_api.cu -- host side of liblbm_gb300.so: the C ABI of include/lbm.h.
//
// The handle keeps the flow constants and the STG tables (built in FP64 on
// the host, Algorithm 1 steps 1-3), carves one device arena into the two
// lattices and the small buffers, and enqueues the kernels of
// lbm_device.cuh on the caller's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_device.cuh"
#include "lbm_staged.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
// sets of segment lattices of the adjoint window: the forward pass fills the
// last kSlotSets segments' sets, the recomputation of the others runs one
// segment ahead of the reverse steps
constexpr int kSlotSets = 3;

// Carves one device allocation into 256-byte aligned buffers.  With guard
// bands on (guard > 0, a debugging aid), a band of at least `guard` bytes sits
// before the first buffer and right after the end of every buffer (up to the
// next aligned start); their (offset, bytes) are recorded in *bands.
struct Arena {
    char *base = nullptr;
    size_t off = 0;
    size_t guard = 0;
    std::vector<std::pair<size_t, size_t>> *bands = nullptr;
    void band() {
        const size_t start = off;
        off = (off + guard + 255) & ~size_t(255);
        if (bands) bands->push_back({start, off - start});
    }
    template <class T>
    T *take(size_t count) {
        if (guard && off == 0) band();
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        if (guard) band();
        return p;
    }
};

// Host FP64 Reichardt law (Sec. 2.3 eq:reichard, textbook coefficients).
double uplus(double yp, double kap, double B) {
    return std::log1p(kap * yp) / kap + B * (1.0 - std::exp(-yp / 11.0) - yp / 11.0 * std::exp(-yp / 3.0));
}

// fractional turns -> 32-bit fixed point
uint32_t turns32(double turns) {
    double fr = turns - std::floor(turns);
    double v = std::floor(fr * 4294967296.0 + 0.5);
    if (v >= 4294967296.0) v -= 4294967296.0;
    return (uint32_t)(uint64_t)v;
}

// Forward-mode dual number (value, derivative) for the derivative tables of
// the adjoint: d/d ell_e of the STG spectrum and of max l_e.
struct Dual {
    double v = 0.0, d = 0.0;
    Dual() = default;
    Dual(double v_, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual dexp(Dual a) { const double e = std::exp(a.v); return {e, e * a.d}; }
inline Dual dsqrt(Dual a) { const double r = std::sqrt(a.v); return {r, a.d / (2.0 * r)}; }
inline Dual dtanh(Dual a) { const double t = std::tanh(a.v); return {t, (1.0 - t * t) * a.d}; }
inline Dual dpow(Dual a, double e) { const double p = std::pow(a.v, e); return {p, e * std::pow(a.v, e - 1.0) * a.d}; }
inline double dexp(double a) { return std::exp(a); }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dtanh(double a) { return std::tanh(a); }
inline double dpow(double a, double e) { return std::pow(a, e); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

}  // namespace

struct lbm_handle;

// Adjoint workspace (FP32 lattices, window T, checkpoint every K steps).
struct AdjointWork {
    bool bound = false, owns = false;
    void *mem = nullptr;
    int T = 0, K = 0;
    float *ckpt = nullptr, *seg = nullptr, *lamA = nullptr, *lamB = nullptr;
    float *ut_init = nullptr, *uthist = nullptr, *ut_scr = nullptr, *fw_scr = nullptr;
    float *vwin = nullptr, *luin = nullptr, *jr_coef = nullptr, *jr_mean = nullptr;
    float *dsq = nullptr, *aunit = nullptr, *dUR = nullptr;
    float4 *kphase = nullptr;
    double *gtheta = nullptr, *objacc = nullptr, *r12 = nullptr;
    float cell_scale = 0.f;
    bool have_lambda0 = false;
};

struct lbm_handle {
    int nx = 0, ny = 0, nz = 0;
    long long ncell = 0;
    // x-slab of a larger channel (lbm_set_slab): global length, global x of
    // local column 0, owned local columns [own_lo, own_hi)
    int nx_global = 0, x_offset = 0, own_lo = 0, own_hi = 0;
    double re_tau = 0;
    lbm_opts opts{};
    int n_modes = 0;
    double k_ratio = 1.01, beta_kmin = 0.5;
    std::vector<double> uniforms;
    double theta[4] = {0.4, 1.0, 0.4, 7.8};
    // flow constants (fixed at creation)
    double delta = 0, utau_ref = 0, nu = 0, tau0 = 0, ubp = 0, maxl = 0;
    // host tables
    std::vector<float> UR, amat, sq, sig;
    std::vector<float> sqsig;                 // [ny][N] x (sqrt(6 q), sigma)
    std::vector<uint32_t> alpha, beta, betaT, phi32;
    std::vector<uint64_t> rate64;
    // row base of the BF16 storage, [ny][RB_W]: f^eq_q(1, (U0(j), 0, 0)) - w_q
    // with U0 the inlet mean profile of creation (fixed for the handle's life:
    // the stored words are relative to it)
    std::vector<float> rowbase;
    // device
    int device = -1;                      // CUDA device of the bound memory (lbm_bind_memory)
    size_t guard_bytes = 0;               // guard bands between arena buffers (lbm_debug_guard_bands)
    std::vector<std::pair<size_t, size_t>> guards, adj_guards;   // (offset, bytes) of the bands
    bool bound = false, owns = false;
    void *mem = nullptr;
    size_t mem_bytes = 0;
    void *lat[2] = {nullptr, nullptr};
    int cur = 0;
    float *d_utau = nullptr, *d_fw = nullptr, *d_uin = nullptr, *d_ubuf = nullptr;
    double *d_st = nullptr, *d_st_utau = nullptr;
    unsigned *d_flags = nullptr;
    float *d_UR = nullptr, *d_amat = nullptr;   // inlet profile in use (one of the two buffers)
    float *d_prof = nullptr;                    // two buffers of 7 ny floats: U_R[ny], amp chol(R)[ny][6]
    int prof_cur = 0;                           // the buffer in use
    float4 *d_sqsig = nullptr;
    uint32_t *d_alpha = nullptr, *d_betaT = nullptr, *d_phi32 = nullptr;
    float *d_rowbase = nullptr;
    // STG ring, two halves of stg_ring time levels: the half in use holds the
    // inlet fluctuations of steps [stg_t0, stg_t0 + stg_len); the other one is
    // refilled on the aux stream, beside those steps, for the steps from
    // stg_next_t0 on (-1: no refill pending)
    int stg_ring = 1;
    int stg_half = 0;
    long long stg_t0 = 0, stg_len = 0, stg_next_t0 = -1;
    cudaEvent_t ev_stg_free = nullptr, ev_stg_ready = nullptr;
    long long check_every = 16;
    int step_kind = LBM_KERNEL_AUTO;    // step kernel variant (lbm_set_step_kernel)
    int sponge_cells = 0;               // outlet sponge (lbm_set_sponge): thickness, added viscosity
    double sponge_nu = 0.0;
    // tensor maps of the lattices the staged kernel has read (base -> map)
    struct MapEntry { const void *base = nullptr; CUtensorMap map; };
    MapEntry maps[32];
    int map_next = 0;
    uint64_t *d_rate64 = nullptr;
    cudaStream_t stream = nullptr;
    long long t = 0;
    long long steps_since_stats = 0;
    long n_samples = 0;
    // inlet profile (RANS input of Algorithm 1 steps 1-3): U[j], R[6j..6j+5]
    bool custom_profile = false;
    std::vector<double> prof_U, prof_R;
    double *d_tw = nullptr;                // [2][nx] wall-shear scratch
    long long *d_gt0 = nullptr;            // start time of the refill inside a graph
    bool fw_side = false;                  // d_fw was last written by the side-stream wall kernel
    cudaEvent_t ev_shear = nullptr;        // wall-shear reduction done on the side stream
    // the wall-row kernel runs beside the interior kernel on a side stream,
    // forked from and joined back into the handle's stream every step
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // a second side stream for the STG work of lbm_adjoint_step
    cudaStream_t aux = nullptr;
    // lbm_adjoint_step: the recomputation of the next segment beside the
    // reverse steps of the current one (its own stream; events per slot set)
    cudaStream_t rstream = nullptr;
    cudaEvent_t ev_rstart = nullptr, ev_rec[kSlotSets] = {}, ev_rev[kSlotSets] = {};
    cudaEvent_t ev_aux_fork = nullptr, ev_aux_join = nullptr;
    // inlet profile uploads (lbm_set_inlet_profile): pinned staging of U_R and
    // amp chol(R), one half per device buffer, copied on their own stream;
    // ev_prof_ready[b]: the upload into buffer b is done (and its staging half
    // free); ev_prof_free[b]: the steps that read buffer b are done
    float *pin_stage = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_prof_ready[2] = {nullptr, nullptr}, ev_prof_free[2] = {nullptr, nullptr};
    // instrumentation
    bool prof_on = false;
    int prof_every = 1;                    // time every prof_every-th step launch
    long long prof_count = 0;
    // CUDA graphs of one STG ring period of steps (lbm_step, see graph_segment)
    struct GraphSeg {
        long long key[9];                  // launch-relevant host state at the segment start
        cudaGraphExec_t exec = nullptr;
        long long d_launches = 0, after_since_stats = 0, d_samples = 0;
    };
    std::vector<GraphSeg> graphs;
    bool graphs_on = true;
    bool capturing = false;
    long long graph_launches = 0;
    long long graph_epoch = 0, graphs_built_epoch = 0;
    cudaStream_t gstream = nullptr;        // capture stream
    // fork / join of the refill inside a graph (events recorded in a capture
    // are waited on only inside it)
    cudaEvent_t ev_gfork = nullptr, ev_gjoin = nullptr;
    std::vector<cudaEvent_t> ev0, ev1;
    std::vector<int> ev_busy;              // steps a busy slot times (0: free)
    size_t ev_next = 0;
    double prof_ms = 0;
    long prof_n = 0, launches = 0;
    size_t elem = 4;

    size_t layout(Arena &ar) {
        const size_t N = (size_t)n_modes > 0 ? (size_t)n_modes : 1;
        lat[0] = ar.take<char>(19 * (size_t)ncell * elem);
        lat[1] = ar.take<char>(19 * (size_t)ncell * elem);
        d_utau = ar.take<float>(2 * (size_t)nz * nx);
        d_fw = ar.take<float>(6 * (size_t)nz * nx);
        // STG ring: two halves of 64 time levels each, fewer where a half
        // would exceed both 8 MB and 1/32 of the two lattices
        const size_t half_budget = std::max<size_t>(8u << 20, 2 * 19 * elem * (size_t)ncell / 32);
        stg_ring = (int)std::max<size_t>(1, std::min<size_t>(64, half_budget / (12 * (size_t)nz * ny)));
        d_uin = ar.take<float>(3 * (size_t)nz * ny * stg_ring * 2);
        d_ubuf = opts.stats_every > 0 ? ar.take<float>(3 * (size_t)ncell) : nullptr;
        d_st = ar.take<double>(7 * (size_t)nx * ny);
        d_st_utau = ar.take<double>(2 * (size_t)nx);
        d_tw = ar.take<double>(2 * (size_t)nx);
        d_gt0 = ar.take<long long>(1);
        d_flags = ar.take<unsigned>(4);
        d_prof = ar.take<float>(14 * (size_t)ny);
        d_UR = d_prof + 7 * (size_t)ny * prof_cur;
        d_amat = d_UR + ny;
        d_sqsig = ar.take<float4>((size_t)ny * N);
        d_alpha = ar.take<uint32_t>((size_t)ny * N);
        d_betaT = ar.take<uint32_t>((size_t)nz * N);
        d_phi32 = ar.take<uint32_t>(N);
        d_rate64 = ar.take<uint64_t>(N);
        d_rowbase = ar.take<float>((size_t)lbmk::RB_W * ny);
        return (ar.off + 255) & ~size_t(255);
    }

    // Row base of the BF16 storage from the current (creation-time) mean profile.
    void make_rowbase() {
        static const int cx[19] = {0, -1, 0, 1, 0, -1, 0, 1, -1, 0, 1, -1, 0, 1, 0, -1, 0, 1, 0};
        static const double w[19] = {1. / 36, 1. / 36, 1. / 18, 1. / 36, 1. / 36, 1. / 36, 1. / 18,
                                     1. / 36, 1. / 18, 1. / 3,  1. / 18, 1. / 36, 1. / 18, 1. / 36,
                                     1. / 36, 1. / 36, 1. / 18, 1. / 36, 1. / 36};
        rowbase.assign((size_t)lbmk::RB_W * ny, 0.f);
        for (int j = 0; j < ny; ++j) {
            const double u = prof_U[j];
            for (int q = 0; q < 19; ++q) {
                const double cu = cx[q] * u;
                rowbase[(size_t)j * lbmk::RB_W + q] = (float)(w[q] * (3.0 * cu + 4.5 * cu * cu - 1.5 * u * u));
            }
        }
    }
    float rb(int j, int q) const { return rowbase[(size_t)j * lbmk::RB_W + q]; }

    // Flow constants (A20): U_b+ = mean of u+ over the cell centres with the
    // creation-time (kappa, B); u_tau = U_b / U_b+, nu = u_tau delta / Re_tau.
    void constants() {
        delta = 0.5 * ny;
        double s = 0;
        for (int j = 0; j < ny; ++j) s += uplus(dwall(j) * re_tau / delta, opts.kappa, opts.B);
        ubp = s / ny;
        utau_ref = opts.u_bulk / ubp;
        nu = utau_ref * delta / re_tau;
        tau0 = 3.0 * nu + 0.5;     // eq:nu with c_s^2 = 1/3
    }
    double dwall(int j) const { return std::min(j + 0.5, ny - j - 0.5); }

    // Inlet tables: mean profile, Cholesky factor of the prescribed Reynolds
    // stress (eq:cholesky), STG modes and spectrum (Sec. 3.1).
    void tables() {
        const double ell_e = theta[0], amp = theta[1], kap = theta[2], B = theta[3];
        const int N = n_modes;
        if (!custom_profile) {
            prof_U.assign(ny, 0.0);
            prof_R.assign(6 * (size_t)ny, 0.0);
            for (int j = 0; j < ny; ++j) {
                const double d = dwall(j);
                prof_U[j] = utau_ref * uplus(d * utau_ref / nu, kap, B);
                // prescribed stress in wall units: -uv+ = (1 - d/delta)(1 - e^{-d+/26})^2,
                // normal stresses 3s + 0.1, s + 0.1, 2s + 0.1; sign of uv flips above the centre
                const double e = 1.0 - std::exp(-d * re_tau / delta / 26.0);
                const double sh = (1.0 - d / delta) * e * e;
                const double u2 = utau_ref * utau_ref;
                double *R = &prof_R[6 * (size_t)j];
                R[0] = (3 * sh + 0.1) * u2; R[1] = (sh + 0.1) * u2; R[2] = (2 * sh + 0.1) * u2;
                R[3] = ((j + 0.5) < 0.5 * ny ? -sh : sh) * u2; R[4] = 0.0; R[5] = 0.0;
            }
        }
        profile_tables(amp);
        const size_t NN = N > 0 ? N : 1;
        sq.assign((size_t)ny * NN, 0.f);
        sig.assign(3 * NN, 0.f);
        sqsig.assign(4 * (size_t)ny * NN, 0.f);
        alpha.assign((size_t)ny * NN, 0u);
        betaT.assign((size_t)nz * NN, 0u);
        phi32.assign(NN, 0u);
        rate64.assign(NN, 0ull);
        if (N == 0) { maxl = 0; return; }
        // l_e(y) = ell_e delta tanh(2 d / (ell_e delta)); largest at the centre rows
        std::vector<double> ell(ny);
        maxl = 0;
        for (int j = 0; j < ny; ++j) {
            ell[j] = ell_e * delta * std::tanh(2.0 * dwall(j) / (ell_e * delta));
            maxl = std::max(maxl, ell[j]);
        }
        std::vector<double> kn(N), dx(N), dy(N), dz(N);
        const double kmin = beta_kmin * 2.0 * kPi / maxl;
        for (int n = 0; n < N; ++n) {
            kn[n] = kmin * std::pow(k_ratio, n);
            const double *U = &uniforms[4 * (size_t)n];
            const double ct = 1.0 - 2.0 * U[0], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
            const double az = 2.0 * kPi * U[1], ang = 2.0 * kPi * U[2];
            dx[n] = st * std::cos(az); dy[n] = st * std::sin(az); dz[n] = ct;
            // sigma_n: unit vector normal to d_n at angle ang from the polar direction
            const double e1[3] = {ct * std::cos(az), ct * std::sin(az), -st};
            const double e2[3] = {-std::sin(az), std::cos(az), 0.0};
            for (int c = 0; c < 3; ++c)
                sig[(size_t)c * N + n] = (float)(std::cos(ang) * e1[c] + std::sin(ang) * e2[c]);
            phi32[n] = turns32(U[3]);
            // time part of the phase: -(d_x U_b / max l_e) turns per step
            const double nu_n = dx[n] * opts.u_bulk / maxl;
            const long long fx = std::llround(-nu_n * 18446744073709551616.0);
            rate64[n] = (uint64_t)fx;
        }
        for (int j = 0; j < ny; ++j)
            for (int n = 0; n < N; ++n) alpha[(size_t)j * N + n] = turns32(kn[n] * dy[n] * (j + 0.5) / (2 * kPi));
        betaT.assign((size_t)nz * NN, 0u);
        for (int k = 0; k < nz; ++k)
            for (int n = 0; n < N; ++n) betaT[(size_t)n * nz + k] = turns32(kn[n] * dz[n] * (k + 0.5) / (2 * kPi));
        // sqrt(6 q_n(y)) from the modified von Karman spectrum (the sqrt6 of
        // eq:aux_vec folded in)
        std::vector<double> sq6;
        double mx = 0.0;
        spectrum<double>(ell_e, sq6, mx);
        for (size_t c = 0; c < sq6.size(); ++c) sq[c] = (float)sq6[c];
        sqsig.assign(4 * (size_t)ny * NN, 0.f);
        for (int j = 0; j < ny; ++j)
            for (int n = 0; n < N; ++n) {
                float *e = &sqsig[4 * ((size_t)j * N + n)];
                e[0] = sq[(size_t)j * N + n];
                e[1] = sig[n]; e[2] = sig[(size_t)N + n]; e[3] = sig[2 * (size_t)N + n];
            }
    }
    double opts_kappa0 = 0.4;   // the creation-time kappa (dissipation estimate of the spectrum)
    AdjointWork adj;
    // host copies of the derivative tables (built with the adjoint workspace)
    std::vector<float> h_dsq, h_aunit, h_dUR, h_kphase;
    float h_cell_scale = 0.f;

    // sqrt(6 q_n(y)) of the modified von Karman spectrum (Sec. 3.1, cited STG
    // method) in scalar type T, with ell_e as the independent variable.
    template <class T>
    void spectrum(T ell_e, std::vector<T> &out, T &maxl_out) const {
        const int N = n_modes;
        std::vector<T> ell(ny);
        T mx(0.0);
        for (int j = 0; j < ny; ++j) {
            ell[j] = ell_e * T(delta) * dtanh(T(2.0 * dwall(j)) / (ell_e * T(delta)));
            if (j == 0 || val(ell[j]) > val(mx)) mx = ell[j];
        }
        maxl_out = mx;
        const T kmin = T(beta_kmin * 2.0 * kPi) / mx;
        const double kcut = kPi;
        out.assign((size_t)ny * N, T(0.0));
        std::vector<T> E(N);
        for (int j = 0; j < ny; ++j) {
            const double d = dwall(j);
            const T ke = T(2.0 * kPi) / ell[j];
            const double eps = utau_ref * utau_ref * utau_ref / (opts_kappa0 * d);
            const double keta = 2.0 * kPi * std::pow(eps / (nu * nu * nu), 0.25);
            T tot(0.0);
            for (int n = 0; n < N; ++n) {
                const T k = kmin * T(std::pow(k_ratio, n));
                const T r = k / ke;
                const T dk = k * T(1.0 - 1.0 / k_ratio);
                const double over = std::max(val(k) - 0.9 * kcut, 0.0);
                T xc = val(k) > 0.9 * kcut ? T(4.0) * (k - T(0.9 * kcut)) / T(kcut) : T(0.0);
                (void)over;
                const T g = T(12.0) * k / T(keta);
                E[n] = r * r * r * r / dpow(T(1.0) + T(2.4) * r * r, 17.0 / 6.0) * dexp(T(0.0) - g * g) *
                       dexp(T(0.0) - xc * xc * xc) * dk;
                tot = tot + E[n];
            }
            for (int n = 0; n < N; ++n) out[(size_t)j * N + n] = dsqrt(T(6.0) * E[n] / tot);
        }
    }

    // derivative tables of the inlet velocity for the adjoint
    void adjoint_tables() {
        const int N = n_modes > 0 ? n_modes : 1;
        h_dsq.assign((size_t)ny * N, 0.f);
        h_kphase.assign(4 * (size_t)N, 0.f);
        h_aunit.assign(6 * (size_t)ny, 0.f);
        h_dUR.assign(2 * (size_t)ny, 0.f);
        h_cell_scale = 0.f;
        if (n_modes > 0) {
            std::vector<Dual> sqd;
            Dual mx;
            spectrum<Dual>(Dual(theta[0], 1.0), sqd, mx);
            for (size_t c = 0; c < sqd.size(); ++c) h_dsq[c] = (float)sqd[c].d;
            h_cell_scale = (float)(mx.d / mx.v);
            const double kmin = beta_kmin * 2.0 * kPi / mx.v;
            for (int n = 0; n < n_modes; ++n) {
                const double kn = kmin * std::pow(k_ratio, n);
                const double *U = &uniforms[4 * (size_t)n];
                const double ct = 1.0 - 2.0 * U[0], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
                const double az = 2.0 * kPi * U[1];
                const double dx = st * std::cos(az), dy = st * std::sin(az), dz = ct;
                h_kphase[4 * n + 0] = (float)(kn * dy);
                h_kphase[4 * n + 1] = (float)(kn * dz);
                h_kphase[4 * n + 2] = (float)(2.0 * kPi * dx * opts.u_bulk / mx.v);
            }
        }
        for (int j = 0; j < ny; ++j) {
            const double *R = &prof_R[6 * (size_t)j];
            const double l11 = std::sqrt(R[0]), l21 = R[3] / l11, l31 = R[4] / l11;
            const double l22 = std::sqrt(R[1] - l21 * l21), l32 = (R[5] - l21 * l31) / l22;
            const double l33 = std::sqrt(R[2] - l31 * l31 - l32 * l32);
            const double L[6] = {l11, l21, l22, l31, l32, l33};
            for (int c = 0; c < 6; ++c) h_aunit[6 * (size_t)j + c] = (float)L[c];
            if (!custom_profile) {
                // U_R = u_tau u+(y+; kappa, B): du+/dkappa, du+/dB at fixed y+
                const double yp = dwall(j) * utau_ref / nu, kap = theta[2];
                const double dk = -std::log1p(kap * yp) / (kap * kap) + yp / (kap * (1.0 + kap * yp));
                const double dB = 1.0 - std::exp(-yp / 11.0) - yp / 11.0 * std::exp(-yp / 3.0);
                h_dUR[j] = (float)(utau_ref * dk);
                h_dUR[ny + j] = (float)(utau_ref * dB);
            }
        }
    }

    size_t adjoint_layout(Arena &ar, int T, int K) {
        const size_t L = 19 * (size_t)ncell, W = 2 * (size_t)nz * nx, I = 3 * (size_t)nz * ny;
        const size_t N = n_modes > 0 ? n_modes : 1;
        adj.ckpt = ar.take<float>(L * (T / K));
        adj.seg = ar.take<float>(L * kSlotSets * (K - 1));   // kSlotSets sets of K - 1 segment slots
        adj.lamA = ar.take<float>(L);
        adj.lamB = ar.take<float>(L);
        adj.ut_init = ar.take<float>(W);
        adj.uthist = ar.take<float>(W * T);
        adj.ut_scr = ar.take<float>(W);
        adj.fw_scr = ar.take<float>(3 * W);
        adj.vwin = ar.take<float>(I * T);
        adj.luin = ar.take<float>(I * T);
        adj.jr_coef = ar.take<float>(ny);
        adj.jr_mean = ar.take<float>(2 * (size_t)ny);
        adj.dsq = ar.take<float>((size_t)ny * N);
        adj.aunit = ar.take<float>(6 * (size_t)ny);
        adj.dUR = ar.take<float>(2 * (size_t)ny);
        adj.kphase = ar.take<float4>(N);
        adj.gtheta = ar.take<double>(4);
        adj.objacc = ar.take<double>(1 + 3 * (size_t)ny);
        adj.r12 = ar.take<double>(ny);
        return (ar.off + 255) & ~size_t(255);
    }

    cudaError_t upload_adjoint_tables() {
        adjoint_tables();
        cudaError_t e;
        if ((e = cudaMemcpyAsync(adj.dsq, h_dsq.data(), h_dsq.size() * 4, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(adj.kphase, h_kphase.data(), h_kphase.size() * 4, cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(adj.aunit, h_aunit.data(), h_aunit.size() * 4, cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(adj.dUR, h_dUR.data(), h_dUR.size() * 4, cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess) return e;
        adj.cell_scale = h_cell_scale;
        return cudaStreamSynchronize(stream);
    }

    // U_R and amp * chol(R) per row (eq:cholesky); false if R is not SPD
    bool profile_tables(double amp) {
        UR.assign(ny, 0.f);
        amat.assign(6 * (size_t)ny, 0.f);
        for (int j = 0; j < ny; ++j) {
            const double *R = &prof_R[6 * (size_t)j];   // 11, 22, 33, 12, 13, 23
            const double r11 = R[0], r22 = R[1], r33 = R[2], r21 = R[3], r31 = R[4], r32 = R[5];
            if (!(r11 > 0)) return false;
            const double l11 = std::sqrt(r11);
            const double l21 = r21 / l11, l31 = r31 / l11;
            const double p22 = r22 - l21 * l21;
            if (!(p22 > 0)) return false;
            const double l22 = std::sqrt(p22);
            const double l32 = (r32 - l21 * l31) / l22;
            const double p33 = r33 - l31 * l31 - l32 * l32;
            if (!(p33 > 0)) return false;
            const double L[6] = {l11, l21, l22, l31, l32, std::sqrt(p33)};
            UR[j] = (float)prof_U[j];
            for (int c = 0; c < 6; ++c) amat[6 * (size_t)j + c] = (float)(amp * L[c]);
        }
        return true;
    }

    // Forget the STG ring (its tables or the time changed); later work on the
    // handle's stream is ordered after a refill still running on the aux stream.
    void stg_reset() {
        if (stg_next_t0 >= 0) cudaStreamWaitEvent(stream, ev_stg_ready, 0);
        stg_len = 0;
        stg_next_t0 = -1;
    }

    // first time level of half b of the STG ring
    float *stg_slot(int b) const { return d_uin + 3 * (size_t)nz * ny * stg_ring * b; }

    cudaError_t upload_tables() {
        const size_t N = n_modes > 0 ? n_modes : 1;
        cudaError_t e;
        stg_reset();                            // the tables feed the ring
        ++graph_epoch;                          // and the step parameters
#define UP(dst, vec) if ((e = cudaMemcpyAsync(dst, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice, stream)) != cudaSuccess) return e
        UP(d_UR, UR); UP(d_amat, amat); UP(d_sqsig, sqsig);
        UP(d_alpha, alpha); UP(d_betaT, betaT); UP(d_phi32, phi32); UP(d_rate64, rate64);
        UP(d_rowbase, rowbase);
#undef UP
        (void)N;
        return cudaStreamSynchronize(stream);   // host vectors may change after return
    }
};

namespace {

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "liblbm_gb300: CUDA error: %s\n", cudaGetErrorString(e));
    return LBM_ECUDA;
}

// Makes the handle's device current for the length of a call and puts the
// caller's device back afterwards (a no-op before lbm_bind_memory, or when the
// handle's device is already current).
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(const lbm_handle *h) {
        if (!h || h->device < 0) return;
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
        if (cur == h->device) return;
        if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
        prev = cur;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};
#define LBM_DEVICE_GUARD(h)                 \
    DeviceGuard device_guard_(h);           \
    if (!device_guard_.ok) return LBM_ECUDA

constexpr size_t kEventPool = 2048;
constexpr int kGuardByte = 0xA5;          // fill of the guard bands

// Harvest a finished event pair into the running total.
void prof_harvest(lbm_handle *h, size_t slot) {
    if (!h->ev_busy[slot]) return;
    float ms = 0.f;
    cudaEventSynchronize(h->ev1[slot]);
    cudaEventElapsedTime(&ms, h->ev0[slot], h->ev1[slot]);
    h->prof_ms += ms;
    h->prof_n += h->ev_busy[slot];
    h->ev_busy[slot] = 0;
}

size_t prof_slot(lbm_handle *h) {
    const size_t slot = h->ev_next;
    h->ev_next = (h->ev_next + 1) % kEventPool;
    prof_harvest(h, slot);
    h->ev_busy[slot] = 1;
    return slot;
}

// Where one step reads and writes: state in / out, wall buffers, STG field.
struct StepIO {
    const void *in;
    void *out;
    const float *utau_in = nullptr;   // warm start; null: utau itself
    float *utau, *fw;
    const float *vprime;
    bool stats;
    // objective sums accumulated by the step (pair and wall kernels; null: none)
    double *obj = nullptr;
    int obj_i0 = 0, obj_i1 = 0, obj_iR = -1;
};

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links no driver library of its own).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The staged kernel needs 16-byte row strides (nx a multiple of 16 / element
// size) and the tensor-map encoder.
bool staged_supported(const lbm_handle *h) {
    return h->nx % (16 / (int)h->elem) == 0 && tensor_map_encoder() != nullptr;
}

int resolve_kind(const lbm_handle *h) {
    if (h->step_kind != LBM_KERNEL_AUTO) return h->step_kind;
    if (h->elem == 2 && h->nx % 4 == 0) return LBM_KERNEL_QUAD;
    return h->nx % 2 == 0 ? LBM_KERNEL_PAIR : LBM_KERNEL_CELL;
}

// 4-d tensor map (x, y, z, q) of a lattice at `base`, box (BW, 2, 1, 1).
template <class S>
const CUtensorMap *lattice_map(lbm_handle *h, const void *base) {
    for (auto &m : h->maps)
        if (m.base == base) return &m.map;
    auto &m = h->maps[h->map_next];
    h->map_next = (h->map_next + 1) % 32;
    const cuuint64_t e = sizeof(typename S::T);
    const CUtensorMapDataType dt = e == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : h->opts.precision == LBM_BF16_DEV ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[4] = {(cuuint64_t)h->nx, (cuuint64_t)h->ny, (cuuint64_t)h->nz, 19};
    const cuuint64_t strides[3] = {h->nx * e, (cuuint64_t)h->nx * h->ny * e, (cuuint64_t)h->ncell * e};
    const cuuint32_t box[4] = {(cuuint32_t)lbmk::Staged<S>::BW, (cuuint32_t)lbmk::SG_TY, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = tensor_map_encoder()(&m.map, dt, 4, const_cast<void *>(base), dims, strides, box, es,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { m.base = nullptr; return nullptr; }
    m.base = base;
    return &m.map;
}

int device_sms() {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 148; }
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 148;
        }
        sms[dev] = v;
    }
    return sms[dev];
}

// Raise the dynamic shared-memory limit of the staged kernel<S, STATS>, once
// per device (one set of flags per instantiation).
template <class S, bool STATS>
cudaError_t allow_staged_smem(int bytes) {
    static unsigned done[2] = {0, 0};   // bit per device
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && (done[dev / 32] >> (dev % 32)) & 1u) return cudaSuccess;
    e = cudaFuncSetAttribute(lbmk::staged_kernel<S, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev < 64) done[dev / 32] |= 1u << (dev % 32);
    return e;
}

template <class S, bool STATS>
cudaError_t launch_staged(lbm_handle *h, const lbmk::StepArgs<S> &a, const void *in) {
    lbmk::StagedArgs<S> g;
    const CUtensorMap *m = lattice_map<S>(h, in);
    if (!m) return cudaErrorInvalidValue;
    std::memcpy(&g.tmap, m, sizeof(CUtensorMap));
    g.s = a;
    g.nxt = (h->nx + lbmk::SG_TX - 1) / lbmk::SG_TX;
    g.nyt = (h->ny - 2) / lbmk::SG_TY;
    g.ntiles = g.nxt * g.nyt * h->nz;
    constexpr int smem = lbmk::staged_smem_bytes<S, lbmk::StagedCfg<S>::STAGES>();
    cudaError_t e = allow_staged_smem<S, STATS>(smem);
    if (e != cudaSuccess) return e;
    if (g.ntiles == 0) return cudaSuccess;          // ny = 4: wall rows only
    const int nb = std::min(g.ntiles, device_sms() * lbmk::StagedCfg<S>::MINB);
    lbmk::staged_kernel<S, STATS><<<nb, lbmk::SG_THREADS, smem, h->stream>>>(g);
    return cudaGetLastError();
}

// The outlet sponge as kernel arguments: zone start, 1 / length, 3 nu_s.
void sponge_args(const lbm_handle *h, float &x0, float &inv, float &s3nu) {
    const int L = h->sponge_cells;
    x0 = (float)(h->nx_global - L - h->x_offset);     // zone start in local columns
    inv = L > 0 ? 1.0f / (float)L : 0.0f;
    s3nu = L > 0 ? (float)(3.0 * h->sponge_nu) : 0.0f;
}

template <class S>
cudaError_t launch_step_t(lbm_handle *h, const StepIO &io) {
    using T = typename S::T;
    lbmk::StepArgs<S> a;
    const size_t N = (size_t)h->ncell;
    for (int q = 0; q < 19; ++q) {
        a.in[q] = (const T *)io.in + q * N;
        a.out[q] = (T *)io.out + q * N;
    }
    a.vprime = io.vprime;
    a.UR = h->d_UR;
    a.amat = h->d_amat;
    a.utau_in = io.utau_in ? io.utau_in : io.utau;
    a.utau = io.utau;
    a.fw = io.fw;
    a.ubuf = h->d_ubuf;
    a.flags = h->d_flags;
    a.rowbase = h->d_rowbase;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.inlet = h->opts.inlet; a.wall_model = h->opts.wall_model;
    a.check = (h->t % h->check_every) == 0;
    a.reverse = (int)(h->t & 1);
    a.tau0 = (float)h->tau0;
    a.csm18 = (float)(18.0 * std::sqrt(2.0) * h->opts.c_smag);
    a.y1_nu = (float)(0.5 / h->nu);
    a.kappa = (float)h->theta[2]; a.B = (float)h->theta[3];
    a.obj = io.obj; a.obj_i0 = io.obj_i0; a.obj_i1 = io.obj_i1; a.obj_iR = io.obj_iR;
    sponge_args(h, a.sp_x0, a.sp_inv, a.sp_3nu);
    const int bxmax = lbmk::STEP_THREADS / lbmk::BY;
    // (steps inside a graph are timed by events around the graph launch)
    const bool timed = h->prof_on && !h->capturing && (h->prof_count++ % h->prof_every) == 0;
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;
    if (timed) {
        const size_t slot = prof_slot(h);
        tev0 = h->ev0[slot];
        tev1 = h->ev1[slot];
    }
    if (timed) cudaEventRecord(tev0, h->stream);
    int kind = resolve_kind(h);
    if (io.obj && kind != LBM_KERNEL_CELL) kind = LBM_KERNEL_PAIR;   // the kernel that sums the objective
    if (io.fw == h->d_fw) h->fw_side = kind != LBM_KERNEL_CELL;
    cudaError_t err = cudaSuccess;
    if (kind == LBM_KERNEL_STAGED || kind == LBM_KERNEL_PAIR || kind == LBM_KERNEL_QUAD) {
        // the wall rows on the side stream, the interior rows on the handle's
        // stream; both read the state of the previous step and write disjoint rows
        const int bx = (h->nx / 2) >= bxmax ? bxmax : 32;
        const int nbx = (h->nx / 2 + bx - 1) / bx;
        const dim3 block(bx, lbmk::BY);
        if ((err = cudaEventRecord(h->ev_fork, h->stream)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess)
            return err;
        // a wall plane takes ~10 us beside the interior kernel: walk up to
        // four planes per block while that stays well inside the interior
        // kernel's time (its bytes at ~6.5 TB/s)
        const double interior_us = (double)h->nx * h->ny * h->nz * (sizeof(typename S::T) * 38.0) / 6.5e6;
        a.wall_planes = std::max(1, std::min(4, (int)(interior_us / 12.0)));
        const dim3 wgrid((h->nx + lbmk::WALL_THREADS - 1) / lbmk::WALL_THREADS,
                         (h->nz + a.wall_planes - 1) / a.wall_planes);
        if (io.stats) lbmk::wall_kernel<S, true><<<wgrid, lbmk::WALL_THREADS, 0, h->side>>>(a);
        else lbmk::wall_kernel<S, false><<<wgrid, lbmk::WALL_THREADS, 0, h->side>>>(a);
        if ((err = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return err;
        if (kind == LBM_KERNEL_STAGED) {
            err = io.stats ? launch_staged<S, true>(h, a, io.in) : launch_staged<S, false>(h, a, io.in);
        } else if (kind == LBM_KERNEL_QUAD) {
            const dim3 qgrid((h->nx + 127) / 128, (h->ny - 2) / lbmk::BY, h->nz), qblock(32, lbmk::BY);
            if (io.stats) lbmk::step4_kernel<S, true><<<qgrid, qblock, 0, h->stream>>>(a);
            else lbmk::step4_kernel<S, false><<<qgrid, qblock, 0, h->stream>>>(a);
        } else {
            const dim3 grid(nbx, (h->ny - 2) / lbmk::BY, h->nz);
            if (io.stats) lbmk::step2_kernel<S, true><<<grid, block, 0, h->stream>>>(a);
            else lbmk::step2_kernel<S, false><<<grid, block, 0, h->stream>>>(a);
        }
        cudaError_t e2 = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
        if (err == cudaSuccess) err = e2;
        h->launches += 1;
    } else {
        const int bx = h->nx >= bxmax ? bxmax : (h->nx >= 64 && bxmax >= 64 ? 64 : 32);
        dim3 block(bx, lbmk::BY), grid((h->nx + bx - 1) / bx, h->ny / lbmk::BY, h->nz);
        if (io.stats) lbmk::step_kernel<S, true><<<grid, block, 0, h->stream>>>(a);
        else lbmk::step_kernel<S, false><<<grid, block, 0, h->stream>>>(a);
    }
    if (timed) cudaEventRecord(tev1, h->stream);
    h->launches += 1;
    return err;
}

// Enqueue one step; a launch that could not be set up (no tensor map) is
// reported here, kernel errors by cudaGetLastError as usual.
cudaError_t launch_step_io(lbm_handle *h, const StepIO &io) {
    switch (h->opts.precision) {
        case LBM_FP16_DEV: return launch_step_t<lbmk::StoreF16>(h, io);
        case LBM_BF16_DEV: return launch_step_t<lbmk::StoreBF16>(h, io);
        case LBM_FP16_ROW: return launch_step_t<lbmk::StoreF16R>(h, io);
        default: return launch_step_t<lbmk::StoreF32>(h, io);
    }
}

// STG field of steps a.t0 .. a.t0 + a.nsteps - 1: four time levels per thread
// when there are enough of them to fill the blocks, else one
void launch_stg_kernel(lbm_handle *h, const lbmk::StgArgs &a, cudaStream_t st) {
    const int n = a.nsteps, nbz = (h->nz + lbmk::STG_KZ - 1) / lbmk::STG_KZ;
    if (n >= 4 * lbmk::STG_KT) {
        const dim3 grid(nbz, h->ny, (n + 4 * lbmk::STG_KT - 1) / (4 * lbmk::STG_KT));
        lbmk::stg_kernel<4><<<grid, lbmk::STG_KZ * lbmk::STG_KT, 0, st>>>(a);
    } else {
        const dim3 grid(nbz, h->ny, (n + lbmk::STG_KT - 1) / lbmk::STG_KT);
        lbmk::stg_kernel<1><<<grid, lbmk::STG_KZ * lbmk::STG_KT, 0, st>>>(a);
    }
    h->launches += 1;
}

// STG inlet velocities of steps t0 .. t0 + n - 1 into the first n slots of
// the ring, on the handle's stream
void launch_stg(lbm_handle *h, long long t0, int n, bool apply_profile) {
    lbmk::StgArgs a;
    a.alpha = h->d_alpha; a.betaT = h->d_betaT; a.phi32 = h->d_phi32; a.rate64 = h->d_rate64;
    a.sqsig = h->d_sqsig; a.amat = h->d_amat; a.UR = h->d_UR; a.out = h->d_uin;
    a.t0 = t0; a.t0_dev = nullptr; a.nsteps = n; a.apply_profile = apply_profile ? 1 : 0;
    a.ny = h->ny; a.nz = h->nz; a.n_modes = h->n_modes;
    launch_stg_kernel(h, a, h->stream);
}

void launch_stg_into(lbm_handle *h, float *out, long long t0, int n, cudaStream_t st);

int one_step(lbm_handle *h) {
    bool stats = false;
    if (h->opts.stats_every > 0) {
        h->steps_since_stats += 1;
        if (h->steps_since_stats >= h->opts.stats_every) { stats = true; h->steps_since_stats = 0; }
    }
    if (h->opts.inlet && (h->t < h->stg_t0 || h->t >= h->stg_t0 + h->stg_len)) {
        if (h->stg_next_t0 >= 0 && h->t == h->stg_next_t0) {
            // the other half was refilled for these steps on the aux stream
            cudaStreamWaitEvent(h->stream, h->ev_stg_ready, 0);
            h->stg_half ^= 1;
        } else {
            h->stg_reset();
            launch_stg_into(h, h->stg_slot(h->stg_half), h->t, h->stg_ring, h->stream);
        }
        h->stg_t0 = h->t;
        h->stg_len = h->stg_ring;
        // refill the other half for the steps after these, beside them; the
        // refill waits for the steps enqueued so far, which read that half
        cudaEventRecord(h->ev_stg_free, h->stream);
        cudaStreamWaitEvent(h->aux, h->ev_stg_free, 0);
        launch_stg_into(h, h->stg_slot(h->stg_half ^ 1), h->stg_t0 + h->stg_ring, h->stg_ring, h->aux);
        cudaEventRecord(h->ev_stg_ready, h->aux);
        h->stg_next_t0 = h->stg_t0 + h->stg_ring;
    }
    StepIO io;
    io.in = h->lat[h->cur];
    io.out = h->lat[h->cur ^ 1];
    io.utau = h->d_utau;
    io.fw = h->d_fw;
    io.vprime = h->opts.inlet ? h->stg_slot(h->stg_half) + 3 * (size_t)h->nz * h->ny * (size_t)(h->t - h->stg_t0)
                              : h->d_uin;
    io.stats = stats;
    if (cudaError_t le = launch_step_io(h, io)) return cuda_fail(le);
    if (stats) {
        h->n_samples += 1;
        const int cols = (h->nx * h->ny + lbmk::ST_COLS - 1) / lbmk::ST_COLS;
        const int tb = lbmk::ST_COLS * lbmk::ST_CHUNKS;
        const int blocks = cols + (h->opts.wall_model ? (2 * h->nx + lbmk::ST_COLS - 1) / lbmk::ST_COLS : 0);
        lbmk::stats_kernel<<<blocks, tb, 0, h->stream>>>(
            h->d_ubuf, h->d_utau, h->d_st, h->d_st_utau, h->nx, h->ny, h->nz, h->ncell, h->opts.wall_model);
        h->launches += 1;
    }
    h->cur ^= 1;
    h->t += 1;
    return cuda_fail(cudaGetLastError());
}

// STG field v' of steps t0 .. t0 + n - 1 into an explicit buffer
void launch_stg_into(lbm_handle *h, float *out, long long t0, int n, cudaStream_t st) {
    lbmk::StgArgs a;
    a.alpha = h->d_alpha; a.betaT = h->d_betaT; a.phi32 = h->d_phi32; a.rate64 = h->d_rate64;
    a.sqsig = h->d_sqsig; a.amat = h->d_amat; a.UR = h->d_UR; a.out = out;
    a.t0 = t0; a.nsteps = n; a.apply_profile = 0;
    // inside a graph the start time comes from device memory, set before every launch
    a.t0_dev = h->capturing ? h->d_gt0 : nullptr;
    a.ny = h->ny; a.nz = h->nz; a.n_modes = h->n_modes;
    launch_stg_kernel(h, a, st);
}

// One adjoint step: s_n (FP32 lattice) and lambda_{n+1} -> lambda_n.
void launch_adjoint(lbm_handle *h, const float *sn, const float *lam, float *lout, const float *utau_n,
                    const float *vprime_n, float *luin_n, bool seeds, const lbm_objective *obj, float jtau_w) {
    lbmk::AdjArgs a;
    const size_t N = (size_t)h->ncell;
    for (int q = 0; q < 19; ++q) a.in[q] = sn + q * N;
    a.lam = const_cast<float *>(lam); a.lout = lout;
    a.utau = utau_n; a.vprime = vprime_n; a.UR = h->d_UR; a.amat = h->d_amat;
    a.luin = luin_n; a.gtheta = h->adj.gtheta;
    a.jr_coef = seeds ? h->adj.jr_coef : nullptr;
    a.jr_mean = h->adj.jr_mean;
    a.jtau_w = seeds ? jtau_w : 0.0f;
    a.i_tau0 = obj ? obj->i_tau0 : 0; a.i_tau1 = obj ? obj->i_tau1 : 0; a.i_R = obj ? obj->i_R : -1;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.inlet = h->opts.inlet; a.wall_model = h->opts.wall_model;
    a.tau0 = (float)h->tau0;
    a.csm18 = (float)(18.0 * std::sqrt(2.0) * h->opts.c_smag);
    a.y1_nu = (float)(0.5 / h->nu);
    a.kappa = (float)h->theta[2]; a.B = (float)h->theta[3];
    sponge_args(h, a.sp_x0, a.sp_inv, a.sp_3nu);
    const bool sponge = a.sp_3nu != 0.0f;
    if (h->nx % 2 == 0) {
        // one launch: the wall rows (two cells per thread; with the inlet on,
        // their inlet / outlet columns one cell per thread), the inlet / outlet
        // columns of the other rows, the packed interior pairs.  With the inlet
        // on and nx < 6 no wall-row pair is away from both ends: the one-cell
        // blocks take all four columns.
        const bool in = h->opts.inlet != 0;
        const int nwp = (in && h->nx < 6) ? 0 : ((h->nx + 127) / 128) * 2 * h->nz;
        const int nwe = in ? 2 * ((h->nz + 15) / 16) : 0;
        const int ne = in && h->ny > 4 ? (4 * (h->ny - 4) * h->nz + 127) / 128 : 0;
        const int ni = h->ny > 4 ? ((h->nx / 2 + 63) / 64) * ((h->ny - 4) / lbmk::BY) * h->nz : 0;
        const dim3 block(64, lbmk::BY);
        const unsigned nb = (unsigned)(nwp + nwe + ne + ni);
        if (sponge) lbmk::adjoint_fused_kernel<true><<<nb, block, 0, h->stream>>>(a, nwp, nwe, ne);
        else lbmk::adjoint_fused_kernel<false><<<nb, block, 0, h->stream>>>(a, nwp, nwe, ne);
        h->launches += 1;
        return;
    }
    // odd nx: wall rows and their second rows on the side stream, the rest
    // (one cell per thread) on the handle's stream, joined before anything
    // that follows
    const int bx = 64;
    const dim3 block(bx, lbmk::BY);
    const int nbx = (h->nx + bx - 1) / bx;
    cudaEventRecord(h->ev_fork, h->stream);
    cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    const dim3 gw(nbx, 2, h->nz), gi(nbx, (h->ny - 4) / lbmk::BY, h->nz);
    if (sponge) lbmk::adjoint_wall_kernel<true><<<gw, block, 0, h->side>>>(a);
    else lbmk::adjoint_wall_kernel<false><<<gw, block, 0, h->side>>>(a);
    cudaEventRecord(h->ev_join, h->side);
    if (h->ny > 4) {
        if (sponge) lbmk::adjoint_kernel<true><<<gi, block, 0, h->stream>>>(a);
        else lbmk::adjoint_kernel<false><<<gi, block, 0, h->stream>>>(a);
    }
    cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    h->launches += 2;
}

// theta gradient through the inlet velocity for nsteps steps from t0
void launch_stg_adjoint(lbm_handle *h, long long t0, int nsteps, const float *luin, cudaStream_t st) {
    if (!h->opts.inlet) return;
    lbmk::StgAdjArgs a;
    a.alpha = h->d_alpha; a.betaT = h->d_betaT; a.phi32 = h->d_phi32; a.rate64 = h->d_rate64;
    a.sqsig = h->d_sqsig; a.dsq = h->adj.dsq; a.kphase = h->adj.kphase; a.aunit = h->adj.aunit;
    a.dUR = h->adj.dUR; a.luin = luin; a.gtheta = h->adj.gtheta;
    a.amp = (float)h->theta[1]; a.cell_scale = h->adj.cell_scale;
    a.t0 = t0; a.nsteps = nsteps; a.ny = h->ny; a.nz = h->nz; a.n_modes = h->n_modes;
    dim3 grid((h->nz + lbmk::STG_KZ - 1) / lbmk::STG_KZ, h->ny, (nsteps + lbmk::STG_KT - 1) / lbmk::STG_KT);
    lbmk::stg_adjoint_kernel<<<grid, lbmk::STG_KZ * lbmk::STG_KT, 0, st>>>(a);
    h->launches += 1;
}

template <class S>
void launch_init(lbm_handle *h, void *lat) {
    const long long n = h->ncell;
    lbmk::init_kernel<S><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>((typename S::T *)lat, h->d_UR,
                                                                               h->d_rowbase, h->nx, h->ny, n);
}

const double kW[19] = {1. / 36, 1. / 36, 1. / 18, 1. / 36, 1. / 36, 1. / 36, 1. / 18, 1. / 36, 1. / 18, 1. / 3,
                       1. / 18, 1. / 36, 1. / 18, 1. / 36, 1. / 36, 1. / 36, 1. / 18, 1. / 36, 1. / 36};

uint16_t f32_to_bf16_rn(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) == 0x7f800000u) return (uint16_t)(b >> 16);   // inf / nan
    b += 0x7fffu + ((b >> 16) & 1u);
    return (uint16_t)(b >> 16);
}
float bf16_to_f32(uint16_t v) {
    uint32_t b = (uint32_t)v << 16;
    float x;
    std::memcpy(&x, &b, 4);
    return x;
}

// ---------------------------------------------------------------------------
// CUDA graphs of whole STG ring periods.  lbm_step launches the stg_ring steps
// that start where the ring swaps halves as one graph: the steps of one
// period, and beside them the refill of the other half, joined at the end.
// The launch parameters of a step depend on the host state at its start
// (lattice parity, ring half, phases of the checks and the statistics,
// inlet-profile buffer), which form the graph's key; equal keys give equal
// graphs except for the refill's start time, which the refill reads from
// device memory set before every launch.  Changes of the tables, the sponge
// or the kernel choice retire all graphs (graph_epoch).
// ---------------------------------------------------------------------------
void graph_key(const lbm_handle *h, long long key[9]) {
    key[0] = h->stg_half;
    key[1] = h->cur;
    key[2] = h->t % h->check_every;
    key[3] = h->t & 1;
    key[4] = h->steps_since_stats;
    key[5] = 0;                            // (timing brackets whole graph launches)
    key[6] = 0;
    key[7] = h->prof_cur;
    key[8] = h->stg_ring;
}

bool graph_usable(const lbm_handle *h) {
    if (!(h->graphs_on && h->opts.inlet && h->stg_ring >= 8 && h->stg_next_t0 >= 0 && h->t == h->stg_next_t0 &&
          resolve_kind(h) != LBM_KERNEL_STAGED))
        return false;
    // not while the caller captures the handle's stream into a graph of its own
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
}

void graphs_clear(lbm_handle *h) {
    if (!h->graphs.empty()) cudaStreamSynchronize(h->stream);   // none may still run
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    h->graphs_built_epoch = h->graph_epoch;
}

// Launch a graph on the handle's stream, its refill starting at the period
// after this one (set in device memory first).  With instrumentation on, a
// pair of events brackets the launch and is booked for the period's steps.
cudaError_t graph_launch(lbm_handle *h, lbm_handle::GraphSeg &g) {
    lbmk::set_time_kernel<<<1, 1, 0, h->stream>>>(h->d_gt0, h->stg_t0 + h->stg_ring);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t slot = 0;
    if (h->prof_on) {
        slot = prof_slot(h);
        h->ev_busy[slot] = h->stg_ring;
        if ((e = cudaEventRecord(h->ev0[slot], h->stream)) != cudaSuccess) return e;
    }
    if ((e = cudaGraphLaunch(g.exec, h->stream)) != cudaSuccess) return e;
    if (h->prof_on) e = cudaEventRecord(h->ev1[slot], h->stream);
    return e;
}

// Capture one ring period as the handle would enqueue it, on a capture stream
// standing in for the handle's stream, and record in g what the period does to
// the host state.  On return the host state is as before the call
// (graph_segment advances it when it launches the graph); false if the
// capture did not succeed.
bool graph_capture(lbm_handle *h, lbm_handle::GraphSeg &g) {
    if (!h->gstream && cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (!h->ev_gfork && cudaEventCreateWithFlags(&h->ev_gfork, cudaEventDisableTiming) != cudaSuccess) return false;
    if (!h->ev_gjoin && cudaEventCreateWithFlags(&h->ev_gjoin, cudaEventDisableTiming) != cudaSuccess) return false;
    const long long t0 = h->t, cur0 = h->cur, since0 = h->steps_since_stats, samples0 = h->n_samples;
    const long long prof0 = h->prof_count, launches0 = h->launches;
    const cudaStream_t real = h->stream;
    h->stream = h->gstream;
    h->capturing = true;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        // the refill of the other half, beside this period's steps
        ok = cudaEventRecord(h->ev_gfork, h->gstream) == cudaSuccess &&
             cudaStreamWaitEvent(h->aux, h->ev_gfork, 0) == cudaSuccess;
        if (ok) {
            launch_stg_into(h, h->stg_slot(h->stg_half ^ 1), h->stg_t0 + h->stg_ring, h->stg_ring, h->aux);
            ok = cudaEventRecord(h->ev_gjoin, h->aux) == cudaSuccess;
        }
        for (int s = 0; ok && s < h->stg_ring; ++s) ok = one_step(h) == LBM_OK;
        if (ok) ok = cudaStreamWaitEvent(h->gstream, h->ev_gjoin, 0) == cudaSuccess;
        const cudaError_t ee = cudaStreamEndCapture(h->gstream, &graph);
        ok = ok && ee == cudaSuccess && graph != nullptr;
    }
    h->stream = real;
    h->capturing = false;
    if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    const long long launches1 = h->launches, since1 = h->steps_since_stats, samples1 = h->n_samples;
    h->t = t0; h->cur = (int)cur0; h->steps_since_stats = since0; h->n_samples = samples0;
    h->prof_count = prof0; h->launches = launches0;
    if (!ok) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        return false;
    }
    // the launch enqueues the work the capture only recorded
    g.d_launches = launches1 - launches0;
    g.after_since_stats = since1;
    g.d_samples = samples1 - samples0;
    return true;
}

// One ring period from the ring swap on: from a graph (built at the first
// period with this key).  Returns LBM_OK, or 1 if no graph could be built
// (the caller then steps one at a time; the swap has been made).
int graph_segment(lbm_handle *h) {
    if (h->graphs_built_epoch != h->graph_epoch) graphs_clear(h);
    cudaError_t e;
    // swap to the other half, filled beside the previous period
    if ((e = cudaStreamWaitEvent(h->stream, h->ev_stg_ready, 0)) != cudaSuccess) return cuda_fail(e);
    h->stg_half ^= 1;
    h->stg_t0 = h->t;
    h->stg_len = h->stg_ring;
    long long key[9];
    graph_key(h, key);
    lbm_handle::GraphSeg *g = nullptr;
    for (auto &c : h->graphs)
        if (std::equal(key, key + 9, c.key)) g = &c;
    if (!g) {
        if (h->graphs.size() >= 32) graphs_clear(h);
        lbm_handle::GraphSeg ng;
        std::copy(key, key + 9, ng.key);
        if (!graph_capture(h, ng)) {
            h->graphs_on = false;                // capture refused: plain launches from now on
            h->stg_next_t0 = -1;                 // the refill was not enqueued
            return 1;
        }
        h->graphs.push_back(ng);
        g = &h->graphs.back();
    }
    if ((e = graph_launch(h, *g)) != cudaSuccess) return cuda_fail(e);
    // the events the captured steps recorded stay inside the graph: those
    // waited on later are recorded again, here on the handle's stream (the
    // refill of the next half is complete with the graph)
    if ((e = cudaEventRecord(h->ev_stg_ready, h->stream)) != cudaSuccess) return cuda_fail(e);
    h->t += h->stg_ring;
    h->cur ^= (h->stg_ring & 1);
    h->steps_since_stats = g->after_since_stats;
    h->n_samples += g->d_samples;
    h->prof_count += h->stg_ring;
    h->launches += g->d_launches + 1;            // and the time setter
    h->stg_next_t0 = h->stg_t0 + h->stg_ring;
    // the graph's wall kernels ran inside it, ordered on the handle's stream
    // and not on the side stream: a wall-shear reduction follows them there
    h->fw_side = false;
    ++h->graph_launches;
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_opts(lbm_opts *o) {
    if (!o) return;
    o->precision = LBM_FP32;
    o->u_bulk = 0.05;
    o->c_smag = 0.01;
    o->kappa = 0.4;
    o->B = 7.8;
    o->wall_model = 1;
    o->inlet = 1;
    o->stats_every = 0;
    o->cuda_stream = nullptr;
}

int lbm_create(const lbm_grid *grid, double re_tau, const lbm_stg_params *stg, const lbm_opts *opts,
               lbm_handle **out) {
    if (!grid || !stg || !opts || !out) return LBM_EINVAL;
    *out = nullptr;
    if (grid->ny < 4 || grid->ny % 2 || grid->nx < 3 || grid->nz < 1) return LBM_EINVAL;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return LBM_EINVAL;
    if (!(re_tau > 0) || stg->n_modes < 0 || (stg->n_modes > 0 && !stg->uniforms)) return LBM_EINVAL;
    if (opts->precision < LBM_FP32 || opts->precision > LBM_FP16_ROW) return LBM_EINVAL;
    if (!(opts->u_bulk > 0) || !(opts->kappa > 0) || opts->stats_every < 0) return LBM_EINVAL;
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ENOMEM;
    h->nx = grid->nx; h->ny = grid->ny; h->nz = grid->nz;
    h->ncell = (long long)h->nx * h->ny * h->nz;
    h->nx_global = h->nx; h->x_offset = 0; h->own_lo = 0; h->own_hi = h->nx;
    h->re_tau = re_tau;
    h->opts = *opts;
    h->stream = (cudaStream_t)opts->cuda_stream;
    h->n_modes = stg->n_modes;
    h->k_ratio = stg->k_ratio;
    h->beta_kmin = stg->beta_kmin;
    h->uniforms.assign(stg->uniforms ? stg->uniforms : nullptr,
                       stg->uniforms ? stg->uniforms + 4 * (size_t)stg->n_modes : nullptr);
    h->theta[0] = stg->ell_e; h->theta[1] = stg->amp; h->theta[2] = opts->kappa; h->theta[3] = opts->B;
    h->opts_kappa0 = opts->kappa;
    h->elem = opts->precision == LBM_FP32 ? 4 : 2;
    h->constants();
    h->tables();
    h->make_rowbase();
    *out = h;
    return LBM_OK;
}

int lbm_required_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_EINVAL;
    Arena ar;
    ar.guard = h->guard_bytes;
    lbm_handle tmp_view = *h;   // layout() only writes pointers of the copy
    *bytes = tmp_view.layout(ar);
    return LBM_OK;
}

int lbm_bind_memory(lbm_handle *h, void *dev_ptr, size_t bytes) {
    if (!h) return LBM_EINVAL;
    if (h->bound) return LBM_ESTATE;
    size_t need = 0;
    lbm_required_bytes(h, &need);
    // the handle lives on the device of its memory from here on: every later
    // call makes that device current while it runs
    int dev = -1;
    if (dev_ptr) {
        if (((uintptr_t)dev_ptr & 255) != 0) return LBM_EINVAL;
        if (bytes < need) return LBM_ENOMEM;
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, dev_ptr) != cudaSuccess ||
            (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return LBM_EINVAL;                   // not device memory
        }
        dev = pa.device;
    } else if (cudaGetDevice(&dev) != cudaSuccess) {
        return cuda_fail(cudaGetLastError());
    }
    h->device = dev;
    LBM_DEVICE_GUARD(h);
    if (dev_ptr) {
        h->mem = dev_ptr;
        h->owns = false;
    } else {
        if (cudaMalloc(&h->mem, need) != cudaSuccess) { cudaGetLastError(); return LBM_ENOMEM; }
        h->owns = true;
    }
    h->mem_bytes = need;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaHostAlloc((void **)&h->pin_stage, 14 * sizeof(float) * h->ny, cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_prof_ready[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_prof_ready[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_prof_free[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_prof_free[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_aux_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_aux_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_stg_free, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_stg_ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_shear, cudaEventDisableTiming) != cudaSuccess) {
        if (h->owns) cudaFree(h->mem);
        h->mem = nullptr;
        return cuda_fail(cudaGetLastError());
    }
    Arena ar;
    ar.base = (char *)h->mem;
    ar.guard = h->guard_bytes;
    h->guards.clear();
    ar.bands = &h->guards;
    h->layout(ar);
    h->bound = true;
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->mem, 0, need, h->stream)) != cudaSuccess) return cuda_fail(e);
    for (const auto &b : h->guards)
        if ((e = cudaMemsetAsync((char *)h->mem + b.first, kGuardByte, b.second, h->stream)) != cudaSuccess)
            return cuda_fail(e);
    if ((e = h->upload_tables()) != cudaSuccess) return cuda_fail(e);
    std::vector<float> ut(2 * (size_t)h->nz * h->nx, (float)h->utau_ref);
    if ((e = cudaMemcpyAsync(h->d_utau, ut.data(), ut.size() * 4, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    switch (h->opts.precision) {
        case LBM_FP16_DEV: launch_init<lbmk::StoreF16>(h, h->lat[0]); break;
        case LBM_BF16_DEV: launch_init<lbmk::StoreBF16>(h, h->lat[0]); break;
        case LBM_FP16_ROW: launch_init<lbmk::StoreF16R>(h, h->lat[0]); break;
        default: launch_init<lbmk::StoreF32>(h, h->lat[0]); break;
    }
    h->cur = 0;
    h->t = 0;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    return cuda_fail(cudaStreamSynchronize(h->stream));
}

int lbm_step(lbm_handle *h, int n) {
    if (!h || n < 0) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    for (int s = 0; s < n;) {
        if (graph_usable(h) && n - s >= h->stg_ring) {
            const int rc = graph_segment(h);
            if (rc == LBM_OK) { s += h->stg_ring; continue; }
            if (rc != 1) return rc;
        }
        const int rc = one_step(h);
        if (rc) return rc;
        ++s;
    }
    return LBM_OK;
}

int lbm_sync(lbm_handle *h) {
    if (!h) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    unsigned fl[3] = {0, 0, 0};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(fl, h->d_flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    if (fl[0] || fl[1] || fl[2]) {
        if ((e = cudaMemsetAsync(h->d_flags, 0, sizeof fl, h->stream)) != cudaSuccess) return cuda_fail(e);
        cudaStreamSynchronize(h->stream);
    }
    if (fl[2]) return LBM_ETIMEOUT;
    if (fl[1]) return LBM_EDIVERGED;
    if (fl[0]) return LBM_ENOTCONV;
    return LBM_OK;
}

int lbm_set_step_kernel(lbm_handle *h, int kind) {
    if (!h) return LBM_EINVAL;
    switch (kind) {
        case LBM_KERNEL_AUTO: case LBM_KERNEL_CELL: break;
        case LBM_KERNEL_PAIR: if (h->nx % 2) return LBM_EINVAL; break;
        case LBM_KERNEL_STAGED: if (!staged_supported(h)) return LBM_EINVAL; break;
        case LBM_KERNEL_QUAD: if (h->nx % 4) return LBM_EINVAL; break;
        default: return LBM_EINVAL;
    }
    h->step_kind = kind;
    ++h->graph_epoch;
    return LBM_OK;
}

int lbm_set_graphs(lbm_handle *h, int on) {
    if (!h) return LBM_EINVAL;
    h->graphs_on = on != 0;
    return LBM_OK;
}

int lbm_probe_wait_timeout(lbm_handle *h) {
    if (!h) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    lbmk::wait_timeout_probe_kernel<<<1, 32, 0, h->stream>>>(h->d_flags, 1 << 14);
    h->launches += 1;
    return cuda_fail(cudaGetLastError());
}

int lbm_graph_info(const lbm_handle *h, int *on, long *launched) {
    if (!h || !on || !launched) return LBM_EINVAL;
    *on = h->graphs_on ? 1 : 0;
    *launched = (long)h->graph_launches;
    return LBM_OK;
}

int lbm_get_step_kernel(const lbm_handle *h, int *kind) {
    if (!h || !kind) return LBM_EINVAL;
    *kind = resolve_kind(h);
    return LBM_OK;
}

int lbm_set_sponge(lbm_handle *h, int cells, double nu_max) {
    if (!h || cells < 0 || cells > h->nx_global || !(nu_max >= 0.0) || !std::isfinite(nu_max)) return LBM_EINVAL;
    h->sponge_cells = nu_max > 0.0 ? cells : 0;
    h->sponge_nu = cells > 0 ? nu_max : 0.0;
    ++h->graph_epoch;
    return LBM_OK;
}

int lbm_set_slab(lbm_handle *h, int nx_global, int x_offset, int own_lo, int own_hi) {
    if (!h || own_lo < 0 || own_hi > h->nx || own_lo >= own_hi || x_offset < 0 ||
        x_offset + h->nx > nx_global)
        return LBM_EINVAL;
    // the global faces are this slab's lattice ends, or not in it at all
    if ((x_offset + own_lo == 0) != (own_lo == 0) || (x_offset + own_hi == nx_global) != (own_hi == h->nx))
        return LBM_EINVAL;
    h->nx_global = nx_global;
    h->x_offset = x_offset;
    h->own_lo = own_lo;
    h->own_hi = own_hi;
    ++h->graph_epoch;                            // the sponge position may move
    return LBM_OK;
}

int lbm_halo_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_EINVAL;
    *bytes = 5 * (size_t)h->ny * h->nz * h->elem;
    return LBM_OK;
}

}  // extern "C"

namespace {
// c_x = -1 and c_x = +1 populations (Sec. 2.1 order)
constexpr int kQxMinus[5] = {1, 5, 8, 11, 15};
constexpr int kQxPlus[5] = {3, 7, 10, 13, 17};

int halo_copy(lbm_handle *h, int face, void *buf, bool pack) {
    if (!h || !buf || (face != LBM_FACE_LEFT && face != LBM_FACE_RIGHT)) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    // left face: the first owned column sends its c_x = -1 populations to the
    // left neighbour; the ghost column before it receives the neighbour's
    // c_x = +1 populations.  The right face mirrors that.
    const bool left = face == LBM_FACE_LEFT;
    lbmk::HaloArgs a;
    const int *qs = (left == pack) ? kQxMinus : kQxPlus;
    for (int p = 0; p < 5; ++p) a.qs[p] = qs[p];
    a.col = pack ? (left ? h->own_lo : h->own_hi - 1) : (left ? h->own_lo - 1 : h->own_hi);
    if (a.col < 0 || a.col >= h->nx) return LBM_EINVAL;          // no neighbour on that side
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.ncell = h->ncell;
    const long long n = 5LL * h->ny * h->nz;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    void *lat = h->lat[h->cur];
    if (h->elem == 4) {
        if (pack) lbmk::halo_pack_kernel<float><<<blocks, 256, 0, h->stream>>>((const float *)lat, (float *)buf, a);
        else lbmk::halo_unpack_kernel<float><<<blocks, 256, 0, h->stream>>>((float *)lat, (const float *)buf, a);
    } else {
        if (pack)
            lbmk::halo_pack_kernel<uint16_t><<<blocks, 256, 0, h->stream>>>((const uint16_t *)lat, (uint16_t *)buf, a);
        else
            lbmk::halo_unpack_kernel<uint16_t><<<blocks, 256, 0, h->stream>>>((uint16_t *)lat, (const uint16_t *)buf, a);
    }
    h->launches += 1;
    return cuda_fail(cudaGetLastError());
}
}  // namespace

extern "C" {

int lbm_halo_pack(lbm_handle *h, int face, void *dev_buf) { return halo_copy(h, face, dev_buf, true); }
int lbm_halo_unpack(lbm_handle *h, int face, const void *dev_buf) {
    return halo_copy(h, face, const_cast<void *>(dev_buf), false);
}

int lbm_set_stream(lbm_handle *h, void *s) {
    if (!h) return LBM_EINVAL;
    h->stream = (cudaStream_t)s;
    h->opts.cuda_stream = s;
    return LBM_OK;
}

int lbm_stats(lbm_handle *h, double *sums, double *utau_sums, long *n_samples) {
    if (!h || !sums || !utau_sums || !n_samples) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(sums, h->d_st, 7 * sizeof(double) * h->nx * h->ny, cudaMemcpyDeviceToHost,
                             h->stream)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(utau_sums, h->d_st_utau, 2 * sizeof(double) * h->nx, cudaMemcpyDeviceToHost,
                             h->stream)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    *n_samples = h->n_samples;
    return LBM_OK;
}

int lbm_reset_stats(lbm_handle *h) {
    if (!h) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->d_st, 0, 7 * sizeof(double) * h->nx * h->ny, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemsetAsync(h->d_st_utau, 0, 2 * sizeof(double) * h->nx, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    h->steps_since_stats = 0;
    h->n_samples = 0;
    return LBM_OK;
}

int lbm_get_fields(lbm_handle *h, double *rho, double *u) {
    if (!h || !rho || !u) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    // the other lattice is free between steps: use it as scratch (>= 16 B per cell)
    float *drho = (float *)h->lat[h->cur ^ 1];
    float *du = drho + h->ncell;
    const long long n = h->ncell;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    h->launches += 1;
    switch (h->opts.precision) {
        case LBM_FP16_DEV:
            lbmk::fields_kernel<lbmk::StoreF16><<<blocks, 256, 0, h->stream>>>(
                (const __half *)h->lat[h->cur], h->d_rowbase, h->d_fw, drho, du, h->nx, h->ny, h->nz, n);
            break;
        case LBM_BF16_DEV:
            lbmk::fields_kernel<lbmk::StoreBF16><<<blocks, 256, 0, h->stream>>>(
                (const __nv_bfloat16 *)h->lat[h->cur], h->d_rowbase, h->d_fw, drho, du, h->nx, h->ny, h->nz, n);
            break;
        case LBM_FP16_ROW:
            lbmk::fields_kernel<lbmk::StoreF16R><<<blocks, 256, 0, h->stream>>>(
                (const __half *)h->lat[h->cur], h->d_rowbase, h->d_fw, drho, du, h->nx, h->ny, h->nz, n);
            break;
        default:
            lbmk::fields_kernel<lbmk::StoreF32><<<blocks, 256, 0, h->stream>>>(
                (const float *)h->lat[h->cur], h->d_rowbase, h->d_fw, drho, du, h->nx, h->ny, h->nz, n);
    }
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    std::vector<float> buf(4 * (size_t)n);
    if ((e = cudaMemcpyAsync(buf.data(), drho, 4 * sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream)) !=
        cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    for (long long c = 0; c < n; ++c) rho[c] = buf[c];
    for (long long c = 0; c < 3 * n; ++c) u[c] = buf[n + c];
    return LBM_OK;
}

int lbm_get_populations(lbm_handle *h, double *f) {
    if (!h || !f) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    const size_t n = 19 * (size_t)h->ncell;
    std::vector<char> buf(n * h->elem);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(buf.data(), h->lat[h->cur], n * h->elem, cudaMemcpyDeviceToHost, h->stream)) !=
        cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    const size_t N = h->ncell;
    for (size_t idx = 0; idx < n; ++idx) {
        const int q = (int)(idx / N);
        if (h->opts.precision == LBM_FP32) f[idx] = ((const float *)buf.data())[idx];
        else if (h->opts.precision == LBM_FP16_DEV)
            f[idx] = kW[q] + (double)__half2float(((const __half *)buf.data())[idx]);
        else {  // row base: f - w as the kernels form it, stored word + row base, in FP32
            const float word = h->opts.precision == LBM_BF16_DEV
                                   ? bf16_to_f32(((const uint16_t *)buf.data())[idx])
                                   : __half2float(((const __half *)buf.data())[idx]);
            f[idx] = kW[q] + (double)(word + h->rb((int)((idx % N) / h->nx % h->ny), q));
        }
    }
    return LBM_OK;
}

int lbm_set_populations(lbm_handle *h, const double *f) {
    if (!h || !f) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    const size_t n = 19 * (size_t)h->ncell, N = h->ncell;
    std::vector<char> buf(n * h->elem);
    for (size_t idx = 0; idx < n; ++idx) {
        const int q = (int)(idx / N);
        if (h->opts.precision == LBM_FP32) ((float *)buf.data())[idx] = (float)f[idx];
        else if (h->opts.precision == LBM_FP16_DEV)
            ((__half *)buf.data())[idx] = __double2half(f[idx] - kW[q]);
        else {
            const float dev = (float)(f[idx] - kW[q] - (double)h->rb((int)((idx % N) / h->nx % h->ny), q));
            if (h->opts.precision == LBM_BF16_DEV) ((uint16_t *)buf.data())[idx] = f32_to_bf16_rn(dev);
            else ((__half *)buf.data())[idx] = __float2half_rn(dev);
        }
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->lat[h->cur], buf.data(), n * h->elem, cudaMemcpyHostToDevice, h->stream)) !=
        cudaSuccess) return cuda_fail(e);
    return cuda_fail(cudaStreamSynchronize(h->stream));
}

int lbm_get_utau(lbm_handle *h, double *utau) {
    if (!h || !utau) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    const size_t n = 2 * (size_t)h->nz * h->nx;
    std::vector<float> buf(n);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(buf.data(), h->d_utau, n * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c < n; ++c) utau[c] = buf[c];
    return LBM_OK;
}

int lbm_get_time(const lbm_handle *h, long *t) {
    if (!h || !t) return LBM_EINVAL;
    *t = (long)h->t;
    return LBM_OK;
}

int lbm_set_time(lbm_handle *h, long t) {
    if (!h || t < 0) return LBM_EINVAL;
    h->t = t;
    return LBM_OK;
}

int lbm_get_constants(const lbm_handle *h, double out[6]) {
    if (!h || !out) return LBM_EINVAL;
    out[0] = h->delta; out[1] = h->utau_ref; out[2] = h->nu; out[3] = h->tau0; out[4] = h->ubp; out[5] = h->maxl;
    return LBM_OK;
}

int lbm_inlet_velocity(lbm_handle *h, long t, double *out) {
    if (!h || !out || t < 0) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    h->stg_reset();                              // the call writes into the ring
    launch_stg(h, t, 1, true);
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    const size_t n = 3 * (size_t)h->ny * h->nz;
    std::vector<float> buf(n);
    if ((e = cudaMemcpyAsync(buf.data(), h->d_uin, n * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c < n; ++c) out[c] = buf[c];
    return LBM_OK;
}

int lbm_set_params(lbm_handle *h, const double theta[4]) {
    if (!h || !theta) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!(theta[0] > 0) || !(theta[2] > 0)) return LBM_EINVAL;
    for (int c = 0; c < 4; ++c) h->theta[c] = theta[c];
    h->tables();
    if (!h->bound) return LBM_OK;
    cudaError_t e = h->upload_tables();
    if (e == cudaSuccess && h->adj.bound) e = h->upload_adjoint_tables();
    return cuda_fail(e);
}

int lbm_set_inlet_profile(lbm_handle *h, const double *U, const double *R) {
    if (!h || !U || !R) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    std::vector<double> oldU = h->prof_U, oldR = h->prof_R;
    h->prof_U.assign(U, U + h->ny);
    h->prof_R.assign(R, R + 6 * (size_t)h->ny);
    if (!h->profile_tables(h->theta[1])) {
        h->prof_U = oldU; h->prof_R = oldR;
        h->profile_tables(h->theta[1]);
        return LBM_EINVAL;
    }
    h->custom_profile = true;
    if (!h->bound) return LBM_OK;
    cudaError_t e;
    // Double-buffered upload: the profile goes into the buffer not in use, on
    // the copy stream, after the steps that last read that buffer (those
    // before the previous call), so that it overlaps the steps in flight; the
    // handle's stream waits for it before the next step.
    const int b = h->prof_cur ^ 1;
    const size_t n7 = 7 * (size_t)h->ny;
    float *stage = h->pin_stage + n7 * b, *dst = h->d_prof + n7 * b;
    // the staging half may still feed the upload of two calls ago
    if ((e = cudaEventSynchronize(h->ev_prof_ready[b])) != cudaSuccess) return cuda_fail(e);
    std::copy(h->UR.begin(), h->UR.end(), stage);
    std::copy(h->amat.begin(), h->amat.end(), stage + h->ny);
    if ((e = cudaStreamWaitEvent(h->copy, h->ev_prof_free[b], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dst, stage, n7 * sizeof(float), cudaMemcpyHostToDevice, h->copy)) != cudaSuccess ||
        (e = cudaEventRecord(h->ev_prof_ready[b], h->copy)) != cudaSuccess ||
        (e = cudaEventRecord(h->ev_prof_free[h->prof_cur], h->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->stream, h->ev_prof_ready[b], 0)) != cudaSuccess)
        return cuda_fail(e);
    h->prof_cur = b;
    h->d_UR = dst;
    h->d_amat = dst + h->ny;
    return LBM_OK;
}

int lbm_get_inlet_profile(const lbm_handle *h, double *U, double *R) {
    if (!h || !U || !R) return LBM_EINVAL;
    std::copy(h->prof_U.begin(), h->prof_U.end(), U);
    std::copy(h->prof_R.begin(), h->prof_R.end(), R);
    return LBM_OK;
}

}  // extern "C"

// z-averaged wall shear of the last step into device memory out[2 * nx]
// (every entry written).
static void launch_wall_shear(lbm_handle *h, double *out, cudaStream_t st) {
    const dim3 grid((h->nx + lbmk::WS_X - 1) / lbmk::WS_X, 2), block(lbmk::WS_X, lbmk::WS_Z);
    lbmk::wall_shear_kernel<<<grid, block, 0, st>>>(h->d_fw, out, h->nx, h->nz);
}

extern "C" {

int lbm_wall_shear_async(lbm_handle *h, double *out) {
    if (!h || !out) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    const int n = 2 * h->nx;
    // page-locked host memory the device can address: the reduction stores
    // straight into it (no separate copy on the stream); other memory gets
    // the device result copied
    cudaPointerAttributes pa;
    double *direct = nullptr;
    if (cudaPointerGetAttributes(&pa, out) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer) direct = static_cast<double *>(pa.devicePointer);
    } else {
        cudaGetLastError();                      // not a pointer CUDA knows: copy
    }
    // When the side-stream wall kernel wrote the forces, the reduction follows
    // it there, beside the interior kernel of the same step; the handle's
    // stream then waits for it, so it still precedes whatever the caller
    // enqueues next (and the next step's wall kernel comes after it on the
    // side stream).
    const cudaStream_t st = h->fw_side ? h->side : h->stream;
    launch_wall_shear(h, direct ? direct : h->d_tw, st);
    h->launches += 1;
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    if (!direct &&
        (e = cudaMemcpyAsync(out, h->d_tw, n * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e);
    if (st != h->stream &&
        ((e = cudaEventRecord(h->ev_shear, st)) != cudaSuccess ||
         (e = cudaStreamWaitEvent(h->stream, h->ev_shear, 0)) != cudaSuccess))
        return cuda_fail(e);
    return LBM_OK;
}

int lbm_wall_shear(lbm_handle *h, double *out) {
    if (!h || !out) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    const int rc = lbm_wall_shear_async(h, out);
    if (rc) return rc;
    return cuda_fail(cudaStreamSynchronize(h->stream));
}

// ---------------------------------------------------------------------------
// Wall shear without any allocation.  The staging buffer of the reduction is
// this fixed array: device code could name it directly, host code needs its
// device address, looked up once per device with that device current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_wall_shear[2 * LBM_NOALLOC_MAX_NX];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

int lbm_wall_shear_noalloc(lbm_handle *h, double *out) {
    if (!h || !out) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    if (h->nx > LBM_NOALLOC_MAX_NX) {
        std::fprintf(stderr, "liblbm_gb300: lbm_wall_shear_noalloc: nx = %d exceeds the fixed scratch "
                     "(LBM_NOALLOC_MAX_NX = %d)\n", h->nx, LBM_NOALLOC_MAX_NX);
        return LBM_ENOSCRATCH;
    }
    // the array's address on the handle's device (made current by the guard)
    const int dev = h->device;
    cudaError_t e;
    if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, g_noalloc_wall_shear)) != cudaSuccess) return cuda_fail(e);
            g_noalloc_ptr[dev] = (double *)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    const int n = 2 * h->nx;
    // every entry read below is written by this launch first
    launch_wall_shear(h, scratch, h->stream);
    h->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(out, scratch, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    return cuda_fail(cudaStreamSynchronize(h->stream));
}

int lbm_debug_guard_bands(lbm_handle *h, int bytes) {
    if (!h || bytes < 0) return LBM_EINVAL;
    if (h->bound) return LBM_ESTATE;
    h->guard_bytes = (size_t)bytes;
    return LBM_OK;
}

int lbm_debug_check_guards(lbm_handle *h, long long *changed) {
    if (!h || !changed) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    cudaError_t e;
    for (cudaStream_t st : {h->stream, h->side, h->aux, h->copy})
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    long long bad = 0;
    std::vector<unsigned char> buf;
    auto scan = [&](void *base, const std::vector<std::pair<size_t, size_t>> &bands) -> cudaError_t {
        for (const auto &b : bands) {
            buf.resize(b.second);
            cudaError_t err = cudaMemcpy(buf.data(), (char *)base + b.first, b.second, cudaMemcpyDeviceToHost);
            if (err != cudaSuccess) return err;
            for (unsigned char c : buf) bad += c != kGuardByte;
        }
        return cudaSuccess;
    };
    if ((e = scan(h->mem, h->guards)) != cudaSuccess) return cuda_fail(e);
    if (h->adj.bound && (e = scan(h->adj.mem, h->adj_guards)) != cudaSuccess) return cuda_fail(e);
    *changed = bad;
    return LBM_OK;
}

int lbm_profile_enable(lbm_handle *h, int on) {
    if (!h || on < 0) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (on && h->ev0.empty()) {
        h->ev0.resize(kEventPool); h->ev1.resize(kEventPool); h->ev_busy.assign(kEventPool, 0);
        for (size_t c = 0; c < kEventPool; ++c) {
            if (cudaEventCreate(&h->ev0[c]) != cudaSuccess || cudaEventCreate(&h->ev1[c]) != cudaSuccess)
                return cuda_fail(cudaGetLastError());
        }
    }
    h->prof_on = on != 0;
    h->prof_every = on > 0 ? on : 1;
    h->prof_count = 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_handle *h, double *ms_total, long *step_launches, long *all_launches) {
    if (!h || !ms_total || !step_launches || !all_launches) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    for (size_t c = 0; c < h->ev_busy.size(); ++c) prof_harvest(h, c);
    *ms_total = h->prof_ms;
    *step_launches = h->prof_n;
    *all_launches = h->launches;
    h->prof_ms = 0;
    h->prof_n = 0;
    h->launches = 0;
    return cuda_fail(cudaGetLastError());
}

int lbm_adjoint_required_bytes(const lbm_handle *h, int window, int ckpt_every, size_t *bytes) {
    if (!h || !bytes || window < 1 || ckpt_every < 1 || window % ckpt_every) return LBM_EINVAL;
    Arena ar;
    ar.guard = h->guard_bytes;
    lbm_handle *m = const_cast<lbm_handle *>(h);
    AdjointWork keep = m->adj;
    *bytes = m->adjoint_layout(ar, window, ckpt_every);
    m->adj = keep;
    return LBM_OK;
}

int lbm_adjoint_bind(lbm_handle *h, int window, int ckpt_every, void *dev_ptr, size_t bytes) {
    if (!h || window < 1 || ckpt_every < 1 || window % ckpt_every) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (h->opts.precision != LBM_FP32) return LBM_EINVAL;
    if (!h->bound) return LBM_ESTATE;
    size_t need = 0;
    lbm_adjoint_required_bytes(h, window, ckpt_every, &need);
    if (h->adj.bound && h->adj.owns && h->adj.mem) cudaFree(h->adj.mem);
    h->adj = AdjointWork();
    void *mem = dev_ptr;
    bool owns = false;
    if (dev_ptr) {
        if (((uintptr_t)dev_ptr & 255) != 0) return LBM_EINVAL;
        if (bytes < need) return LBM_ENOMEM;
    } else {
        if (cudaMalloc(&mem, need) != cudaSuccess) { cudaGetLastError(); return LBM_ENOMEM; }
        owns = true;
    }
    Arena ar;
    ar.base = (char *)mem;
    ar.guard = h->guard_bytes;
    h->adj_guards.clear();
    ar.bands = &h->adj_guards;
    h->adjoint_layout(ar, window, ckpt_every);
    h->adj.mem = mem; h->adj.owns = owns; h->adj.bound = true;
    h->adj.T = window; h->adj.K = ckpt_every;
    cudaError_t e;
    if ((e = cudaMemsetAsync(mem, 0, need, h->stream)) != cudaSuccess) return cuda_fail(e);
    for (const auto &b : h->adj_guards)
        if ((e = cudaMemsetAsync((char *)mem + b.first, kGuardByte, b.second, h->stream)) != cudaSuccess)
            return cuda_fail(e);
    return cuda_fail(h->upload_adjoint_tables());
}

int lbm_adjoint_step(lbm_handle *h, int window, int ckpt_every, const lbm_objective *obj, double *J,
                     double dJ_dtheta[4]) {
    if (!h || !obj || !J || !dJ_dtheta) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    if (!h->adj.bound || h->adj.T != window || h->adj.K != ckpt_every) {
        const int rc = lbm_adjoint_bind(h, window, ckpt_every, nullptr, 0);
        if (rc) return rc;
    }
    if (obj->i_tau0 < 0 || obj->i_tau1 > h->nx || obj->i_tau0 > obj->i_tau1 || obj->i_R < 0 || obj->i_R >= h->nx)
        return LBM_EINVAL;
    AdjointWork &A = h->adj;
    const int T = window, K = ckpt_every, nx = h->nx, ny = h->ny, nz = h->nz;
    const size_t L = 19 * (size_t)h->ncell, W = 2 * (size_t)nz * nx, I = 3 * (size_t)nz * ny;
    const long long t0 = h->t;
    cudaStream_t st = h->stream;
    cudaError_t e;
    // STG field of the window on the aux stream, beside the copies below
    if (h->opts.inlet) {
        if ((e = cudaEventRecord(h->ev_aux_fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->aux, h->ev_aux_fork, 0)) != cudaSuccess)
            return cuda_fail(e);
        launch_stg_into(h, A.vwin, t0, T, h->aux);
        if ((e = cudaEventRecord(h->ev_aux_join, h->aux)) != cudaSuccess) return cuda_fail(e);
    }
    // prescribed R12 of the J_R target, accumulators
    std::vector<double> r12(ny);
    for (int j = 0; j < ny; ++j) r12[j] = h->prof_R[6 * (size_t)j + 3];
    if ((e = cudaMemcpyAsync(A.r12, r12.data(), ny * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemsetAsync(A.objacc, 0, (1 + 3 * (size_t)ny) * sizeof(double), st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemsetAsync(A.gtheta, 0, 4 * sizeof(double), st)) != cudaSuccess) return cuda_fail(e);
    // ---- forward over the window: s_0 copied to checkpoint 0, every K-th state
    // written straight into its checkpoint, u_tau of step n into uthist[n] ----
    if ((e = cudaMemcpyAsync(A.ut_init, h->d_utau, W * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpyAsync(A.ckpt, h->lat[h->cur], L * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if (h->opts.inlet && (e = cudaStreamWaitEvent(st, h->ev_aux_join, 0)) != cudaSuccess) return cuda_fail(e);
    const int obj_blocks = ny + (2 * nz * (obj->i_tau1 - obj->i_tau0) + 127) / 128;
    // the objective sums ride along in the step kernels, except in the
    // one-cell kernel (nx odd), which leaves them to objective_kernel
    const bool fused_obj = resolve_kind(h) != LBM_KERNEL_CELL;
    const void *cur = A.ckpt;
    int pp = 0;                                  // next lattice buffer of the ping-pong
    // the K - 1 recomputed states of segment s sit in slot set s % kSlotSets
    auto slots = [&](int sgm) { return A.seg + (size_t)(sgm % kSlotSets) * (K - 1) * L; };
    // the states inside the last kSlotSets segments go straight to their slot
    // sets (one each), so that the reverse sweep recomputes none of them
    const int S = T / K;
    auto stored = [&](int sgm) { return sgm >= S - kSlotSets; };
    for (int n = 0; n < T; ++n) {
        void *out;
        const int m = n + 1, sg = m / K;
        if (m < T && m % K == 0) out = A.ckpt + (size_t)sg * L;
        else if (m < T && stored(sg)) out = slots(sg) + (size_t)(m % K - 1) * L;
        else { out = h->lat[pp]; pp ^= 1; }
        if (out == cur) { out = h->lat[pp]; pp ^= 1; }
        StepIO io;
        io.in = cur; io.out = out;
        io.utau_in = n == 0 ? A.ut_init : A.uthist + (size_t)(n - 1) * W;
        io.utau = A.uthist + (size_t)n * W;
        io.fw = h->d_fw; io.vprime = A.vwin + (size_t)n * I; io.stats = false;
        if (fused_obj) { io.obj = A.objacc; io.obj_i0 = obj->i_tau0; io.obj_i1 = obj->i_tau1; io.obj_iR = obj->i_R; }
        if (cudaError_t le = launch_step_io(h, io)) return cuda_fail(le);
        h->t += 1;
        cur = out;
        if (!fused_obj) {
            lbmk::objective_kernel<<<obj_blocks, 128, 0, st>>>((const float *)cur, h->d_fw, A.objacc, nx, ny, nz,
                                                               obj->i_tau0, obj->i_tau1, obj->i_R);
            h->launches += 1;
        }
    }
    h->cur = cur == h->lat[0] ? 0 : 1;          // s_T is in a lattice buffer
    if ((e = cudaMemcpyAsync(h->d_utau, A.uthist + (size_t)(T - 1) * W, W * 4, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess) return cuda_fail(e);
    // ---- J_R seeds on the device (no host round trip between the sweeps) ----
    const double ur2 = h->utau_ref * h->utau_ref;
    const double nw = 2.0 * (obj->i_tau1 - obj->i_tau0) * nz;
    lbmk::objective_seed_kernel<<<(ny + 63) / 64, 64, 0, st>>>(A.objacc, A.r12, A.jr_coef, A.jr_mean, ny,
                                                               (double)T * nz, ur2);
    h->launches += 1;
    const float jtau_w = nw > 0 ? (float)(1.0 / (T * nw * ur2)) : 0.0f;
    // ---- reverse: segments from the last, recompute from the checkpoint ----
    if ((e = cudaMemsetAsync(A.lamA, 0, L * 4, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(A.lamB, 0, L * 4, st)) != cudaSuccess) return cuda_fail(e);
    float *lam = A.lamA, *lout = A.lamB;
    const long long t_end = h->t;
    // The recomputation of segment s - 1 is independent of the reverse steps
    // of segment s: with one-launch adjoint steps (nx even) it runs on its own
    // stream beside them, into its slot set, once the reverse steps of
    // segment s - 1 + kSlotSets (which read that set) are done.  Same kernels,
    // same inputs: the results do not depend on the overlap.
    const bool overlap = h->nx % 2 == 0 && S > kSlotSets;
    if (overlap) {
        if (!h->rstream && (e = cudaStreamCreateWithFlags(&h->rstream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e);
        if (!h->ev_rstart && (e = cudaEventCreateWithFlags(&h->ev_rstart, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e);
        for (int c = 0; c < kSlotSets; ++c)
            for (cudaEvent_t *ev : {&h->ev_rec[c], &h->ev_rev[c]})
                if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
                    return cuda_fail(e);
        // the checkpoints, u_tau history and STG field of the forward pass are ready
        if ((e = cudaEventRecord(h->ev_rstart, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->rstream, h->ev_rstart, 0)) != cudaSuccess)
            return cuda_fail(e);
    }
    auto recompute = [&](int sgm, cudaStream_t on) -> cudaError_t {
        const int base = sgm * K;
        const float *prev = A.ckpt + (size_t)sgm * L;
        float *sl = slots(sgm);
        const cudaStream_t keep = h->stream;
        h->stream = on;
        cudaError_t err = cudaSuccess;
        for (int m = 1; m < K && err == cudaSuccess; ++m) {
            const int n = base + m - 1;
            StepIO io;
            io.in = prev; io.out = sl + (size_t)(m - 1) * L;
            io.utau_in = n == 0 ? A.ut_init : A.uthist + (size_t)(n - 1) * W;
            io.utau = A.ut_scr; io.fw = A.fw_scr; io.vprime = A.vwin + (size_t)n * I; io.stats = false;
            h->t = t0 + n;
            err = launch_step_io(h, io);
            prev = sl + (size_t)(m - 1) * L;
        }
        h->stream = keep;
        return err;
    };
    for (int sgm = S - 1; sgm >= 0; --sgm) {
        const int base = sgm * K;
        // this segment's states: from the forward pass (the last kSlotSets),
        // from the recomputation enqueued beside the previous segment, or
        // recomputed here
        if (!stored(sgm)) {
            if (overlap) {
                if ((e = cudaStreamWaitEvent(st, h->ev_rec[sgm % kSlotSets], 0)) != cudaSuccess) return cuda_fail(e);
            } else if (cudaError_t le = recompute(sgm, st)) {
                return cuda_fail(le);
            }
        }
        if (overlap && sgm >= 1 && !stored(sgm - 1)) {
            const int last_reader = sgm - 1 + kSlotSets;      // the previous user of that set
            if (last_reader <= S - 1 &&
                (e = cudaStreamWaitEvent(h->rstream, h->ev_rev[last_reader % kSlotSets], 0)) != cudaSuccess)
                return cuda_fail(e);
            if (cudaError_t le = recompute(sgm - 1, h->rstream)) return cuda_fail(le);
            if ((e = cudaEventRecord(h->ev_rec[(sgm - 1) % kSlotSets], h->rstream)) != cudaSuccess)
                return cuda_fail(e);
        }
        for (int n = base + K - 1; n >= base; --n) {
            const float *sn = n == base ? A.ckpt + (size_t)sgm * L : slots(sgm) + (size_t)(n - base - 1) * L;
            launch_adjoint(h, sn, lam, lout, A.uthist + (size_t)n * W, A.vwin + (size_t)n * I,
                           h->opts.inlet ? A.luin + (size_t)n * I : nullptr, true, obj, jtau_w);
            std::swap(lam, lout);
        }
        if (overlap && (e = cudaEventRecord(h->ev_rev[sgm % kSlotSets], st)) != cudaSuccess) return cuda_fail(e);
        // theta gradient through this segment's inlet velocities, beside the
        // next segment's reverse steps
        if (h->opts.inlet) {
            if ((e = cudaEventRecord(h->ev_aux_fork, st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(h->aux, h->ev_aux_fork, 0)) != cudaSuccess)
                return cuda_fail(e);
            launch_stg_adjoint(h, t0 + base, K, A.luin + (size_t)base * I, h->aux);
        }
    }
    h->t = t_end;
    if (lam != A.lamA) std::swap(A.lamA, A.lamB);   // lambda_0 in lamA
    if (h->opts.inlet) {
        if ((e = cudaEventRecord(h->ev_aux_join, h->aux)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, h->ev_aux_join, 0)) != cudaSuccess)
            return cuda_fail(e);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    // ---- J (FP64, on the host) from the window sums, and dJ/dtheta ----
    std::vector<double> acc(1 + 3 * (size_t)ny);
    if ((e = cudaMemcpyAsync(acc.data(), A.objacc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(dJ_dtheta, A.gtheta, 4 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    const double Jt = nw > 0 ? acc[0] / (T * nw * ur2) : 0.0;
    double JR = 0.0;
    for (int j = 0; j < ny; ++j) {
        const double cnt = (double)T * nz;
        const double mu = acc[1 + 3 * j] / cnt, mv = acc[2 + 3 * j] / cnt, muv = acc[3 + 3 * j] / cnt;
        const double r = (muv - mu * mv) / ur2 - h->prof_R[6 * (size_t)j + 3] / ur2;
        JR += r * r;
    }
    *J = Jt + JR;
    A.have_lambda0 = true;
    return LBM_OK;
}

int lbm_adjoint_state_gradient(lbm_handle *h, double *lambda0) {
    if (!h || !lambda0) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->adj.bound || !h->adj.have_lambda0) return LBM_ESTATE;
    const size_t L = 19 * (size_t)h->ncell;
    std::vector<float> buf(L);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(buf.data(), h->adj.lamA, L * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c < L; ++c) lambda0[c] = buf[c];
    return LBM_OK;
}

int lbm_vjp_step(lbm_handle *h, const double *lambda_next, double *lambda_prev, double dtheta[4]) {
    if (!h || !lambda_next || !lambda_prev || !dtheta) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    if (!h->adj.bound) {
        const int rc = lbm_adjoint_bind(h, 1, 1, nullptr, 0);
        if (rc) return rc;
    }
    AdjointWork &A = h->adj;
    const size_t L = 19 * (size_t)h->ncell, W = 2 * (size_t)h->nz * h->nx;
    cudaStream_t st = h->stream;
    cudaError_t e;
    if (h->opts.inlet) launch_stg_into(h, A.vwin, h->t, 1, h->stream);
    if ((e = cudaMemsetAsync(A.gtheta, 0, 4 * sizeof(double), st)) != cudaSuccess) return cuda_fail(e);
    // forward step into scratch for this step's u_tau (the state stays)
    if ((e = cudaMemcpyAsync(A.ut_scr, h->d_utau, W * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    StepIO io;
    io.in = h->lat[h->cur]; io.out = A.lamB; io.utau = A.ut_scr; io.fw = A.fw_scr; io.vprime = A.vwin;
    io.stats = false;
    if (cudaError_t le = launch_step_io(h, io)) return cuda_fail(le);
    std::vector<float> buf(L);
    for (size_t c = 0; c < L; ++c) buf[c] = (float)lambda_next[c];
    if ((e = cudaMemcpyAsync(A.lamA, buf.data(), L * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemsetAsync(A.lamB, 0, L * 4, st)) != cudaSuccess) return cuda_fail(e);
    launch_adjoint(h, (const float *)h->lat[h->cur], A.lamA, A.lamB, A.ut_scr, A.vwin,
                   h->opts.inlet ? A.luin : nullptr, false, nullptr, 0.0f);
    launch_stg_adjoint(h, h->t, 1, h->adj.luin, h->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(buf.data(), A.lamB, L * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpyAsync(dtheta, A.gtheta, 4 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c < L; ++c) lambda_prev[c] = buf[c];
    A.have_lambda0 = false;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint files: a fixed header, then the payload -- the stored lattice
// (raw FP32 or 16-bit words), u_tau, the statistics accumulators and, if one
// was set, the inlet profile -- with a 64-bit FNV-1a checksum over the payload
// folded eight bytes at a time.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

constexpr char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};
constexpr uint32_t kFileVersion = 2;

struct FileHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t nx, ny, nz, precision, n_modes, inlet, wall_model, stats_every, custom_profile, sponge_cells;
    int64_t t, n_samples, steps_since_stats;
    double re_tau, u_bulk, c_smag, kappa0, B0, theta[4], sponge_nu;
    uint64_t uniforms_hash, payload_bytes, checksum;
};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        size_t i = 0;
        for (; i + 8 <= n; i += 8) {
            uint64_t w;
            std::memcpy(&w, b + i, 8);
            h = (h ^ w) * 1099511628211ull;
        }
        for (; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

uint64_t hash_doubles(const std::vector<double> &v) {
    Fnv f;
    f.add(v.data(), v.size() * sizeof(double));
    return f.h;
}

struct Payload {            // device ranges of the payload, in file order
    std::vector<std::pair<void *, size_t>> dev;
};

Payload payload_of(lbm_handle *h) {
    Payload p;
    p.dev.push_back({h->lat[h->cur], 19 * (size_t)h->ncell * h->elem});
    p.dev.push_back({h->d_utau, 2 * (size_t)h->nz * h->nx * sizeof(float)});
    p.dev.push_back({h->d_st, 7 * (size_t)h->nx * h->ny * sizeof(double)});
    p.dev.push_back({h->d_st_utau, 2 * (size_t)h->nx * sizeof(double)});
    return p;
}

constexpr size_t kChunk = 64u << 20;   // host staging of device ranges

}  // namespace

extern "C" {

int lbm_save(lbm_handle *h, const char *path) {
    if (!h || !path) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e);
    FileHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = kFileVersion; hd.header_bytes = sizeof(FileHeader);
    hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.precision = h->opts.precision;
    hd.n_modes = h->n_modes; hd.inlet = h->opts.inlet; hd.wall_model = h->opts.wall_model;
    hd.stats_every = h->opts.stats_every; hd.custom_profile = h->custom_profile ? 1 : 0;
    hd.sponge_cells = h->sponge_cells; hd.sponge_nu = h->sponge_nu;
    hd.t = h->t; hd.n_samples = h->n_samples; hd.steps_since_stats = h->steps_since_stats;
    hd.re_tau = h->re_tau; hd.u_bulk = h->opts.u_bulk; hd.c_smag = h->opts.c_smag;
    hd.kappa0 = h->opts_kappa0; hd.B0 = h->opts.B;
    for (int c = 0; c < 4; ++c) hd.theta[c] = h->theta[c];
    hd.uniforms_hash = hash_doubles(h->uniforms);
    const Payload pl = payload_of(h);
    size_t total = 0;
    for (auto &r : pl.dev) total += r.second;
    if (h->custom_profile) total += (h->prof_U.size() + h->prof_R.size()) * sizeof(double);
    hd.payload_bytes = total;
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return LBM_EINVAL;
    int rc = LBM_OK;
    Fnv f;
    std::vector<char> buf(kChunk);
    if (std::fwrite(&hd, sizeof hd, 1, fp) != 1) rc = LBM_EINVAL;   // checksum patched below
    for (auto &r : pl.dev) {
        for (size_t off = 0; rc == LBM_OK && off < r.second; off += kChunk) {
            const size_t n = std::min(kChunk, r.second - off);
            if ((e = cudaMemcpyAsync(buf.data(), (char *)r.first + off, n, cudaMemcpyDeviceToHost, h->stream)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
                rc = cuda_fail(e);
                break;
            }
            f.add(buf.data(), n);
            if (std::fwrite(buf.data(), 1, n, fp) != n) rc = LBM_EINVAL;
        }
    }
    if (rc == LBM_OK && h->custom_profile) {
        for (const std::vector<double> *v : {&h->prof_U, &h->prof_R}) {
            f.add(v->data(), v->size() * sizeof(double));
            if (std::fwrite(v->data(), sizeof(double), v->size(), fp) != v->size()) rc = LBM_EINVAL;
        }
    }
    if (rc == LBM_OK) {
        hd.checksum = f.h;
        if (std::fseek(fp, 0, SEEK_SET) != 0 || std::fwrite(&hd, sizeof hd, 1, fp) != 1) rc = LBM_EINVAL;
    }
    if (std::fclose(fp) != 0 && rc == LBM_OK) rc = LBM_EINVAL;
    return rc;
}

int lbm_load(lbm_handle *h, const char *path) {
    if (!h || !path) return LBM_EINVAL;
    LBM_DEVICE_GUARD(h);
    if (!h->bound) return LBM_ESTATE;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return LBM_EINVAL;
    FileHeader hd;
    int rc = LBM_OK;
    if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, kMagic, 8) != 0 ||
        hd.version != kFileVersion || hd.header_bytes != sizeof(FileHeader))
        rc = LBM_EINVAL;
    // the file must come from a channel created like this one
    if (rc == LBM_OK &&
        (hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.precision != h->opts.precision ||
         hd.n_modes != h->n_modes || hd.inlet != h->opts.inlet || hd.wall_model != h->opts.wall_model ||
         hd.stats_every != h->opts.stats_every || hd.re_tau != h->re_tau || hd.u_bulk != h->opts.u_bulk ||
         hd.c_smag != h->opts.c_smag || hd.kappa0 != h->opts_kappa0 || hd.B0 != h->opts.B ||
         hd.uniforms_hash != hash_doubles(h->uniforms)))
        rc = LBM_EINVAL;
    // read and check the whole payload before touching the handle
    const Payload pl = payload_of(h);
    size_t dev_bytes = 0;
    for (auto &r : pl.dev) dev_bytes += r.second;
    const size_t prof_n = hd.custom_profile ? 7 * (size_t)h->ny : 0;
    if (rc == LBM_OK && hd.payload_bytes != dev_bytes + prof_n * sizeof(double)) rc = LBM_EINVAL;
    if (rc == LBM_OK && (hd.sponge_cells < 0 || hd.sponge_cells > h->nx_global || !(hd.sponge_nu >= 0.0))) rc = LBM_EINVAL;
    std::vector<char> data;
    std::vector<double> prof(prof_n);
    if (rc == LBM_OK) {
        data.resize(dev_bytes);
        Fnv f;
        for (size_t off = 0; off < dev_bytes; off += kChunk) {
            const size_t n = std::min(kChunk, dev_bytes - off);
            if (std::fread(data.data() + off, 1, n, fp) != n) { rc = LBM_EINVAL; break; }
            f.add(data.data() + off, n);
        }
        if (rc == LBM_OK && prof_n) {
            if (std::fread(prof.data(), sizeof(double), prof_n, fp) != prof_n) rc = LBM_EINVAL;
            else f.add(prof.data(), prof_n * sizeof(double));
        }
        if (rc == LBM_OK && (f.h != hd.checksum || std::fgetc(fp) != EOF)) rc = LBM_EINVAL;
    }
    std::fclose(fp);
    if (rc) return rc;
    // nothing the handle enqueued may still run when its state is replaced:
    // steps, wall rows and wall-shear reductions (side stream), STG refills
    // (aux) and profile uploads (copy) all write the buffers restored below
    cudaError_t e;
    for (cudaStream_t s : {h->stream, h->side, h->aux, h->copy})
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
    // parameters and inlet profile (host tables, uploaded), then the device state
    h->custom_profile = false;
    if ((rc = lbm_set_params(h, hd.theta)) != LBM_OK) return rc;
    if (prof_n && (rc = lbm_set_inlet_profile(h, prof.data(), prof.data() + h->ny)) != LBM_OK) return rc;
    size_t off = 0;
    for (auto &r : pl.dev) {
        if ((e = cudaMemcpyAsync(r.first, data.data() + off, r.second, cudaMemcpyHostToDevice, h->stream)) !=
            cudaSuccess) return cuda_fail(e);
        off += r.second;
    }
    h->sponge_cells = hd.sponge_cells;
    h->sponge_nu = hd.sponge_nu;
    ++h->graph_epoch;
    h->t = hd.t;
    h->n_samples = (long)hd.n_samples;
    h->steps_since_stats = hd.steps_since_stats;
    h->stg_reset();                              // the STG ring is refilled at the next step
    return cuda_fail(cudaStreamSynchronize(h->stream));
}

void lbm_destroy(lbm_handle *h) {
    if (!h) return;
    DeviceGuard device_guard(h);
    // no work of the handle may still run when its memory goes
    if (h->copy) cudaStreamSynchronize(h->copy);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->adj.owns && h->adj.mem) { cudaStreamSynchronize(h->stream); cudaFree(h->adj.mem); }
    if (h->bound) cudaStreamSynchronize(h->stream);
    for (size_t c = 0; c < h->ev0.size(); ++c) { cudaEventDestroy(h->ev0[c]); cudaEventDestroy(h->ev1[c]); }
    if (h->owns && h->mem) cudaFree(h->mem);
    if (h->copy) { cudaStreamSynchronize(h->copy); cudaStreamDestroy(h->copy); }
    if (h->pin_stage) cudaFreeHost(h->pin_stage);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_prof_ready[b]) cudaEventDestroy(h->ev_prof_ready[b]);
        if (h->ev_prof_free[b]) cudaEventDestroy(h->ev_prof_free[b]);
    }
    if (h->side) { cudaStreamSynchronize(h->side); cudaStreamDestroy(h->side); }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) { cudaStreamSynchronize(h->aux); cudaStreamDestroy(h->aux); }
    if (h->ev_aux_fork) cudaEventDestroy(h->ev_aux_fork);
    if (h->ev_aux_join) cudaEventDestroy(h->ev_aux_join);
    if (h->ev_stg_free) cudaEventDestroy(h->ev_stg_free);
    if (h->ev_stg_ready) cudaEventDestroy(h->ev_stg_ready);
    if (h->ev_shear) cudaEventDestroy(h->ev_shear);
    graphs_clear(h);
    if (h->rstream) { cudaStreamSynchronize(h->rstream); cudaStreamDestroy(h->rstream); }
    if (h->ev_rstart) cudaEventDestroy(h->ev_rstart);
    for (int c = 0; c < kSlotSets; ++c)
        for (cudaEvent_t ev : {h->ev_rec[c], h->ev_rev[c]})
            if (ev) cudaEventDestroy(ev);
    if (h->ev_gfork) cudaEventDestroy(h->ev_gfork);
    if (h->ev_gjoin) cudaEventDestroy(h->ev_gjoin);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    delete h;
}

const char *lbm_error_string(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "not enough device memory";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_EDIVERGED: return "lattice diverged (non-finite or |u| > 0.3)";
        case LBM_ENOTCONV: return "u_tau Newton solve did not converge";
        case LBM_ESTATE: return "call out of order";
        case LBM_ENOSCRATCH: return "size exceeds the fixed scratch of a no-allocation call";
        case LBM_ETIMEOUT: return "a device-side wait timed out";
        default: return "unknown error";
    }
}

}  // extern "C"

/*
 * lbm.h -- C ABI of liblbm_gb300.so, a GB300 (sm_103a) implementation of the
 * per-time-step hot path of the STG wall-modelled LES lattice Boltzmann channel
 * method of Xue, Yao & Davidson, "Synthetic turbulence generator for the
 * wall-modeled LES lattice Boltzmann method" (arXiv 2304.04214):
 *
 *   D3Q19 multiple-relaxation-time collide-and-stream (Sec. 2.1, App. A.1),
 *   Smagorinsky eddy viscosity folded into the viscous rates (Sec. 2.2),
 *   force-based Reichardt wall model on the first off-wall cells (Sec. 2.3),
 *   synthetic-turbulence inlet plane with regularized reconstruction (Sec. 3.1),
 *   in the order of Algorithm 1.
 *
 * Geometry.  Lattice nx x ny x nz, x streamwise (inlet at x = 0, zero-gradient
 * outlet at x = nx-1), y wall-normal (specular slip walls half a cell below
 * j = 0 and above j = ny-1, so the first cell centre sits at y = 1/2), z
 * spanwise and periodic.  delta = ny/2.  Requirements: ny even and >= 4,
 * nx >= 3, nz >= 1.
 *
 * Layout.  Populations are structure-of-arrays f[q][k][j][i], i fastest, with
 * the velocity order of Sec. 2.1 (eq:vel-set): q = 9 is the rest velocity and
 * q and 18 - q are opposite.  The lattice state between steps is the
 * post-collision population set (pull streaming happens at the start of the
 * next step).  Host arrays passed to the calls below use the same layout in
 * FP64; device storage is FP32 (f), or FP16 / BF16 deviations f - w_q.
 *
 * Conventions.  Every call returns 0 (LBM_OK) or a negative LBM_E* code and
 * never throws.  All work is enqueued on the handle's CUDA stream; calls that
 * return host data synchronize that stream first.  Host pointers are owned
 * by the caller.  Device memory is either bound by the caller
 * (lbm_bind_memory with a pointer) or allocated by the library (pointer NULL).
 * A handle belongs to one CUDA device, the device of its memory: while a call
 * runs, that device is current (the caller's current device is put back
 * before the call returns), so a handle may be used from any current device;
 * its stream (lbm_opts.cuda_stream, lbm_set_stream) must belong to that
 * device.
 *
 * Errors common to the calls (each declaration lists only its own):
 * LBM_EINVAL for a NULL handle or a NULL pointer argument; LBM_ESTATE for a
 * call that needs device memory before lbm_bind_memory; LBM_ECUDA when a CUDA
 * runtime call fails (its message is printed to stderr).  Device-side
 * conditions found while steps run (divergence, a Newton solve that did not
 * converge, a wait that gave up) are deferred to lbm_sync.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LBM_OK          0
#define LBM_EINVAL     -1   /* invalid argument (bad grid, NULL pointer, size) */
#define LBM_ENOMEM     -2   /* bound memory too small or allocation failed */
#define LBM_ECUDA      -3   /* a CUDA runtime call failed */
#define LBM_EDIVERGED  -4   /* non-finite or |u| > 0.3 seen on the lattice */
#define LBM_ENOTCONV   -5   /* the u_tau Newton solve did not converge */
#define LBM_ESTATE     -6   /* call out of order (e.g. step before memory) */
#define LBM_ENOSCRATCH -7   /* larger than the fixed scratch of lbm_wall_shear_noalloc */
#define LBM_ETIMEOUT   -8   /* a device-side wait gave up (the step's output is invalid) */

/* ---- storage of the populations ----
 * The 16-bit storages keep a deviation, rounded to nearest, and compute in
 * FP32.  "Row base": the deviation from the equilibrium of the row's mean
 * flow, f_q - f^eq_q(1, (U0(y_j), 0, 0)), U0 the inlet mean profile (a 19 x ny
 * table); values about ten times smaller than f_q - w_q in the core flow, so
 * the rounding noise is that much smaller. */
#define LBM_FP32      0     /* f_q in FP32 */
#define LBM_FP16_DEV  1     /* f_q - w_q in IEEE FP16 */
#define LBM_BF16_DEV  2     /* row base in BF16 */
#define LBM_FP16_ROW  3     /* row base in IEEE FP16 */

typedef struct lbm_handle lbm_handle;

typedef struct {
    int nx, ny, nz;
} lbm_grid;

/* Synthetic turbulence generator (Sec. 3.1, eq:aux_vec).  The modes use
 * k_n = k_min r^(n-1) with k_min = beta_kmin 2 pi / max_y l_e(y) and
 * l_e(y) = ell_e delta tanh(2 d_w / (ell_e delta)); u' = amp * a v' with a the
 * Cholesky factor of the prescribed Reynolds stress (eq:cholesky). */
typedef struct {
    int n_modes;              /* N, >= 0 (0: no fluctuations) */
    double k_ratio;           /* r, default 1.01 */
    double beta_kmin;         /* default 0.5 */
    double ell_e;             /* length-scale factor (theta_0), default 0.4 */
    double amp;               /* amplitude A (theta_1), default 1 */
    const double *uniforms;   /* host, n_modes x 4 values in [0,1): the STG's
                                 random draws (polar angle and azimuth of d_n,
                                 angle of sigma_n about d_n, phase phi_n).
                                 Copied at creation. */
} lbm_stg_params;

typedef struct {
    int precision;            /* LBM_FP32 | LBM_FP16_DEV | LBM_BF16_DEV | LBM_FP16_ROW */
    double u_bulk;            /* bulk velocity U_b (lattice units), default 0.05 */
    double c_smag;            /* C_smag Delta^2 of eq:smogrinsky_model, default 0.01 */
    double kappa;             /* Reichardt kappa (theta_2), default 0.4 */
    double B;                 /* Reichardt B (theta_3), default 7.8 */
    int wall_model;           /* 1: Reichardt wall force (Sec. 2.3); 0: off */
    int inlet;                /* 1: STG inlet + zero-gradient outlet; 0: periodic x */
    int stats_every;          /* accumulate statistics every s steps; 0: off */
    void *cuda_stream;        /* cudaStream_t to enqueue on; NULL: default stream */
} lbm_opts;

/* Fill *opts with the defaults listed above (FP32, stream NULL); NULL is
 * ignored. */
void lbm_default_opts(lbm_opts *opts);

/* Create a channel.  Computes the flow constants in FP64 on the host:
 * delta = ny/2, U_b+ = mean of the Reichardt law over the cell centres,
 * u_tau = U_b / U_b+, nu = u_tau delta / Re_tau, tau0 = 3 nu + 1/2 (eq:nu),
 * and the STG tables (Algorithm 1, steps 1-3).  No device memory is touched:
 * bind memory next.  *out receives the handle (free with lbm_destroy).
 * Errors: LBM_EINVAL for NULL pointers, ny odd or < 4, nx < 3, nz < 1,
 * re_tau <= 0, n_modes < 0, uniforms NULL while n_modes > 0. */
int lbm_create(const lbm_grid *grid, double re_tau, const lbm_stg_params *stg,
               const lbm_opts *opts, lbm_handle **out);

/* Device bytes the handle needs (both lattices, tables, wall and inlet
 * buffers, statistics) into *bytes.  Alignment of the bound pointer: 256
 * bytes.  No device work; works before lbm_bind_memory. */
int lbm_required_bytes(const lbm_handle *h, size_t *bytes);

/* Bind device memory: dev_ptr of at least lbm_required_bytes bytes, owned by
 * the caller (the library never frees it); or dev_ptr NULL to let the library
 * cudaMalloc it on the current device (freed by lbm_destroy).  The device of
 * that memory becomes the handle's device.  Uploads the tables and
 * initializes the lattice to f^eq(1, (U_R(y), 0, 0)) with U_R the inlet mean
 * profile.  Errors: LBM_ENOMEM if bytes is too small, LBM_EINVAL if
 * misaligned or not device memory, LBM_ESTATE if already bound, LBM_ECUDA. */
int lbm_bind_memory(lbm_handle *h, void *dev_ptr, size_t bytes);

/* Enqueue n time steps of Algorithm 1 on the handle's stream and return
 * without synchronizing.  Each step: the inlet velocity of steps 4-5 comes
 * from a ring of STG time levels filled ahead of the steps (on a second
 * stream of the handle); then two kernels read the previous state and write
 * disjoint rows of the next one: the interior kernel (rows 1..ny-2, on the
 * handle's stream) does pull streaming with the boundary rules, the
 * regularized inlet (steps 6-8) and the collision (step 15); the wall-row
 * kernel (rows 0 and ny-1, on a side stream forked from and joined back into
 * the handle's stream) does the same for the first off-wall cells with the
 * wall model (steps 9-14).  (Odd nx, or LBM_KERNEL_CELL: one kernel for all
 * rows.)
 * With CUDA graphs on (the default, lbm_set_graphs), whole periods of the STG
 * ring (64 steps where the inlet plane allows) that fit in n are launched as
 * one graph each, built the first time a period's launch state occurs; the
 * steps and their results are the same as with separate launches.
 * Errors: LBM_ESTATE before lbm_bind_memory, LBM_EINVAL if n < 0, LBM_ECUDA. */
int lbm_step(lbm_handle *h, int n);

/* Launch ring periods of steps as CUDA graphs (on != 0, the default) or every
 * kernel separately (on = 0).  Errors: LBM_EINVAL. */
int lbm_set_graphs(lbm_handle *h, int on);

/* Failure-detection check: enqueue one block that waits, with the bounded
 * wait of the staged kernel's copy ring (here 2^14 polls), on a barrier that
 * nothing completes; it gives up and raises the device timeout flag, so the
 * next lbm_sync returns LBM_ETIMEOUT (and clears the flag).  Nothing else is
 * touched.  Errors: LBM_EINVAL, LBM_ESTATE before lbm_bind_memory,
 * LBM_ECUDA. */
int lbm_probe_wait_timeout(lbm_handle *h);

/* Whether graphs are on (*on; 0 also after a capture the runtime refused),
 * and how many graph launches lbm_step has made (*launched; each also
 * launches one single-thread kernel that sets the period's start time, which
 * the launch counts of lbm_profile_read include).  Errors: LBM_EINVAL. */
int lbm_graph_info(const lbm_handle *h, int *on, long *launched);

/* Synchronize the stream and report deferred device errors:
 * LBM_EDIVERGED, LBM_ENOTCONV, LBM_ETIMEOUT (the counters are cleared when
 * read). */
int lbm_sync(lbm_handle *h);

/* Checkpoint / resume (the paper has none; this is for long statistics runs).
 * lbm_save writes the channel's state to the file at path: a header (grid,
 * storage, creation options, a hash of the STG draws, time, parameters,
 * statistics sample counters), then the stored populations as raw FP32 or
 * 16-bit words, u_tau, the FP64 statistics accumulators and, if one was set,
 * the inlet profile, with a 64-bit FNV-1a checksum over that payload.  It
 * synchronizes the stream.  lbm_load restores a handle created with the same
 * grid, storage, Re_tau, options and STG draws: the next steps are
 * bit-identical to those of the run that saved.  It reads and checks the
 * whole file before it changes the handle, then waits for all work the handle
 * has enqueued (on any of its streams) before it replaces the state, so it
 * may follow lbm_step without a synchronization.  Errors: LBM_ESTATE before
 * lbm_bind_memory; LBM_EINVAL for a file that cannot be opened, read or
 * written, a foreign or corrupted file (magic, version, sizes, checksum), or
 * one saved by a channel created differently; LBM_ECUDA. */
int lbm_save(lbm_handle *h, const char *path);
int lbm_load(lbm_handle *h, const char *path);

/* Set the CUDA stream later calls enqueue on (cudaStream_t; NULL = default).
 * Work already enqueued stays on the previous stream; the caller orders the
 * two.  Errors: LBM_EINVAL for a NULL handle. */
int lbm_set_stream(lbm_handle *h, void *cuda_stream);

/* ---- step kernel variants (all compute the same step of Algorithm 1) ---- */
#define LBM_KERNEL_AUTO    0  /* QUAD for the 16-bit storages and PAIR for FP32 where the
                                 grid allows, else PAIR (nx even), else CELL */
#define LBM_KERNEL_CELL    1  /* one cell per thread, direct loads */
#define LBM_KERNEL_PAIR    2  /* two x-adjacent cells per thread, packed FP32x2; nx even */
#define LBM_KERNEL_STAGED  3  /* PAIR arithmetic with the pulled populations copied into
                                 shared memory by the tensor memory accelerator (a
                                 persistent grid, 128 x 2-cell tiles, multi-stage ring);
                                 nx a multiple of 4 (FP32) or 8 (16-bit storage) */
#define LBM_KERNEL_QUAD    4  /* four x-adjacent cells per thread, the x halo by warp
                                 shuffle, PAIR arithmetic; nx a multiple of 4 */

/* Choose the kernel of later steps (also the forward and recomputed steps of
 * lbm_adjoint_step).  PAIR, QUAD and STAGED run the same arithmetic and give
 * bit-identical states; CELL evaluates the same collision one cell at a time
 * (the same formulas, a different FP32 operation order).  Errors: LBM_EINVAL
 * for an unknown kind or a grid the kind does not support. */
int lbm_set_step_kernel(lbm_handle *h, int kind);

/* The kernel later steps will run (AUTO resolved) into *kind.  Errors:
 * LBM_EINVAL for NULL pointers. */
int lbm_get_step_kernel(const lbm_handle *h, int *kind);

/* Outlet sponge zone (Sec. 4.1 places one before the outlet; its form is not
 * given, reading A24): over the last `cells` cells the kinematic viscosity
 * rises by nu_max r^2, r in [0, 1] the position of the cell centre in the
 * zone, so tau0 of those cells is tau0 + 3 nu_max r^2 (the Smagorinsky part
 * is added on top as everywhere).  Damps what the outlet would reflect.
 * cells = 0 or nu_max = 0: none (the default).  Applies to later steps and
 * to the forward and adjoint steps of lbm_adjoint_step; saved in checkpoint
 * files.  Errors: LBM_EINVAL for cells outside [0, nx] or nu_max negative or
 * not finite. */
int lbm_set_sponge(lbm_handle *h, int cells, double nu_max);

/* ---- x-slab domain decomposition (one handle per rank; no counterpart in
 * the paper, whose Algorithm 1 runs the cell loop over one domain) ----
 *
 * A channel of nx_global cells along x is cut into slabs of consecutive x
 * columns, one handle each.  A handle is created with its local lattice:
 * its owned columns plus ghost columns on each side that has a neighbouring
 * slab (the inlet and outlet stay the global faces: the first slab starts with
 * the inlet column, the last ends with the outlet column).  Before every step,
 * the innermost ghost column on each side must hold the neighbour's
 * post-collision populations that stream into this slab: the five with
 * c_x = +1 on the left, the five with c_x = -1 on the right (every other
 * population of a ghost column is never read by an owned cell).  The kernels
 * step ghost columns like any cell of the lattice ends (left: inlet, right:
 * zero-gradient outlet); their results are not used.  With the halo moved
 * exactly, the owned columns are bit for bit those of the undivided channel.
 *
 * lbm_set_slab: local column c is global column c + x_offset; this handle owns
 * local columns [own_lo, own_hi).  Call before lbm_set_sponge (whose zone is
 * in global columns).  Errors: LBM_EINVAL for a range outside the lattice, or
 * a slab whose lattice ends are not the global faces where it holds them.
 *
 * lbm_halo_bytes: bytes of one face's halo buffer, 5 x ny x nz stored words
 * (FP32: 4 bytes, 16-bit storage: 2 bytes), layout [5][nz][ny].
 *
 * lbm_halo_pack (enqueued): copy the populations this slab sends across
 * `face` (LBM_FACE_LEFT: the c_x = -1 populations of its first owned column;
 * LBM_FACE_RIGHT: the c_x = +1 populations of its last owned column) into the
 * caller's device buffer.  lbm_halo_unpack (enqueued): copy a neighbour's
 * buffer into the ghost column next to the owned range on `face`.  Moving the
 * buffers between ranks (NCCL, a peer copy, host staging) is the caller's.
 * Errors: LBM_EINVAL for a bad face, or a face with no ghost column
 * (unpack) or no neighbour to send to; LBM_ESTATE before lbm_bind_memory. */
#define LBM_FACE_LEFT  0
#define LBM_FACE_RIGHT 1
int lbm_set_slab(lbm_handle *h, int nx_global, int x_offset, int own_lo, int own_hi);
int lbm_halo_bytes(const lbm_handle *h, size_t *bytes);
int lbm_halo_pack(lbm_handle *h, int face, void *dev_buf);
int lbm_halo_unpack(lbm_handle *h, int face, const void *dev_buf);

/* Statistics accumulated every stats_every steps since the last reset:
 * sums[(j*nx + i)*7 + c], c = (u, v, w, uu, vv, ww, uv), each summed over z
 * and samples in FP64; utau_sums[w*nx + i] (w = 0 bottom, 1 top) summed over z
 * and samples; *n_samples the number of samples.  Host buffers of nx*ny*7 and
 * 2*nx doubles.  Synchronizes.  lbm_reset_stats zeroes the accumulators and
 * the sample count (enqueued, no synchronization).  Errors: the common ones. */
int lbm_stats(lbm_handle *h, double *sums, double *utau_sums, long *n_samples);
int lbm_reset_stats(lbm_handle *h);

/* Macroscopic fields of the last collision, eq:density and eq:momentum:
 * rho[c] and u[3*c + a] for cell c = (k*ny + j)*nx + i, host FP64.
 * rho u = sum_q f*_q c_q - F/2 with F the wall force of that collision.
 * Synchronizes.  Errors: the common ones. */
int lbm_get_fields(lbm_handle *h, double *rho, double *u);

/* Copy the post-collision populations out / in (host FP64, 19*ncell, layout
 * f[q][k][j][i]).  set rounds to the storage type (FP16/BF16 deviations are
 * rounded to nearest after subtracting w_q in FP64); both synchronize.
 * Errors: the common ones. */
int lbm_get_populations(lbm_handle *h, double *f);
int lbm_set_populations(lbm_handle *h, const double *f);

/* Friction velocity of every wall cell from the last step, host FP64,
 * utau[(w*nz + k)*nx + i] (w = 0 bottom, 1 top).  Synchronizes.  Errors: the
 * common ones. */
int lbm_get_utau(lbm_handle *h, double *utau);

/* Time counter t (the STG time of the next step, eq:aux_vec); set moves it
 * (the STG ring is refilled from the new time).  Errors: LBM_EINVAL for
 * t < 0. */
int lbm_get_time(const lbm_handle *h, long *t);
int lbm_set_time(lbm_handle *h, long t);

/* Flow constants: out[0..5] = delta, u_tau,ref, nu, tau0, U_b+, max l_e
 * (host values of lbm_create; works before lbm_bind_memory). */
int lbm_get_constants(const lbm_handle *h, double out[6]);

/* STG inlet velocity u_in(j, k, t) = (U_R(j), 0, 0) + amp a(j) v'(j, k, t)
 * (eq:u_couple, eq:v_fluc, eq:aux_vec) computed by the device kernel for time
 * t; host FP64 out[(k*ny + j)*3 + a].  Synchronizes.  Errors: LBM_EINVAL
 * for t < 0. */
int lbm_inlet_velocity(lbm_handle *h, long t, double *out);

/* Inlet mean profile and Reynolds stress, the RANS input of Algorithm 1
 * steps 1-3 (eq:u_couple, eq:cholesky).  U[j]: streamwise mean velocity of
 * row j; R[6*j + c] = (R11, R22, R33, R12, R13, R23) of row j, lattice units.
 * set copies the host buffers, recomputes amp * chol(R) in FP64 on the host
 * and uploads the result into the device profile buffer not in use, on a
 * copy stream of the handle, so that the upload overlaps the steps in flight;
 * the handle's stream waits for it before the next step (no host
 * synchronization, except when the staging buffer of two calls ago is still
 * being copied).  It returns LBM_EINVAL if some R(j) is not positive
 * definite.  The defaults are the Reichardt profile and the analytic stress
 * of lbm_create. */
int lbm_set_inlet_profile(lbm_handle *h, const double *U, const double *R);
int lbm_get_inlet_profile(const lbm_handle *h, double *U, double *R);

/* Wall shear stress tau_w = rho u_tau^2 (Sec. 2.3) of the last step,
 * averaged over z: host out[w*nx + i], w = 0 bottom, 1 top.  Synchronizes.
 * Errors: the common ones. */
int lbm_wall_shear(lbm_handle *h, double *out);

/* The same reduction enqueued without synchronizing: out (2*nx doubles,
 * owned by the caller) holds the result once the handle's stream has passed
 * this point (after lbm_sync, a stream synchronize, or an event recorded after
 * this call).  Page-locked host memory the device can address (cudaHostAlloc,
 * a registered range) is written by the reduction kernel itself; any other
 * memory gets a copy from device scratch on the stream (synchronous for
 * pageable memory).
 * Successive calls are stream-ordered, so two output buffers used in turn let
 * a coupling loop read step n while step n + 1 runs.  Errors: LBM_EINVAL,
 * LBM_ESTATE before lbm_bind_memory, LBM_ECUDA. */
int lbm_wall_shear_async(lbm_handle *h, double *out);

/* Wall shear for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this is a property of the library, not of the method.)
 *
 * Same result and arguments as lbm_wall_shear, but the device staging buffer
 * the reduction writes before the copy to `out` is a fixed array compiled into
 * the library (file-scope static __device__ memory of LBM_NOALLOC_MAX_NX * 2
 * doubles = 512 KiB) rather than part of the handle's memory, and the call
 * allocates nothing at all: no cudaMalloc, no cudaFree, no library routine
 * that allocates.  It is meant for code that must not allocate at that point,
 * e.g. a coupling loop inside a host application whose memory manager owns
 * every device allocation, or a real-time loop where an allocation could
 * synchronize the device or fail under memory pressure.  Every GPU that loads
 * the library holds the 512 KiB until the process exits.
 *
 * The first call for a handle on a given device looks the array's address on
 * that device up (cudaGetSymbolAddress, with the handle's device current);
 * make that first call before any stream capture.  All calls share the one array and it keeps the
 * last call's contents; each call overwrites the 2*nx entries it uses before
 * reading them, and copies them to `out` before it returns.  Two calls whose
 * GPU work overlaps (different streams with no ordering between them) race on
 * the array.  Errors: LBM_ENOSCRATCH if 2*nx > 2*LBM_NOALLOC_MAX_NX,
 * LBM_EINVAL, LBM_ESTATE, LBM_ECUDA as for lbm_wall_shear. */
#define LBM_NOALLOC_MAX_NX 32768
int lbm_wall_shear_noalloc(lbm_handle *h, double *out);

/* Debugging aid: guard bands (a stand-in for a memory checker, which is not
 * available everywhere).  lbm_debug_guard_bands, before lbm_bind_memory, puts
 * a band of at least `bytes` bytes before the first buffer of the device
 * arena and right after the end of every buffer (and likewise in the adjoint
 * workspace), filled with the byte 0xA5; lbm_required_bytes and
 * lbm_adjoint_required_bytes count them.  bytes = 0 (the default): none.
 * lbm_debug_check_guards waits for all work of the handle and sets *changed
 * to the number of band bytes that no longer hold the pattern: a write past
 * the end (or before the start) of a buffer shows there.  Errors:
 * LBM_EINVAL for bytes < 0; LBM_ESTATE for guard bands after
 * lbm_bind_memory or a check before it. */
int lbm_debug_guard_bands(lbm_handle *h, int bytes);
int lbm_debug_check_guards(lbm_handle *h, long long *changed);

/* Instrumentation.  While enabled (on > 0), every on-th separately launched
 * step (interior and wall-row kernels, from the first one after the call) is
 * bracketed by CUDA events on the handle's stream: on = 1 times every step,
 * a larger on samples them (each event pair costs the stream a few
 * microseconds); a graph of a ring period (lbm_step) is bracketed as a whole
 * and counts for its steps (their kernels, the statistics reductions and the
 * ring refill).  on = 0 disables; on < 0 is LBM_EINVAL.  read synchronizes
 * and returns the summed time in ms and the number of timed steps since the
 * last read, and the number of kernels of any kind the handle launched. */
int lbm_profile_enable(lbm_handle *h, int on);
int lbm_profile_read(lbm_handle *h, double *ms_total, long *step_launches, long *all_launches);

/* ---- Adjoint (gradients of a downstream objective) ----
 *
 * Objective over a window of T steps starting at the current state s_0
 * (FP32 storage only):  J = J_tau + J_R with
 *   J_tau = mean over the T steps and over the wall cells of both walls with
 *           i_tau0 <= i < i_tau1 of tau_w / u_tau,ref^2 (tau_w = rho u_tau^2,
 *           Sec. 2.3, eq:force_wm);
 *   J_R   = sum_j ( <u'v'>(i_R, j) / u_tau,ref^2 - R12+(j) )^2, <.> the mean over
 *           z and the T steps, <u'v'> = <uv> - <u><v>, R12+ the prescribed
 *           inlet shear stress (Sec. 3.1, eq:cholesky input).
 * u is the physical velocity of each collision (eq:momentum).  theta =
 * (ell_e, amp, kappa, B): the STG length-scale factor and amplitude and the
 * Reichardt constants (eq:reichard) of the wall model and the inlet mean. */
typedef struct {
    int i_tau0, i_tau1;   /* wall cells with i_tau0 <= i < i_tau1 enter J_tau */
    int i_R;              /* x station of the Reynolds-stress mismatch */
} lbm_objective;

/* Device bytes of the adjoint workspace for a window of `window` steps with a
 * checkpoint every `ckpt_every` steps (window a multiple of ckpt_every):
 * window/ckpt_every checkpoint lattices, three sets of ckpt_every - 1 segment
 * lattices (the forward pass fills them for the last three segments; the
 * next segment is recomputed beside the reverse steps of the current one),
 * two adjoint lattices, u_tau of every step, the STG field and
 * the inlet adjoint of every step.  No device work.  Errors: LBM_EINVAL for
 * window < 1, ckpt_every < 1 or window not a multiple of ckpt_every. */
int lbm_adjoint_required_bytes(const lbm_handle *h, int window, int ckpt_every, size_t *bytes);

/* Bind the adjoint workspace (caller-owned, 256-byte aligned, at least
 * lbm_adjoint_required_bytes), or dev_ptr NULL to let the library cudaMalloc it.
 * Errors: LBM_EINVAL (bad window, storage not FP32), LBM_ENOMEM, LBM_ESTATE. */
int lbm_adjoint_bind(lbm_handle *h, int window, int ckpt_every, void *dev_ptr, size_t bytes);

/* Advance the state `window` steps (exactly as lbm_step would), evaluate J over
 * them and its gradient by the hand-written adjoint of the fused step: store
 * s_0 and every ckpt_every-th state (and all states of the last three
 * segments, in the three sets of segment lattices), then for each segment in
 * reverse recompute its states from the checkpoint (except the last three) and
 * run the adjoint steps backwards (for even nx, a segment's recomputation
 * runs on a stream of the handle beside the reverse steps of the segment
 * after it).  *J and dJ_dtheta[4] are host FP64.  dJ/ds_0 is kept for
 * lbm_adjoint_state_gradient.  Synchronizes.  Errors: LBM_EINVAL for a
 * window or objective range the workspace or the grid does not fit, the
 * common ones otherwise (binds a workspace first if none is bound). */
int lbm_adjoint_step(lbm_handle *h, int window, int ckpt_every, const lbm_objective *obj, double *J,
                     double dJ_dtheta[4]);

/* dJ/ds_0 of the last lbm_adjoint_step, host FP64 [19][ncell].
 * Errors: LBM_ESTATE before a completed lbm_adjoint_step. */
int lbm_adjoint_state_gradient(lbm_handle *h, double *lambda0);

/* One vector-Jacobian product of the time step at the current state (which
 * is left unchanged): given lambda_next = a row vector on s_{t+1} (host FP64
 * [19][ncell]) return lambda_prev = lambda_next ds_{t+1}/ds_t and
 * dtheta = lambda_next ds_{t+1}/dtheta.  Needs an adjoint workspace
 * (lbm_adjoint_bind).  Errors: the common ones (LBM_ESTATE without one). */
int lbm_vjp_step(lbm_handle *h, const double *lambda_next, double *lambda_prev, double dtheta[4]);

/* Replace the model parameters theta = (ell_e, amp, kappa, B) and rebuild
 * the tables that depend on them (the flow constants of lbm_create stay);
 * synchronizes after the upload.  Errors: LBM_EINVAL for ell_e <= 0 or
 * kappa <= 0. */
int lbm_set_params(lbm_handle *h, const double theta[4]);

/* Free the handle, after the work it enqueued has finished; device memory is
 * freed only if the library allocated it.  NULL is ignored. */
void lbm_destroy(lbm_handle *h);

/* Static string for an error code (a generic text for unknown codes). */
const char *lbm_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */

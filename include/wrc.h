/*
 * wrc.h -- C ABI of the GB300 library for the Deslauriers-Dubuc (DD)
 * wavelet-collocation solver of filtered 2-D incompressible flow with a
 * Krylov-projected time step (Walsh & Alam, "Fujiwhara interaction of
 * tropical cyclone scale vortices using a weighted residual collocation
 * method", arXiv:1604.08159).
 *
 * Problem (Sec. 2.2-2.5 in their barotropic, incompressible reading): the
 * vorticity omega on the doubly periodic square [-pi, pi)^2 obeys
 *     d omega/dt + U . grad omega = nu_eff lap omega + g_SGS - r omega,
 *     lap psi = -(omega - mean omega),  U = dpsi/dy,  V = -dpsi/dx,
 * with nu = 1/Re, the Smagorinsky model of Eq. 5 (constant |S| "a priori",
 * or pointwise |S| as a vorticity forcing g_SGS), and Rayleigh friction r.
 * omega is held on an adaptive grid: the finest lattice is NJ x NJ with
 * NJ = n0 * 2^J, h_J = 2 pi / NJ; the grid is the epsilon-thresholded set of
 * DD wavelet coefficients of order 2p (Eq. 6; wrc_config.p) plus its
 * adjacent zone and closure.  One
 * time step is the exponential-Euler step
 *     omega^{n+1} = omega^n + dt phi_1(dt A_n) (A_n omega^n + g_n)
 * with A_n the frozen linear operator (Sec. 2.1: projection of the discrete
 * system onto a Krylov subspace), followed by grid adaptation.
 *
 * Conventions common to every call:
 *  - Lattice arrays are NJ*NJ, row-major, index p = k*NJ + i with
 *    x_i = -pi + i h_J, y_k = -pi + k h_J.
 *  - "Active" vectors are ordered by increasing lattice index p.
 *  - A pointer argument with device_ptr = 0 is a host pointer; with
 *    device_ptr = 1 it is CUDA device memory that the run's stream may read
 *    or write.  The caller owns every buffer it passes; nothing is retained
 *    after the call returns.
 *  - Every call returns a wrc_status; nothing is thrown across the ABI.
 *    wrc_last_error() gives a message for the last failing call on a run.
 *  - Calls on one run are not thread-safe; distinct runs are independent.
 *  - wrc_step is asynchronous on the run's stream; every query
 *    synchronises that stream before it returns.
 */
#ifndef WRC_H
#define WRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wrc_run wrc_run;

typedef enum {
    WRC_OK = 0,
    WRC_ERR_ARG = -1,            /* invalid argument or configuration */
    WRC_ERR_OOM = -2,            /* a device allocation failed */
    WRC_ERR_CUDA = -3,           /* a CUDA call or kernel launch failed */
    WRC_ERR_BREAKDOWN_NAN = -4,  /* a non-finite value appeared in the Arnoldi process */
    WRC_ERR_TIMEOUT = -5,        /* a bounded wait ran out */
    WRC_ERR_BUSY = -6,           /* the server has no free slot or memory */
    WRC_ERR_STATE = -7           /* call out of order (e.g. step before init) */
} wrc_status;

typedef enum { WRC_FP64 = 0, WRC_MIXED = 1 } wrc_precision;
/* Time integration (Sec. 1 and 2.1, the Krylov projection of the step):
 *  WRC_SCHEME_FROZEN      exponential Euler with the linearisation frozen at
 *                         t^n, omega^{n+1} = omega^n + dt phi_1(dt A_n)(A_n omega^n + g_n)
 *                         (first order in time; one persistent kernel per step)
 *  WRC_SCHEME_ROSENBROCK  exponential Rosenbrock-Euler with the Jacobian of the
 *                         advection, omega^{n+1} = omega^n + dt phi_1(dt J_n) F(omega^n),
 *                         J_n q = A_n q - U[q] . grad omega^n with U[q] the
 *                         velocity of q's own streamfunction (a reconstruction
 *                         and a Poisson solve per Krylov vector; second order in
 *                         time without subgrid forcing, which is held at t^n);
 *                         the Arnoldi process runs as host-driven launches.
 *                         wrc_step only (an ensemble or the server refuses it). */
typedef enum { WRC_SCHEME_FROZEN = 0, WRC_SCHEME_ROSENBROCK = 1 } wrc_scheme;
typedef enum { WRC_SGS_OFF = 0, WRC_SGS_APRIORI = 1, WRC_SGS_DYNAMIC = 2 } wrc_sgs;
/* The equations a run solves:
 *  WRC_MODEL_VORTICITY  the barotropic vorticity-streamfunction form above
 *  WRC_MODEL_EXNER      the compressible velocity-Exner form of Eqs. 1-2
 *                       (see "Compressible velocity-Exner form" below) */
typedef enum { WRC_MODEL_VORTICITY = 0, WRC_MODEL_EXNER = 1 } wrc_model;
typedef enum { WRC_FIELD_OMEGA = 0, WRC_FIELD_PSI = 1, WRC_FIELD_U = 2,
               WRC_FIELD_V = 3, WRC_FIELD_NUT = 4 } wrc_field;

#define WRC_MAX_M 31       /* largest Krylov dimension */
#define WRC_MAX_NJ 4096    /* largest finest lattice (NJ*NJ < 2^24) */
#define WRC_MAX_VORTICES 64

/* Run parameters.
 *  n0        coarsest points per direction: a power of two, >= 4
 *  J         refinement levels, >= 1, with n0 * 2^J <= WRC_MAX_NJ
 *  krylov_m  Krylov dimension m, 1..WRC_MAX_M
 *  sgs       wrc_sgs; prec: wrc_precision
 *  p         half the DD order 2p (Sec. 2.4, 2.6.2): 2 (2p = 4, also for 0),
 *            3 or 4; the predictor interpolates 2p coarser neighbours, the
 *            first derivative is the DD interpolant's (Sec. 2.5), the second
 *            the central stencil of order 2p
 *  eps       threshold on |d| (absolute), >= 0 (Eq. 6)
 *  re        Reynolds number; nu = 1/re
 *  cs        Smagorinsky constant C_s (Eq. 5), filter width Delta = h_J
 *  s_apriori the constant |S| used when sgs == WRC_SGS_APRIORI
 *  rayleigh_r linear damping coefficient r (Sec. 2.3), >= 0
 *  dt        time step, > 0
 *  scheme    wrc_scheme (0: frozen linearisation)
 *  model     wrc_model (0: vorticity form)
 *  cpt, coriolis, gx, gy   (WRC_MODEL_EXNER only, else ignored) C = c_p theta_0
 *            of Eq. 2 (>= 0), the Coriolis parameter f of the f-plane and the
 *            mean geostrophic wind (G_x, G_y); finite                   */
typedef struct {
    int32_t n0, J, krylov_m, sgs, prec, p;
    double eps, re, cs, s_apriori, rayleigh_r, dt;
    int32_t scheme, model;      /* wrc_scheme, wrc_model */
    double cpt, coriolis, gx, gy;
} wrc_config;

/* Create a run on the current CUDA device, bound to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Allocates the run's
 * device state.  Errors: WRC_ERR_ARG for an invalid config or out == NULL,
 * WRC_ERR_OOM, WRC_ERR_CUDA.  On error *out is NULL. */
wrc_status wrc_create(const wrc_config* cfg, void* cuda_stream, wrc_run** out);

/* Initial condition (Sec. 3.1): the sum of n Gaussian vortices
 * omega = gamma/(pi s^2) exp(-r^2/s^2), r the minimum-image distance to
 * (xc, yc), sampled on the full lattice; then the full-lattice forward
 * transform, thresholding and adaptation (Eq. 6).  Host arrays of length n,
 * 1 <= n <= WRC_MAX_VORTICES, s > 0. */
wrc_status wrc_init_vortices(wrc_run* run, int32_t n, const double* xc, const double* yc,
                             const double* gamma, const double* s);

/* Initial condition from a sampled lattice field omega_lattice (NJ*NJ),
 * then transform, thresholding and adaptation as above. */
wrc_status wrc_init_field(wrc_run* run, const double* omega_lattice, int32_t device_ptr);

/* Set the adaptive grid directly: `active` (NJ*NJ bytes, 0/1) and the values
 * omega_lattice (NJ*NJ, read at active points only).  The grid must contain
 * every level-0 point and be closed under DD prediction (every active point's
 * predictor points active); otherwise WRC_ERR_ARG.  No thresholding is done;
 * stencil levels and ghost points are rebuilt. */
wrc_status wrc_set_grid(wrc_run* run, const uint8_t* active, const double* omega_lattice,
                        int32_t device_ptr);

/* Rebuild the grid from the current omega with threshold eps (which becomes
 * the run's eps): details on the grid, significance, adjacent zone, closure,
 * values at new points from the reconstruction (Eq. 6). */
wrc_status wrc_threshold(wrc_run* run, double eps);

/* Advance nsteps time steps (each: reconstruction, streamfunction, velocity
 * and SGS forcing, Krylov projection, phi_1 update, adaptation).  Returns
 * after the launches are queued; one host synchronisation per step reads the
 * new grid's sizes. */
wrc_status wrc_step(wrc_run* run, int32_t nsteps);

/* Wait for the run's stream: without a limit for timeout_ms < 0, else for at
 * most timeout_ms milliseconds (0 polls once).  WRC_ERR_TIMEOUT if the
 * queued work has not finished by then; it stays queued and a later call can
 * wait for it again.  Returns WRC_ERR_BREAKDOWN_NAN if a step met a
 * non-finite Arnoldi coefficient since the last call. */
wrc_status wrc_sync(wrc_run* run, int32_t timeout_ms);

/* Bound of every device-side wait of the run's kernels (the grid barriers of
 * the cooperative Krylov kernel; in the grid rebuild, a ghost's wait for the
 * interpolation rows of its coarser ghost predictors), in seconds,
 * 0 < seconds <= 60; default 2 s.  A wait that runs out sets an error word
 * and the kernel returns; the step (for a rebuild's wait: the next step)
 * then fails with WRC_ERR_TIMEOUT and the run's state is undefined until a
 * new initial condition (wrc_init_*, wrc_set_grid) or wrc_destroy.
 * WRC_ERR_ARG outside the range. */
wrc_status wrc_set_wait_limit(wrc_run* run, double seconds);

/* Thread-block cluster size (1, 2 or 4) of the run's next Krylov launch on
 * its current grid.  Clusters of 2 or 4 blocks pre-add their dot sums in
 * distributed shared memory; they are used when the device can hold the
 * launch with them, the environment variable WRC_KRYLOV_CLUSTER (1 or 2,
 * read at wrc_create) does not cap them, and the launch path forms them: a
 * probe launch at the device's first wrc_create and the check of the
 * device's first clustered launch switch them off for the device otherwise,
 * e.g. under a profiler that replays cooperative launches without
 * clusters; a launch whose clusters were not formed runs as the unclustered
 * kernel and computes the same step. */
wrc_status wrc_query_krylov_form(wrc_run* run, int32_t* cluster_size);

/* Sizes of the current grid: active points, ghost points and active points
 * per level (per_level has J+1 entries; any pointer may be NULL). */
wrc_status wrc_query_counts(wrc_run* run, int64_t* n_active, int64_t* n_ghost, int64_t* per_level);

/* The active set: lattice indices (int32) and omega values, ordered by
 * lattice index; at most `cap` entries are written (WRC_ERR_ARG if cap is
 * smaller than the active count).  Either output may be NULL. */
wrc_status wrc_query_active(wrc_run* run, int32_t* idx_out, double* omega_out, int64_t cap,
                            int32_t device_ptr);

/* Masks of the current grid as NJ*NJ bytes (0/1): active points, ghost
 * points, and the significant points of the last thresholding.  Any output
 * may be NULL. */
wrc_status wrc_query_masks(wrc_run* run, uint8_t* active, uint8_t* ghost, uint8_t* significant,
                           int32_t device_ptr);

/* Wavelet details d = u - Pred(u) of the last thresholding (Eq. 6), one per
 * active point of the grid it was computed on (0 at level-0 points), in that
 * grid's order; cap as in wrc_query_active. */
wrc_status wrc_query_details(wrc_run* run, double* d_out, int64_t cap, int32_t device_ptr);

/* Per active point the stencil level j* along x and y (Sec. 2.5: the finest
 * level at which the point has an active neighbour), as bytes. */
wrc_status wrc_query_stencil_levels(wrc_run* run, uint8_t* jx_out, uint8_t* jy_out, int64_t cap,
                                    int32_t device_ptr);

/* Lattice field (NJ*NJ) for the current state: WRC_FIELD_OMEGA the
 * reconstruction R(omega) (Eq. 6), PSI the streamfunction, U and V the
 * velocity, NUT the Smagorinsky eddy viscosity (C_s h_J)^2 |S| (Eq. 5). */
wrc_status wrc_query_field(wrc_run* run, int32_t which, double* out, int32_t device_ptr);

/* Freeze the linearisation at the current state (reconstruction,
 * streamfunction, velocity, SGS forcing), as the first part of a step does. */
wrc_status wrc_freeze(wrc_run* run);

/* w = A_n q at the active points for the frozen linearisation (Sec. 2.5
 * derivatives at each point's stencil level, ghost values by DD prediction):
 * A_n q = -U Dx q - V Dy q + nu_eff (Dxx + Dyy) q - r q.  Optionally also
 * the SGS forcing g_n at the active points (g_out may be NULL).  q and w
 * hold n_active values.  Requires wrc_freeze after the last grid change. */
wrc_status wrc_apply_operator(wrc_run* run, const double* q, double* w, double* g_out,
                              int32_t device_ptr);

/* Krylov data of the last step: beta = |b|, k = dimension used (< m after
 * a happy breakdown), h_last = h_{k+1,k}, H ((m+1) x m row-major, may be
 * NULL) and y = phi_1(dt H_k) e_1 (m entries, may be NULL). */
wrc_status wrc_query_krylov(wrc_run* run, double* beta, int32_t* k, double* h_last, double* H,
                            double* y);

/* Diagnostics of the current state, out[0..8] = energy E = 1/2 int |U|^2,
 * enstrophy Z = 1/2 int omega^2, palinstrophy P = 1/2 int |grad omega|^2,
 * circulation int omega (rectangle rule on the reconstructed lattice
 * fields), time t, step count, active count, ghost count, and the Krylov
 * error estimate of the last step, dt beta h_{k+1,k} |y_k| with
 * y = phi_1(dt H_k) e_1 (the residual-based estimate of the projection's
 * error in the increment; 0 after a breakdown at k = 0 or before any step;
 * the paper gives no estimate -- this is the standard one for Krylov
 * approximations of phi_1). */
wrc_status wrc_diagnostics(wrc_run* run, double out[9]);

/* Counters: out[0] kernel launches made by the library in this process,
 * out[1] steps taken by this run, out[2] host synchronisations made by its
 * steps and grid rebuilds, out[3] current active count. */
wrc_status wrc_query_stats(wrc_run* run, int64_t out[4]);

/* Event timing of the Krylov part of each step (the cooperative Arnoldi
 * kernel, phi_1 and the update): when enabled, each step's Krylov launches
 * are bracketed by CUDA events on the run's stream; enabling or disabling
 * clears the record.  enable = 2 also traces the phases of the cooperative
 * kernel (wrc_query_phase_trace); 0 disables, 1 times only.  enable = 3
 * times the stages of each step instead (wrc_query_stages): an event at each
 * stage boundary, with the step's phases launched directly rather than
 * replayed as CUDA graphs while it is on.  WRC_ERR_ARG for other values.
 * Synchronises. */
wrc_status wrc_profile(wrc_run* run, int32_t enable);

/* Stages of a step timed by wrc_profile(run, 3), in the order a step runs
 * them (the reconstruction twice: R(omega) before the Poisson solve, and the
 * new omega's before thresholding; the adaptation in two parts around the
 * host's read of the new grid's sizes):
 *   RECONSTRUCT  inverse DD4 transform onto the finest lattice (Sec. 2.3)
 *   POISSON      the FFT streamfunction solve (and, in the mixed mode, the
 *                spectral velocity and strain)
 *   VELOCITY     U, V at the active points
 *   SGS          the Smagorinsky forcing (Eq. 5), empty without it
 *   KRYLOV       the cooperative Arnoldi / phi_1 / update launch(es)
 *   ADAPT        details, threshold, adjacent zone, closure, ghosts,
 *                compaction, the new compact arrays and interpolation rows
 *   HOST         from the end of the first adaptation part to the start of
 *                the second: the host's wait for the new sizes and the
 *                launch latency after it (no kernel of the step runs) */
enum {
    WRC_STAGE_RECONSTRUCT = 0,
    WRC_STAGE_POISSON = 1,
    WRC_STAGE_VELOCITY = 2,
    WRC_STAGE_SGS = 3,
    WRC_STAGE_KRYLOV = 4,
    WRC_STAGE_ADAPT = 5,
    WRC_STAGE_HOST = 6,
    WRC_STAGE_COUNT = 7
};

/* Stage record since wrc_profile(run, 3): out[0] the steps timed, out[1 + s]
 * the total device time of stage s over them in ms (CUDA events on the run's
 * stream).  WRC_ERR_ARG if cap < 1 + WRC_STAGE_COUNT; WRC_ERR_STATE when
 * stage timing is off.  Synchronises. */
wrc_status wrc_query_stages(wrc_run* run, double* out, int32_t cap);

/* Phase trace of the last cooperative Krylov launch of the run (profiling
 * mode 2): for each grid barrier p it passed, out[4p..4p+3] = the first and
 * the last arrival of its blocks, the index of the last block to arrive, and
 * the release of block 0, in microseconds from the start of block 0 (device
 * global timer).  Barrier 0 follows b = A_n omega + g, barrier 1 the ghost
 * values of v_0, barriers 2 and 3 the first projection of A v_0; then each
 * further Arnoldi step has two: after its one reduction (the second pass of
 * the previous vector and the first of the new one) and after the new
 * vectors (the last step stops after its reduction); the final barrier
 * follows phi_1, before the update.
 * *nphases receives the count.  WRC_ERR_ARG if cap < 4 * count; WRC_ERR_STATE without a traced
 * launch.  Synchronises. */
wrc_status wrc_query_phase_trace(wrc_run* run, double* out, int32_t cap, int32_t* nphases);

/* Profile record since wrc_profile(run, 1): out[0] Krylov launches timed,
 * out[1] their total device time in ms, out[2] their algorithmic bytes (per
 * active point: 4 words per operator application, 2(j+1)+3 words at Arnoldi
 * step j, k+2 words for the combination), out[3] their algorithmic FP64
 * operations (30 per operator application, 8(j+1)+4 at step j, 3k more).
 * Synchronises. */
wrc_status wrc_query_profile(wrc_run* run, double out[4]);

/* Message of the last failing call on `run` ("" if none); for a NULL run,
 * the last failure of wrc_create on this thread. */
const char* wrc_last_error(const wrc_run* run);

/* Release the run's device memory (synchronises its stream first). */
void wrc_destroy(wrc_run* run);

/* ---- Passive scalar ----------------------------------------------------------
 * The vapour mixing ratio r_v of the paper's section on the transport of
 * water vapor: Eq. (vapour) with only a diffusion term on its right-hand
 * side, D r_v / Dt = kappa (Dxx + Dyy) r_v, carried by the run's flow.  Each
 * wrc_step then advances r_v with the same Krylov projection and the same
 * frozen velocity as omega, r_v^{n+1} = r_v^n + dt phi_1(dt A_r) A_r r_v^n with
 * A_r = -U Dx - V Dy + kappa (Dxx + Dyy) (no Rayleigh friction, no subgrid
 * forcing), and the adaptive grid adapts to both fields: the significant
 * sets of omega and r_v (same eps) are joined before the adjacent zone and
 * the closure.  Supported by wrc_step only (a batched ensemble or the server
 * refuses such a run); a new initial condition (wrc_init_*, wrc_set_grid)
 * drops the scalar. */

/* Enable the passive scalar with diffusivity kappa >= 0 and its initial
 * field: NJ*NJ doubles, row-major [k * NJ + i] (host or device memory per
 * device_ptr; not kept).  The run must have an initial condition.  The grid
 * is thresholded once more with omega's details on the current grid and the
 * field's details on every lattice point; r_v at the new grid is the field
 * there.  Synchronises.  WRC_ERR_ARG for a NULL field or kappa < 0;
 * WRC_ERR_STATE without an initial condition; WRC_ERR_OOM, WRC_ERR_CUDA. */
wrc_status wrc_scalar_init(wrc_run* run, double kappa, const double* field, int32_t device_ptr);

/* The active lattice indices and r_v at them, in the order of
 * wrc_query_active (cap >= the active count).  Synchronises.  WRC_ERR_STATE
 * when the scalar is not enabled; WRC_ERR_ARG if cap is too small. */
wrc_status wrc_query_scalar(wrc_run* run, int32_t* idx_out, double* r_out, int64_t cap, int32_t device_ptr);

/* ---- Compressible velocity-Exner form ---------------------------------------
 * A run created with model = WRC_MODEL_EXNER holds the velocity (u, v) and
 * the Exner function pi on the adaptive grid and solves Eqs. 1-2 of the
 * paper on the f-plane (Sec. 2.2), with Rayleigh friction standing for the
 * balance of Eq. 4:
 *     pi_t = -(u pi_x + v pi_y) - pi (u_x + v_y)
 *     u_t  = -(u u_x + v u_y) - C pi_x + f (v - G_y) - r u + nu_eff lap u
 *     v_t  = -(u v_x + v v_y) - C pi_y - f (u - G_x) - r v + nu_eff lap v
 * (Eq. 1 as printed, coefficient one on pi div u; nu_eff = 1/re plus the
 * constant eddy viscosity of the a-priori Smagorinsky model, Eq. 5; the
 * dynamic model is not available here).  Linearised about rest it is an
 * acoustic system with sound speed sqrt(C pi_0): the Krylov projection of the
 * step (Sec. 2.1) takes its stiff part exactly.  One step is
 *     U^{n+1} = U^n + dt phi_1(dt M) F(U^n),  U = [u; v; pi] at the active points,
 * M the exact Jacobian of F (scheme WRC_SCHEME_ROSENBROCK, second order) or
 * the operator with the coefficients u, v, pi frozen at t^n
 * (WRC_SCHEME_FROZEN), unweighted l2 inner product over the stacked vector;
 * no Poisson solve.  The grid adapts to all three fields: the union of their
 * significant sets (same eps), the adjacent zone, the closure.  FP64 only
 * (prec = WRC_FP64), wrc_step only (ensembles and the server refuse the
 * model).  wrc_step, wrc_sync, wrc_query_counts, wrc_query_masks,
 * wrc_query_stencil_levels, wrc_query_krylov, wrc_query_stats, wrc_profile
 * (modes 0, 1 and 3), wrc_set_wait_limit and wrc_destroy apply to such a run;
 * wrc_query_active returns its indices only (omega_out must be NULL); the
 * other calls of the vorticity form return WRC_ERR_STATE. */

/* Initial condition from sampled lattice fields u, v, pi (NJ*NJ doubles
 * each, host or device per device_ptr; not kept): the full-lattice transform
 * of each, their joint thresholding and the adaptation (Eq. 6).  WRC_ERR_ARG
 * for a NULL field; WRC_ERR_STATE for a vorticity-form run. */
wrc_status wrc_exner_init(wrc_run* run, const double* u, const double* v, const double* pi, int32_t device_ptr);

/* Initial condition of n Gaussian vortices (as wrc_init_vortices) in the
 * velocity form: the vorticity sampled on the full lattice, its
 * streamfunction from the library's Poisson solve (the exact inverse of the
 * collocation Laplacian), u = D_y psi, v = -D_x psi by the finest-lattice
 * stencils, pi = pi0 everywhere (pi0 > 0); then as wrc_exner_init. */
wrc_status wrc_exner_init_vortices(wrc_run* run, int32_t n, const double* xc, const double* yc,
                                   const double* gamma, const double* s, double pi0);

/* The active lattice indices and u, v, pi at them, in the order of
 * wrc_query_active (cap >= the active count); any output may be NULL.
 * Synchronises.  WRC_ERR_STATE for a vorticity-form run. */
wrc_status wrc_query_exner(wrc_run* run, int32_t* idx_out, double* u_out, double* v_out, double* pi_out,
                           int64_t cap, int32_t device_ptr);

/* ---- Diagnostics without allocation ------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code running while a stream is captured
 * into a CUDA graph, host frameworks that own all device memory through their
 * own pool, real-time loops that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.
 * Same quantities as wrc_diagnostics out[0..3] (E, Z, P, circulation) for a
 * reconstructed vorticity lattice omega_lattice and its streamfunction
 * psi_lattice (device arrays, NJ*NJ doubles, e.g. from wrc_query_field with
 * device_ptr = 1), written to the device array out[0..3]; asynchronous on
 * cuda_stream.  It allocates nothing: its scratch (one row of 4 partial sums
 * per reduction block, 1216 blocks at most, and a counter: 39 KB) is a fixed
 * array in the library that every GPU using the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address, so make it before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams, or devices' views of one
 * call) race and give wrong sums; serialise them.  NJ must be a power of two,
 * 8 <= NJ <= WRC_MAX_NJ, and cuda_stream must belong to the current device;
 * otherwise WRC_ERR_ARG.  WRC_ERR_CUDA if a launch fails. */
wrc_status wrc_lattice_diagnostics_noalloc(const double* omega_lattice, const double* psi_lattice, int32_t NJ,
                                           double* out, void* cuda_stream);

/* ---- Batched ensemble ------------------------------------------------------
 * Uneven members (different lattices, parameters and initial conditions;
 * one precision for all) advanced together.  Each step runs the members'
 * reconstruction, streamfunction and adaptation phases as captured CUDA
 * graphs spread over eight member streams, and the Krylov part of all members
 * in ONE cooperative launch whose blocks are shared out in proportion to the
 * members' active counts (a member's partial sums, barrier and breakdown
 * decisions are its own).  The path of a member is the single-run path
 * (Sec. 2.1-2.5 as in wrc_step); only the block decomposition of its
 * reductions differs, so a member's result equals its solo run to rounding.
 * There is one host synchronisation per ensemble step. */
typedef struct wrc_ensemble wrc_ensemble;

/* Create n members from cfgs[0..n) (all with the same prec) on the current
 * device; the batched launch runs on cuda_stream (NULL = legacy default
 * stream; member phases always run on the ensemble's own streams).  Errors
 * as wrc_create; wrc_ensemble_last_error(NULL) explains a failed create. */
wrc_status wrc_ensemble_create(int32_t n, const wrc_config* cfgs, void* cuda_stream, wrc_ensemble** out);

/* The run handle of a member, for initial conditions (wrc_init_vortices,
 * wrc_init_field, wrc_set_grid) and every query.  Owned by the ensemble: do
 * not destroy it and do not call wrc_step on it while the ensemble is used. */
wrc_status wrc_ensemble_member(wrc_ensemble* e, int32_t member, wrc_run** run);

/* Advance every member nsteps steps (all members need an initial condition). */
wrc_status wrc_ensemble_step(wrc_ensemble* e, int32_t nsteps);

/* Block shape of the batched Krylov kernel: threads per block (64, 128 or
 * 256) and target active points per thread (1..64). */
wrc_status wrc_ensemble_set_shape(wrc_ensemble* e, int32_t threads_per_block, int32_t points_per_thread);

/* Autotuner: time the batched Krylov launch over steps_per_candidate real
 * steps for each of the 9 shapes {64,128,256} x {1,2,4} (those with at least
 * one co-resident block per member), keep the fastest and
 * cache it for this process per (precision, member-count bucket,
 * active-count bucket); a cached choice is applied without stepping.  The
 * chosen shape is written to out_shape[0..1] (may be NULL). */
wrc_status wrc_ensemble_tune(wrc_ensemble* e, int32_t steps_per_candidate, int32_t out_shape[2]);

/* out[0] members, out[1] total active points, out[2] ensemble steps taken,
 * out[3] blocks of the last batched launch, out[4..5] the block shape. */
wrc_status wrc_ensemble_stats(wrc_ensemble* e, int64_t out[6]);

/* Event timing of the batched Krylov launches: returns in *ms (may be NULL)
 * the device time recorded since the last call and clears it; enable != 0
 * keeps recording. */
wrc_status wrc_ensemble_profile(wrc_ensemble* e, int32_t enable, double* ms);

const char* wrc_ensemble_last_error(const wrc_ensemble* e);

/* Destroy the members and the ensemble (synchronises). */
void wrc_ensemble_destroy(wrc_ensemble* e);

/* ---- Request server (continuous batching) ----------------------------------
 * The paper has no counterpart: a host-side scheduler for many independent
 * runs (Sec. 3 initial conditions of 1..WRC_MAX_VORTICES Gaussian vortices,
 * any lattice and parameters) that arrive over time.  A worker thread owns
 * all GPU work.  Each admitted run keeps its whole adaptive-grid state on the
 * device until its last step; only its final result (diagnostics and active
 * set) is copied to the host, after which its device memory is freed.
 *
 * Admission, in arrival order (a request that does not fit blocks the ones
 * behind it): a request is admitted once it has arrived, fewer than max_slots
 * runs are resident, and the HBM charged to the resident runs plus the
 * request's estimate (wrc_server_estimate) stays within hbm_budget_bytes.  A
 * resident run is charged the larger of its estimate and the bytes it holds.
 * If creating a run still finds the device out of memory, the request goes
 * back to the head of the queue and nothing more is admitted until a resident
 * run finishes.
 *
 * WRC_SERVE_BATCHED (continuous batching): every worker iteration advances
 * every resident run by one step -- the runs of each precision in one batched
 * step as wrc_ensemble_step does (one cooperative Krylov launch for all of
 * them) -- then retires the runs that reached their step count and admits
 * new arrivals, so runs join and leave the batch between steps.  A run's
 * result equals its solo wrc_step result to rounding (only the block
 * decomposition of its reductions differs).  A run whose step fails is
 * retired as failed; the others carry on.
 * WRC_SERVE_FIFO: the plain per-run form for comparison -- one run at a
 * time, in arrival order, stepped with wrc_step.
 *
 * Times are seconds on a monotonic clock since wrc_server_create. */
typedef struct wrc_server wrc_server;

typedef enum { WRC_SERVE_BATCHED = 0, WRC_SERVE_FIFO = 1 } wrc_serve_policy;
typedef enum { WRC_REQ_QUEUED = 0, WRC_REQ_RUNNING = 1, WRC_REQ_DONE = 2, WRC_REQ_FAILED = 3 } wrc_request_state;

typedef struct {
    int32_t policy;               /* wrc_serve_policy */
    int32_t max_slots;            /* resident runs at most, 1..1024 (FIFO: 1) */
    int32_t threads_per_block;    /* batched kernel shape: 64/128/256, or 0 for the */
    int32_t points_per_thread;    /* autotuned shape if one is cached, else 128 x 1 */
    double hbm_budget_bytes;      /* admission budget, > 0 (e.g. 150e9) */
} wrc_server_config;

typedef struct {
    int32_t state;                /* wrc_request_state */
    int32_t status;               /* wrc_status of a failed request, else WRC_OK */
    int64_t steps;                /* steps taken so far */
    int64_t n_active, n_ghost;    /* grid sizes at the end (DONE) */
    double t_arrival;             /* when the request counts as arrived */
    double t_admit;               /* when its run was created (-1 before) */
    double t_done;                /* when its result was ready (-1 before) */
    double diag[4];               /* E, Z, P, circulation at the end (as wrc_diagnostics) */
    double time;                  /* simulated time at the end */
    double updates;               /* active-point updates: sum of the active count over its steps */
    double charged_bytes;         /* HBM charged while resident */
} wrc_request_info;

/* Device bytes charged on admission for a run of configuration cfg: the
 * allocations wrc_create makes for its lattice (exact) plus the compact
 * arrays for an active-count bound N_a,max = min(NJ^2, 8192 + NJ^2/16) and
 * N_a,max/2 ghost points, at the capacity the run grows them to.  Host
 * arithmetic only.  WRC_ERR_ARG for an invalid cfg. */
wrc_status wrc_server_estimate(const wrc_config* cfg, double* bytes);

/* Start a server (and its worker thread) on the current CUDA device.
 * WRC_ERR_ARG for an invalid config; wrc_server_last_error(NULL) explains. */
wrc_status wrc_server_create(const wrc_server_config* cfg, wrc_server** out);

/* Queue a run: configuration, nv vortices (host arrays, as
 * wrc_init_vortices), nsteps >= 0 steps, and its arrival time arrival_s in
 * server seconds (a time in the past, e.g. 0, means now; a later time holds
 * the request until then, which replays a trace without host timing jitter).
 * Writes the request id.  WRC_ERR_ARG for invalid arguments, WRC_ERR_BUSY if
 * the estimate exceeds the whole budget, WRC_ERR_STATE after a fatal server
 * error. */
wrc_status wrc_server_submit(wrc_server* srv, const wrc_config* cfg, int32_t nv, const double* xc, const double* yc,
                             const double* gamma, const double* s, int64_t nsteps, double arrival_s, int64_t* id);

/* State, timing and (once DONE) result of a request.  WRC_ERR_ARG for an
 * unknown or released id. */
wrc_status wrc_server_query(wrc_server* srv, int64_t id, wrc_request_info* out);

/* The final active set of a DONE request (as wrc_query_active, host arrays,
 * either may be NULL; WRC_ERR_ARG if cap < n_active, WRC_ERR_STATE if the
 * request is not DONE). */
wrc_status wrc_server_result_active(wrc_server* srv, int64_t id, int32_t* idx_out, double* omega_out, int64_t cap);

/* Message of a FAILED request, copied into buf (cap bytes, NUL-terminated). */
wrc_status wrc_server_request_error(wrc_server* srv, int64_t id, char* buf, int64_t cap);

/* Wait until request id (or, for id = -1, every request submitted so far) is
 * DONE or FAILED; WRC_ERR_TIMEOUT after timeout_s seconds. */
wrc_status wrc_server_wait(wrc_server* srv, int64_t id, double timeout_s);

/* Forget a finished request and its host result. */
wrc_status wrc_server_release(wrc_server* srv, int64_t id);

/* out[0] submitted, out[1] done, out[2] failed, out[3] queued, out[4]
 * resident now, out[5] most resident at once, out[6] HBM charged now, out[7]
 * most HBM charged at once, out[8] worker iterations that stepped runs,
 * out[9] active-point updates of all steps, out[10] server clock now,
 * out[11] 1 after a fatal server error. */
wrc_status wrc_server_stats(wrc_server* srv, double out[12]);

/* Message of the last server-level failure ("" if none); for NULL, the last
 * failure of wrc_server_create on this thread. */
const char* wrc_server_last_error(const wrc_server* srv);

/* Stop the worker after its current iteration, fail the requests still
 * queued or resident, free every run and the server. */
void wrc_server_destroy(wrc_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* WRC_H */

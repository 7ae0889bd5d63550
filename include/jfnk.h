/*
 * jfnk.h -- C ABI of the GB300 (sm_103a) symmetry-preserving JFNK hot path.
 *
 * The library evaluates, on one GPU, the matrix-free pieces of the implicit
 * solver of Hossain & Alam, "Assessment of a symmetry-preserving JFNK method
 * for atmospheric convection":
 *
 *   F(u)   semi-discrete right-hand side of the dry nonhydrostatic equations
 *          (Section 2.1, Eqs. ch2_28-ch2_30; Eq. ds), discretised with the
 *          Deslauriers-Dubuc collocation derivative (Section 2.3), the
 *          skew-symmetric convective form (Section 2.2) and constant or
 *          Smagorinsky exchange coefficients (Section 2.4, Table 1);
 *   R(u)   trapezoidal residual 2u/dt - F(u) - [2u^n/dt + F(u^n)] (Eq. ns);
 *   J v    finite-difference Jacobian-vector product (Eq. fd);
 *   M^-1 r field-block physics-based preconditioner (Section 2.5.2);
 *   step   one implicit step by inexact Newton + restarted right-preconditioned
 *          GMRES(m) (Section 2.5.1, Eq. jv).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - State vectors are float64, field-major, x fastest:
 *     2D: [field][z][x], fields (u, w, theta, p)
 *     3D: [field][z][y][x], fields (u, v, w, theta, p)
 *   theta is the potential-temperature perturbation, p the c_p-scaled Exner
 *   perturbation.  n = n_fields * nx * ny * nz values (ny = 1 in 2D).
 * - Grid: x (and y) periodic with nodes x_i = -lx/2 + i lx/nx; z cell-centred,
 *   z_k = (k + 1/2) lz/nz, mirror walls at z = 0 and z = lz (w odd; theta, p
 *   even; u, v even for free slip, odd for no slip).
 * - Unless stated otherwise, vector arguments are DEVICE pointers owned by the
 *   caller (e.g. torch tensor data pointers), 8-byte aligned, not aliased with
 *   each other.  The library owns its workspace, allocated once in
 *   jfnk_create; no entry point allocates afterwards.
 * - Every call is enqueued on the handle's CUDA stream.  Calls that fill a
 *   host struct (jfnk_step, jfnk_budgets, jfnk_get_*) synchronise that stream
 *   before returning; the others return without synchronising.
 * - Errors are returned as jfnk_status; nothing is thrown across the ABI.
 *   On JFNK_ERR_INVALID_ARG nothing was enqueued and no state changed.
 *   On JFNK_ERR_CUDA the handle should be destroyed.
 * - A handle is not thread-safe: one host thread at a time, one stream.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JFNK_OK = 0,
    JFNK_ERR_INVALID_ARG = 1,   /* bad size, pointer, option; nothing enqueued   */
    JFNK_ERR_CUDA = 2,          /* a CUDA runtime call failed                     */
    JFNK_ERR_OOM = 3,           /* workspace allocation failed in jfnk_create     */
    JFNK_ERR_NOT_CONVERGED = 4, /* Newton hit max_newton above tolerance          */
    JFNK_ERR_BREAKDOWN = 5,     /* GMRES found no descent (zero Krylov space)     */
    JFNK_ERR_NAN = 6,           /* a residual norm was not finite                 */
    JFNK_ERR_TIMEOUT = 7,       /* a bounded device loop hit its iteration cap    */
    JFNK_ERR_UNSUPPORTED = 8    /* valid request the library does not implement   */
} jfnk_status;

enum { JFNK_FREESLIP = 0, JFNK_NOSLIP = 1 };
enum { JFNK_SGS_CONST = 0, JFNK_SGS_SMAGORINSKY = 1, JFNK_SGS_DEARDORFF = 2 };
enum { JFNK_FP64 = 0, JFNK_MIXED = 1 };
enum { JFNK_PC_NONE = 0, JFNK_PC_BLOCK = 1, JFNK_PC_UNET = 2, JFNK_PC_SCHUR = 3, JFNK_PC_NONLINEAR = 4 };

/* Largest Krylov dimension m accepted by jfnk_create. */
#define JFNK_MAX_KRYLOV 32
/* Length of the per-step history arrays in jfnk_stats. */
#define JFNK_MAX_NEWTON 32

/* Grid (Section 3.1 / 3.2 domains).  dim = 2 or 3; ny = 1 when dim = 2.
 * nx, ny >= 1 and nz >= 2(2p-2) (one mirror reflection must cover the
 * stencil's two-level halo).  Lengths in metres.  bc_* select the parity of
 * the horizontal velocity at the bottom / top wall. */
typedef struct {
    int dim, nx, ny, nz;
    double lx, ly, lz;
    int bc_bottom, bc_top;
} jfnk_grid;

/* Stratification and thermodynamics (Section 2.1).  theta0 [K] background
 * potential temperature; beta = d(theta_bar)/dz [K/m]; pbar the constant base
 * Exner value multiplying div(u) in Eq. ch2_28 (c_p = 1004 by default);
 * gamma_p the coefficient of that term (R/c_v); g [m/s^2]; rho0 [kg/m^3] and
 * cp [J/(kg K)] convert the surface heat flux into a theta source. */
typedef struct {
    double theta0, beta, pbar, g, gamma_p, rho0, cp;
} jfnk_strat;

/* Sub-grid closure (Section 2.4).  mode JFNK_SGS_CONST uses K_M, K_H [m^2/s]
 * (Table 1); JFNK_SGS_SMAGORINSKY uses nu = (Cs Delta)^2 sqrt(2 S:S),
 * Delta = (dx dz)^(1/2) in 2D, (dx dy dz)^(1/3) in 3D, K_M = nu, K_H = nu/Pr.
 * JFNK_SGS_DEARDORFF is the anisotropic closure of Section 2.4 (Eq. KmM):
 * with s = sqrt(2 S:S) and
 * eps = nu S:S, K_m = Cs^(4/3) eps^(1/3) (dx dy)^(2/3) acts along x (and y)
 * and K_M = Cs^(4/3) eps^(1/3) dz^(4/3) along z for momentum; heat takes
 * K_h = (1 + 2l/sqrt(dx dy)) K_m and K_H = (1 + 2l/dz) K_M, with the mixing
 * length l = min(Delta, 0.75 sqrt(e)/N), sqrt(e) = nu/(0.1 Delta) and N the
 * background Brunt-Vaisala frequency (l = Delta where beta <= 0); dy reads as
 * dx in 2-D.  K_M, K_H and Pr are not used by this mode (Pr must still be > 0). */
typedef struct {
    int mode;
    double K_M, K_H, Cs, Pr;
} jfnk_sgs;

/* Solver options.
 * precision   JFNK_FP64: every kernel in float64.
 *             JFNK_MIXED: stencils of the Jacobian-vector product, Krylov basis
 *             and preconditioner in float32; the Newton residual, the FD
 *             difference quotient, Hessenberg/Givens and the update in float64.
 * wavelet_p   order p of the Deslauriers-Dubuc derivative (2 supported).
 * krylov_m    restart length m (1..JFNK_MAX_KRYLOV).
 * flexible    accepted for compatibility; the library always stores the
 *             preconditioned directions (FGMRES form), identical in exact
 *             arithmetic to right-preconditioned GMRES for a linear M.
 * pc_sweeps   Chebyshev steps of the preconditioner, 1..64.
 * precond     JFNK_PC_NONE, JFNK_PC_BLOCK (pc_sweeps Chebyshev steps per block),
 *             JFNK_PC_UNET (the block preconditioner plus a learned
 *             correction, see "Learned right preconditioner" below) or
 *             JFNK_PC_SCHUR (pc_sweeps >= 2: the acoustic Schur
 *             complement of the semi-implicit elimination Section 2.5
 *             follows -- only (2/dt) I and the pressure gradient / divergence
 *             couplings linearised about pbar are kept, the velocities are
 *             eliminated, the pressure Helmholtz operator
 *             H = (2/dt) I - gamma_p pbar theta0 (dt/2) sum_j D_j D_j gets
 *             pc_sweeps Chebyshev steps on its Gershgorin interval, the
 *             velocities are back-substituted, theta gets r_theta / theta_c
 *             of its field block; advection, diffusion and buoyancy are
 *             dropped) or
 *             JFNK_PC_NONLINEAR (the nonlinear preconditioning of Section
 *             2.5.2 with P the field-block operator frozen at the Newton
 *             iterate: Newton on the preconditioned residual M^{-1} W R, i.e.
 *             GMRES on M^{-1} J applied from the left, M^{-1} the same
 *             pc_sweeps-step Chebyshev field-block inverse as JFNK_PC_BLOCK.
 *             The paper's form u - P^{-1}[f - L(u) + P u] equals P^{-1} R for
 *             an exact inverse; M^{-1} R keeps the root of R for the
 *             approximate one.  The Newton test stays on ||W R||; GMRES
 *             stops at ||M^{-1} W(R + J du)|| <= eta ||M^{-1} W R||).
 * newton_rtol, newton_atol_factor, eta, max_newton, max_restarts: stopping rules
 *             ||W R|| <= max(rtol ||W R_0||, atol_factor ||W 2u^n/dt||);
 *             GMRES stops at ||W(R + J du)|| <= eta ||W R||.
 * dt          time step [s].
 * scale_*     field scales U, Theta, P of the diagonal scaling W used for
 *             norms, the FD step and the Krylov inner product. */
typedef struct {
    int precision, wavelet_p, krylov_m, flexible, precond, pc_sweeps;
    double newton_rtol, newton_atol_factor, eta;
    int max_newton, max_restarts;
    double dt, scale_u, scale_theta, scale_p;
} jfnk_opts;

/* Per-step report filled by jfnk_step / jfnk_step_host. */
typedef struct {
    int newton_iters;                        /* Newton corrections taken            */
    int gmres_iters;                         /* Krylov iterations over all Newtons  */
    int restarts;                            /* GMRES restarts over all Newtons     */
    int converged;                           /* 1 if the Newton test was met        */
    double res0, res_final, tol;             /* ||W R|| at start / end, threshold   */
    double res_hist[JFNK_MAX_NEWTON + 1];    /* ||W R|| after each correction       */
    int gmres_per_newton[JFNK_MAX_NEWTON];   /* Krylov iterations per correction    */
    int pc_fallback;                         /* 1: the learned preconditioner failed
                                                and the step was redone with the
                                                field-block one (counts above are
                                                those of the redone step)           */
    int pc_switches;                         /* Newton corrections whose GMRES solve
                                                switched from the learned to the
                                                field-block preconditioner          */
} jfnk_stats;

/* Budgets of Section 3.1.3 (literal E_k, E_p) plus conservation diagnostics. */
typedef struct {
    double E_k, E_p, sum_theta, sum_div;
    double max[5], min[5];
} jfnk_budget;

typedef struct jfnk_handle jfnk_handle;

/* Create a solver for one grid.  Validates every field of the four structs,
 * allocates all device workspace on the current device and binds the handle
 * to `cuda_stream` (a cudaStream_t, NULL for the legacy default stream).
 * *out receives the handle, or NULL on error. */
jfnk_status jfnk_create(const jfnk_grid* grid, const jfnk_strat* strat,
                        const jfnk_sgs* sgs, const jfnk_opts* opts,
                        void* cuda_stream, jfnk_handle** out);

/* Free the workspace and the handle (NULL is accepted). */
jfnk_status jfnk_destroy(jfnk_handle* h);

/* Surface heat-flux anomaly H [W/m^2] of Section 3.2, device float64 array of
 * nx (2D) or ny*nx (3D) values; it adds H/(rho0 cp dz) to the theta tendency
 * of the bottom row.  The array is copied into the workspace; NULL clears it. */
jfnk_status jfnk_set_surface_flux(jfnk_handle* h, const double* H);

/* F(u) of Eq. ds for all fields: u, F are n-vectors (see conventions).
 * Evaluated in the handle's stencil precision (float32 when MIXED, with u
 * rounded to float32; float64 otherwise). */
jfnk_status jfnk_rhs(jfnk_handle* h, const double* u, double* F);

/* Trapezoidal residual R(u) = 2u/dt - F(u) - 2u_n/dt - F(u_n) (Eq. ns), always float64. */
jfnk_status jfnk_residual(jfnk_handle* h, const double* u_n, const double* u, double* R);

/* Forward-difference Jacobian-vector product of R (Eq. fd), unscaled units:
 *   Jv = 2 v/dt - (F(u + eps v) - F(u)) / eps.
 * F_u may be NULL (then F(u) is evaluated here) or F(u) from jfnk_rhs.
 * eps > 0 is used as given; eps <= 0 selects the rule
 *   eps = sqrt(eps_mach (1 + ||W u||)) / ||W v||,  eps_mach = 2^-52,
 * for both precisions (MIXED evaluates the difference F(u + eps v) - F(u)
 * term by term without cancellation, so float32 stencils do not need a
 * larger step).  *eps_out (host pointer, may be NULL) receives the step
 * used; this synchronises the stream. */
jfnk_status jfnk_jv(jfnk_handle* h, const double* u, const double* F_u, const double* v,
                    double eps, double* Jv, double* eps_out);

/* Field-block preconditioner z = M^-1 r (Section 2.5.2) with the exchange
 * coefficients frozen at state u; r and z in scaled units (W applied).
 * With JFNK_PC_NONE z = r. */
jfnk_status jfnk_precond_apply(jfnk_handle* h, const double* u, const double* r, double* z);

/* One implicit step u^n -> u^{n+1} in place on the device vector u.
 * Returns JFNK_ERR_NOT_CONVERGED (u holds the last iterate) when the Newton
 * test is not met within max_newton corrections.  `out` may be NULL. */
jfnk_status jfnk_step(jfnk_handle* h, double* u, jfnk_stats* out);

/* Same as jfnk_step for a HOST state vector: copies u_host to the device,
 * steps, and copies the result back (pinned memory recommended). */
jfnk_status jfnk_step_host(jfnk_handle* h, double* u_host, jfnk_stats* out);

/* Energy budgets and extremes of the device state u (Section 3.1.3).
 * Extrema propagate NaN (a NaN anywhere in a field makes its max and min NaN). */
jfnk_status jfnk_budgets(jfnk_handle* h, const double* u, jfnk_budget* out);

/* Number of this library's kernel launches enqueued since the handle was created. */
jfnk_status jfnk_get_launch_count(jfnk_handle* h, long long* out);

/* Kernel families whose launches can be timed (roofline reports). */
enum {
    JFNK_KF_ARNOLDI_A = 0,   /* pass A: h1 = V^T w                         */
    JFNK_KF_ARNOLDI_B = 1,   /* pass B: w' = w - V h1, h2 = V^T w', Givens  */
    JFNK_KF_ARNOLDI_C = 2,   /* pass C: v_{j+1} = (w - V h) / h_{j+1,j}     */
    JFNK_KF_JV = 3,          /* Jacobian-vector product stencil             */
    JFNK_KF_PRECOND = 4,     /* preconditioner sweeps (one apply)           */
    JFNK_KF_RESIDUAL = 5,    /* Newton residual stencil (float64)           */
    JFNK_KF_UNET = 6,        /* learned preconditioner network (one apply)  */
    JFNK_KF_COUNT = 7
};

/* Device time and algorithmic bytes of one kernel family. */
typedef struct {
    long long launches;
    double ms;          /* summed CUDA-event time of the launches            */
    double bytes;       /* summed algorithmic HBM bytes (inputs read once,   */
                        /* outputs written once) of the same launches        */
} jfnk_kernel_time;

/* Enable (mask != 0, bit i = family i) or disable event timing of kernel
 * families on the handle's stream; enabling resets the accumulators.  The
 * events add a few microseconds of host work per timed launch.  Launches of
 * a GMRES cycle's Krylov steps after the cycle has ended (they return at
 * entry) are not counted. */
jfnk_status jfnk_kernel_timing(jfnk_handle* h, unsigned int mask);

/* jfnk_kernel_timing with the launches inside GMRES cycles timed only at
 * Krylov steps j with j % every == every / 2 (every >= 1; other launches are
 * always timed; the offset centres the sample on the cycle, whose passes
 * grow with j).  Each pair of events splits the programmatic dependent
 * launch of its kernel from its neighbours; sampling keeps that cost off most
 * steps.  Returns JFNK_ERR_INVALID_ARG for h NULL or every < 1. */
jfnk_status jfnk_kernel_timing_sampled(jfnk_handle* h, unsigned int mask, int every);

/* Drain the outstanding events (synchronises the stream) and copy the
 * accumulators of all JFNK_KF_COUNT families into out[0 .. JFNK_KF_COUNT). */
jfnk_status jfnk_kernel_timing_read(jfnk_handle* h, jfnk_kernel_time* out);

/* ------------------------------------------------------------------ batch
 * Many independent grids stepped together (e.g. heat-island instances of
 * uneven sizes and surface fluxes, Section 3.2).  Each instance gets its own
 * handle (full workspace) and a non-blocking stream created by the batch; a
 * batch step forks the caller's stream into the instance streams, runs every
 * instance's Newton / GMRES sequence concurrently from one host thread per
 * instance, and joins back, so independent instances overlap on the GPU.
 * Instance handles launch their GMRES cycles as stream launches
 * (jfnk_set_cycle_graph(h, 0)); jfnk_batch_handle gives access to change it. */
#define JFNK_MAX_BATCH 256
typedef struct jfnk_batch jfnk_batch;

/* n instances; grids, strats, sgs, opts are host arrays of n structs (same
 * validation as jfnk_create).  cuda_stream: the caller's stream. */
jfnk_status jfnk_create_batch(int n, const jfnk_grid* grids, const jfnk_strat* strats,
                              const jfnk_sgs* sgs, const jfnk_opts* opts, void* cuda_stream,
                              jfnk_batch** out);
jfnk_status jfnk_destroy_batch(jfnk_batch* b);

/* The handle of instance i (owned by the batch; e.g. for jfnk_set_surface_flux). */
jfnk_status jfnk_batch_handle(jfnk_batch* b, int i, jfnk_handle** out);

/* One implicit step of every instance: u is a host array of n device state
 * pointers (layout of instance i's grid).  stats / status (host arrays of n,
 * may be NULL) receive each instance's report and status.  Returns JFNK_OK
 * when every instance converged, otherwise the first error or
 * JFNK_ERR_NOT_CONVERGED.  Blocks the calling thread until all instances
 * finish; the caller's stream waits for them. */
jfnk_status jfnk_step_batch(jfnk_batch* b, double* const* u, jfnk_stats* stats, jfnk_status* status);

/* ----------------------------------------------- learned preconditioner
 * Not in the paper (its preconditioner is the field-block one of Section
 * 2.5.2, which stays the fallback).  A linear convolutional U-Net N acts on
 * the scaled field planes of a Krylov vector (4 in 2-D, 5 in 3-D) and corrects the block
 * preconditioner M: with precond = JFNK_PC_UNET the flexible-GMRES direction
 * of v is z = M^-1 v + N(v).
 *
 * Network (no biases, no activations, zero padding; rows z, columns x):
 *   L0a 3x3 16->16 (input: the 4 planes, zero-padded to 16 channels),
 *   L0b 3x3 16->16 = s0, 2x2 average pool, L1a 3x3 16->32, L1b 3x3 32->32
 *   = s1, 2x2 average pool, L2a 3x3 32->64, L2b 3x3 64->64, nearest
 *   upsampling, concat [up, s1], L1c 3x3 96->32, nearest upsampling, concat
 *   [up, s0], L0c 3x3 48->16, L0d 1x1 16->16 (first 4 channels = N(v)).
 * 3-D grids: input and output have 5 channels (u, v, w, theta, p); every 3x3
 * convolution acts on each horizontal (y, x) plane (rows y, columns x, zero
 * padding at the plane's edges), pooling averages 2x2x2 blocks and the
 * upsampling repeats each point 2x2x2, so that the vertical coupling enters
 * through the coarser levels.
 * Flat weight order (float32): layers in that order, each [tap][cout][cin]
 * with tap = ky * k + kx reading the input at offset (ky - k/2, kx - k/2).
 * Convolutions run on the tensor cores with bfloat16 operands and float32
 * accumulation; training keeps float32 master weights (Adam).
 *
 * The convolutions work in balanced units: N(v) = B^-1 net(B v) with
 * B = diag(1, 1, s_theta / Theta_b, s_p / P_b) (3-D: diag(1, 1, 1, s_theta /
 * Theta_b, s_p / P_b)), s_* = scale_* of jfnk_opts,
 * Theta_b = s_u sqrt(|beta| theta0 / g) and P_b = s_u sqrt(gamma_p pbar /
 * theta0) (factor 1 where beta or gamma_p pbar is 0): the units in which the
 * linearised buoyancy and acoustic couplings of Eqs. ch2_28-ch2_30 are
 * skew-adjoint, so that errors of the network are weighted as the Jacobian
 * weights them.
 *
 * Training pairs come from the solver's own GMRES solves (Section 2.5.1),
 * the field-block M frozen at the Newton iterate u_k:
 *   JFNK_PAIRS_ARNOLDI  every Arnoldi step: w = J_hat z_j is an exact inverse
 *                       pair, X = w / ||w||, T = (z_j - M^-1 w) / ||w||;
 *   JFNK_PAIRS_NEWTON   every converged Newton correction: b = -W R(u_k),
 *                       beta = ||b||, x_hat the scaled correction,
 *                       X = b / beta, T = x_hat / beta - M^-1 X.
 * The loss of a pair is 1/2 ||B (N(X) - T)||^2 / ||B X||^2.
 *
 * Only handles with precision JFNK_MIXED on 2-D grids with nx, nz multiples of
 * 32, or on 3-D grids with nx a multiple of 32, ny of 64 and nz of 4, accept
 * these calls (and precond = JFNK_PC_UNET); others get
 * JFNK_ERR_UNSUPPORTED.  Safeguards: a GMRES cycle of m steps with the learned
 * preconditioner that reduces the residual by less than a factor 2 hands the
 * rest of that Newton solve to the field-block preconditioner (restarting from
 * the correction reached; jfnk_stats.pc_switches counts such solves), and a
 * step with JFNK_PC_UNET that ends in JFNK_ERR_NOT_CONVERGED,
 * JFNK_ERR_BREAKDOWN or JFNK_ERR_NAN is redone from u^n with the field-block
 * preconditioner (jfnk_stats.pc_fallback = 1).
 * Until a network is attached JFNK_PC_UNET behaves as JFNK_PC_BLOCK. */

/* Attach a network with seeded random weights (N(0, 1/fan-in), last layer
 * zero so that N = 0 until trained); replaces an attached one. */
jfnk_status jfnk_unet_init(jfnk_handle* h, unsigned long long seed);

/* Number of float32 weights of the network. */
jfnk_status jfnk_unet_num_weights(jfnk_handle* h, size_t* count);

/* Copy the float32 master weights to / from host memory (count must equal
 * jfnk_unet_num_weights; setting resets the Adam moments). */
jfnk_status jfnk_unet_get_weights(jfnk_handle* h, float* host, size_t count);
jfnk_status jfnk_unet_set_weights(jfnk_handle* h, const float* host, size_t count);

enum { JFNK_PAIRS_NEWTON = 1, JFNK_PAIRS_ARNOLDI = 2 };

/* Record training pairs of the kinds in the bit mask `kinds` during later
 * jfnk_step calls, until `capacity` pairs are held (device memory:
 * 2 * capacity * 4 * nx * nz floats; every pair adds one field-block
 * preconditioner apply to the step).  Drops the pairs held; capacity 0 or
 * kinds 0 stops recording and frees them. */
jfnk_status jfnk_unet_capture(jfnk_handle* h, int capacity, int kinds);

/* Number of recorded pairs. */
jfnk_status jfnk_unet_pair_count(jfnk_handle* h, int* count);

/* Copy recorded pair i into device float32 arrays X, T of 4 * nx * nz. */
jfnk_status jfnk_unet_get_pair(jfnk_handle* h, int i, float* X, float* T);

/* `epochs` passes of Adam (step lr, beta1 = 0.9, beta2 = 0.999, one update
 * per pair, fixed pair order per epoch) over the recorded pairs.
 * loss_hist: host array of `epochs` doubles (may be NULL) receiving the mean
 * loss of each epoch (measured before each update).  Synchronises. */
jfnk_status jfnk_unet_train(jfnk_handle* h, int epochs, float lr, double* loss_hist);

/* y = N(x) for device float32 arrays of 4 * nx * nz (field planes, x fastest). */
jfnk_status jfnk_unet_forward(jfnk_handle* h, const float* x, float* y);

/* Loss of one pair (device x, t) and, when grads (host, jfnk_unet_num_weights
 * floats) is not NULL, its gradient with respect to the flat weights.
 * Synchronises; JFNK_ERR_TIMEOUT as for jfnk_unet_status. */
jfnk_status jfnk_unet_loss_grad(jfnk_handle* h, const float* x, const float* t, double* loss,
                                float* grads);

/* Engine of the network's convolutions (not in the paper; the network itself
 * is this project's addition): JFNK_UNET_TCGEN05 (default) runs them as
 * implicit GEMMs on the tcgen05 tensor cores with TMEM accumulators,
 * JFNK_UNET_MMA_SYNC on the mma.sync path; both compute the same layers in
 * bfloat16 with float32 accumulation.  Synchronises the handle's stream. */
#define JFNK_UNET_TCGEN05 0
#define JFNK_UNET_MMA_SYNC 1
jfnk_status jfnk_unet_set_engine(jfnk_handle* h, int engine);

/* Synchronises the stream and returns JFNK_ERR_TIMEOUT when a tensor-core
 * wait inside a network convolution ran past its iteration limit since the
 * network was created (that convolution's output is not valid; the flag
 * stays set), else JFNK_OK. */
jfnk_status jfnk_unet_status(jfnk_handle* h);

/* Change the preconditioner between steps: any JFNK_PC_* value accepted by
 * jfnk_create (JFNK_PC_UNET only where the calls above are supported). */
jfnk_status jfnk_set_precond(jfnk_handle* h, int precond);

/* Number of tile shapes jfnk_set_tiles accepts per kernel family. */
#define JFNK_NUM_TILE_SHAPES 4

/* Choose the tile shapes of the float32 Jacobian-product and preconditioner
 * stencils for this handle's grid: every candidate is timed on the handle's
 * stream with inputs derived from the device state u (unchanged), and the
 * fastest is kept.  tiles (host, may be NULL) receives {jv, pc} indices.
 * Synchronises the stream; results of the kernels are unaffected (every
 * shape computes the same values).  A float64 handle keeps its single shape. */
jfnk_status jfnk_autotune(jfnk_handle* h, const double* u, int* tiles);

/* Set the tile-shape indices (0 .. JFNK_NUM_TILE_SHAPES-1) directly. */
jfnk_status jfnk_set_tiles(jfnk_handle* h, int tile_jv, int tile_pc);

/* Launch the Krylov steps of GMRES cycles as CUDA graphs (Section 2.5.1's
 * restarted FGMRES(m), every preconditioner, float32 or float64).
 * steps > 0: the cycle's m steps are captured once into segments of
 * `steps` steps each (steps > m is taken as m) and each segment
 * is one graph launch; the host polls for the end of the cycle once per
 * segment instead of once per step.  steps = 0: every kernel is a separate
 * stream launch.  steps = JFNK_CYCLE_GRAPH_AUTO (the default of jfnk_create):
 * one step per segment with the Schur complement, two with the learned
 * correction, min(m, JFNK_CYCLE_GRAPH_SEGMENT) on grids of at most
 * JFNK_CYCLE_GRAPH_SEGMENT_POINTS points and m above.  Results are
 * bit-identical either way: every kernel of a step returns at entry once the
 * cycle has ended, so steps launched past the end change nothing.  The
 * segments are captured on a private stream (the first cycle with each
 * preconditioner runs as stream launches) and again whenever the grid
 * description, tiles, surface flux, sweep count, preconditioner or
 * kernel-timing settings or the learned network's weights change; timed
 * families are timed by event nodes inside the graphs.  Pair recording uses
 * stream launches.  Returns JFNK_ERR_INVALID_ARG for h NULL or steps < -1. */
jfnk_status jfnk_set_cycle_graph(jfnk_handle* h, int steps);

#define JFNK_CYCLE_GRAPH_AUTO (-1)
/* Default segment length (not the Schur complement) and the grid size up to which it applies. */
#define JFNK_CYCLE_GRAPH_SEGMENT 8
#define JFNK_CYCLE_GRAPH_SEGMENT_POINTS 262144

/* Largest grid (nx * nz points) accepted by jfnk_budgets_static. */
#define JFNK_BUDGETS_STATIC_MAX_POINTS 8388608

/* Budgets without a handle and without any device allocation.
 *
 * For callers that cannot call cudaMalloc: code that runs where device
 * allocation is not allowed (for example inside a stream capture that must
 * not allocate, under an allocator that owns all device memory, or in a
 * service with a fixed memory budget) cannot create a handle, because
 * jfnk_create allocates workspace.  This entry point computes the same
 * values as jfnk_budgets from a 2-D grid description alone.  The paper has
 * no counterpart; it is a deployment variant.
 *
 * u:   device float64 state [4][nz][nx] (2-D only; 3-D is JFNK_ERR_UNSUPPORTED).
 * out: device float64 array of 12 values, written by the last kernel block:
 *      E_k, E_p, sum theta dV, sum div(u) dV, max(u, w, theta, p), min(u, w, theta, p).
 * Grids above JFNK_BUDGETS_STATIC_MAX_POINTS are rejected with
 * JFNK_ERR_INVALID_ARG before anything is enqueued.
 * Scratch: a file-scope device array of about 393 KB (one float64 partial per
 * kernel block and value, plus a counter) that every GPU which loads the
 * library holds until the process exits.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 * The array's device address belongs to a CUDA context: the first call in
 * each context (the primary context of a device, or any context the caller
 * has made current) looks it up with cudaGetSymbolAddress and caches it
 * under that context's id; make that first call before any stream capture.
 * A device reset (cudaDeviceReset) creates a new context, whose first call
 * looks the address up again.  All calls in a context share the array and
 * it keeps the last call's contents (the counter is reset by every call);
 * calls that overlap on the GPU (different streams without ordering) race.
 * Extrema propagate NaN: a NaN anywhere in a field makes its max and min NaN.
 * Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy default stream):
 * out is complete only once cuda_stream has reached the kernel (synchronise
 * the stream, or order later work after it, before reading out). */
jfnk_status jfnk_budgets_static(const jfnk_grid* grid, const double* u, double* out,
                                void* cuda_stream);

/* Static description of a status code. */
const char* jfnk_status_str(jfnk_status s);

#ifdef __cplusplus
}
#endif
#endif /* JFNK_H */

/*
 * ase_df.h -- C ABI of the GB300 (sm_103a) FP64 library for the per-stage spatial
 * residual of a finite-volume Euler solver with ASE-DF reconstruction
 * (arXiv 2410.05489, "An Adaptive Reconstruction Method for Arbitrary High-Order
 * Accuracy Using Discontinuity Feedback").
 *
 * The residual (Sec. 2.1, semi-discrete form) of one RK stage is
 *     L(W) = -(1/|Omega|) sum_faces |l| sum_k eta_k F(x_k) . n
 * with, on every face, (r-1)/2 Gauss points (Sec. 2.1; one point in 1D), the
 * Lax-Friedrichs flux of Sec. 2.3 between reconstructed states, and the states from the
 * adaptive stencil extension of Sec. 3 (Algorithm 1) driven by the discontinuity
 * feedback factor of Sec. 3.1, Eq. (3.2): linear 5th/7th/9th order where the stencil is
 * smooth, WENOZ-AO(5,3) with DF damping (Sec. 3.2) otherwise.  Time stepping is the
 * SSP-RK3 of Sec. 2.3.  Also here: the paper's gas-kinetic flux with S2O4 time stepping
 * (Sec. 2.2, ase_df_gks_*), vector-Jacobian products of the residual and of a step
 * (ase_df_residual_adjoint, ase_df_step_adjoint), batched solves of many independent
 * problems (ase_df_batch_*), and a residual entry point that allocates nothing
 * (ase_df_residual_noalloc).
 *
 * Conventions (all entry points):
 *   - Arrays are DEVICE pointers owned by the caller, FP64, C-contiguous:
 *       W      [C][ny][nx]   conservative cell averages; C = 3 in 1D (rho, rho u, E),
 *                            C = 4 in 2D (rho, rho u, rho v, E); 1D uses ny = 1.
 *       sx     [ny][nx+1]    discontinuity strength sigma of the x-faces; x-face f lies
 *                            between cells f-1 and f.
 *       sy     [ny+1][nx]    sigma of the y-faces (2D only; pass NULL in 1D).
 *       L      [C][ny][nx]   residual dW/dt.
 *   - sigma is solver state: the sigma a residual consumes is the one the previous
 *     residual (previous RK stage) produced; ase_df_prime_sigma gives sigma^0.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     stream-ordered and asynchronous; the status readers (ase_df_get_status,
 *     ase_df_get_repair_stats, ase_df_batch_get_status), the benchmark helpers and the
 *     batch schedule setters synchronise, as their comments say.  A 2D context runs
 *     its y-face sweeps on a stream of its own, forked from and joined back to the
 *     caller's stream within each call (also under graph capture), so the ordering
 *     seen from the caller's stream is unchanged.
 *   - The context owns its scratch memory (face fluxes, RK stage states, sigma
 *     ping-pong buffers); one context per host thread.
 *   - Errors: argument and launch errors are returned at once (ase_df_last_error gives
 *     the message); conditions found on the device (non-physical states, non-finite
 *     values) are OR-ed into a device status word read by ase_df_get_status.  Nothing
 *     traps or asserts on the device.
 */
#ifndef ASE_DF_H
#define ASE_DF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ASE_DF_OK = 0,
  ASE_DF_E_INVAL = 1,       /* bad argument or parameter */
  ASE_DF_E_NOMEM = 2,       /* device allocation failed */
  ASE_DF_E_CUDA = 3,        /* a CUDA call or launch failed */
  ASE_DF_E_NONPHYSICAL = 4, /* the device status word reports a non-physical state */
  ASE_DF_E_TIMEOUT = 5,     /* a bounded device wait ran out */
  ASE_DF_E_BOUNDS = 6       /* a size exceeds a documented limit */
} ase_df_status;

typedef enum {
  ASE_DF_BC_PERIODIC = 0,   /* ghost cells wrap around */
  ASE_DF_BC_OUTFLOW = 1,    /* zero-gradient: ghost cells copy the nearest interior cell */
  ASE_DF_BC_INFLOW_BAND = 2, /* x-lo only: ghost cells whose centre y lies in
                               (inflow_lo, inflow_hi) hold inflow_state; outflow elsewhere */
  ASE_DF_BC_REFLECT = 3,    /* reflecting wall: ghost cells mirror the interior about the wall
                               face with the normal momentum negated (needs (r+1)/2 cells or
                               more in that direction; not supported by the adjoint) */
  ASE_DF_BC_WALL_AFTER = 4, /* y-lo only (2D; the double Mach reflection of Sec. 4.3): ghost
                               cells whose centre x is below wall_x hold inflow_state, the
                               others a reflecting wall (needs (r+1)/2 rows or more) */
  ASE_DF_BC_MOVING_SHOCK = 5 /* y-hi only (2D): ghost cells whose centre x is below
                               shock_x0 + shock_speed t hold inflow_state, the others state_b;
                               t is the time of the stage being evaluated (the device time of
                               the context plus the stage's offset: SSP-RK3 stages at t,
                               t + dt, t + dt/2; gas-kinetic S2O4 stages at t, t + dt/2) */
} ase_df_bc;

/* Device status word bits (ase_df_get_status). */
#define ASE_DF_FLAG_NONPHYSICAL 0x1u   /* a cell average with rho <= 0, p <= 0 or non-finite */
#define ASE_DF_FLAG_POSITIVITY  0x2u   /* informational: a Gauss point took the first-order
                                          states (non-physical reconstructed state) */
#define ASE_DF_FLAG_DT          0x4u   /* the CFL step came out non-positive or non-finite */
#define ASE_DF_FLAG_FROZEN      0x8u   /* informational: to stay physical, a cell kept its stage's
                                          combination of W^n and W^(s) without the flux update
                                          (last resort of the positivity repair; that cell is
                                          not conservative in that stage) */
#define ASE_DF_FLAG_SYNC        0x10u  /* internal error: a grid barrier of the positivity repair
                                          gave up waiting (the stage's repair is incomplete) */

/* Problem statement (Sec. 2: 1D/2D Euler on a uniform Cartesian grid). */
typedef struct {
  int32_t ndim;            /* 1 or 2 */
  int32_t order;           /* scheme order r: 3, 5, 7 or 9 */
  int64_t nx, ny;          /* cells; ny is ignored (taken as 1) in 1D */
  double x0, x1, y0, y1;   /* domain [x0,x1] x [y0,y1] */
  double gamma;            /* ratio of specific heats, > 1 */
  double sigma_thres;      /* DF threshold of Eq. (3.2); the paper uses 2.0 (Sec. 4.1) */
  double cfl;              /* CFL number for dt = cfl / max((|u|+c)/dx + (|v|+c)/dy) */
  int32_t bc[4];           /* ase_df_bc of x-lo, x-hi, y-lo, y-hi */
  double inflow_state[4];  /* primitive (rho, u, v, p) of an x-lo inflow band */
  double inflow_lo, inflow_hi;
  double t_end;            /* > 0: CFL steps are shortened so that t never passes t_end */
  double gks_c1, gks_c2;   /* gas-kinetic path: tau_n = c1 dt + c2 |p_l - p_r| / (p_l + p_r) dt
                              (Sec. 2.2); <= 0 takes 0.05 and 1.0, the values of the paper's
                              figure captions for Configuration 3, Shu-Osher and the double Mach
                              reflection (5.0 for c2 in its blast wave) */
  double state_b[4];       /* primitive (rho, u, v, p) beyond the moving shock (ASE_DF_BC_MOVING_SHOCK) */
  double wall_x;           /* ASE_DF_BC_WALL_AFTER: x where the wall starts */
  double shock_x0, shock_speed;  /* ASE_DF_BC_MOVING_SHOCK: shock at x = shock_x0 + shock_speed t */
} ase_df_params;

typedef struct ase_df_ctx ase_df_ctx;

/* Validates p and allocates the context and its device scratch on the current device.
 * Limits: nx, ny <= 2^20 and C*(nx+1)*(ny+1) < 2^31.  Returns ASE_DF_E_INVAL /
 * ASE_DF_E_BOUNDS / ASE_DF_E_NOMEM without allocating anything on failure; *out is
 * NULL then. */
ase_df_status ase_df_init(const ase_df_params* p, ase_df_ctx** out);

/* Frees the context and its device memory (synchronises the device first). */
void ase_df_destroy(ase_df_ctx* ctx);

/* sigma^0 (Sec. 3.1, feedback): the face strengths of a residual evaluated with
 * sigma_in = 0, i.e. from all-linear r-th order states.  Writes sx (and sy in 2D). */
ase_df_status ase_df_prime_sigma(ase_df_ctx* ctx, const double* W, double* sx, double* sy,
                                 void* stream);

/* One residual evaluation (Sec. 2.1 Eq. 2.3 with Sec. 3 reconstruction and the Sec. 2.3
 * flux): reads W and sigma_in, writes L and sigma_out (sx_out, sy_out must not alias
 * sx_in, sy_in).  The Gauss-averaged face fluxes stay in the context
 * (ase_df_copy_face_fluxes). */
ase_df_status ase_df_residual(ase_df_ctx* ctx, const double* W, const double* sx_in,
                              const double* sy_in, double* L, double* sx_out, double* sy_out,
                              void* stream);

/* Copies the face fluxes of the last residual evaluation on this context:
 * Fx [C][ny][nx+1], Fy [C][ny+1][nx] (NULL in 1D). */
ase_df_status ase_df_copy_face_fluxes(ase_df_ctx* ctx, double* Fx, double* Fy, void* stream);

/* One SSP-RK3 step (Sec. 2.3, Eq. SSP-RK3) in place: W holds W^n on entry and W^{n+1}
 * on exit; sx/sy hold sigma^n on entry and the third stage's sigma on exit (each stage
 * consumes the sigma of the stage before).  dt > 0: that step; dt <= 0: the CFL step of
 * W^n (including the inflow state, if any), shortened to t_end.  The device keeps the
 * time t and the last dt (ase_df_get_status).  After every stage, cells whose new
 * average is non-physical are updated again with first-order Lax-Friedrichs fluxes on
 * their faces (the paper's transition to first order for positivity, Sec. 1; up to 8
 * passes, each re-doing the neighbours of newly failing cells); a cell still
 * non-physical after that keeps its stage's combination of W^n and W^(s) without the
 * flux update, with E raised to give p = 1e-13 of the kinetic energy density where
 * rounding leaves a near-vacuum p <= 0 (ASE_DF_FLAG_FROZEN); ASE_DF_FLAG_NONPHYSICAL is
 * raised only if that still fails (rho <= 0 or non-finite values). */
ase_df_status ase_df_step(ase_df_ctx* ctx, double* W, double* sx, double* sy, double dt,
                          void* stream);

/* Runs nsteps ase_df_step calls as one CUDA graph replay when possible (captured on the
 * first call for the given pointers and dt mode, replayed afterwards). */
ase_df_status ase_df_run(ase_df_ctx* ctx, double* W, double* sx, double* sy, double dt,
                         int32_t nsteps, void* stream);

/* Adjoint (vector-Jacobian product) of one residual evaluation
 * (L, sigma_out) = R(W, sigma_in) of ase_df_residual:
 *   Wbar     += (dL/dW)^T Lbar + (dsigma_out/dW)^T sigma_bar_out
 *   sxbar_in += (dL/dsx_in)^T Lbar + (dsigma_out/dsx_in)^T sigma_bar_out   (same for y)
 * The derivative is that of the scheme as defined, taken on the branch the forward
 * evaluation takes: Algorithm 1's branch choice (Sec. 3) is held fixed; linear
 * reconstructions have constant weights; on the WENOZ-AO(5,3) fallback (Sec. 3.2) the
 * WENO-Z weights (beta, tau_Z, |.| piecewise) and the DF factors alpha = sigma_thres / A
 * of Eq. (3.2) are differentiated; the Lax-Friedrichs flux of Sec. 2.3 takes the
 * derivative of the larger wave speed; sigma of Sec. 3.1 is differentiated as written;
 * a Gauss point that took the first-order states passes its adjoint to the two cell
 * averages (its sigma, 1e30, is constant).
 * Arrays are device pointers in the layouts of ase_df_residual: W, Lbar, Wbar
 * [C][ny][nx]; sx_*, sxbar_* [ny][nx+1]; sy_*, sybar_* [ny+1][nx] (NULL in 1D).  Lbar,
 * sxbar_out and sybar_out may be NULL (zero adjoint); sxbar_in and sybar_in may be NULL
 * (that adjoint is not formed).  Outputs are accumulated, not overwritten; they must not
 * alias the inputs.  The first call allocates the context's adjoint scratch (about
 * (4r + 12) C doubles per cell in 2D); ASE_DF_E_NOMEM if that fails.  Deterministic: the
 * kernels gather, without atomics. */
ase_df_status ase_df_residual_adjoint(ase_df_ctx* ctx, const double* W, const double* sx_in,
                                      const double* sy_in, const double* Lbar, const double* sxbar_out,
                                      const double* sybar_out, double* Wbar, double* sxbar_in,
                                      double* sybar_in, void* stream);

/* Adjoint of one ase_df_step of fixed dt > 0 (Sec. 2.3, SSP-RK3 in Shu-Osher form, each
 * stage consuming the sigma of the stage before).  W, sx, sy hold W^n and sigma^n (as
 * passed to that step; read only).  On entry Wbar = dJ/dW^{n+1} and sxbar/sybar =
 * dJ/dsigma^{n+1} (the third stage's sigma_out); on exit they hold dJ/dW^n and
 * dJ/dsigma^n.  The step's first two stages are recomputed on the device (the same
 * launches as ase_df_step, so the stage states are bit-identical) and three residual
 * adjoints run backwards.  The positivity repair of ase_df_step is not differentiated:
 * if a recomputed stage needed it, the step's repaired-cell count grows
 * (ase_df_get_repair_stats) and the result is the adjoint of the unrepaired update. */
ase_df_status ase_df_step_adjoint(ase_df_ctx* ctx, const double* W, const double* sx, const double* sy,
                                  double dt, double* Wbar, double* sxbar, double* sybar, void* stream);

/* Synchronises the stream of the last call and reads the device status word (ASE_DF_FLAG_*),
 * the last dt and the time t.  Returns ASE_DF_E_TIMEOUT if ASE_DF_FLAG_SYNC is set (a
 * device wait gave up), else ASE_DF_E_NONPHYSICAL if that bit is set. */
ase_df_status ase_df_get_status(ase_df_ctx* ctx, uint32_t* flags, double* last_dt, double* t);

/* Self-test of the bounded device waits (failure detection without a GPU fault): launches on
 * `stream` a cooperative kernel of two CTAs whose grid barrier (the one the positivity repair
 * uses between its passes) waits for one CTA more than the grid has.  The wait gives up after
 * about a second, the kernel raises ASE_DF_FLAG_SYNC in the status word and returns, and the
 * barrier's arrival count is cleared; ase_df_get_status then returns ASE_DF_E_TIMEOUT until
 * ase_df_reset.  The context stays usable. */
ase_df_status ase_df_selftest_wait(ase_df_ctx* ctx, void* stream);

/* Diagnostics of the positivity repair of the stage updates (ase_df_step): synchronises,
 * then writes into last_stage[18] (may be NULL) the counts of the most recent stage --
 * [0]: cells the high-order update left non-physical, [p] (p = 1..8): cells newly
 * non-physical after repair pass p, [9 + p] (p = 1..8): cells still non-physical after
 * pass p -- into *total (may be NULL) the number of cells marked since the last
 * ase_df_reset, and into *frozen (may be NULL) the number of cells that took the last
 * resort since then. */
ase_df_status ase_df_get_repair_stats(ase_df_ctx* ctx, uint32_t* last_stage, uint64_t* total,
                                      uint64_t* frozen);

/* Clears the device status word and sets the device time t. */
ase_df_status ase_df_reset(ase_df_ctx* ctx, double t, void* stream);

/* Message of the last error on this context (or, when ctx is NULL, of the last failed
 * ase_df_init or ase_df_residual_noalloc). */
const char* ase_df_last_error(const ase_df_ctx* ctx);

/* Kernel timing with CUDA events recorded on the launching stream around every sweep,
 * combine and wave-speed launch of this context (enable != 0 starts a new record, 0
 * stops recording; while it records, the two sweeps of a stage run one after the
 * other on the caller's stream, so that each launch is timed alone).  ase_df_profile_read synchronises, then returns per kernel kind
 * (0: x-face sweep, 1: y-face sweep, 2: combine, 3: wave-speed reduction, 4: positivity
 * repair, one launch per stage) the summed milliseconds ms[5] and the launch counts n[5]; at most 65536
 * launches are recorded. */
ase_df_status ase_df_profile_enable(ase_df_ctx* ctx, int32_t enable);
ase_df_status ase_df_profile_read(ase_df_ctx* ctx, double* ms, int64_t* n);

/* Branch histogram of Algorithm 1 on the device (a metric of the method's behaviour).
 * While enabled (enable != 0), every sweep of this context counts, per face and side, the
 * branch that the normal reconstruction and (2D) the tangential reconstruction of the
 * state took, and every Gauss point whose reconstructed state was non-physical and took
 * the cell averages (reading G21).  Counting costs a few shared-memory atomics per face;
 * when disabled the sweeps count nothing.  Counts accumulate on the device until read.
 * ase_df_hist_read synchronises the context's streams, writes the counts into counts[7]
 * -- linear 9th, 7th, 5th order, WENOZ-AO(5,3)+DF (Sec. 3.2), linear 3rd order, DF-damped
 * 3rd order, first-order Gauss points -- and clears them.  The gas-kinetic sweeps and the
 * adjoint do not count. */
ase_df_status ase_df_hist_enable(ase_df_ctx* ctx, int32_t enable);
ase_df_status ase_df_hist_read(ase_df_ctx* ctx, uint64_t* counts);

/* The residual of ase_df_residual for callers that cannot allocate device memory (code
 * running inside someone else's CUDA graph capture, real-time loops that must not
 * synchronise the device, frameworks that own every device byte through their own
 * pool).  The paper has no counterpart: this is a library-integration entry point.
 * It takes no context: the face-flux scratch is one file-scope __device__ array of
 * 2^21 doubles (16 MiB, held by every GPU that loads the library until exit), so it
 * calls no cudaMalloc / cudaFree and no allocating library routine.  Arguments as
 * ase_df_residual plus the problem p, validated exactly as ase_df_init validates it;
 * the results equal ase_df_residual's bit for bit.  Every boundary of ase_df_bc is
 * accepted except ASE_DF_BC_MOVING_SHOCK, which needs the solver time that only a
 * context holds (ASE_DF_E_INVAL).  Limit: C*ny*(nx+1) + C*(ny+1)*nx (2D) or 3*(nx+1)
 * (1D) face-flux doubles <= 2^21 - 32, e.g. 2D grids up to 511 x 511; larger grids
 * return ASE_DF_E_BOUNDS.  Each call outside stream capture looks up the array's device
 * address (cudaGetSymbolAddress, with the caller's device current; this also follows the
 * array to a new address after cudaDeviceReset); a call during capture uses the address
 * found by an earlier call on that device, so make one call on each device before
 * capturing (otherwise ASE_DF_E_INVAL).  All calls share the array, which keeps the last
 * call's contents: calls that overlap on the GPU race and must not be issued.
 * Device-side conditions (status flags) are not reported.  On failure the message is
 * in ase_df_last_error(NULL) (one process-wide buffer, shared with ase_df_init). */
ase_df_status ase_df_residual_noalloc(const ase_df_params* p, const double* W, const double* sx_in,
                                      const double* sy_in, double* L, double* sx_out, double* sy_out,
                                      void* stream);

/* ---------------------------------------------------------------------------------
 * Gas-kinetic flux and two-stage fourth-order time stepping (Sec. 2.2 with Appendix A):
 * the paper's primary solver.  The reconstruction (Sec. 3, Algorithm 1, the same sigma
 * feedback) also provides the normal and tangential derivatives of each side's state at
 * the Gauss points; the flux of the BGK distribution function of Eq. (GKS flux), with
 * the physical collision time 0 (inviscid flow) and the numerical collision time
 * tau_n = C1 dt + C2 |p_l - p_r| / (p_l + p_r) dt, is integrated over
 * [0, dt] and [0, dt/2], giving the face flux F and its time derivative F_t; C1, C2 are
 * ase_df_params.gks_c1, gks_c2.  A Gauss
 * point with a non-physical state takes the two cell averages with zero derivatives
 * (sigma 1e30, ASE_DF_FLAG_POSITIVITY).  There is no positivity repair on this path.
 * --------------------------------------------------------------------------------- */

/* One gas-kinetic evaluation for the step size dt > 0: L (as ase_df_residual) and its time
 * derivative Lt (both [C][ny][nx]), sigma_out as ase_df_residual. */
ase_df_status ase_df_gks_residual(ase_df_ctx* ctx, const double* W, const double* sx_in, const double* sy_in,
                                  double dt, double* L, double* Lt, double* sx_out, double* sy_out, void* stream);

/* One S2O4 step in place: W* = W^n + dt/2 L(W^n) + dt^2/8 Lt(W^n), then
 * W^{n+1} = W^n + dt L(W^n) + dt^2/6 (Lt(W^n) + 2 Lt(W*)); each stage consumes the sigma
 * of the stage before (sx, sy: sigma^n on entry, the second stage's on exit).  dt > 0:
 * that step; dt <= 0: the CFL step of W^n (as ase_df_step), fixed before the first flux
 * evaluation.  A non-physical cell average raises ASE_DF_FLAG_NONPHYSICAL. */
ase_df_status ase_df_gks_step(ase_df_ctx* ctx, double* W, double* sx, double* sy, double dt, void* stream);

/* ---------------------------------------------------------------------------------
 * Batched solves (no counterpart in the paper, whose solver advances one problem): n
 * independent problems, 1D and 2D, of mixed order, advanced together, each with its own
 * CFL dt, time and status.  Every sweep direction of every RK stage is ONE persistent
 * launch over the tiles of all problems (work list ordered by cost, atomic work counter);
 * the combination, positivity repair and CFL reduction run over per-problem cell chunks.
 *
 * State: the caller owns three packed device arrays -- W (each problem's [C][ny][nx]
 * block back to back), sx (each [ny][nx+1]) and sy (each 2D problem's [ny+1][nx]; 1D
 * problems take no room; may be NULL if all problems are 1D) -- laid out as
 * ase_df_batch_layout reports.  The batch owns its scratch.  Limits: each problem as in
 * ase_df_init, fewer than 2^31 cells in total.
 * --------------------------------------------------------------------------------- */
typedef struct ase_df_batch ase_df_batch;

/* Validates the n problems p[0..n-1] and allocates the batch (descriptors, work lists,
 * scratch) on the current device.  p[i].t_end bounds each problem's time. */
ase_df_status ase_df_batch_init(const ase_df_params* p, int32_t n, ase_df_batch** out);
void ase_df_batch_destroy(ase_df_batch* b);

/* Offsets (in doubles) of problem i in the packed arrays: W block [w_off[i], w_off[i+1]),
 * sx block [sx_off[i], sx_off[i+1]), sy block [sy_off[i], sy_off[i+1]); n+1 entries each
 * (any pointer may be NULL). */
ase_df_status ase_df_batch_layout(const ase_df_batch* b, int64_t* w_off, int64_t* sx_off, int64_t* sy_off);

/* sigma^0 of every problem (as ase_df_prime_sigma), then every problem's time, dt and
 * status are reset (as ase_df_reset with t = 0). */
ase_df_status ase_df_batch_prime_sigma(ase_df_batch* b, const double* W, double* sx, double* sy,
                                       void* stream);

/* One SSP-RK3 CFL step of every problem, in place (as ase_df_step with dt <= 0, including
 * the positivity repair). */
ase_df_status ase_df_batch_step(ase_df_batch* b, double* W, double* sx, double* sy, void* stream);

/* nsteps batch steps as replays of one CUDA graph (captured on the first call for these
 * pointers and the current schedule). */
ase_df_status ase_df_batch_run(ase_df_batch* b, double* W, double* sx, double* sy, int32_t nsteps,
                               void* stream);

/* Synchronises; per problem: status flags (ASE_DF_FLAG_*), time, last dt (arrays of n;
 * any may be NULL).  Returns ASE_DF_E_NONPHYSICAL if any problem reports that flag. */
ase_df_status ase_df_batch_get_status(ase_df_batch* b, uint32_t* flags, double* t, double* last_dt);

/* Schedule: persistent sweep CTAs per SM (1 or 2), work items ordered by cost (1) or by
 * problem (0), cells per chunk of the per-cell kernels (256 .. 2^24).  Chosen by the
 * autotuner of the Python package; results do not depend on it.  Synchronises the device
 * when the work lists change. */
ase_df_status ase_df_batch_set_schedule(ase_df_batch* b, int32_t ctas_per_sm, int32_t order_by_cost,
                                        int32_t chunk_cells);

/* Tile shape of the 2D sweeps per scheme order: lines[k] (k = 0..3 for orders 3, 5, 7, 9) is
 * 64 (tiles of 8 x 64 faces, two faces per thread) or 32 (8 x 32, one face per thread).
 * Chosen by the autotuner of the Python package; results do not depend on it.  Synchronises
 * the device when the tiles change. */
ase_df_status ase_df_batch_set_tiles(ase_df_batch* b, const int32_t* lines);

/* Message of the last error on this batch (or of the last failed ase_df_batch_init when
 * b is NULL). */
const char* ase_df_batch_last_error(const ase_df_batch* b);

/* FP64 throughput microbenchmark used as the roofline denominator: independent FMA
 * chains on every SM; writes the achieved FP64 FMA instructions per second into
 * *fma_per_s (flops = 2x).  Synchronises the device. */
ase_df_status ase_df_fp64_fma_rate(double* fma_per_s);

/* Check of the face kernel's own FP64 reciprocal and reciprocal square root (an FP32
 * approximation refined by one third-order Newton-Raphson step; the paper has no
 * counterpart): for the n device doubles x[i] writes out[4i .. 4i+3] = (own 1/x, CUDA's
 * 1/x, own 1/sqrt(x), CUDA's rsqrt(x)).  out holds 4n device doubles.  Asynchronous on
 * stream. */
ase_df_status ase_df_check_recip(const double* x, double* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ASE_DF_H */

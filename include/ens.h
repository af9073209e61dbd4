/*
 * ens.h -- C ABI of the GB300-native ensemble ODE solver.
 *
 * The library integrates very many independent, low-dimensional, non-stiff
 * ODE systems, one parameter set each, the workload of Nagy, Plavecz &
 * Hegedus, arXiv 2011.01740 ("Solving large number of non-stiff,
 * low-dimensional ordinary differential equation systems on GPUs and CPUs").
 * One GPU thread owns one system at a time (the "per-thread approach",
 * Sec. 3.2.1); state, Runge-Kutta stages and parameters live in registers.
 *
 * Conventions shared by every entry point:
 *   - Arrays are structure-of-arrays: element k of system i sits at
 *     [k * n + i].  All floating-point data are IEEE double.
 *   - Input pointers may be host or device memory (told apart with
 *     cudaPointerGetAttributes); the library copies what it needs and the
 *     caller keeps ownership.  Output buffers are caller-owned; `dst` of
 *     ens_read may likewise be host or device memory.
 *   - Every call returns an ens_status.  Nothing aborts, traps or prints; the
 *     text of the last failure is available through ens_last_error.  Per-system
 *     failures (step-size underflow, step budget, ...) are reported as status
 *     words (ENS_SYS_*), not as call failures.
 *   - A context is bound to the CUDA device that was current at ens_create and
 *     must be used from one host thread at a time.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Work is enqueued asynchronously; ens_sync waits.
 */
#ifndef ENS_H
#define ENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ens_ctx ens_ctx;

/* Call status. */
typedef enum {
    ENS_OK = 0,
    ENS_EINVAL = 1,    /* bad argument (sizes, enums, NULL pointers, tolerances) */
    ENS_ENOMEM = 2,    /* device or host allocation failed                        */
    ENS_ECUDA = 3,     /* a CUDA runtime call failed (message in ens_last_error)   */
    ENS_ETIMEOUT = 4,  /* the solve hit its wall-clock budget (systems flagged)    */
    ENS_ESYSTEM = 5,   /* the solve finished but some systems carry a status word  */
    ENS_ENOTSUP = 6    /* combination not supported (e.g. RK4 with events)         */
} ens_status;

/* Built-in right-hand sides (inlined device functions).
 *   ENS_SYS_TOY_X2P        x' = x^2 - p                      (Sec. 3, Eq. exemplary_system)
 *                          dim 1, params [p]
 *   ENS_SYS_LORENZ         x1' = sigma (x2 - x1), x2' = rho x1 - x2 - x1 x3,
 *                          x3' = x1 x2 - b x3                (Sec. 4.1, Eqs. Lorenz1-3)
 *                          dim 3, params [rho, sigma, b]
 *   ENS_SYS_KELLER_MIKSIS  dimensionless Keller-Miksis, y1' = y2, y2' = N_KM / D_KM
 *                          (Sec. 4.2, Eqs. dimensionless_system1-2, numerator,
 *                          denominator); dim 2, params [C0..C12] (Eq. coefficients,
 *                          see ens_km_coefficients); tau is the phase-local time.
 *   ENS_SYS_RELIEF_VALVE   y1' = y2, y2' = -kappa y2 - (y1 + delta) + y3,
 *                          y3' = beta (q - y1 sqrt(y3))     (Sec. 4.3, Eqs.
 *                          pressure_relief_valve_1-3) with the impact law
 *                          y1 <- 0, y2 <- -r y2 (Eqs. impact_law_1-3);
 *                          dim 3, params [q, kappa, delta, beta, r]
 *   ENS_SYS_KELLER_MIKSIS_TANGENT
 *                          Keller-Miksis with its tangent (variational)
 *                          equation v' = J(y) v for the largest Lyapunov
 *                          exponent; dim 4 (y1, y2, v1, v2), params as
 *                          Keller-Miksis; phase mode only, FP64.  v is scaled
 *                          to unit length at the start and at every phase end
 *                          (renormalisation between phases, Sec. 1), and
 *                          ln |v| at each recorded phase end is an extra
 *                          accessory row (see ens_acc_rows).                */
typedef enum {
    ENS_SYS_TOY_X2P = 0,
    ENS_SYS_LORENZ = 1,
    ENS_SYS_KELLER_MIKSIS = 2,
    ENS_SYS_RELIEF_VALVE = 3,
    ENS_SYS_KELLER_MIKSIS_TANGENT = 4
} ens_system;

/* Steppers: classic RK4 with fixed steps (Sec. 3, Sec. 4.1), the adaptive
 * Cash-Karp 4(5) pair with error control (Sec. 4.2.1, Sec. 4.3.1; tableau of
 * Cash & Karp, ACM TOMS 16(3), 1990), and the Dormand-Prince 5(4) pair of the
 * paper's Julia runs (Sec. 4.2; Dormand & Prince, J. Comput. Appl. Math. 6,
 * 1980) with the same controller, reusing its seventh stage as the next
 * step's first (ENS_NRHS counts 6 per trial plus one per fresh start). */
typedef enum { ENS_RK4 = 0, ENS_RKCK45 = 1, ENS_DOPRI5 = 2 } ens_solver;

/* Arithmetic of the kernels.
 *   ENS_FP64         IEEE double with fused multiply-add (the default path).
 *   ENS_FP64_STRICT  IEEE double, no contraction, operations in the order the
 *                    equations are written: bit-reproducible against a plain
 *                    C evaluation of the same formulas (RK4 systems only).
 *   ENS_FP32_COMP    right-hand side and stage sums in float with compensated
 *                    (Kahan) stage combination and a float-pair (hi + lo)
 *                    state; time, error norm, controller and event root in
 *                    double (Keller-Miksis / Cash-Karp only).
 *   ENS_FP32X2       double-float: every value of the step (state, stages,
 *                    right-hand side, error estimate, controller) is a pair
 *                    of floats, about 48 significant bits, on the FP32
 *                    pipes; the time, the step and the forcing sin / cos are
 *                    double.  Keller-Miksis phase mode with Cash-Karp and
 *                    C10 = 21/5 only (else ENS_ENOTSUP from ens_solve).     */
typedef enum { ENS_FP64 = 0, ENS_FP32_COMP = 1, ENS_FP64_STRICT = 2, ENS_FP32X2 = 3 } ens_precision;

/* Per-system status bits (ENS_STATUS). */
enum {
    ENS_SYS_DT_UNDERFLOW = 1,        /* rejected step proposal fell below dt_min  */
    ENS_SYS_MAX_STEPS = 2,           /* trial-step budget max_steps exhausted      */
    ENS_SYS_NONFINITE = 4,           /* final state not finite (fixed-step solve)  */
    ENS_SYS_EVENT_NO_CONVERGE = 8,   /* more than 40 event-location retries        */
    ENS_SYS_TIMEOUT = 16             /* solve budget timeout_s ran out             */
};

/* ens_read selectors and the layout each returns (n = ensemble size). */
enum {
    ENS_STATE = 0,    /* double [dim][n]   state at the end of the solve          */
    ENS_ACC = 1,      /* double [rows][n]  accessories, see ens_acc_rows          */
    ENS_STATUS = 2,   /* int32  [n]        ENS_SYS_* bits                         */
    ENS_NSTEPS = 3,   /* int64  [n]        accepted steps                         */
    ENS_NREJ = 4,     /* int64  [n]        steps rejected by the error test       */
    ENS_NRHS = 5,     /* int64  [n]        right-hand-side evaluations            */
    ENS_TIME = 6,     /* double [n]        final time (phase-local for phases)    */
    ENS_DT = 7        /* double [n]        final step-size proposal               */
};

/* Solver settings.
 *   rtol, atol     error test: accept iff max_i |y5_i - y4_i| /
 *                  (atol + rtol max(|y_i|, |y5_i|)) <= 1.  The new step is
 *                  h * clamp(0.9 E^(-1/5), 0.2, 5) bounded by [dt_min, dt_max]
 *                  (the paper states tolerances only; this controller is the
 *                  library's reading).
 *   dt0            first step (adaptive) or the fixed step (RK4).
 *   n_steps        RK4 only: number of fixed steps (t_span[1] is ignored).
 *   event_tol      absolute event tolerance (relief valve, Sec. 4.3.1).
 *   max_steps      cap on trial steps per system (ENS_SYS_MAX_STEPS).
 *   n_phases       > 0: phase mode (Keller-Miksis, Sec. 4.2): n_phases
 *                  integrations over tau in [t_span[0], t_span[0] + phase_len],
 *                  tau reset at each phase start; accessories per phase.
 *   acc_t_start    relief valve: the y1 minimum accessory covers t >= it.
 *   n_transient    phase mode: the first n_transient phases are integrated but
 *                  not recorded (the paper's transient phases, Sec. 4.2);
 *                  0 <= n_transient < n_phases (0 outside phase mode).
 *   prec           ens_precision.
 *   timeout_s      wall-clock budget of one ens_solve on the device; systems
 *                  still running are stopped with ENS_SYS_TIMEOUT (<= 0: 600 s). */
typedef struct {
    double rtol, atol;
    double dt0, dt_min, dt_max;
    double event_tol;
    int64_t max_steps;
    int64_t n_steps;
    int32_t n_phases;
    int32_t prec;
    double phase_len;
    double acc_t_start;
    double timeout_s;
    int32_t n_transient;
} ens_tol;

/* Launch configuration (see ens_set_launch / ens_autotune).
 *   mode           ENS_LAUNCH_PLAIN: one system per thread, grid covers n.
 *                  ENS_LAUNCH_PERSISTENT: a fixed grid of lanes; every lane
 *                  claims its next system from a device counter (atomicAdd)
 *                  when its current one finishes (work stealing), so uneven
 *                  adaptive step counts do not idle warps.
 *   block          threads per block (multiple of 32, 32..256).
 *   blocks_per_sm  persistent mode: resident blocks per SM (grid = SMs x this).
 *   use_graph      capture the launch sequence of ens_solve in a CUDA graph on
 *                  the first call and replay it afterwards.
 *   cost_order     persistent mode: claim systems in decreasing order of their
 *                  step count in a one-phase pilot solve (longest first).
 *   systems_per_thread  systems integrated by each thread, their steps
 *                  interleaved in one instruction stream (0 means 1); each
 *                  system's arithmetic is that of one per thread, so results
 *                  do not change.  RK4: 1, 2 or 4.  Adaptive: 1, or 2 for the
 *                  FP64 Cash-Karp phase mode of the Keller-Miksis model with
 *                  one driving frequency and C10 = 21/5, persistent mode, at
 *                  most 128 threads per block (both slots of a lane claim
 *                  systems; each iteration computes both slots' trials).
 *                  Other combinations: ENS_ENOTSUP from ens_set_launch, or
 *                  from ens_solve where the parameters decide (a second
 *                  frequency or another exponent). */
enum { ENS_LAUNCH_PLAIN = 0, ENS_LAUNCH_PERSISTENT = 1 };
typedef struct {
    int32_t mode;
    int32_t block;
    int32_t blocks_per_sm;
    int32_t use_graph;
    int32_t cost_order;
    int32_t systems_per_thread;
    int32_t reserved[2];
} ens_launch;

/* One candidate of the last ens_autotune: its launch, the device time in
 * milliseconds of the main kernel of the shortened solve it was timed on, and
 * the fraction of the horizon that solve covered. */
typedef struct {
    ens_launch launch;
    double ms;
    double horizon_frac;
} ens_tune_row;

/* Liquid and gas constants of the Keller-Miksis model (SI units):
 * density rho_L, sound speed c_L, viscosity mu_L, surface tension sigma,
 * vapour pressure p_V, ambient pressure P_inf, polytropic exponent gamma. */
typedef struct {
    double rho, c, mu, sigma, pv, pinf, gamma;
} ens_liquid;

/* ------------------------------------------------------------------------ */

/* Create a solver context for n systems of kind `sys`.
 *   params   SoA [npar][n] (host or device), copied.
 *   y0       SoA [dim][n]  (host or device), copied: the state at t_span[0].
 *   t_span   {t0, t1} on the host: integration interval (event mode / plain
 *            adaptive), or t0 = phase start for phase mode.
 *   solver   ens_solver; tol: settings above (copied).
 * n = 0 is valid (every later call is a no-op).  Errors: ENS_EINVAL for a
 * NULL out/params/y0/tol (when n > 0), unknown enums, non-positive tolerances
 * or steps; ENS_ENOMEM; ENS_ECUDA.  On failure *out is NULL. */
ens_status ens_create(ens_ctx **out, ens_system sys, int64_t n, const double *params,
                      const double *y0, const double t_span[2], ens_solver solver,
                      const ens_tol *tol);

/* Replace the parameters and initial states of an existing context (same
 * layout and sizes as ens_create; host or device pointers), enqueued on
 * `stream`.  Either pointer may be NULL to keep the current values. */
ens_status ens_set_inputs(ens_ctx *ctx, const double *params, const double *y0, void *stream);

/* Select the launch configuration.  NULL restores the built-in default. */
ens_status ens_set_launch(ens_ctx *ctx, const ens_launch *cfg);

/* Read back the launch configuration in use. */
ens_status ens_get_launch(const ens_ctx *ctx, ens_launch *cfg);

/* Integrate every system from its initial state (the inputs are not
 * modified, so repeated calls give repeated results).  Asynchronous on
 * `stream`; results become readable in stream order. */
ens_status ens_solve(ens_ctx *ctx, void *stream);

/* Wait for the context's last solve.  Returns ENS_OK, ENS_ETIMEOUT when any
 * system hit the wall-clock budget, ENS_ESYSTEM when any system carries
 * another status bit, or ENS_ECUDA. */
ens_status ens_sync(ens_ctx *ctx);

/* Device time in milliseconds of the main solve kernel of the context's last
 * solve (CUDA events recorded on the solve's stream right before and after
 * that launch, also when the solve replays a CUDA graph).  It excludes the
 * planning work that ens_solve may run first (the one-phase pilot and the
 * claim-order sort of cost_order).  The paper has no counterpart: a
 * measurement hook for the kernel-level roofline.  Call after ens_sync;
 * ENS_EINVAL before the first solve, ENS_ECUDA if the events are not
 * complete. */
ens_status ens_kernel_ms(ens_ctx *ctx, double *ms);

/* Copy one output (selector ENS_*) into dst (host or device), which must hold
 * at least the size the selector's layout gives; dst_bytes smaller than that
 * is ENS_EINVAL.  Synchronous with respect to the context's last stream. */
ens_status ens_read(ens_ctx *ctx, int which, void *dst, size_t dst_bytes);

/* Number of accessory rows of ENS_ACC for this context:
 *   phase mode (Keller-Miksis): 2 * (n_phases - n_transient), row 2k = max y1
 *     in phase n_transient + k, row 2k+1 = its min y1, taken over the natural
 *     step points and the phase start (no dense output, Sec. 4.2.1);
 *   tangent system: 3 * R with R = n_phases - n_transient, the 2R rows above
 *     and then row 2R + k = ln |v| at the end of recorded phase k (the
 *     tangent vector's growth over that phase; their mean over phases divided
 *     by phase_len estimates the largest Lyapunov exponent);
 *   relief valve: 35 rows: rows 0..31 ring of the last Poincare maxima of y1
 *     (slot m mod 32 holds maximum number m; NaN if unused), row 32 the
 *     minimum of y1 for t >= acc_t_start, row 33 the number of maxima, row 34
 *     the number of impacts (Sec. 4.3);
 *   otherwise 0. */
int64_t ens_acc_rows(const ens_ctx *ctx);

/* Ensemble size, state dimension and parameter count of a context. */
int64_t ens_size(const ens_ctx *ctx);
int32_t ens_dim(const ens_ctx *ctx);
int32_t ens_npar(const ens_ctx *ctx);

/* Autotuner (the paper tunes block size and registers by hand, Sec. 3.2.2
 * and Sec. 4.1.2).  Times candidate launches on this context with shortened
 * solves on `stream`, keeps the fastest as the context's launch (use_graph is
 * kept) and writes it to *best (may be NULL).
 *   RK4: block 32..256 x systems_per_thread 1, 2, 4, each timed twice (the
 *   faster time counts and is the one in the table), on the whole solve up
 *   to 1e9 system-steps, else on 1/8 of the steps.
 *   Adaptive: persistent launches of 3 to 24 warps per SM with longest-first
 *   claiming, the best residency without it, a plain launch and, where the
 *   kernel exists, two systems per thread at 6 and 8 warps per SM, each on
 *   1/8 of the phases (or of the time span) of every system -- the horizon is
 *   cut, not the ensemble, so the balance between throughput and the
 *   longest system's chain stays that of the full solve; the fraction is
 *   halved while one shortened solve takes over 0.6 s.  The two fastest
 *   candidates are then timed again on twice that horizon (rows with the
 *   doubled horizon_frac), and the faster of those two is the choice: shapes
 *   with different tails can trade places as the horizon grows.  The claim
 *   order comes from the full solve's one-phase pilot, computed once.
 * The context's outputs hold the last candidate's shortened solve afterwards.
 * The choice and its table are cached per (system, solver, precision, n,
 * phases, transient phases, horizon, device) for the process. */
ens_status ens_autotune(ens_ctx *ctx, void *stream, ens_launch *best);

/* The candidates timed by the context's last ens_autotune, in the order
 * tried: copies up to `cap` rows into `rows` (may be NULL) and returns how
 * many there are (0 for a NULL ctx or before any tuning). */
int32_t ens_autotune_table(const ens_ctx *ctx, ens_tune_row *rows, int32_t cap);

/* Text of the context's last failure ("" if none).  ctx may be NULL: then the
 * last failure of a call that had no context (ens_create) is returned. */
const char *ens_last_error(const ens_ctx *ctx);

/* Free the context and its device buffers (NULL is a no-op). */
void ens_destroy(ens_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Host planner                                                              */

/* Keller-Miksis coefficients C0..C12 of Sec. 4.2 (Eq. coefficients) for n
 * systems from physical SI parameters: pressure amplitudes pA1, pA2 [Pa],
 * frequencies f1, f2 [Hz], phase shift theta [rad], equilibrium radius RE [m].
 * C8 is taken with omega2 (the time derivative of the second driving term);
 * the printed C8 carries omega1, which is the same whenever pA2 = 0.
 * All arrays live on the same side (all host or all device); out is SoA
 * [13][n].  Device arrays are processed by a kernel on `stream`. */
ens_status ens_km_coefficients(int64_t n, const double *pA1, const double *f1, const double *pA2,
                               const double *f2, const double *theta, const double *RE,
                               const ens_liquid *liquid, double *out, void *stream);


/* ------------------------------------------------------------------------ */
/* Surrogate screening (learned extension of the Keller-Miksis sweep)         */
/*
 * A small ensemble of multilayer perceptrons maps the driving of a bubble,
 * x = (log p_A, log f) scaled to [-1, 1] (ens_km_features), to
 * y0 = ln(max y1 over the recorded periods) and the logit of y1 = "period-1
 * response" (ens_km_labels).  Each member is 2 -> 128 -> 128 -> 128 -> 128 -> 2
 * with GELU (erf form) after the first four layers; weights are kept as FP32
 * masters with BF16 copies, the 128 x 128 products run on the tensor cores
 * with FP32 accumulation.  The screening forward returns the mean and the
 * population standard deviation of y0 over the members and the mean
 * period-1 probability; points whose spread exceeds a threshold are handed
 * back to the FP64 solver (ens_select_above, ens_gather_f64, the solver
 * calls above, ens_scatter_labels).  The paper has no surrogate: this part
 * is an extension of its parameter sweeps (Sec. 4.2).
 *
 * Parameter vector of one member (floats, in this order, W stored [out][in]):
 *   W1[128][2] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
 *   W4[128][128] b4[128] W5[2][128] b5[2]              (ens_mlp_param_count())
 * Loss per sample: (out0 - y0)^2 + binary cross-entropy with logits of
 * (out1, y1), averaged over the batch; Adam on every parameter.
 * Unless stated otherwise, array arguments are device memory
 * (ENS_EINVAL otherwise) and work is enqueued on `stream`.
 */
typedef struct ens_mlp ens_mlp;

typedef struct {
    int32_t epochs;        /* passes over the training set                      */
    int32_t batch;         /* samples per Adam step                             */
    float lr, beta1, beta2, eps;   /* Adam (Kingma & Ba 2015)                    */
    uint64_t seed;         /* shuffle stream (splitmix64)                        */
    float lr_final;        /* > 0: cosine decay of the Adam step size from lr
                              (first step) to lr_final (last step) over all
                              epochs (Loshchilov & Hutter 2017, no restarts);
                              0: constant lr                                     */
} ens_train_cfg;

/* Create `members` (1..8) networks; weights uniform in +-1/sqrt(fan_in),
 * biases 0, member k drawn from the splitmix64 stream seed + k. */
ens_status ens_mlp_create(ens_mlp **out, int32_t members, uint64_t seed);
/* Number of floats in one member's parameter vector (50,178). */
int64_t ens_mlp_param_count(void);
/* Copy all members' parameters in / out ([members][param_count] floats,
 * host or device); set_params also resets the Adam moments. */
ens_status ens_mlp_set_params(ens_mlp *m, const float *params, size_t bytes);
ens_status ens_mlp_get_params(ens_mlp *m, float *params, size_t bytes);
/* Raw outputs of every member: x [n][2] -> out [members][n][2]. */
ens_status ens_mlp_forward(ens_mlp *m, int64_t n, const float *x, float *out, void *stream);
/* Loss (per member, host array [members]) and gradient ([members][param_count],
 * host or device) of one batch; synchronous. */
ens_status ens_mlp_loss_grad(ens_mlp *m, int64_t n, const float *x, const float *y, float *loss,
                             float *grad, void *stream);
/* Train on n samples (x [n][2], y [n][2]) with shuffled mini-batches; loss_hist
 * (host, may be NULL) receives the mean per-sample loss of each epoch and
 * member ([epochs][members]).  Synchronous. */
ens_status ens_mlp_train(ens_mlp *m, int64_t n, const float *x, const float *y, const ens_train_cfg *cfg,
                         float *loss_hist, void *stream);
/* Fused ensemble inference: mean[n], stdv[n] (population standard deviation
 * of output 0 over the members), p1[n] (mean sigmoid of output 1). */
ens_status ens_mlp_screen(ens_mlp *m, int64_t n, const float *x, float *mean, float *stdv, float *p1,
                          void *stream);
/* Choose the screening kernel: 1 (default) the tcgen05 kernel (accumulators
 * in tensor memory, one CTA per SM per member), 0 the mma.sync kernel that
 * fuses all members in one block.  If wait_expired is not NULL it receives
 * 1 when a tcgen05 launch since the last call gave up waiting for its tensor
 * cores (its outputs are then invalid), else 0. */
ens_status ens_mlp_set_screen_impl(ens_mlp *m, int32_t impl, int32_t *wait_expired);
/* Choose the training products (ens_mlp_forward, ens_mlp_loss_grad,
 * ens_mlp_train): 1 (default) the tcgen05 kernels (forward, input gradients
 * and the weight gradients of the three 128 x 128 layers with accumulators in
 * tensor memory), 0 the mma.sync kernels.  Both take BF16 operands with FP32
 * accumulation; the 2-wide first and last layers are FP32 in both.  If
 * wait_expired is not NULL it receives 1 when a tcgen05 training launch gave
 * up waiting for its tensor cores since the flag was last cleared (by each
 * ens_mlp_loss_grad and ens_mlp_train call, which then return ENS_ECUDA),
 * else 0. */
ens_status ens_mlp_set_train_impl(ens_mlp *m, int32_t impl, int32_t *wait_expired);
const char *ens_mlp_last_error(const ens_mlp *m);
void ens_mlp_destroy(ens_mlp *m);

/* Features x[n][2] = 2 (ln v - ln lo) / (ln hi - ln lo) - 1 for v = pA and f
 * with range = {pA_lo, pA_hi, f_lo, f_hi} (host array, all > 0). */
ens_status ens_km_features(int64_t n, const double *pA, const double *f, const double range[4], float *x,
                           void *stream);
/* Targets y[n][2] from phase-mode accessories acc[2 n_phases][n]: y0 = ln of
 * the largest per-phase maximum over phases [first_phase, n_phases), y1 = 1
 * if those per-phase maxima spread by less than spread_tol (relative). */
ens_status ens_km_labels(int64_t n, const double *acc, int32_t n_phases, int32_t first_phase,
                         double spread_tol, float *y, void *stream);
/* idx[0..*count) = increasing indices i with v[i] > thr (idx holds n
 * entries); *count is written on the host; synchronous. */
ens_status ens_select_above(int64_t n, const float *v, float thr, int32_t *idx, int64_t *count, void *stream);
/* The same with two gates: i is selected when v[i] > thr or, if w is not
 * NULL, w[i] > thr_w (the screening fallback: ensemble spread above its
 * threshold, or a steep region of the predicted map). */
ens_status ens_select_gate(int64_t n, const float *v, float thr, const float *w, float thr_w, int32_t *idx,
                           int64_t *count, void *stream);
/* Steepness of a map v on a rows x cols grid (row-major, columns fastest)
 * with feature-space spacings d_row, d_col > 0 between adjacent points:
 * g = the largest |v(neighbour) - v| / distance over the up to four points
 * `stride` >= 1 rows or columns away.  Where the predicted map is steep the
 * training grid resolves the response least, so the screen hands those
 * points to the solver as well; a stride that keeps the distance near the
 * training grid's spacing measures the map's slope rather than the
 * rounding noise of the network's output. */
ens_status ens_grid_gradient(int64_t rows, int64_t cols, int64_t stride, const float *v, float d_row, float d_col,
                             float *g, void *stream);
/* out [5][n][2]: for each feature point x[n][2], the points x, x +- d0 e0,
 * x +- d1 e1 (e0, e1 the feature axes); with ens_mlp_screen over the 5 n
 * points and ens_stencil_gradient it gives the grid gradient's steepness at
 * scattered points (the calibration sample of the screening gate). */
ens_status ens_feature_stencil(int64_t n, const float *x, float d0, float d1, float *out, void *stream);
/* g[i] = max(|v[n+i] - v[i]|, |v[2n+i] - v[i]|) / d0 max'ed with
 * max(|v[3n+i] - v[i]|, |v[4n+i] - v[i]|) / d1, for v [5][n] evaluated at the
 * points of ens_feature_stencil. */
ens_status ens_stencil_gradient(int64_t n, const float *v, float d0, float d1, float *g, void *stream);
/* dst[i] = src[idx[i]] for i < k. */
ens_status ens_gather_f64(int64_t k, const int32_t *idx, const double *src, double *dst, void *stream);
/* dst[idx[i]] = y[i][0] for i < k (writes re-solved values into a screened map). */
ens_status ens_scatter_labels(int64_t k, const int32_t *idx, const float *y, float *dst, void *stream);

/* One right-hand-side evaluation per system with the device code the solvers
 * inline: dy[dim][n] = f(t[i], y[:, i]; params[:, i]).  All arrays device
 * memory; for Keller-Miksis the same kernel variant as the solver is chosen
 * (second frequency, rational exponent).  Synchronous for the variant choice,
 * the evaluation itself is enqueued on `stream`. */
ens_status ens_eval_rhs(ens_system sys, int64_t n, const double *params, const double *t, const double *y,
                        double *dy, void *stream);

/* Allocation-free adaptive solve (the paper has no counterpart: it concerns
 * how the library is embedded, not the method).
 *
 * For callers that cannot allocate device memory themselves or through this
 * library: processes whose device memory belongs to another allocator (a
 * framework's caching pool, a preallocated arena of a real-time or embedded
 * deployment) that must not be bypassed or fragmented, and plugins that are
 * only handed device buffers by their host.  ens_create allocates; this call
 * does not.  It runs the same persistent, work-stealing Cash-Karp kernel as
 * ens_solve (FP64; Keller-Miksis in phase mode, or the relief valve with
 * events) directly on caller-owned device buffers laid out as ens_read
 * returns them:
 *   params [npar][n], y0 [dim][n]                       inputs (not modified)
 *   y [dim][n], t_out [n], dt_out [n], acc [rows][n],
 *   status [n] (int32), nacc, nrej, nrhs [n] (int64)    outputs
 * (rows as ens_acc_rows would give: 2 (n_phases - n_transient), or 35 for
 * the relief valve).
 * cost_order != 0 claims systems longest first after a one-phase pilot
 * (written into the output buffers, then overwritten).
 *
 * Its only other memory is a fixed ~4.2 MB array in the library's device
 * globals (claim counter, status OR, claim order): every GPU that loads the
 * library holds it until the process exits, which caps n at 1,048,576
 * systems (larger n is ENS_EINVAL with a message in ens_last_error(NULL)).
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with that device current); make it before any
 * stream capture.  Calls share the array: the counter and the status OR are
 * cleared at the start of every call, and calls that overlap on the GPU (on
 * different streams, or from different host threads) race on it.  No call
 * to cudaMalloc, cudaFree or any allocating routine is made.  Work is
 * enqueued on `stream` (one small synchronous read selects the
 * Keller-Miksis kernel variant).  The solver settings are validated as
 * ens_create validates them.  Every array must be device memory of the
 * current device, or managed memory; device memory of another GPU is
 * refused, since the kernel would reach it as a peer address.  Returns
 * ENS_OK, ENS_EINVAL (arguments, n above the cap, arrays that are not
 * addressable as above), ENS_ENOTSUP (other systems or precisions) or
 * ENS_ECUDA. */
ens_status ens_solve_noalloc(ens_system sys, int64_t n, const double *params, const double *y0,
                             const double t_span[2], const ens_tol *tol, double *y, double *t_out,
                             double *dt_out, double *acc, int32_t *status, int64_t *nacc, int64_t *nrej,
                             int64_t *nrhs, int32_t cost_order, void *stream);

/* Library version string. */
const char *ens_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ENS_H */

/*
 * kzk.h -- C ABI of the B300 (sm_103a) ExpRK22 / WENO5 / FFT propagator for the
 * KZK-type sonic-boom equation of Einkemmer, Ostermann & Residori,
 * "An exponential integrator/WENO discretization for sonic-boom simulation on
 * modern computer hardware" (arXiv:2103.06080).
 *
 * The operation advanced by kzk_advance is one step of the second-order
 * exponential Runge-Kutta scheme ExpRK22 (Eq. 5), evaluated in Fourier space
 * (Eq. 11, Algorithm 2 STEP 1-4), for
 *     d_sigma V = L V + b(sigma, V),                                 (Eq. 2a)
 *     L = diffraction * d_tau^{-1} d_y^2 + A d_tau^2                 (Eq. 2)
 *     b = (B(sigma)/2) d_tau V^2 + (A(sigma) - A) d_tau^2 V          (Eq. 3)
 * on a grid periodic in retarded time tau (x, contiguous) and transverse y
 * (Sec. 3.3).  b's flux derivative is discretised with WENO5 (Jiang-Shu
 * weights, global Lax-Friedrichs splitting with alpha = B(sigma) * lf_umax)
 * on the gradient form of Eq. 7; L is applied exactly through the diagonal
 * tables E = e^z, Phi1 = (e^z - 1)/z, Phi2 = (e^z - 1 - z)/z^2 with
 *     z = dsigma * ( -diffraction * k_y^2 / (i k_tau + reg_eps * diffraction)
 *                    - A k_tau^2 )                                   (Eq. 11)
 * (the regularised multiplier of the paper; at the tau-Nyquist frequency only
 * the even part -A k_tau^2 is kept).  Wavenumbers are physical:
 * k = 2 pi m / (max - min) for the signed FFT index m.
 *
 * Conventions for every entry point:
 *   - All state buffers are owned by the caller, contiguous, row-major
 *     [batch][ny][nx] (tau fastest), of the plan's precision (double for
 *     KZK_FP64, float for KZK_FP32).  "device" pointers must be CUDA device
 *     memory of the current device; "host" pointers ordinary host memory.
 *   - The plan owns its tables and workspace (device memory, allocated in
 *     kzk_plan_create, freed in kzk_plan_destroy).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; calls that return host data synchronise it.
 *   - No exception crosses the ABI.  Every function returns a kzk_status;
 *     kzk_last_error() gives a one-line description of the last failure on
 *     the calling thread.  CUDA errors map to KZK_ERR_CUDA.
 *   - A plan is not thread-safe: use it from one host thread and one stream
 *     at a time.
 */
#ifndef KZK_H
#define KZK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KZK_OK = 0,
    KZK_ERR_ARG = 1,        /* null pointer, bad enum, non-positive extent, bad dt      */
    KZK_ERR_SIZE = 2,       /* grid size not supported (see kzk_grid)                   */
    KZK_ERR_CFL = 3,        /* max|u| exceeded lf_umax (LF splitting no longer upwind)  */
    KZK_ERR_NONFINITE = 4,  /* a NaN or Inf appeared in the state                       */
    KZK_ERR_CUDA = 5,       /* a CUDA runtime call failed                                */
    KZK_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up                       */
    KZK_ERR_OOM = 7,        /* device allocation failed                                 */
    KZK_ERR_STATE = 8       /* call not valid for this plan (e.g. wrong plan kind)      */
} kzk_status;

typedef enum { KZK_FP64 = 0, KZK_FP32 = 1 } kzk_precision;

/* Grid of Sec. 3.3: tau_k = tau_min + k (tau_max - tau_min)/nx, y_j likewise. */
typedef struct {
    int32_t nx, ny;                 /* nx: tau points (contiguous), ny: y points; either
                                       powers of two in [8, 8192] x [2, 4096], or even
                                       sizes in [8, 16384] x [2, 32768] with nx/2 and ny
                                       free of prime factors above 7 (the paper's
                                       7*2^k x 1250*2^k grids, Table 1: mixed-radix
                                       transforms) */
    double tau_min, tau_max, y_min, y_max;
    int32_t prec;                   /* kzk_precision of state and bulk arithmetic.
                                       KZK_FP32 plans keep the spectral state as a
                                       compensated pair hi + lo (FP32 hi, bf16 lo) by
                                       default: the column passes transform only the
                                       increment of a stage ((E - 1) V + dsigma Phi1 b1 of
                                       Eq. 11) and add it to hi + lo exactly (TwoSum), so the
                                       rounding of a full-state transform pair does not
                                       accumulate over thousands of steps (kzk_options
                                       selects a plain FP32 state instead). */
} kzk_grid;

#define KZK_MAX_RELAX 2

/* Coefficients of Eq. 0 / Eq. 2a.  B(sigma) = B * pB(sigma) and
 * A(sigma) = A * pA(sigma) with cubic pX(sigma) = c0 + c1 s + c2 s^2 + c3 s^3
 * when has_profile != 0 (stratified atmosphere), else constant.
 * Relaxation (optional, n_relax processes): each adds C_r d_tau^2 q_r to the
 * linear operator, q_r the causal solution of theta_r dq_r/dtau + q_r = V,
 * i.e. the multiplier C_r (i k_tau)^2 / (1 + i theta_r k_tau) in z of Eq. 11
 * (at the tau-Nyquist frequency its real part only).  The paper's operator
 * has none (n_relax = 0). */
typedef struct {
    double B;                       /* nonlinearity, > 0                             */
    double A;                       /* absorption, >= 0 (kept exactly in L)          */
    double diffraction;             /* 1/(4 pi) in the paper; <= 0 selects 1/(4 pi)   */
    double reg_eps;                 /* epsilon of z; <= 0 selects 2^-53, the epsilon of the FP64 table
                                       generation used by both plan precisions */
    double weno_eps;                /* Jiang-Shu epsilon; <= 0 selects 1e-6          */
    double lf_umax;                 /* M of the LF speed alpha = B(sigma) * M, > 0   */
    double B_prof[4];
    double A_prof[4];
    int32_t has_profile;
    int32_t n_relax;                /* relaxation processes, 0 .. KZK_MAX_RELAX      */
    double relax_C[KZK_MAX_RELAX];  /* strengths C_r >= 0                            */
    double relax_theta[KZK_MAX_RELAX]; /* relaxation times theta_r > 0 (tau units)   */
    int32_t method;                 /* KZK_EXPRK22 (0, Eq. 5) or KZK_EXPEULER (1: the
                                       exponential Euler scheme of Sec. 3.2, first order:
                                       the first stage of Eq. 5 taken as the step) */
} kzk_coeffs;

#define KZK_EXPRK22 0
#define KZK_EXPEULER 1

/* Diagnostics (FP64): of the state after the last step, and over the run. */
typedef struct {
    double mean;                    /* sum u / (nx ny)                               */
    double energy;                  /* dtau dy sum u^2                               */
    double max_abs;                 /* max |u|                                       */
    double nonfinite;               /* number of NaN/Inf values                      */
    double run_max_abs;             /* max over the states at the start of each step and the final one */
    double run_nonfinite;           /* NaN/Inf count summed over those states        */
} kzk_diag;

typedef struct kzk_plan_s kzk_plan;

/* Kernel and state choices of a plan (kzk_plan_create_ex).  Zero-initialise
 * and set only what should be pinned: all zero (KZK_AUTO) gives the defaults
 * below, which are what kzk_plan_create uses.  A choice the grid or the
 * precision cannot take is refused with KZK_ERR_SIZE (kernel choices) or
 * KZK_ERR_ARG (unknown values).  kzk_plan_info reports the choices in effect. */
#define KZK_AUTO 0
/* row_kernel: the tau passes (C2R, WENO5, R2C of one row)                    */
#define KZK_ROW_PAIR 1          /* KZK_FP32, even ny: two rows per CTA as the lanes of
                                   packed FP32 values (default for those plans)        */
#define KZK_ROW_SINGLE 2        /* one row per CTA (default and only choice for KZK_FP64
                                   and mixed-radix grids)                               */
/* col_kernel: the y passes (transforms fused with the phi-multiplies)        */
#define KZK_COL_PAIR 1          /* KZK_FP32 with the compensated state, 256 <= ny <= 4096,
                                   nx >= 8: two spectral columns per CTA in packed FP32,
                                   in-place transforms, tiles staged by the tensor memory
                                   accelerator (default for those plans)               */
#define KZK_COL_TMA 2           /* Stockham tiles staged by the tensor memory
                                   accelerator (default for the other KZK_FP32 plans it
                                   fits: ny >= 16, ny * TC / 8 <= 512 threads)          */
#define KZK_COL_TILE 3          /* per-tile Stockham kernels with plain loads (default for
                                   KZK_FP64 and for the plans no other kernel fits)     */
/* fp32_state (KZK_FP32 plans)                                                 */
#define KZK_STATE_COMPENSATED 1 /* hi + lo spectral state (default)                 */
#define KZK_STATE_PLAIN 2       /* plain FP32 state; its propagator E and the state
                                   transforms' twiddles are two-float (hi + lo)        */
/* transforms                                                                  */
#define KZK_TRANSFORMS_MIXED 1  /* the mixed-radix kernels for every grid (default:
                                   radix-8/16 kernels for powers of two, mixed radix for
                                   the other grids); row_kernel / col_kernel then take
                                   no other value than KZK_AUTO / KZK_ROW_SINGLE        */
/* graph                                                                       */
#define KZK_GRAPH_ON 1          /* kzk_advance replays CUDA graphs of captured steps
                                   (default): chunks of 16 steps and single steps, each
                                   captured once per plan (at the first kzk_advance) and
                                   replayed for any sigma0, the sigma-dependent
                                   coefficients of each chunk written to device memory by
                                   one kernel before it                                  */
#define KZK_GRAPH_OFF 2         /* kzk_advance launches every kernel directly        */
typedef struct {
    int32_t row_kernel;         /* KZK_AUTO, KZK_ROW_PAIR, KZK_ROW_SINGLE            */
    int32_t col_kernel;         /* KZK_AUTO, KZK_COL_PAIR, KZK_COL_TMA, KZK_COL_TILE */
    int32_t fp32_state;         /* KZK_AUTO, KZK_STATE_COMPENSATED, KZK_STATE_PLAIN  */
    int32_t transforms;         /* KZK_AUTO, KZK_TRANSFORMS_MIXED                    */
    int32_t autotune;           /* nonzero: every kernel choice left at KZK_AUTO is
                                   made by timing instead -- each eligible (row_kernel,
                                   col_kernel) combination advances a zero state for one
                                   untimed and two timed steps (CUDA events) at plan
                                   creation, and the fastest is kept                   */
    int32_t graph;              /* KZK_AUTO (= KZK_GRAPH_ON), KZK_GRAPH_ON, KZK_GRAPH_OFF */
} kzk_options;

/* Create a plan for `batch` independent propagations sharing grid,
 * coefficients and step dt (= dsigma of Eq. 5).  Builds the FP64 phi tables of
 * Eq. 11 on the device (rounded once to float for KZK_FP32), the twiddle
 * tables, and the workspace (4 spectral arrays per instance).
 * Errors: KZK_ERR_ARG (null, dt <= 0, B <= 0, A < 0, lf_umax <= 0, batch < 1,
 * n_relax outside [0, KZK_MAX_RELAX], some C_r < 0 or theta_r <= 0, unknown
 * method),
 * KZK_ERR_SIZE (see kzk_grid; also a grid whose column or row does not fit
 * the device's shared memory), KZK_ERR_OOM, KZK_ERR_CUDA.  *out is NULL on
 * failure. */
kzk_status kzk_plan_create(const kzk_grid *grid, const kzk_coeffs *coeffs, double dt,
                           int32_t batch, kzk_plan **out);

/* kzk_plan_create with explicit kernel and state choices (opts, host,
 * nullable: NULL = all KZK_AUTO, which is kzk_plan_create).  Errors as
 * kzk_plan_create, plus KZK_ERR_SIZE for a kernel choice the grid or precision
 * cannot take, and KZK_ERR_ARG for an unknown option value. */
kzk_status kzk_plan_create_ex(const kzk_grid *grid, const kzk_coeffs *coeffs, double dt, int32_t batch,
                              const kzk_options *opts, kzk_plan **out);

/* The choices in effect for a (non-batched) plan: every field resolved (no
 * KZK_AUTO; fp32_state is KZK_AUTO for KZK_FP64 plans, transforms KZK_AUTO
 * for the radix-8/16 kernels; autotune echoes the request).  out: host. */
kzk_status kzk_plan_info(kzk_plan *plan, kzk_options *out);

/* Random inhomogeneous medium (Sec. 2, Algorithm 1): the velocity field
 *   U(sigma, y) = sum_n U~_n cos(|K_n| lambda (sigma cos theta_n + y sin theta_n) + phi_n),
 *   U~_n = |U~(K_n)| (-sin theta_n, cos theta_n) = (U_par, U_perp) components,
 * enters b of Eq. 3 as 2 pi U_par d_tau V - U_perp d_y V, computed in the flux
 * form that follows Eq. 7: WENO5 along tau of -2 pi U_par u - B u^2/2 (global
 * Lax-Friedrichs speed per row |2 pi U_par| + B(sigma) lf_umax), WENO5 along y
 * of U_perp u (speed max_y |U_perp|), and the source (d_y U_perp) u with the
 * derivative of the mode sum.  The mode data (|K_n| lambda, theta_n, phi_n,
 * |U~(K_n)| / c0, host arrays of n_modes doubles) are inputs; the caller keeps
 * ownership (they are copied).  n_modes = 0 removes the medium. */
#define KZK_MAX_MODES 1024
typedef struct {
    int32_t n_modes;
    const double *klam;             /* |K_n| lambda                                  */
    const double *theta;            /* theta_n: angle of K_n to the sigma axis       */
    const double *phase;            /* phi_n                                         */
    const double *amp;              /* |U~(K_n)| / c0                                */
} kzk_medium;

/* Attach a random medium to a (non-batched) plan.  Afterwards every step of
 * kzk_advance / kzk_step_stages and kzk_rhs includes the medium terms, and
 * the adjoint entry points transpose them (the tau-flux with 2 pi U_par, the
 * y-WENO5 -- its weights differentiated like the tau ones -- and the source).
 * Allocates two physical work arrays of the state's size and an
 * [n_modes][ny] FP64 table.
 * Errors: KZK_ERR_ARG (NULL, n_modes outside [0, KZK_MAX_MODES], NULL or
 * non-finite arrays), KZK_ERR_STATE (batched plan), KZK_ERR_OOM, KZK_ERR_CUDA. */
kzk_status kzk_plan_set_medium(kzk_plan *plan, const kzk_medium *medium);

/* The medium's coefficients at sigma as the kernels use them: out (host,
 * [ny][3]) = U_par, U_perp, d U_perp / dy at y_j = y_min + j dy; max_uperp
 * (host, nullable) = max_j |U_perp|.  Synchronises the stream.
 * Errors: KZK_ERR_ARG, KZK_ERR_STATE (no medium), KZK_ERR_CUDA. */
kzk_status kzk_medium_eval(kzk_plan *plan, double sigma, double *out, double *max_uperp, void *stream);

/* Advance u (device, [batch][ny][nx], in place, physical space) by n_steps
 * ExpRK22 steps from sigma0 (Eq. 11 / Algorithm 2).  n_steps = 0 is a no-op.
 * diag_out (host, nullable, `batch` entries): when given, the call
 * synchronises the stream, fills the diagnostics and returns
 * KZK_ERR_NONFINITE if any NaN/Inf was seen, else KZK_ERR_CFL if max|u|
 * exceeded lf_umax, else KZK_OK.  Without diag_out the call is asynchronous
 * and performs no host synchronisation.  Unless the plan's options say
 * KZK_GRAPH_OFF, the steps are replayed from CUDA graphs that the first call
 * captures (on a plan-owned stream; that first call must not itself be inside
 * a stream capture); results equal the direct launches bit for bit. */
kzk_status kzk_advance(kzk_plan *plan, void *u, int64_t n_steps, double sigma0, void *stream,
                       kzk_diag *diag_out);

/* Per-step diagnostics of the last kzk_advance call: hist (host) receives
 * min(n, steps of that call) records [step][batch] of {mean, energy, max|u|,
 * nonfinite} (4 doubles each) of the state at the start of each step.
 * Synchronises the stream. */
kzk_status kzk_diag_history(kzk_plan *plan, double *hist, int64_t n, void *stream);

/* Nonlinear term b(sigma, u) of Eq. 3 in physical space, discretised as in
 * kzk_advance (WENO5 flux derivative plus the absorption-deviation term).
 * u, b: device, [batch][ny][nx]; b may not alias u. */
kzk_status kzk_rhs(kzk_plan *plan, const void *u, void *b, double sigma, void *stream);

/* One step from u (device) into u_next (device) that also returns the first
 * stage V^{n,*} of Eq. 5 (device, physical; for KZK_EXPEULER the step itself,
 * u_star = u_next).  u_next may alias u. */
kzk_status kzk_step_stages(kzk_plan *plan, const void *u, void *u_star, void *u_next,
                           double sigma0, void *stream);

/* tau-direction real FFT of every row (Sec. 3.3): forward (dir = -1) maps
 * physical u [batch][ny][nx] to the packed half spectrum v [batch][ny][nx/2]
 * complex (interleaved re, im) with v[m] = F(u)[m] / nx for 0 < m < nx/2 and
 * v[0] = (F(u)[0] / nx, F(u)[nx/2] / nx); dir = +1 is its exact inverse.
 * Both pointers device, precision of the plan, no aliasing. */
kzk_status kzk_tau_fft(kzk_plan *plan, const void *in, void *out, int32_t dir, void *stream);

/* Copy the plan's tables back, unscaled: E, Phi1, Phi2 (host, each
 * (ny/2+1) * (nx/2+1) complex128 interleaved, row l = |k_y| index, column m =
 * k_tau index 0..nx/2).  Synchronises. */
kzk_status kzk_get_tables(kzk_plan *plan, double *E, double *Phi1, double *Phi2);

/* Gradient of a loss with respect to the initial state u0 (device), given its
 * gradient g_end (device) with respect to the state after n_steps steps from
 * sigma0: g0 (device) = (d u_end / d u0)^T g_end.  Reverse sweep of the exact
 * transpose of the ExpRK22 step (transposed WENO5 including the derivatives
 * of the nonlinear weights, conjugated multipliers, adjoint FFTs), with a
 * checkpoint of the forward state every ckpt_every steps (>= 1) and
 * recomputation of each segment.  u0 is not modified.  g0 may alias g_end.
 * Mixed-radix plans: KZK_ERR_SIZE when nx has no divisor in [4, 16] with
 * nx / divisor <= 512 (the transposed row pass's chunks). */
kzk_status kzk_adjoint(kzk_plan *plan, const void *u0, const void *g_end, void *g0,
                       int64_t n_steps, double sigma0, int32_t ckpt_every, void *stream);

/* Flags of kzk_plan_create_batched. */
#define KZK_BATCH_AUTOTUNE 1
/* Each kzk_advance_batched call replays a CUDA graph in which every instance
 * runs the launches of kzk_advance (its own plan's kernels, sized for its
 * grid) on its own captured stream, the instances concurrently.  The graph is
 * cached per (n_steps, sigma0, state pointers).  This is the default mode (no
 * mode flag). */
#define KZK_BATCH_STREAMS 2
/* Instead: one persistent cooperative kernel launch per call for all
 * instances (captured once per step count in a CUDA graph and replayed). */
#define KZK_BATCH_PERSISTENT 4

/* Plan for n independent propagations with their own grids (same precision),
 * coefficients and steps dts[i], advanced together by one graph launch per
 * kzk_advance_batched call.
 * Streams mode (default, or KZK_BATCH_STREAMS): the graph holds every
 * instance's kzk_advance launches on its own captured stream; any grid
 * kzk_plan_create accepts.  With KZK_BATCH_AUTOTUNE every instance's kernel
 * choices are made by timing (kzk_options.autotune).
 * KZK_BATCH_PERSISTENT: the graph holds one persistent cooperative kernel that
 * runs every pass of every step for all instances -- rows of all instances for
 * the row passes, column tiles of all instances for the column passes, the
 * same computation as kzk_advance (KZK_FP32: with the plans' compensated
 * state, on the single-row and per-tile column bodies, as plans with
 * KZK_ROW_SINGLE and KZK_COL_TILE compute it) -- separated by grid barriers
 * whose waits are bounded (KZK_ERR_TIMEOUT).  With KZK_BATCH_AUTOTUNE the
 * column-tile width is chosen by timing two steps of each candidate at
 * creation.  Each grid must be a power of two, nx <= 8192.
 * Errors as kzk_plan_create, and KZK_ERR_ARG for both mode flags. */
kzk_status kzk_plan_create_batched(const kzk_grid *grids, const kzk_coeffs *coeffs, const double *dts,
                                   int32_t n, int32_t flags, kzk_plan **out);

/* kzk_plan_create_batched whose instances take the kernel and state choices
 * opts (host, nullable; as kzk_plan_create_ex).  In the persistent mode only
 * fp32_state matters (the persistent kernel has its own bodies). */
kzk_status kzk_plan_create_batched_ex(const kzk_grid *grids, const kzk_coeffs *coeffs, const double *dts,
                                      int32_t n, int32_t flags, const kzk_options *opts, kzk_plan **out);

/* Advance the n states u[i] (device pointers, [ny_i][nx_i], in place) by
 * n_steps steps each from sigma0.  diag_out (host, n entries, nullable)
 * behaves as in kzk_advance.  KZK_ERR_STATE for a non-batched plan. */
kzk_status kzk_advance_batched(kzk_plan *plan, void *const *u, int64_t n_steps, double sigma0, void *stream,
                               kzk_diag *diag_out);

/* Launch configuration of a batched plan: CTAs of the persistent launch,
 * log2 cap on the column-tile width (the autotuner's choice), dynamic shared
 * memory per CTA (all 0 for a plan in streams mode). */
kzk_status kzk_batch_info(kzk_plan *plan, int32_t *grid_ctas, int32_t *tile_cap, int64_t *smem_bytes);

/* Testing hook of the bounded grid barrier: later batched launches of this
 * plan wait for extra_blocks more CTAs than they launch (extra_blocks > 0
 * makes every barrier wait run out) with a wait bound of timeout_ms; such
 * launches are not graph-captured.  extra_blocks = 0 restores normal
 * operation (the bound stays timeout_ms).  KZK_ERR_STATE for a plan in
 * streams mode. */
kzk_status kzk_batch_test_barrier(kzk_plan *plan, int32_t extra_blocks, int64_t timeout_ms);

/* kzk_advance that also keeps, inside the plan, the spectral state every
 * ckpt_every steps (the checkpoints kzk_adjoint would recompute).  u is
 * advanced in place; no diagnostics.  A later kzk_adjoint_checkpointed on the
 * same plan reuses the checkpoints until the next kzk_advance_checkpointed or
 * kzk_adjoint call on the plan (which replace them). */
kzk_status kzk_advance_checkpointed(kzk_plan *plan, void *u, int64_t n_steps, double sigma0,
                                    int32_t ckpt_every, void *stream);

/* Adjoint of the last kzk_advance_checkpointed run of this plan: g0 (device)
 * = (d u_end / d u0)^T g_end, recomputing each segment from its checkpoint
 * (the reverse half of kzk_adjoint).  KZK_ERR_STATE without such a run. */
kzk_status kzk_adjoint_checkpointed(kzk_plan *plan, const void *g_end, void *g0, void *stream);

/* Release the plan and all device memory it owns.  NULL is accepted. */
kzk_status kzk_plan_destroy(kzk_plan *plan);

/* Static description of a status code. */
const char *kzk_status_string(kzk_status s);

/* One-line description of the last failure on the calling thread. */
const char *kzk_last_error(void);

/* Number of kernels the library has launched since load (all plans), counting
 * every kernel of a replayed graph. */
int64_t kzk_launch_count(void);

/* Measurement helper (no counterpart in the paper).  Advances u (device,
 * physical, modified like kzk_advance) by n_steps steps with a CUDA event
 * recorded on `stream` around every kernel of the step, and returns in ms[4]
 * the mean device duration of one launch of each kernel: ms[0] row pass of
 * stage 1, ms[1] column pass of stage 1, ms[2] row pass of stage 2, ms[3]
 * column pass of stage 2 (0 for KZK_EXPEULER; with a random medium a "row
 * pass" is its coefficient, C2R and b launches together).  Synchronises the
 * stream. */
kzk_status kzk_kernel_times(kzk_plan *plan, void *u, int64_t n_steps, double sigma0, void *stream,
                            double *ms);

/* Measurement helper (no counterpart in the paper): sustained fused
 * multiply-add throughput of the device in FLOP/s (2 per FMA) for the given
 * precision, from a kernel of independent FMA chains on every SM timed with
 * CUDA events (KZK_FP32: the faster of scalar and packed-pair FMA chains).
 * Synchronises the stream. */
kzk_status kzk_alu_peak(int32_t prec, void *stream, double *flops_per_s);

/* Patterns of kzk_tile_copy_rate. */
#define KZK_COPY_STRIP 0       /* column strips: 16-byte rows, ny rows at a pitch of 8 n bytes */
#define KZK_COPY_CONTIGUOUS 1  /* the same bytes per CTA as one contiguous run */

/* Measurement helper (no counterpart in the paper): the rate, in bytes per
 * second, at which this device's tensor memory accelerator copies the tiles
 * of the FP32 column passes from HBM into shared memory, with no arithmetic.
 * Two arrays of [ny][n] complex FP32 values (n complex columns, n even; ny a
 * power of two in [256, 4096]; n * ny <= 2^28), allocated here and released
 * before returning; one CTA per column pair copies that pair's tile of both
 * arrays -- KZK_COPY_STRIP: in the boxes the column-pair kernels use (ny rows
 * of 16 bytes at a pitch of 8 n bytes), KZK_COPY_CONTIGUOUS: the same number
 * of bytes as contiguous runs -- with as many CTAs per SM as the stage-1
 * column pass, then leaves.  The L2 cache is overwritten before every timed
 * launch; the result is the best of 7 launches (bytes of both arrays / event
 * time).  Errors: KZK_ERR_ARG (null output, bad pattern), KZK_ERR_SIZE (n or ny
 * out of range), KZK_ERR_OOM / KZK_ERR_CUDA, KZK_ERR_TIMEOUT (a bounded wait of
 * the copy kernel ran out).  Synchronises the stream. */
kzk_status kzk_tile_copy_rate(int32_t n, int32_t ny, int32_t pattern, void *stream, double *bytes_per_s);

/* Largest batch * nx * ny accepted by kzk_rhs_noalloc. */
#define KZK_NOALLOC_MAX_POINTS (1 << 18)

/* kzk_rhs without any device allocation.  The paper has no counterpart: this
 * serves callers that cannot let a library call cudaMalloc -- a process that
 * hands all device memory to its own pool allocator up front (a cudaMalloc
 * here would fail or bypass the pool), or a latency-critical path that cannot
 * take cudaMalloc's implicit device synchronisation.  No plan is needed: grid,
 * coeffs (host) and batch describe the problem as for kzk_plan_create, and
 * u, b (device, [batch][ny][nx], plan precision, b not aliasing u) are the
 * caller's input and output; b = b(sigma, u) exactly as kzk_rhs computes it.
 * The intermediates live in one file-scope device array of
 * 2 * 8 * KZK_NOALLOC_MAX_POINTS + 16 * 12288 bytes (about 4.2 MB) that every
 * GPU loading the library keeps until the process exits.  The first call in a
 * CUDA context (per device; again after cudaDeviceReset re-creates the
 * context, which the call notices by the context's id) looks up that array's
 * device address and lifts the kernels' shared-memory limit; make that first
 * call before any stream capture.  The array keeps the last call's contents:
 * the twiddle tables of the last (nx, precision) stay and are reused by the
 * next call with the same pair; everything else a call reads it writes first.
 * All calls share the array, so calls whose GPU work overlaps (different
 * streams or host threads) race: serialise them.  A CUDA error already pending
 * on entry (cudaPeekAtLastError) is left pending and the call returns
 * KZK_ERR_CUDA without launching.  Errors: KZK_ERR_ARG (null, aliasing, bad
 * precision or coefficients), KZK_ERR_SIZE (nx not a power of two in
 * [8, 8192], ny not a power of two, or batch * nx * ny above
 * KZK_NOALLOC_MAX_POINTS), KZK_ERR_CUDA.  Calls no cudaMalloc / cudaFree. */
kzk_status kzk_rhs_noalloc(const kzk_grid *grid, const kzk_coeffs *coeffs, int32_t batch,
                           const void *u, void *b, double sigma, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KZK_H */

/*
 * sunb.h -- C ABI of a batched stiff-ODE integrator for NVIDIA B300 (sm_103a).
 *
 * It integrates many small, independent ODE systems y_c' = f(t, y_c; p_c),
 * one per cell, the setting of arXiv 2405.01713 (Balos et al., "SUNDIALS
 * Time Integrators for Exascale Applications with Many Independent ODE
 * Systems"): operator splitting (Sec. 1, Sec. 3.1 Eq. chemODE, Sec. 3.2
 * Eq. nyxODE) leaves one decoupled ODE per cell to be advanced over the
 * outer step dt_CFD.  Each cell runs a variable-order (1..5), variable-step
 * BDF method of the CVODE kind (Sec. 2, Eq. 1) with the WRMS error test of
 * Eq. wrms, the modified Newton iteration and stopping test of
 * Eq. stop_newton, a dense Jacobian and a pivoted LU (Table 1, approach 2A;
 * Sec. 4.1.4, 4.1.6).  Unlike the paper's batches, cells do not advance in
 * lock-step: every cell chooses its own steps and orders.  The variants
 * the paper compares are options of a context: typical-value absolute
 * tolerances (Sec. 4.1.3), difference-quotient Jacobians (approaches
 * 3A/3B), matrix-free GMRES linear solves (approaches 1A/1B) and an
 * explicit Runge-Kutta method (Sec. 4.1.5).
 *
 * Conventions
 *  - State arrays are cell-contiguous ("CY" order, Sec. 4.1.2): y[c*N + i].
 *  - Pointers named dev_* are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers named host_* (and the tables of
 *    sunb_problem) are host memory, read during the call only.
 *  - All device work is enqueued on the stream given to sunb_create and is
 *    asynchronous unless stated; the caller must keep device buffers alive
 *    until the stream has passed the work.
 *  - Every function returns an int status (sunb_status).  Invalid arguments
 *    return SUNB_ILL_INPUT before anything is launched; CUDA failures return
 *    SUNB_CUDA_ERROR.  sunb_last_error() describes the last failure.  No
 *    function aborts or throws.
 *  - A context is not thread-safe; use one context per stream.
 */
#ifndef SUNB_H
#define SUNB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sunb_ctx sunb_ctx;

typedef enum {
    SUNB_SUCCESS = 0,
    SUNB_TOO_MUCH_WORK = -1,   /* a cell hit max_steps before tout          */
    SUNB_ERR_FAILURE = -3,     /* seven error-test failures in one step     */
    SUNB_CONV_FAILURE = -4,    /* ten Newton failures in one step           */
    SUNB_H_TOO_SMALL = -5,     /* the step no longer advances t             */
    SUNB_NONFINITE = -6,       /* f(t0, y0) or y0 not finite                */
    SUNB_MEM_FAIL = -20,       /* device or host allocation failed          */
    SUNB_ILL_INPUT = -22,      /* invalid argument                          */
    SUNB_CUDA_ERROR = -30,     /* a CUDA call failed                        */
    SUNB_NO_RECORD = -31       /* adjoint asked without a recorded forward  */
} sunb_status;

typedef enum {
    SUNB_ROBERTSON = 0,  /* N = 3, params [C,3] = (k1, k2, k3)                     */
    SUNB_MECHANISM = 1,  /* N = K+1 (Y_1..Y_K, T), params [C,1] = pressure (dyn/cm2) */
    SUNB_COSMOLOGY = 2,  /* N = 1 (e, with T = e), params [C,2] = (rho, F)          */
    SUNB_MIXED = 3       /* cosmology cells followed by mechanism cells, one launch */
} sunb_kind;

typedef enum { SUNB_FP64 = 0, SUNB_MIXED32 = 1 } sunb_precision;
typedef enum { SUNB_SCHED_QUEUE = 0, SUNB_SCHED_STATIC = 1 } sunb_schedule;

/* Reaction mechanism (Sec. 3.1): K species, M reversible reactions with
 * modified-Arrhenius forward rates and equilibrium constants from
 * single-range NASA-7 thermodynamics.  Host arrays, copied at create. */
typedef struct {
    int32_t n_species;        /* K, 1..63                                   */
    int32_t n_reactions;      /* M, 1..4096                                 */
    const double *W;          /* [K] molecular weights, g/mol               */
    const double *nasa;       /* [K,7] a1..a7: cp/R = a1+a2T+a3T^2+a4T^3+a5T^4 */
    const int32_t *react;     /* [M,3] reactant species (repeats allowed), -1 = none */
    const int32_t *prod;      /* [M,3] product species, -1 = none           */
    const double *lnA;        /* [M] ln of the pre-exponential factor (cgs, mol) */
    const double *beta;       /* [M] temperature exponent                   */
    const double *Ea;         /* [M] activation energy, cal/mol             */
} sunb_mechanism;

/* Piecewise power-law cooling curve (Sec. 3.2): knots strictly increasing
 * in ln T; the heating term is gamma_heat * (T/1e4)^-0.7 per unit density. */
typedef struct {
    int32_t n_knots;          /* 2..256                                     */
    const double *lnT;        /* [n_knots]                                  */
    const double *lnLam;      /* [n_knots] ln Lambda at the knots           */
    double gamma_heat;
} sunb_cooling_table;

typedef struct {
    int32_t kind;             /* sunb_kind                                   */
    int64_t n_cells;          /* cells (for SUNB_MIXED: mechanism cells)     */
    int64_t n_cells_cosmo;    /* SUNB_MIXED only: cosmology cells            */
    int32_t max_order;        /* 1..5 (0 = 5)                                */
    int32_t max_steps;        /* per cell and call (0 = 100000)              */
    int32_t precision;        /* sunb_precision: FP32 Newton matrix/LU if MIXED32 */
    int32_t lanes_per_cell;   /* mechanism cells: 8, 16, 32, or 0 = autotune  */
    int32_t schedule;         /* sunb_schedule                                */
    int32_t record_adjoint;   /* 0, or the tape capacity (accepted steps per
                                 cell): SUNB_MECHANISM records for sunb_adjoint;
                                 SUNB_ROBERTSON and SUNB_COSMOLOGY record the
                                 step history only (sunb_get_tapes; their
                                 records carry no column map, NaN there);
                                 not for SUNB_MIXED                           */
    const sunb_mechanism *mech;        /* SUNB_MECHANISM, SUNB_MIXED */
    const sunb_cooling_table *table;   /* SUNB_COSMOLOGY, SUNB_MIXED */
} sunb_problem;

/* Totals over all cells of the last sunb_integrate (the work counters the
 * paper uses as cost measures, Sec. 4.1.1 and 4.1.5). */
typedef struct sunb_stats_t {
    int64_t nst, nfe, nje, nni, ncf, nef;   /* steps, f evals, Newton-matrix
                                               builds, Newton iterations,
                                               Newton failures, error-test failures */
    int32_t max_nst;          /* largest per-cell step count                 */
    int32_t worst_status;     /* most negative per-cell status               */
    int64_t n_failed;         /* cells with a nonzero status                 */
} sunb_stats_t;

/* Create a context: validates the problem, copies the tables to the device
 * and allocates all workspace once (the pooled-memory lesson of Sec. 4.3.1:
 * nothing is allocated per call).  stream is a cudaStream_t (NULL = legacy
 * default stream).  On failure *out is NULL. */
int sunb_create(const sunb_problem *prob, void *stream, sunb_ctx **out);

/* Relative tolerance and per-component absolute tolerances of Eq. wrms,
 * w_i = 1/(rtol |y_i^{n-1}| + atol_i).  host_atol has N entries (for
 * SUNB_MIXED: the N mechanism entries then one cosmology entry); NULL
 * means atol_scalar for every component.  Default: 1e-6 and 1e-10. */
int sunb_set_tolerances(sunb_ctx *ctx, double rtol, double atol_scalar, const double *host_atol);

/* Typical-value absolute tolerances (Sec. 4.1.3, Eq. eta): from the state
 * dev_y (the layout of sunb_integrate) the library reduces, on the
 * context's stream, each component's minimum and maximum over the batch
 * (for SUNB_MIXED: the mechanism components over the mechanism cells, the
 * cosmology component over the cosmology cells) and sets
 *   atol_i = eta * (min_i + max_i) / 2
 * with rtol, as sunb_set_tolerances would.  Where (min + max)/2 is not a
 * positive finite number (a component zero or negative everywhere, NaN in
 * some cell) the typical value is the paper's default 1.  host_atol_out
 * (nullable) receives the N (N + 1 for SUNB_MIXED) tolerances.  The
 * paper resets typical values at user-chosen intervals: call this between
 * outer steps as often as wanted.  Synchronises the stream (the tolerances
 * come back to the host).  SUNB_ILL_INPUT for NULL y or eta <= 0. */
int sunb_set_typical_tolerances(sunb_ctx *ctx, const double *dev_y, double rtol, double eta,
                                double *host_atol_out);

/* Newton-matrix Jacobian of mechanism cells: mode 0 analytic (default,
 * Table 1 approach 2A), mode 1 forward difference quotients (approaches
 * 3A/3B, Sec. 4.1.4): column j from f(y + inc e_j) with inc =
 * max(sqrt(eps) |y_j|, sqrt(eps)/w_j), N right-hand sides per matrix build.
 * Takes effect at the next sunb_integrate.  SUNB_ILL_INPUT for other modes,
 * for kinds without mechanism cells, and with adjoint tapes (the adjoint
 * differentiates the analytic Jacobian). */
int sunb_set_jacobian(sunb_ctx *ctx, int mode);

/* Linear solver of the Newton iteration of mechanism cells (SUNB_MIXED:
 * its mechanism cells; thread-per-cell cells always use LU).
 * SUNB_LS_DIRECT (default): LU factors of the Newton matrix M = I - gamma J,
 * rebuilt as the modified Newton iteration asks.  SUNB_LS_GMRES: the
 * matrix-free inexact Newton iteration of Table 1 approaches 1A/1B (Sec. 2,
 * Eqs. linear and stop_linear): each Newton correction by GMRES on the
 * system scaled by the error weights, unpreconditioned, Jacobian-vector
 * products by a forward difference of f along the Krylov vector (increment
 * 1/||v||_wrms), stopping once the scaled residual's WRMS norm is at most
 * 0.05 of the Newton tolerance 0.1/C_q, after at most min(N, 64) iterations
 * (no restarts).  No Newton matrix is built (nje stays 0) and every
 * iteration costs one more right-hand side (counted in nfe).  The library
 * allocates 8 * (resident lane groups) * ((l+1)(N+l) + 4l + 1 + 2N) bytes
 * of device scratch (each group's share rounded up to 4 doubles),
 * l = min(N, 64), on the first switch to GMRES, grows it when a later
 * configuration has more resident groups, and frees it in sunb_destroy.  Takes effect at the next sunb_integrate or
 * sunb_graph_capture.  SUNB_ILL_INPUT for other values, for kinds without
 * mechanism cells, and with adjoint tapes (the adjoint differentiates the
 * direct solver's iteration); SUNB_MEM_FAIL if the scratch cannot be
 * allocated (the previous solver then stays selected).  A later
 * configuration change (the autotuner's) that cannot grow the scratch makes
 * sunb_integrate and sunb_graph_capture fail with SUNB_MEM_FAIL before any
 * launch. */
#define SUNB_LS_DIRECT 0
#define SUNB_LS_GMRES 1
int sunb_set_linear_solver(sunb_ctx *ctx, int solver);

/* Integration method of thread-per-cell kinds (SUNB_ROBERTSON,
 * SUNB_COSMOLOGY).  SUNB_METHOD_BDF (default): the variable-order BDF.
 * SUNB_METHOD_ERK: the explicit alternative of Sec. 4.1.5, a fourth-order
 * adaptive Runge-Kutta method: Merson's five-stage pair with an embedded
 * third-order estimate under the same WRMS test (||E||_wrms < 1, weights
 * from y_n), step factor 0.9 ||E||^(-1/4) within [0.1, 10] (1e4 after the
 * first step, 1 after a rejection, 0.3 from a step's second rejection),
 * the BDF's starting step, exact landing on tout.  Its counters: nst
 * accepted steps, nfe every f (1 + 5 nst + 4 nef), nef rejections, nje =
 * nni = ncf = 0, qlast = 4; seven rejections of one step give
 * SUNB_ERR_FAILURE.  On stiff cells its step is held to the stability bound,
 * so expect SUNB_TOO_MUCH_WORK there (the paper's finding).  Takes effect at
 * the next sunb_integrate or sunb_graph_capture.  SUNB_ILL_INPUT for other
 * values and for kinds with mechanism cells (not built for lane groups). */
#define SUNB_METHOD_BDF 0
#define SUNB_METHOD_ERK 1
int sunb_set_method(sunb_ctx *ctx, int method);

/* Per-cell parameters p_c of y_c' = f(t, y_c; p_c) (Sec. 2, Eq. 1; for
 * chemistry the cell's pressure, Sec. 3.1; for heating-cooling its density
 * and forcing, Sec. 3.2): a caller-owned device array [C, P] of doubles in
 * the layout of sunb_kind (SUNB_MIXED: the cosmology cells' (rho, F) pairs,
 * then the mechanism cells' pressures).  bytes is the array's size and must
 * equal 8 * C * P for the context's cells (3 per Robertson cell, 1 per
 * mechanism cell, 2 per cosmology cell); any other value returns
 * SUNB_ILL_INPUT and keeps the previous array.  The pointer is kept, not
 * copied: it must stay valid while integrations that use it are in
 * flight. */
int sunb_set_params(sunb_ctx *ctx, const double *dev_params, size_t bytes);

/* Advance every cell from t0 to tout (one outer step dt_CFD; Sec. 2) in
 * place in dev_y [C, N].  Each call is a cold start at order 1 and lands
 * exactly on tout.  dev_status (nullable, int32 [C]) receives per-cell
 * statuses; a cell that fails keeps its last accepted state.  Asynchronous:
 * the return value only reports launch problems; see sunb_stats. */
int sunb_integrate(sunb_ctx *ctx, double *dev_y, double t0, double tout, int32_t *dev_status);

/* Same from host memory: copies host_y [C, N] to a library buffer,
 * integrates, copies back, and waits for the stream.  host_status is
 * nullable.  Returns the most negative per-cell status. */
int sunb_integrate_host(sunb_ctx *ctx, double *host_y, double t0, double tout, int32_t *host_status);

/* Work counters of the last sunb_integrate, the paper's cost measures
 * (steps, right-hand sides, Jacobians, Newton iterations and failures;
 * Sec. 4.1.1, 4.1.5) and its statuses (Sec. 2: a cell that fails keeps its
 * last accepted state).  Waits for the context's stream, then fills
 * *host_totals (nullable; sums over all cells) and copies the per-cell
 * counters to dev_per_cell (nullable, caller-owned device int32 [C, 8]:
 * nst, nfe, nje, nni, ncf, nef, last order, status; for SUNB_MIXED the
 * cosmology cells first).  Returns the most negative per-cell status, or a
 * CUDA failure as SUNB_CUDA_ERROR. */
int sunb_stats(sunb_ctx *ctx, sunb_stats_t *host_totals, int32_t *dev_per_cell);

/* Evaluate the right-hand side f(y) for n_cells cells (step a5 on its own):
 * dev_y, dev_f [n_cells, N], cell c uses parameters of cell c. */
int sunb_rhs(sunb_ctx *ctx, const double *dev_y, double *dev_f, int64_t n_cells);

/* Evaluate the dense Jacobian df/dy (row-major [n_cells, N, N]) of the
 * mechanism or Robertson right-hand side (step a6 on its own). */
int sunb_jac(sunb_ctx *ctx, const double *dev_y, double *dev_J, int64_t n_cells);

/* Batched dense LU with row partial pivoting (first row of largest
 * magnitude) and solve (step a7, Sec. 4.1.6): for each of batch systems,
 * factor dev_A [batch, n, n] in place (unit-lower L below the diagonal,
 * U on and above it), write the row exchanges LAPACK-style to dev_piv
 * [batch, n] (0-based), overwrite dev_b [batch, n] with the solution, and
 * set dev_info [batch] to 0 or k+1 for a zero pivot in column k.  n <= 64.
 * Runs on the given stream (a cudaStream_t). */
int sunb_lu_solve_batched(int32_t n, int64_t batch, double *dev_A, int32_t *dev_piv,
                          double *dev_b, int32_t *dev_info, void *stream);

/* FP32 version of sunb_lu_solve_batched (the matrix precision of the
 * mixed form). */
int sunb_lu_solve_batched_f32(int32_t n, int64_t batch, float *dev_A, int32_t *dev_piv,
                              float *dev_b, int32_t *dev_info, void *stream);

/* The exponential that the right-hand-side kernels use (a table-driven
 * method after Tang 1989: 64-entry table of 2^(j/64), degree-5 polynomial
 * on |r| <= ln2/128; the library exp for |x| >= 704 and NaN), applied to
 * dev_x [n] into dev_y [n] on the given stream; returns after the result is
 * written.  For checking its accuracy against exp.  SUNB_ILL_INPUT for
 * n < 0 or NULL arrays with n > 0 (message via sunb_last_error(NULL)). */
int sunb_exp_check(const double *dev_x, double *dev_y, int64_t n, void *stream);

/* The logarithm that the right-hand-side kernels use (table-driven after
 * Tang 1990: 128 entries of 1/F and log F, F = 1 + j/128, degree-7
 * polynomial for log1p on |r| < 1/128; the library log for zero, negative,
 * subnormal, infinite and NaN x), applied to dev_x [n] into dev_y [n] on
 * the given stream; returns after the result is written.  For checking its
 * accuracy against log.  Errors as sunb_exp_check. */
int sunb_log_check(const double *dev_x, double *dev_y, int64_t n, void *stream);

/* Discrete adjoint (a differentiation extension of the path; the paper only
 * names the sensitivity-capable packages CVODES/IDAS, Sec. 2).  With
 * record_adjoint = cap > 0 at create, sunb_integrate records per cell and
 * accepted step the state, the Nordsieck column map applied since the
 * previous step, the update vector, gamma and 1/l_1 (at most cap steps; a
 * cell that needs more is marked and gets NaN results below).  The
 * differentiated map freezes step sizes, orders and column maps and treats
 * every corrector as solved exactly.
 * sunb_adjoint_replay recomputes the step history from the tapes with each
 * corrector solved by full Newton to rounding level (fresh analytic
 * Jacobian per iteration) and writes the final states of that map to
 * dev_y_final (nullable, [C, N]): evaluate the loss there. */
int sunb_adjoint_replay(sunb_ctx *ctx, double *dev_y_final);

/* Gradient of a loss L(y_final) with dev_dLdy = dL/dy_final ([C, N], device)
 * with respect to (ln A_j, Ea_j): dev_grad [M, 2] = sum over cells (fixed
 * summation order, so repeated calls give the same bytes); dev_grad_cells
 * (nullable, [C, M, 2]) receives the per-cell gradients.  Replays first if
 * sunb_adjoint_replay was not called after the last sunb_integrate.
 * Returns SUNB_NO_RECORD for a context without tapes. */
int sunb_adjoint(sunb_ctx *ctx, const double *dev_dLdy, double *dev_grad, double *dev_grad_cells);

/* The recorded step history (a context with record_adjoint = cap > 0;
 * thread-per-cell kinds fill the column map with NaN, the rest as below):
 * copies the tapes of cells first_cell .. first_cell + n_cells - 1 into
 * host_out (caller-owned host memory, n_cells * sunb_tape_stride(ctx)
 * doubles) and waits for the stream.  Per cell, with N unknowns and
 * R = N + 49: a header of 8 + N doubles [count, h0, overflow (0 or 1),
 * 5 unused, y0 (N)], then cap records of R doubles, of which the first
 * count hold the accepted steps in order: y_n (N; the forward run's
 * state, or the exact corrector's after sunb_adjoint_replay), the column
 * map P (6 x 6, row = output Nordsieck column, applied to the previous
 * step's array: rescales and order decreases), the update vector c (6),
 * gamma, 1/l_1, q (the step's order), q_out (the order of the array after
 * the step: q + 1 after an order increase), h_n (the step size), and the
 * Newton and error-test failures of the step's rejected attempts.  These
 * are the control decisions of Sec. 2's adaptive step and order
 * selection (Eq. wrms, Eq. stop_newton), exported so that they can be
 * replayed.  SUNB_NO_RECORD without tapes; SUNB_ILL_INPUT for a range
 * outside the cells. */
int sunb_get_tapes(sunb_ctx *ctx, int64_t first_cell, int64_t n_cells, double *host_out);

/* Doubles per cell of sunb_get_tapes' output (0 without tapes). */
int64_t sunb_tape_stride(const sunb_ctx *ctx);

/* Replace the Arrhenius parameters ln A_j and Ea_j (host arrays [M]) of a
 * mechanism context; synchronises the context's stream. */
int sunb_set_arrhenius(sunb_ctx *ctx, const double *host_lnA, const double *host_Ea);

/* CUDA graph of outer steps: sunb_graph_capture builds (without running
 * it) a graph of nsteps consecutive outer steps on dev_y, [t0 + k dt,
 * t0 + (k+1) dt] for k < nsteps, each a cold start as in sunb_integrate
 * (queue reset, then the persistent kernel); the autotuner's trials, if
 * pending, run first (synchronously).  sunb_graph_launch re-times the
 * captured steps to start at t0 (kernel-node parameter updates, no
 * re-capture) and launches the graph on the context's stream; dev_y and
 * dev_status stay those given at capture.  Not available with
 * record_adjoint.  A new capture replaces the previous graph. */
int sunb_graph_capture(sunb_ctx *ctx, double *dev_y, double t0, double dt, int32_t nsteps,
                       int32_t *dev_status);
int sunb_graph_launch(sunb_ctx *ctx, double t0);

/* Lanes per mechanism cell chosen by the context (autotuned when asked). */
int sunb_get_lanes_per_cell(const sunb_ctx *ctx);

/* Mechanism mapping in use: lanes per cell, cells per CTA, CTAs per SM;
 * trial_ms (nullable, 6 floats) receives, for L = 8, 16, 32 in turn, the
 * autotuner's trial time in ms and the number of cells of that trial (0 =
 * not run, -1 = mapping does not fit).  With lanes_per_cell = 0 at create,
 * the first sunb_integrate runs the trials (synchronously, each on a
 * scratch copy of eight waves of the first cells) and keeps the mapping
 * with the least time per cell for the context's lifetime. */
int sunb_get_mapping(const sunb_ctx *ctx, int32_t *lanes_per_cell, int32_t *cells_per_cta,
                     int32_t *ctas_per_sm, float *trial_ms);

/* Number of the library's kernel launches enqueued so far by this context. */
int64_t sunb_get_launch_count(const sunb_ctx *ctx);

int sunb_destroy(sunb_ctx *ctx);

/* Integrate n_cells Robertson cells (the kind SUNB_ROBERTSON integrates)
 * from t0 to tout without allocating anything: no context, no cudaMalloc,
 * cudaFree or other allocating call.  It is meant for callers that own all
 * device memory themselves and may not allocate once their time loop runs.
 * The paper has no counterpart; the method is the one of sunb_integrate.
 *  - dev_k [n_cells,3] (k1, k2, k3) and dev_y [n_cells,3] (advanced in
 *    place) are caller-owned device arrays; host_atol points to 3 host
 *    doubles; dev_status (nullable, int32 [n_cells]) receives the per-cell
 *    statuses; max_steps <= 0 means 100000; stream is a cudaStream_t.
 *  - The work queue and the per-cell counters live in one static device
 *    array of 2 MiB + 256 bytes that every GPU loading the library keeps
 *    until the process exits; it limits n_cells to 65536 (larger batches
 *    return SUNB_ILL_INPUT before anything is enqueued).
 *  - The first call on a device looks up that array's device address (with
 *    the device current) and caches it, and copies the step-size choice's
 *    exp and log tables (3.6 KB of constants, into static device arrays)
 *    with a synchronous copy; make that first call before any stream
 *    capture.  The counter is cleared on every call.
 *  - All calls share the array: calls whose work overlaps on the GPU (on
 *    different streams, or from several host threads) race; serialise them.
 *  - The set-up is cached per device index for the life of the process: a
 *    cudaDeviceReset (or anything else that destroys the device's primary
 *    context) invalidates it, and calling this entry point on that device
 *    afterwards is not supported.
 *  - Asynchronous on stream; returns launch errors only; errors are
 *    described by sunb_last_error(NULL). */
int sunb_integrate_robertson_noalloc(const double *dev_k, double *dev_y, int64_t n_cells,
                                     double t0, double tout, double rtol, const double *host_atol,
                                     int32_t max_steps, int32_t *dev_status, void *stream);

/* Description of the last failure of ctx (or of a failed create when ctx is
 * NULL); never NULL. */
const char *sunb_last_error(const sunb_ctx *ctx);

const char *sunb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SUNB_H */

/*
 * crkdg.h -- C ABI of the GB300 (sm_103a) compact RKDG time step.
 *
 * The library advances hyperbolic conservation laws u_t + div f(u) = 0 with
 * the compact Runge--Kutta discontinuous Galerkin (cRKDG) method of Chen, Sun
 * and Xing (arXiv 2307.06471), on uniform Cartesian meshes in 1D and 2D:
 *   inner stages (eq. (2.8), first line):
 *       u^(i) = u^n - dt sum_{j<i} a_ij div^loc f(u^(j))
 *     with the cell-local operator of eq. (2.7) (no neighbour data);
 *   final stage (eq. (2.8), second line):
 *       u^{n+1} = u^n - dt sum_i b_i div^DG f(u^(i))
 *     with the DG operator of eq. (2.3) and the Lax--Friedrichs flux of
 *     Sec. 2.1 (alpha local to each face point and stage);
 *   a TVB-minmod limiter applied once per step, after the final stage
 *     (Remark 2.2; Sec. 4.2).
 *
 * Conventions (all calls):
 *   - every call returns a crkdg_status; nothing throws across the ABI;
 *     crkdg_last_error() gives a thread-local message for the last failure;
 *   - host arrays are owned by the caller and only read/written during the
 *     call; device memory is owned by the context;
 *   - calls run asynchronously on the context's CUDA stream unless marked
 *     "synchronises";
 *   - device-side failures (non-physical states, NaN, bounded waits that ran
 *     out) are recorded in a device status word read by crkdg_sync(); no
 *     kernel traps.
 *
 * State layout (host and device): planes [v][m][y][x], x fastest, with
 *   v   the conserved variable (advection: u; 1D Euler: rho, rho w, E;
 *       2D Euler: rho, rho w, rho v, E),
 *   m   the Legendre mode on the reference cell [-1,1]^d:
 *       1D: P_m(xi), m = 0..k;
 *       2D: P_i(xi) P_j(eta) ordered by total degree i + j ascending and,
 *       within one degree, by i descending; P^k takes i + j <= k, Q^k takes
 *       i, j <= k (so P^k is a prefix of Q^k and modes 0, 1, 2 are
 *       (0,0), (1,0), (0,1)).  Mode 0 is the cell average.
 *   1D meshes use ny = 1.
 */
#ifndef CRKDG_H
#define CRKDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRKDG_MAX_STAGES 6

typedef enum {
    CRKDG_OK = 0,
    CRKDG_EINVAL = -1,         /* bad argument (message in crkdg_last_error) */
    CRKDG_ENOMEM = -2,         /* device or host allocation failed */
    CRKDG_ECUDA = -3,          /* a CUDA runtime call failed */
    CRKDG_ENONPHYSICAL = -4,   /* device saw rho <= 0, p <= 0 or NaN */
    CRKDG_ETIMEOUT = -5,       /* a bounded device wait ran out */
    CRKDG_EUNSUPPORTED = -6    /* combination not built (e.g. k > 3) */
} crkdg_status;

/* device status bits returned by crkdg_sync */
#define CRKDG_ST_NONPHYSICAL 0x1u
#define CRKDG_ST_NAN 0x2u
#define CRKDG_ST_TIMEOUT 0x4u

/* boundary condition of one side */
enum { CRKDG_BC_PERIODIC = 0, CRKDG_BC_OUTFLOW = 1, CRKDG_BC_REFLECT = 2, CRKDG_BC_DIRICHLET = 3 };
/* built-in exterior data for CRKDG_BC_DIRICHLET sides (bc_params per side):
 *   CONST       params[0..nv-1] = exterior state
 *   SINE        advection: A sin(kx x + ky y - w t + phi); params A, kx, ky, w, phi
 *   SINE_PROD   advection: A sin(kx (x - cx t)) sin(ky (y - cy t)); params A, kx, cx, ky, cy
 *   DMR_BOTTOM  x < x0: post-shock state, else reflecting wall; params post[4], x0
 *   DMR_TOP     x < x0 + s_y y + s_t t: post-shock, else pre-shock;
 *               params post[4], pre[4], x0, s_y, s_t
 * Exterior data for stage i are evaluated at t^n + c_i dt (Sec. 2.1, 3.4). */
enum { CRKDG_FN_CONST = 0, CRKDG_FN_SINE = 1, CRKDG_FN_SINE_PROD = 2, CRKDG_FN_DMR_BOTTOM = 3,
       CRKDG_FN_DMR_TOP = 4 };

enum { CRKDG_SIDE_W = 0, CRKDG_SIDE_E = 1, CRKDG_SIDE_S = 2, CRKDG_SIDE_N = 3 };
enum { CRKDG_ADVECTION = 0, CRKDG_EULER = 1 };
enum { CRKDG_BASIS_P = 0, CRKDG_BASIS_Q = 1 };
/* Precision of the state and of the step's arithmetic.
 * CRKDG_F32   FP32 state and arithmetic, FP64 reductions.
 * CRKDG_F64   FP64 throughout.
 * CRKDG_F32C  compensated FP32 state, 2D Euler without limiters.  The state
 *             is kept as hi + lo FP32 pairs; all stage arithmetic runs in
 *             FP32 on hi and only the final update u^{n+1} = u^n + Delta is
 *             accumulated exactly (TwoSum), which removes the per-step
 *             rounding of the state itself; Delta keeps the FP32 rounding of
 *             the fluxes, O(eps |f|) per point.
 * CRKDG_F32D  compensated FP32 state with deviation-form fluxes, 2D Euler
 *             without limiters: every stage state is held as its deviation
 *             from the cell's base state (the hi part of its average) and
 *             every flux as f(c + d) - f(c) by exact algebraic differences,
 *             so the inner-stage operators, the final stage and Delta carry
 *             FP32 errors of a few ulps of their own size.  The final stage
 *             is then evaluated to full accuracy in the sense of the
 *             perturbed-RK estimate of Sec. 3.3 (Grant), at FP32 speed, and
 *             the run keeps the convergence order of FP64 (boundary data of
 *             non-affine Dirichlet sides are formed from FP32-rounded full
 *             states: exact deviations on periodic, outflow, wall and
 *             constant-state sides only).  Same planes as CRKDG_F32C. */
enum { CRKDG_F32 = 0, CRKDG_F64 = 1, CRKDG_F32C = 2, CRKDG_F32D = 3 };
enum { CRKDG_FLUX_LLF = 0 };   /* Lax--Friedrichs, alpha per face point and stage */

typedef struct {
    int dim;                   /* 1 or 2 */
    int nx, ny;                /* cells; ny = 1 when dim = 1 */
    double x0, x1, y0, y1;     /* domain [x0,x1] x [y0,y1] */
    int bc[4];                 /* CRKDG_BC_* for W, E, S, N (periodic pairs) */
    int bc_fn[4];              /* CRKDG_FN_* for Dirichlet sides */
    double bc_params[4][16];   /* per-side parameters of bc_fn */
} crkdg_mesh;

/* Butcher tableau of eq. (2.5): a strictly lower triangular, row-major s x s
 * in a[CRKDG_MAX_STAGES * CRKDG_MAX_STAGES] (row i at a[i*CRKDG_MAX_STAGES]),
 * weights b[s], nodes c[s]. */
typedef struct {
    int s;
    double a[CRKDG_MAX_STAGES * CRKDG_MAX_STAGES];
    double b[CRKDG_MAX_STAGES];
    double c[CRKDG_MAX_STAGES];
} crkdg_tableau;

typedef struct crkdg_ctx crkdg_ctx;   /* opaque; owns all device buffers */

/* Create a solver context (eq. (2.1) on `mesh`, space P^k/Q^k, Sec. 2.1).
 *   k          polynomial degree 0..3
 *   basis      CRKDG_BASIS_P or _Q (ignored in 1D)
 *   flux       CRKDG_FLUX_LLF
 *   tab        explicit Butcher tableau, 1 <= s <= CRKDG_MAX_STAGES
 *   gamma      ratio of specific heats (Euler)
 *   physics    CRKDG_ADVECTION (phys_params = beta_x, beta_y) or CRKDG_EULER
 *   precision  CRKDG_F32 (bulk FP32, FP64 reductions), CRKDG_F64, or the
 *              compensated forms CRKDG_F32C / CRKDG_F32D (2D Euler)
 *   stream     cudaStream_t to run on (NULL: the legacy default stream)
 * Allocates the state (two ping-pong copies) and scratch on the current
 * device.  Returns CRKDG_EINVAL / CRKDG_EUNSUPPORTED / CRKDG_ENOMEM. */
int crkdg_create(const crkdg_mesh* mesh, int k, int basis, int flux, const crkdg_tableau* tab,
                 double gamma, int physics, int precision, const double* phys_params,
                 void* stream, crkdg_ctx** out);
void crkdg_destroy(crkdg_ctx* ctx);

/* Bytes of one copy of the state of the context crkdg_create makes for these
 * arguments: cells x variables x modes values of 4 bytes (CRKDG_F32,
 * CRKDG_F32C / CRKDG_F32D twice: hi planes then lo planes) or 8 (CRKDG_F64),
 * laid out as planes [v][m][y][x].  Host arithmetic only.  EINVAL for a
 * null pointer or arguments crkdg_create rejects as out of range. */
int crkdg_state_bytes(const crkdg_mesh* mesh, int k, int basis, int physics, int precision, size_t* bytes);

/* crkdg_create with the state's two ping-pong copies in device memory the
 * caller owns (for example two PyTorch tensors): state_a and state_b each
 * hold crkdg_state_bytes bytes on the current device, 16-byte aligned and
 * not overlapping, and stay allocated until crkdg_destroy, which does not
 * free them.  The context reads and writes them on its stream only; the
 * state starts as the contents of state_a at t = 0 (nothing is zeroed).
 * Each step writes the other copy: crkdg_current_state says which holds the
 * current state.  EINVAL for null, misaligned, overlapping or non-device
 * buffers; otherwise as crkdg_create. */
int crkdg_create_on_buffers(const crkdg_mesh* mesh, int k, int basis, int flux, const crkdg_tableau* tab,
                            double gamma, int physics, int precision, const double* phys_params, void* stream,
                            void* state_a, void* state_b, crkdg_ctx** out);

/* The copy that holds the current state -- which = 0 (state_a, the first
 * copy) or 1 -- and its device address, as of the calls made so far (work
 * queued on the stream included): read it after synchronising the stream.
 * A pending limit (crkdg_limit) is not yet applied to it. */
int crkdg_current_state(const crkdg_ctx* ctx, int* which, void** dev_ptr);

/* Sizes: cells = nx*ny, modes per cell, variables, volume points per cell. */
int crkdg_sizes(const crkdg_ctx* ctx, int* n_cells, int* n_modes, int* n_vars, int* n_qp);

/* Coordinates of the volume quadrature points (tensor Gauss--Legendre, k+1
 * per direction), host array xy[cell][q][dim], cell = y*nx + x.  Pure host
 * computation. */
int crkdg_quadrature_points(const crkdg_ctx* ctx, double* xy);

/* L2 projection (Sec. 2.2, the Pi of eq. (2.7)) of point values of the
 * initial data, values[cell][q][v] (FP64, host), by the volume Gauss rule;
 * replaces the state, sets t = 0 and clears any pending limit.  Synchronises. */
int crkdg_project_ic(crkdg_ctx* ctx, const double* values);

/* Replace / read the state, host FP64 planes [v][m][y][x].  get_state first
 * applies a pending limit (see crkdg_limit).  FP32 states travel as FP64 and
 * are rounded (set) or widened (get) on the GPU, through a staging buffer of
 * the state's size in FP64 that the context allocates on first use (ENOMEM if
 * it cannot).  Both synchronise. */
int crkdg_set_state(crkdg_ctx* ctx, const double* host_state, double t);
int crkdg_get_state(crkdg_ctx* ctx, double* host_state);

/* FP64 CFL time step dt = cfl / max_K (s_x(ubar)/dx + s_y(ubar)/dy) over cell
 * averages (1D: cfl * dx / max |f'|).  Synchronises. */
int crkdg_cfl_dt(crkdg_ctx* ctx, double cfl, double* dt_out);

/* One full cRKDG step of size dt (eq. (2.8)), asynchronous: all inner
 * stages, the final DG stage with boundary data at t^n + c_i dt, the limiter
 * of a previous step (applied on load) and the FP64 reductions of the new
 * cell averages (max wave speed, totals).  t advances by dt. */
int crkdg_step(crkdg_ctx* ctx, double dt);

/* March n_steps steps with dt computed on the device from the previous
 * step's FP64 wave-speed reduction, dt = min(cfl/maxspeed, t_end - t); no
 * host synchronisation between steps.  Steps whose dt would be <= 0 copy the
 * state.  With capture != 0 the n_steps launches are recorded once into a
 * CUDA graph and replayed on later calls with the same n_steps. */
int crkdg_advance(crkdg_ctx* ctx, int n_steps, double cfl, double t_end, int capture);

/* Limiter control (Remark 2.2).  M >= 0: enable the TVB-minmod limiter with
 * parameter M for the end of every following step, and mark the current
 * state as pending a limit (it is limited before its next use: on load by
 * the next step, or by get_state).  M < 0: disable for following steps (a
 * pending limit of an earlier step is still applied). */
int crkdg_limit(crkdg_ctx* ctx, double M_tvb);

/* Positivity-preserving scaling (Zhang and Shu, J. Comput. Phys. 229, 2010;
 * not part of the paper's method).  eps > 0: after the TVB limiter (if on)
 * at the end of every following step, scale each cell's non-constant modes
 * so that density and pressure are >= eps at the volume and face Gauss
 * points; cell averages are unchanged.  Marks the current state pending like
 * crkdg_limit.  eps <= 0: off.  2D Euler only (CRKDG_EUNSUPPORTED otherwise). */
int crkdg_positivity(crkdg_ctx* ctx, double eps);

/* One step with dt taken from the device run state: the dt that the fused
 * reduction of the previous step (or of crkdg_advance's first reduction)
 * computed, dt = min(cfl / maxspeed, t_end - t) with the cfl and t_end of the
 * last crkdg_advance.  No host synchronisation (2D only). */
int crkdg_step_device(crkdg_ctx* ctx);

/* One step of the original RKDG method for comparison (eq. (2.6) in the
 * Shu--Osher SSP form of Sec. 3.2.1: order 2 or 3), with every stage using
 * div^DG f and the final-stage limiters (crkdg_limit / crkdg_positivity)
 * applied after every stage, as the paper does for RKDG (Sec. 4.2).  Runs as
 * order forward-Euler DG passes (each needs neighbour data), limiter passes
 * and linear combinations; needs a third state copy (allocated on first use).
 * Boundary data of the stages at t, t + dt (and t + dt/2 for order 3).
 * 2D FP32/FP64.  The device dt of crkdg_step_device is not updated: use
 * crkdg_cfl_dt. */
int crkdg_rkdg_step(crkdg_ctx* ctx, double dt, int order);

/* Fixed-dt run of n_steps steps.  1D meshes of up to 960 cells run the whole
 * sequence in one single-block launch (block barrier between steps). */
int crkdg_run_fixed(crkdg_ctx* ctx, int n_steps, double dt);

/* Totals sum_K |K| ubar_K per variable (FP64, eq. (3.4)).  Synchronises. */
int crkdg_conservation(crkdg_ctx* ctx, double* sums);

/* Number of cells the limiter flagged as troubled in the last limited step
 * (counted on the device).  Synchronises. */
int crkdg_troubled_count(crkdg_ctx* ctx, unsigned long long* count);

/* Wait for the stream; return the device status bits seen so far (and
 * clear them).  Returns CRKDG_ENONPHYSICAL if any bit is set. */
int crkdg_sync(crkdg_ctx* ctx, unsigned* device_status);

/* Current simulation time (host copy). */
int crkdg_time(const crkdg_ctx* ctx, double* t);

/* Number of 2D steps with dt > 0 the context has completed since its
 * creation, counted by each step's device reduction (steps past t_end of a
 * device-driven run, which leave the state unchanged, are not counted).
 * Synchronises.  CRKDG_EUNSUPPORTED in 1D. */
int crkdg_step_count(crkdg_ctx* ctx, unsigned long long* steps);

/* Monitor a device-driven run without stalling it: enqueue on the context
 * stream a copy of the device run state into out[5] = {t, dt of the next
 * step, t_end, cfl, maximum wave speed (max_K (|u|+c)/dx + (|v|+c)/dy of the
 * last step's new averages, eq. (3.4)'s FP64 reduction)}.  out is host
 * memory owned by the caller; it is written when the stream reaches the copy,
 * so read it after crkdg_sync (or another synchronisation of the stream).
 * With page-locked (pinned) memory the call returns at once; with pageable
 * memory the copy waits for the stream.  Returns EINVAL for null. */
int crkdg_run_state_async(crkdg_ctx* ctx, double* out);

/* Launch shape of the fused 2D step: rows per warp segment and warps per
 * block (0 = keep).  crkdg_autotune times candidates on the current state
 * (run state restored afterwards; a limit pending in CRKDG_LIMIT_PASS mode is
 * applied first, as the next step would apply it) and keeps the fastest; the
 * candidates include the current shape, so tuning never selects a shape
 * slower in its own timing.  Returns the kept shape's time per step (the step
 * kernel and its one-block finalize) in microseconds.  Synchronises. */
int crkdg_set_launch(crkdg_ctx* ctx, int seg_rows, int warps_per_block);
int crkdg_get_launch(const crkdg_ctx* ctx, int* seg_rows, int* warps_per_block);
int crkdg_autotune(crkdg_ctx* ctx, double* best_us);

/* Where the pending limiter of the previous step's final stage (Remark 2.2)
 * runs when a 2D step loads u^n: CRKDG_LIMIT_FUSED inside the fused step
 * (each warp limits the cells it loads), CRKDG_LIMIT_PASS (default) in a
 * separate in-place pass over all cells, one thread per cell, just before
 * the step.  Both compute the same limiter (same arithmetic; results agree to
 * rounding, which can differ where the compiler fuses multiply-adds
 * differently in the two kernels); the pass costs one extra read of u^n but
 * spreads the limiter's uneven work (troubled cells gather at shocks) over
 * the whole GPU instead of the few warps that hold the shock.  The learned
 * indicator (crkdg_set_indicator) follows the mode: evaluated in the pass
 * (a grid of a few blocks per SM, each loading the weights once) or fused
 * into the step's load.  EINVAL for another mode. */
enum { CRKDG_LIMIT_FUSED = 0, CRKDG_LIMIT_PASS = 1 };
int crkdg_set_limit_mode(crkdg_ctx* ctx, int mode);
int crkdg_get_limit_mode(const crkdg_ctx* ctx, int* mode);

/* How the 2D step evaluates its operators for linear advection.
 * CRKDG_FORM_AUTO (default): where the flux is linear (CRKDG_ADVECTION, FP32
 * or FP64) and every non-periodic side is outflow, wall or a constant state,
 * the step uses the modal form of the operators — the local operator (eq.
 * (2.7)) is beta . grad of the modal polynomial, the final stage's
 * sum_i b_i div^DG f(u^(i)) equals the DG operator of sum_i b_i u^(i) (the
 * linearity behind Theorem 3.3), applied once with the upwind flux — which
 * the quadrature form computes exactly as well; results agree to rounding.
 * The modal step takes its own launch shape (crkdg_set_launch and
 * crkdg_autotune tune the quadrature step).  CRKDG_FORM_QUADRATURE: always
 * the quadrature form.  EINVAL for another value. */
enum { CRKDG_FORM_QUADRATURE = 0, CRKDG_FORM_AUTO = 1 };
int crkdg_set_operator_form(crkdg_ctx* ctx, int form);
int crkdg_get_operator_form(const crkdg_ctx* ctx, int* form);

/* Apply the pending limiter (2D) to the stored state now, in place on the
 * device, as the separate pass above; async on the context stream.  The next
 * step then loads the state without limiting it again and reports the cells
 * this pass flagged through crkdg_troubled_count.  No-op when nothing is
 * pending. */
int crkdg_apply_limit(crkdg_ctx* ctx);

/* Checkpoint: header + FP64 state; load restores state, t and limiter. */
int crkdg_save(crkdg_ctx* ctx, const char* path);
int crkdg_load(crkdg_ctx* ctx, const char* path);

const char* crkdg_last_error(void);
const char* crkdg_version(void);

/* ------------------------------------------------------------------------
 * Batched ensembles (no counterpart in the paper: many independent 2D Euler
 * problems advanced together).  Problems have their own mesh size and domain
 * and share the scheme (k, basis, tableau, gamma, precision), the boundary
 * types (periodic / outflow / reflect) and the final-stage limiters.  One
 * batched step launch covers every problem's tiles; each problem keeps its
 * own t, dt (from its own FP64 wave-speed reduction, eq. (3.4) style), t_end
 * and status, and stops costing work once it reaches t_end.
 * ------------------------------------------------------------------------ */
typedef struct crkdg_batch crkdg_batch;
typedef struct {
    int nx, ny;                 /* cells */
    double x0, x1, y0, y1;      /* domain */
} crkdg_batch_problem;

/* bc[4]: W, E, S, N types shared by all problems.  Allocates one state for
 * all problems (two copies), the problem and task tables, per-problem run
 * states.  stream must be a non-default stream for crkdg_batch_run. */
int crkdg_batch_create(const crkdg_batch_problem* probs, int n, const int* bc, int k, int basis,
                       const crkdg_tableau* tab, double gamma, int precision, void* stream, crkdg_batch** out);
void crkdg_batch_destroy(crkdg_batch* b);
/* n_problems, total cells, modes per cell, warp tasks per step */
int crkdg_batch_sizes(const crkdg_batch* b, int* n_problems, long long* total_cells, int* n_modes, int* n_tasks);
/* per problem: quadrature points xy[cell][q][2]; projection of point values
 * values[cell][q][4] (sets t = 0); FP64 host planes [v][m][y][x] in and out
 * (get_state applies a pending limit to the returned copy) */
int crkdg_batch_quadrature_points(const crkdg_batch* b, int problem, double* xy);
int crkdg_batch_project_ic(crkdg_batch* b, int problem, const double* values);
int crkdg_batch_set_state(crkdg_batch* b, int problem, const double* host_state, double t);
int crkdg_batch_get_state(crkdg_batch* b, int problem, double* host_state);
/* final-stage limiters for every problem, as crkdg_limit / crkdg_positivity */
int crkdg_batch_limit(crkdg_batch* b, double M_tvb);
int crkdg_batch_positivity(crkdg_batch* b, double eps);
/* Run every problem to t_end with dt = min(cfl / maxspeed, t_end - t) per
 * problem: a CUDA graph of steps_per_graph batched steps (captured once per
 * shape, replayed) is launched until all problems are done or max_graphs
 * graphs ran; *n_done = problems that reached t_end.  Synchronises once per
 * graph (reads one counter). */
int crkdg_batch_run(crkdg_batch* b, double cfl, double t_end, int steps_per_graph, int max_graphs, int* n_done);
int crkdg_batch_problem_info(crkdg_batch* b, int problem, double* t, unsigned long long* steps, unsigned* status);
/* where the pending limiter of every problem runs (as crkdg_set_limit_mode):
 * CRKDG_LIMIT_PASS (default) one in-place pass over every running problem's
 * cells (tiles of 128 cells of a row) before the batched step, which then
 * loads the limited states; CRKDG_LIMIT_FUSED inside the batched step's
 * load.  Problems that reached t_end are not limited by the pass (their
 * stored state keeps its pending limit, which get_state applies).  EINVAL
 * for another mode. */
int crkdg_batch_set_limit_mode(crkdg_batch* b, int mode);
/* launch shape (rows per warp segment, warps per block) and its autotuner,
 * which times one batched step per candidate on the current states (run
 * states restored afterwards) */
int crkdg_batch_set_launch(crkdg_batch* b, int seg_rows, int warps_per_block);
int crkdg_batch_autotune(crkdg_batch* b, double cfl, double* best_us);
const char* crkdg_batch_last_error(void);
/* features and TVB labels of one problem's stored state (see crkdg_features) */
int crkdg_batch_features(crkdg_batch* b, int problem, float* X_dev, float* y_dev, double M_tvb);

/* ------------------------------------------------------------------------
 * Learned troubled-cell indicator (no counterpart in the paper).  A network
 * 40 -> 64 -> 64 -> 64 -> 1 (ReLU) gives a logit per cell from 40 features
 * of the cell: per conserved variable q, the four neighbour-average
 * differences (E, W, N, S) and the five non-constant P^2 modes divided by
 * their largest magnitude s_q, then log10(s_q / (M h^2)) clipped to [-8, 8]
 * (h = max(dx, dy)).  Parameters: FP32 vector of crkdg_mlp_n_params() values,
 * order W1 b1 W2 b2 W3 b3 W4 b4, W row-major (out x in).  Training runs FP32
 * kernels (class-weighted BCE, Adam); inference runs BF16 weights and
 * activations with FP32 accumulation on the tensor cores.
 * ------------------------------------------------------------------------ */
typedef struct crkdg_mlp crkdg_mlp;
int crkdg_mlp_create(unsigned long long seed, void* stream, crkdg_mlp** out);   /* He-normal init */
void crkdg_mlp_destroy(crkdg_mlp* m);
int crkdg_mlp_n_params(void);
int crkdg_mlp_set_params(crkdg_mlp* m, const float* host_params);   /* also resets Adam state */
int crkdg_mlp_get_params(const crkdg_mlp* m, float* host_params);
/* mean loss -[pw y log s(z) + (1-y) log(1-s(z))] over n samples (X_dev
 * [n][40], y_dev [n] in {0,1}, device FP32) and its gradient (host, may be NULL) */
int crkdg_mlp_loss_grad(crkdg_mlp* m, const float* X_dev, const float* y_dev, int n, double pos_weight,
                        double* loss, float* grad_host);
/* epochs of minibatch Adam (lr, beta = 0.9/0.999, eps = 1e-8) over a seeded
 * shuffle; *last_epoch_loss = mean minibatch loss of the last epoch */
int crkdg_mlp_train(crkdg_mlp* m, const float* X_dev, const float* y_dev, int n, int epochs, int batch, double lr,
                    double pos_weight, unsigned long long seed, double* last_epoch_loss);
/* logits_dev[n] from X_dev[n][40] (tensor-core inference) */
int crkdg_mlp_predict(crkdg_mlp* m, const float* X_dev, int n, float* logits_dev);
/* The same logits on the fifth-generation tensor cores (tcgen05): tiles of
 * 512 samples per block, each layer four M = 128 products with BF16
 * operands in shared memory and the FP32 accumulators in tensor memory.  The
 * biases enter the products in BF16 (a ones column of the activations against
 * a bias column of the weights; crkdg_mlp_predict adds them in FP32), so the
 * two agree to BF16 rounding of the biases and the accumulation order.  Its
 * waits for the tensor core are bounded: CRKDG_ETIMEOUT (logits NaN) if one
 * runs out.  Synchronises. */
int crkdg_mlp_predict_tc(crkdg_mlp* m, const float* X_dev, int n, float* logits_dev);
const char* crkdg_mlp_last_error(void);
/* features X_dev[cell][40] and TVB labels y_dev[cell] (1 = the TVB-minmod
 * test with parameter M flags the cell) of the context's stored state */
int crkdg_features(crkdg_ctx* ctx, float* X_dev, float* y_dev, double M_tvb);
/* Use the network as the troubled-cell test of the final-stage limiter:
 * limit when the logit > z_hi, keep when < z_lo, TVB test in between (the
 * reconstruction is always the TVB-minmod one).  net = NULL: TVB test only.
 * 2D Euler, k = 2, FP32; net must outlive its use. */
int crkdg_set_indicator(crkdg_ctx* ctx, const crkdg_mlp* net, double z_lo, double z_hi);
/* Which tensor-core path evaluates the network in the limiter pass (the
 * default limit mode): CRKDG_MLP_TCGEN05 (default) tiles of 512 cells per
 * block, each layer four tcgen05 products of 128 rows with the accumulators
 * in tensor memory (a bounded wait that runs out leaves the TVB test deciding
 * and sets CRKDG_ST_TIMEOUT for crkdg_sync); CRKDG_MLP_MMA_SYNC one warp per
 * 32 cells with mma.sync.  The indicator fused into the step's load always uses
 * mma.sync.  EINVAL for another value. */
enum { CRKDG_MLP_TCGEN05 = 0, CRKDG_MLP_MMA_SYNC = 1 };
int crkdg_set_indicator_engine(crkdg_ctx* ctx, int engine);

/* Measured arithmetic peak of the current device (no counterpart in the
 * paper: the denominator of the step kernel's roofline, which is bound by
 * FP32 fused multiply-adds rather than by memory).  A grid of 8 warps' worth
 * of blocks per SM runs 8 independent FMA chains per thread; the median of
 * `reps` launches timed by CUDA events on `stream` (NULL: legacy default
 * stream; synchronises) gives
 *   tflops         FMA flops (2 per FMA; 4 per packed FP32x2 FMA) per second / 1e12,
 *   ms_per_launch  the median launch time (may be NULL),
 *   n_sms          the SM count the grid covered (may be NULL).
 * kind: CRKDG_PEAK_F32 (scalar FFMA), CRKDG_PEAK_F32X2 (packed __ffma2_rn),
 * CRKDG_PEAK_F64 (DFMA).  Allocates a few KiB for a result sink.  Errors:
 * crkdg_probe_last_error(). */
enum { CRKDG_PEAK_F32 = 0, CRKDG_PEAK_F32X2 = 1, CRKDG_PEAK_F64 = 2 };
int crkdg_alu_peak(int kind, int reps, void* stream, double* tflops, double* ms_per_launch, int* n_sms);
const char* crkdg_probe_last_error(void);

/* No-allocation reduction (no counterpart in the paper; an interface for
 * callers that cannot allocate device memory: code inside a framework that
 * owns the device memory pool, or code that must not allocate while a graph
 * is captured or inside a real-time loop).  Computes, like crkdg_cfl_dt and
 * crkdg_conservation, the FP64 maximum wave speed over cell averages
 * (2D: max (|u|+c)/dx + (|v|+c)/dy; 1D: max (|w|+c)/dx; advection: |beta|/dx
 * terms) and the totals sum_K |K| ubar_K, without allocating:
 *   u_dev    device state planes [v][m][y][x] of n_modes modes (caller-owned,
 *            FP32 or FP64 per `precision`), only read;
 *   dim      1 or 2; in 1D ny and dy are ignored (one row of unit height,
 *            as crkdg_create lays out a 1D mesh);
 *   out_dev  device array of 2 + nv doubles (caller-owned), written on
 *            `stream`: out[0] = max wave speed, out[1 + v] = total of
 *            variable v, out[1 + nv] = the status bits the reduction saw
 *            (an integer value: CRKDG_ST_NONPHYSICAL for a cell average with
 *            rho <= 0 or p <= 0, CRKDG_ST_NAN for a NaN wave speed; 0 when
 *            the state is physical) -- a NaN cell does not show in out[0],
 *            since the maximum skips NaN, so check out[1 + nv];
 *   beta     host pointer to (beta_x, beta_y) for advection, else may be NULL.
 * Asynchronous on `stream`.  Scratch: a file-scope device array of about
 * 64 KiB (1024 per-warp slots) that every GPU loading the library holds until
 * the process exits.  Its device address is looked up, with the stream's
 * device current, at every call made outside a stream capture; a call made
 * while `stream` is being captured reuses the address of the last uncaptured
 * call on that device, so the first call on a device must come before any
 * capture (CRKDG_EINVAL otherwise), and after cudaDeviceReset make one
 * uncaptured call before capturing again.  Every call shares the array and
 * clears its counter first, so calls that overlap on the GPU (other streams,
 * other threads) race: serialise them.  Meshes above 2^30 cells are rejected
 * with CRKDG_EINVAL; errors are reported by crkdg_noalloc_last_error().
 * Calls no cudaMalloc/cudaFree. */
int crkdg_reduce_state_noalloc(const void* u_dev, int dim, int nx, int ny, int n_modes, int physics, int precision,
                               double dx, double dy, double gamma, const double* beta, double* out_dev,
                               void* stream);
const char* crkdg_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CRKDG_H */

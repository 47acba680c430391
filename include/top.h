/*
 * top.h -- C ABI of the GB300 (sm_103a) consensus-ADMM trajectory optimiser.
 *
 * The library solves, for a batch of B trajectories, the piecewise-polynomial
 * minimum-control-effort problem of arXiv 2507.10290 ("TOP: Trajectory
 * Optimization via Parallel Optimization towards Constant Time Complexity"),
 * Sec. III-B, Eq. 2:
 *
 *   min  sum_i int_0^{T_i} ||sigma_i^{(p)}(t)||^2 dt          (p = 4, min snap)
 *   s.t. sigma_i^{[d-1]}(T_i) = sigma_{i+1}^{[d-1]}(0)        (continuity, orders 0..6)
 *        sigma_1^{[p-1]}(0) = start, sigma_N^{[p-1]}(T_N) = end (orders 0..3)
 *        G_i(sigma_i, ...) <= 0                                (sampled constraints)
 *
 * by the consensus ADMM iteration of Sec. III-D (Algorithm 1, Eq. 18a-g): a
 * per-segment closed-form local QP solve (or the numerical L-BFGS step of
 * Sec. III-C.3, Eq. 15-17), the junction consensus average, the scaled dual
 * updates, the slack and projection steps for linear / quadratic
 * constraints, the primal / dual residuals of Eq. 19-20 and the stopping rule
 * of Eq. 21.  Each segment's flat output is a degree-7 polynomial per axis
 * (m = 3 axes, 8 coefficients, Sec. III-D.1, Eq. 18 with d = 2p-1).
 *
 * Conventions for every entry point:
 *   - return TOP_OK (0) on success, a negative TOP_E_* code on error; no
 *     C++ exception crosses the ABI; top_strerror() names a code.
 *   - the caller owns every input and output buffer; the handle owns its
 *     device workspace (allocated by top_create, freed by top_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; top_solve synchronises it once to
 *     read the batch layout unless the problem's memory is TOP_MEM_HOST.
 *   - one handle serves one stream at a time (calls on a handle are not
 *     thread-safe).
 *   - every floating-point input and output is IEEE double.
 *
 * Basis of the returned coefficients (the paper's, Sec. III-D.1):
 *   sigma_i(t)[a] = sum_{k=0}^{7} coeffs[i][a][k] * (t - t_{i-1})^k.
 */
#ifndef TOP_H
#define TOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TOP_API_VERSION 1

/* return codes */
#define TOP_OK          0
#define TOP_E_INVAL    -1  /* invalid argument (sizes, NULL, T <= 0, non-monotone offsets, ...) */
#define TOP_E_NOMEM    -2  /* workspace allocation failed or the batch exceeds the handle's capacity */
#define TOP_E_CUDA     -3  /* a CUDA runtime call failed (the CUDA error is kept for top_last_cuda_error) */
#define TOP_E_TIMEOUT  -4  /* a bounded device wait ran out */
#define TOP_E_NOTSUP   -5  /* a valid but unsupported combination (e.g. numeric step with box rows) */
#define TOP_E_STATE    -6  /* call out of order (e.g. top_grad without a matching top_solve) */
#define TOP_E_NUMERIC  -7  /* a local KKT matrix was not positive definite in FP64 */
#define TOP_E_LIMIT    -8  /* the problem exceeds the fixed scratch of top_solve_noalloc, or 32-bit
                               indexing of per-segment state (S x rows per segment >= 2^31, rows =
                               max(108, 6 M_box, 3 M_ball, 3 M_vn, 2 M_gen, F_poly M_poly)) */
#define TOP_E_BOUNDS   -9  /* the bounds-checked build (libtop_checked.so, compiled with TOP_CHECKED)
                               found an index outside its array; the access was skipped */

/* fixed limits of top_solve_noalloc */
#define TOP_NOALLOC_MAX_SEGMENTS 16384
#define TOP_NOALLOC_MAX_BATCH    1024

/* per-trajectory status written to top_result.status */
#define TOP_CONVERGED      0  /* ||r_p|| < N eps and ||r_d|| < N eps (Eq. 21) */
#define TOP_NOT_CONVERGED  1  /* max_iters reached first (always the case for eps = 0) */
#define TOP_NONFINITE      2  /* a residual became NaN or Inf; results are those of that iteration */
#define TOP_STALLED        3  /* the stall rule stopped it (top_problem.stall_checks): the iteration
                                 precision's residual floor is above N eps; results and the saved
                                 state (top_resume) are those of that iteration */

enum top_precision { TOP_FP32 = 0, TOP_FP64 = 1 };     /* arithmetic of the iteration */
enum top_mode      { TOP_PIN = 0, TOP_FREE = 1 };      /* interior waypoints pinned or free */
enum top_inner     { TOP_CLOSED_FORM = 0, TOP_NUMERIC = 1 };
enum top_memory    { TOP_MEM_DEVICE = 0, TOP_MEM_HOST = 1 };
enum top_schedule  { TOP_SCHED_AUTO = 0, TOP_SCHED_RESIDENT = 1, TOP_SCHED_STREAM = 2 };
enum top_numeric_form { TOP_NUMERIC_AUTO = 0, TOP_NUMERIC_WARP = 1, TOP_NUMERIC_THREAD = 2 };
enum top_gemm_form { TOP_GEMM_CUDA_CORES = 0, TOP_GEMM_TENSOR = 1 };
enum top_stream_form { TOP_STREAM_FUSED = 0, TOP_STREAM_PHASES = 1 };

typedef struct top_handle top_handle;

/* Fixed at creation: capacities of the device workspace and the precision. */
typedef struct top_config {
  int32_t precision;      /* TOP_FP32: FP32 iteration with FP64 KKT inverse and FP64 cost;
                             TOP_FP64: everything in FP64 */
  int32_t max_batch;      /* largest B a call may pass */
  int32_t max_segments;   /* largest total segment count S a call may pass */
  int32_t max_samples;    /* largest M (samples per segment) of any constraint family */
  int32_t schedule;       /* TOP_SCHED_AUTO: trajectories that fit one CTA run resident (packed),
                             longer ones in a thread-block cluster of up to 16 CTAs with distributed
                             shared memory (closed-form families), the rest streaming;
                             TOP_SCHED_RESIDENT: resident only (longer: TOP_E_NOTSUP);
                             TOP_SCHED_STREAM: streaming only */
  int32_t segs_per_cta;   /* resident-form capacity per CTA; 0 = chosen from shared-memory size */
  int32_t ckpt_interval;  /* adjoint checkpoint interval in iterations (0 = 10) */
  int32_t numeric_form;   /* how the numerical local step (Sec. III-C.3) runs, enum top_numeric_form:
                             TOP_NUMERIC_WARP: a segment whose general bound is violated at the minimiser
                             of the quadratic part is solved by one warp (lanes over axis x coefficient and
                             over the (sample, bound) pairs), at the price of one more (short) launch per
                             iteration; TOP_NUMERIC_THREAD: one thread per segment, no extra launch;
                             TOP_NUMERIC_AUTO: WARP.  Results agree within the L-BFGS tolerance, not bit
                             for bit (identical where no bound is violated). */
  int32_t gemm_form;      /* enum top_gemm_form, for the product (D K D)^-1 rhs of the closed-form local
                             step (Eq. 18a) in the resident form: where all 32 segments of a warp share one
                             inverse (interior segments of one trajectory with one duration, Sec. III-D.1)
                             TOP_GEMM_TENSOR runs the warp's 96 products as mma.sync m16n8k8 TF32 tiles
                             with the operands split into high and low TF32 parts (FP32 accuracy);
                             TOP_FP32, no inequality rows and fixed rho only, elsewhere ignored.
                             TOP_GEMM_CUDA_CORES (the default) keeps every product on the FP32 pipe. */
  int32_t stream_form;    /* enum top_stream_form, for trajectories in the streaming form:
                             TOP_STREAM_FUSED (the default): between two residual evaluations one launch
                             per iteration applies the previous iteration's junction update (Eq. 18b-c)
                             and then the local step, the junction state and the segments' end values
                             alternating between two halves of the workspace;
                             TOP_STREAM_PHASES: one launch per phase (local step, junction update).
                             Both give the same results bit for bit. */
  int32_t reserved[6];    /* must be zero */
} top_config;

/* One batch.  Pointers are device pointers for TOP_MEM_DEVICE and host
 * pointers for TOP_MEM_HOST (the library then stages them through its
 * workspace; a page-locked, mapped top_result.coeffs buffer is written by the
 * kernels directly instead, with no copy after the solve); optional families
 * pass M_* = 0 and NULL pointers. */
typedef struct top_problem {
  int32_t B;                  /* trajectories */
  int32_t memory;             /* enum top_memory */
  const int32_t *seg_offset;  /* [B+1] CSR: trajectory b owns segments seg_offset[b] .. seg_offset[b+1]-1;
                                 N_b = 0 is allowed (empty trajectory) */
  const double *waypoints;    /* [S+B][3] path P (Algorithm 1 input): trajectory b owns rows
                                 seg_offset[b]+b .. seg_offset[b+1]+b (N_b+1 points) */
  const double *durations;    /* [S] segment durations T_i > 0 (Sec. III-B) */
  const double *start_state;  /* [B][4][3] boundary state, derivative order r = 0..3 x axis (Eq. 2b) */
  const double *end_state;    /* [B][4][3] */
  int32_t mode;               /* enum top_mode: PIN fixes interior junction positions to the waypoints */
  int32_t inner;              /* enum top_inner (Algorithm 1: ClosedFormSolve / NumericSolve) */
  double rho;                 /* ADMM penalty rho > 0 (fixed) */
  double eps;                 /* stopping tolerance of Eq. 21 (E_r = E_d = N_b eps); 0 = run max_iters */
  int32_t max_iters;          /* >= 0 */
  int32_t check_every;        /* evaluate residuals / stop every this many iterations (>= 1) */
  /* linear box rows |v_axis(t_ij)| <= vbox[b] (Sec. III-C.1, Eq. 8-10, 18d-e) */
  int32_t M_box;  const double *vbox;     /* [B] */
  /* ball corridor ||p(t_ij) - ball_c[i]|| <= ball_r[i] (Sec. III-C.2, Eq. 11-14, shifted) */
  int32_t M_ball; const double *ball_c;   /* [S][3] */
  const double *ball_r;                   /* [S] */
  /* velocity norm ||v(t_ij)|| <= vnorm[b] by projection (Eq. 18f-g) */
  int32_t M_vn;   const double *vnorm;    /* [B] */
  /* general convex bounds through the numerical step (Eq. 15-17): ||v|| <= gen_vmax, ||a|| <= gen_amax */
  int32_t M_gen;  const double *gen_vmax; /* [B] */
  const double *gen_amax;                 /* [B] */
  int32_t lbfgs_mem;          /* numerical step: L-BFGS memory (0 = 8) */
  int32_t lbfgs_max_iters;    /* numerical step: iteration cap per local solve (0 = 50) */
  double lbfgs_tol;           /* numerical step: relative gradient tolerance (0 = 1e-6 FP32 / 1e-12 FP64) */
  /* Residual balancing of rho (UpdateRho of Algorithm 1, Eq. 22), per
   * trajectory.  0 keeps rho fixed.  1: after the stopping test of every
   * iteration, rho <- rho * rho_tau_incr when ||r_p|| > rho_mu ||r_d||, and
   * rho <- rho / rho_tau_decr when ||r_d|| > rho_mu ||r_p||; the unscaled
   * duals are kept across a change (every scaled dual is multiplied by
   * rho_old / rho_new) and the local matrix inverse follows the new rho.
   * Residuals are then evaluated at every iteration (check_every is ignored).
   * Not available in top_grad and top_solve_noalloc (TOP_E_NOTSUP). */
  int32_t adaptive_rho;
  double rho_mu;              /* >= 1 (0 = 10) */
  double rho_tau_incr;        /* >= 1 (0 = 1.1) */
  double rho_tau_decr;        /* >= 1 (0 = 1.1) */
  /* Polytope corridors (Sec. III-C.1, Eq. 8-10, 18d-e): segment i must satisfy
   * n_f . p(t_ij) <= h_f for its F_poly faces at the M_poly sample times
   * t_ij = j T_i / M_poly, each row with its own slack and dual.  The rows
   * couple the axes; the library factorises each segment's local matrix in
   * the eigenbasis of sum_f n_f n_f^T, where it is block diagonal.  Closed-form
   * step only, fixed rho (adaptive_rho: TOP_E_NOTSUP); such problems run in the
   * cluster-resident form (one thread-block cluster per trajectory, up to 16 CTAs;
   * longer trajectories stream).  M_poly = 0: no polytopes. */
  int32_t M_poly;
  int32_t F_poly;             /* faces per segment (>= 1 when M_poly > 0) */
  const double *poly_n;       /* [S][F_poly][3] face normals (any length; rows scale with it) */
  const double *poly_h;       /* [S][F_poly] offsets */
  /* Stall rule (an extension for precision hand-off; the paper has none): with
   * eps > 0, a trajectory for which neither ||r_p|| nor ||r_d|| has fallen
   * below 0.99 of its best value for stall_checks consecutive residual checks
   * stops with status TOP_STALLED (0 = off).  Resident (fixed rho) and
   * cluster-resident forms; the streaming form ignores it. */
  int32_t stall_checks;
} top_problem;

/* Outputs (same memory kind as the problem).  history may be NULL. */
typedef struct top_result {
  double *coeffs;    /* [S][3][8] paper basis (see above) */
  double *cost;      /* [B] J = sum_i c_i^T Qt(T_i) c_i of the returned coefficients */
  double *r_primal;  /* [B] ||r_p|| (Eq. 19) at the last evaluated iteration */
  double *r_dual;    /* [B] ||r_d|| (Eq. 20) at the last evaluated iteration */
  int32_t *iters;    /* [B] iterations run */
  int32_t *status;   /* [B] TOP_CONVERGED | TOP_NOT_CONVERGED | TOP_NONFINITE | TOP_STALLED */
  double *history;   /* optional [max_iters][B][2]: (||r_p||, ||r_d||) at every evaluated iteration
                        (entries of iterations that were not evaluated are left untouched) */
  double *rho;       /* optional [B]: rho after the last update (adaptive_rho), else the fixed rho */
} top_result;

/* Allocate a handle and its device workspace on the current CUDA device.
 * Errors: TOP_E_INVAL (NULL or non-positive capacities), TOP_E_NOMEM, TOP_E_CUDA. */
int top_create(const top_config *cfg, top_handle **out);

/* Run the CADMM iteration (Algorithm 1 / Eq. 18-21) on every trajectory of
 * the batch and write the coefficients, costs, residuals, iteration counts
 * and statuses.  Trajectories are independent; each stops on its own.
 * Errors: TOP_E_INVAL, TOP_E_NOMEM (batch above capacity), TOP_E_NOTSUP,
 * TOP_E_NUMERIC, TOP_E_CUDA, TOP_E_TIMEOUT. */
int top_solve(top_handle *h, const top_problem *pb, top_result *res, void *stream);

/* Gradient of sum_b dJ[b] * J_b, J_b the cost of trajectory b after exactly
 * pb->max_iters iterations of the closed-form iteration (Eq. 18a-g, eps
 * ignored, fixed rho), with respect to the waypoints and the durations, by a
 * hand-written adjoint through the unrolled iterations with checkpoints every
 * ckpt_interval iterations.  The box, ball and velocity-norm rows are
 * differentiated through their slack / projection steps (Eq. 18d-g); at a
 * kink (a slack exactly 0, a projected point exactly on its sphere) the
 * inactive branch is taken.  Without rows, trajectories of up to 256
 * segments (FP32; fewer in FP64) run the whole sweep resident in one launch.
 * dJ: [B]; dwaypoints: [S+B][3]; ddurations: [S] (same memory kind as the
 * problem; outputs are overwritten; a trajectory's first and last waypoint
 * get 0, they enter only through the boundary states).  The paper has no
 * gradient; this is an extension.
 * Errors: as top_solve; TOP_E_NOTSUP with polytope rows, the numerical step or adaptive rho. */
int top_grad(top_handle *h, const top_problem *pb, const double *dJ, double *dwaypoints,
             double *ddurations, void *stream);

/* Sample trajectories: for each trajectory b, the derivative of order
 * `order` (0 = position .. 3 = jerk) of the piecewise polynomial given by
 * `coeffs` ([S][3][8], the layout of top_result.coeffs) at the M times
 * t_m = m T_b / (M - 1), m = 0..M-1, T_b the trajectory's total duration
 * (Sec. III-D.1: sigma_i(t) = c_i^T beta(t - t_{i-1}); at a junction the
 * later segment is used).  Only B, memory, seg_offset and durations of `pb`
 * are read.  out: [B][M][3]; coeffs and out in the memory kind of `pb`.
 * An empty trajectory gets zeros.  The paper evaluates its similarity metric
 * e_simi on such samples (Sec. IV-A.2, M = 8192).
 * Errors: TOP_E_INVAL (M < 2, order outside 0..3, bad offsets), TOP_E_NOMEM
 * (B or S above the handle's capacity), TOP_E_CUDA. */
int top_sample(top_handle *h, const top_problem *pb, const double *coeffs, int32_t M, int32_t order, double *out,
               void *stream);

/* Outer time allocation (an extension: the paper takes the durations as
 * given).  Minimises F(T) = sum_b J_b(T) + k_T sum_i T_i over the durations,
 * J_b the cost after pb->max_iters iterations as in top_grad, by `steps`
 * gradient steps in log T:  T_i <- T_i exp(-clamp(lr T_i dF/dT_i, -0.5, 0.5)),
 * dF/dT_i = dJ/dT_i + k_T from top_grad.  durations_io: [S] initial durations
 * in, final durations out; pb->durations is not read.  res (may be NULL) gets
 * a top_solve with the final durations.  Same restrictions as top_grad
 * (closed-form step, box / ball / velocity-norm rows, fixed rho).  Memory kind of pb.
 * Errors: as top_grad; TOP_E_INVAL for k_T < 0, lr <= 0 or steps < 0. */
int top_time_alloc(top_handle *h, const top_problem *pb, double k_T, double lr, int32_t steps,
                   double *durations_io, top_result *res, void *stream);

/* Capture-safe mode (an extension: lets a caller record a whole top_solve
 * into a CUDA graph and replay it).  After top_set_layout(h, B, host_off)
 * (host_off: [B+1] host copy of the batch's seg_offset), top_solve calls whose
 * problem is in device memory with that B take the layout from this copy
 * instead of reading seg_offset back from the device, and return without
 * synchronising the stream: every operation they issue is asynchronous on it.
 * Their device-side error flag (bad durations, a non-positive-definite local
 * matrix) is read by top_sync(h, stream), which synchronises the stream and
 * returns TOP_OK, TOP_E_INVAL or TOP_E_NUMERIC for the most recent such call.
 * Workspace is allocated on first need: make one call with the same problem
 * kind before beginning a capture.  top_set_layout(h, 0, NULL) leaves the mode.
 * Errors: TOP_E_INVAL (bad offsets), TOP_E_NOMEM (above the capacities). */
int top_set_layout(top_handle *h, int32_t B, const int32_t *host_seg_offset);
int top_sync(top_handle *h, void *stream);

/* Autotuner for the resident capacity (segments per CTA; an extension, the
 * paper has none): times a solve of `iters` iterations (eps = 0) of the given
 * batch at every capacity from 512 down to 128 in steps of 64 that fits the
 * shared memory (trajectories longer than the capacity run in clusters or
 * streaming), after one untimed solve each, and keeps the fastest in the
 * handle in place of top_config.segs_per_cta.  Where top_config.gemm_form
 * applies (FP32, closed form, no inequality rows, fixed rho) it then times
 * both gemm forms at the chosen capacity and keeps the faster in the handle.
 * out_segs_per_cta (may be NULL) gets the capacity; ms (may be NULL) gets up
 * to n_ms timings: entries 0..6 the capacities 512, 448, ..., 128 (negative
 * for one that does not fit), entries 7 and 8 the CUDA-core and tensor-core
 * forms at the chosen capacity (negative where the choice does not apply).
 * Results of the trial solves are discarded.  Errors: as top_solve. */
int top_autotune(top_handle *h, const top_problem *pb, int32_t iters, int32_t *out_segs_per_cta, float *ms,
                 int32_t n_ms, void *stream);

/* Kernel timing.  With profiling enabled, top_solve records CUDA events on
 * the launching stream around each kernel it launches; top_kernel_times then
 * returns, for the last top_solve, ms[0] = local-matrix precompute, ms[1] =
 * resident iteration kernel, ms[2] = streaming iteration kernels, ms[3] =
 * cluster-resident kernels (0 for a kernel that did not run), for up to n
 * entries.  After top_grad: ms[0] = precompute, ms[1] = resident adjoint,
 * ms[2] = streaming adjoint (forward, recomputation and reverse sweep).  Returns the number of entries written, or TOP_E_INVAL /
 * TOP_E_STATE (profiling off). */
int top_set_profiling(top_handle *h, int enable);
int top_kernel_times(const top_handle *h, float *ms, int n);

/* Kernels this handle's top_solve calls have launched so far (instrumentation
 * with no counterpart in the paper; a host-side
 * count: each launch the library issues, and each kernel node of a CUDA graph
 * it replays, counts once; library copies and memsets do not count).  The
 * difference across a region is the number of the library's kernels that ran
 * in it.  Returns -1 for a NULL handle. */
int64_t top_launch_count(const top_handle *h);

/* A solve for callers that cannot allocate device memory (a framework whose
 * allocator forbids side allocations, a real-time loop that must not call
 * cudaMalloc, a process with a memory budget fixed at start-up): it needs no
 * handle and calls no cudaMalloc, cudaFree or allocating library routine.
 * The paper has no counterpart; it is the same computation as top_solve with
 * the resident kernel.  Its scratch (local-matrix inverses, CTA pack table,
 * error flag) is one file-scope device array of about 5 MB that every GPU
 * which loads the library keeps until the process exits.
 *   pb, res    device memory only (TOP_MEM_DEVICE); closed-form step only.
 *   precision  TOP_FP32 or TOP_FP64.
 * Limits: S <= TOP_NOALLOC_MAX_SEGMENTS, B <= TOP_NOALLOC_MAX_BATCH and every
 * trajectory short enough for one CTA of the resident kernel; otherwise
 * TOP_E_LIMIT.  The first call on a device looks up the array's device
 * address (once, with that device current) and keeps it for the life of the
 * device's primary context: do not call it on a device after cudaDeviceReset.  All calls share
 * the array; calls whose GPU work overlaps race on it and must be serialised
 * by the caller.  Synchronises `stream` like
 * top_solve.  Errors: TOP_E_INVAL, TOP_E_NOTSUP, TOP_E_LIMIT, TOP_E_NUMERIC,
 * TOP_E_CUDA. */
int top_solve_noalloc(const top_problem *pb, top_result *res, int precision, void *stream);

/* Iteration state of a batch (an extension for warm starts and resumption;
 * the paper has none), in the memory kind of the problem, FP64 whatever the
 * handle's precision.  For junction j of trajectory b (row seg_offset[b] + b + j
 * of the [S+B] arrays, as the waypoints) and derivative row (axis a, order r)
 * at index a * 7 + r:
 *   p  the consensus target z_j - u (Eq. 18b-c) that the local step of the
 *      segment starting at j reads (its start side)
 *   m  the target that the segment ending at j reads (its end side)
 * At the trajectory's first junction m holds the fixed start state (orders
 * < 4) and p the first segment's target; at its last junction p holds the
 * fixed end state and m the last segment's target; rows of order >= 4 there
 * are 0 (they are dropped from the consensus).  On free interior rows
 * z = (p + m) / 2 and the two scaled duals are -(p - z) and -(m - z).
 *   ybox   [S][6 M_box]   box rows in the compressed form y = A c - b + v of
 *                         Eq. 18d-e (s = max(0, -y), v = max(0, y)), row
 *                         order (sample, axis, sign)
 *   qball  [S][M_ball][3] ball rows q = A c + w of Eq. 18f-g (phi = P(q), w = q - P(q))
 *   qvn    [S][M_vn][3]   velocity-norm rows, likewise
 *   iters  [B]            iterations run so far
 * Pointers of absent families may be NULL. */
typedef struct top_state {
  double *p;
  double *m;
  double *ybox;
  double *qball;
  double *qvn;
  int32_t *iters;
} top_state;

/* top_solve from a saved state instead of Init, and/or saving the state
 * after the last iteration: `from` (may be NULL: Init) is read before the
 * first iteration, `to` (may be NULL) written after the last; pb->max_iters
 * more iterations run, and res->iters counts these.  A run of K1 iterations
 * saved and resumed for K2 more gives the coefficients, costs and state of one
 * run of K1 + K2 iterations bit for bit (the states are exact in FP64 for
 * either precision; the stopping rule of Eq. 21 is applied per call), so a
 * state saved by an FP32 handle can continue on an FP64 handle.  Fixed rho, the
 * closed-form step with box / ball / velocity-norm rows, and trajectories that
 * run resident or in a thread-block cluster (not the streaming form).
 * Errors: as top_solve; TOP_E_NOTSUP outside that set. */
int top_resume(top_handle *h, const top_problem *pb, const top_state *from, top_result *res, top_state *to,
               void *stream);

/* Free the workspace and the handle (NULL is a no-op). */
void top_destroy(top_handle *h);

/* Static description of a return code. */
const char *top_strerror(int code);

/* The last CUDA error seen by the handle (as a cudaError_t value), 0 if none. */
int top_last_cuda_error(const top_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* TOP_H */

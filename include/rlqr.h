/*
 * rlqr.h -- C ABI of the B300 dual-regularized LQR solver.
 *
 * The library solves the first-order optimality system of a dual-regularized
 * LQR problem (Section "Dual-Regularized LQR", eq. min-max-with-ys), i.e. the
 * linear system of eq. primal-dual-linear-system specialised as in eq.
 * optimal-control-specialization:
 *
 *     [ P  C^T ] [x]     [s]        x = (x_0, u_0, x_1, u_1, ..., x_N)
 *     [ C  -D  ] [y] = - [c]        y = (y_0, ..., y_N)
 *
 * with P = blkdiag([Q_i M_i; M_i^T R_i], Q_N), C the bidiagonal dynamics
 * matrix (-I on the diagonal, [A_i B_i] below it), D = blkdiag(Delta_i) with
 * Delta_i = delta * I for i = 0..N, s = (q_0, r_0, ..., q_N), c = (c_0..c_N).
 *
 * It returns x, u, the costates y and a per-stage pivot-PD certificate
 * (Section "Inertia Certification", Theorem
 * riccati-inertia-certification-theorem): for delta > 0 the KKT matrix has
 * inertia (N(n+m)+n, (N+1)n, 0) iff every flag byte equals 3.
 *
 * Conventions shared by every entry point
 *   - All problem arrays are DEVICE pointers to FP64 values, row-major
 *     matrices, stage-major and contiguous:
 *       Q (N+1)*nx*nx   M N*nx*nu   R N*nu*nu   q (N+1)*nx   r N*nu
 *       A N*nx*nx       B N*nx*nu   c (N+1)*nx
 *     Q_i and R_i must be symmetric: only their upper triangle (row <= column)
 *     is read.  c_0 is the initial-state term,
 *     c_{i+1} the offset of the dynamics x_{i+1} = A_i x_i + B_i u_i + c_{i+1}.
 *   - Outputs x (N+1)*nx, u N*nu, y (N+1)*nx (FP64) and pivot_pd (N+1 bytes)
 *     are DEVICE pointers.  pivot_pd[i] bit0 = (I + delta P_i) is PD,
 *     bit1 = G_i is PD (set for i = N, which has no control pivot).
 *   - The caller owns every buffer.  The library never allocates device
 *     memory: scratch lives in a caller-provided workspace whose size the
 *     *_workspace_bytes functions return.
 *   - Every call is asynchronous on the given stream (a cudaStream_t; NULL =
 *     the legacy default stream) and issues no host synchronisation.  The
 *     host return value covers argument validation and launch errors only;
 *     per-instance outcomes (status, relative residual, refinement
 *     iterations) are written to device arrays.
 *   - A zero or non-finite pivot makes the recursion undefined: that
 *     instance's status becomes RLQR_ERR_SINGULAR and its outputs are
 *     unspecified.  A pivot that is merely not PD gives RLQR_NOT_PD, which is
 *     informational: by Theorem riccati-rational-identity-theorem the result
 *     is still the unique KKT solution.
 */
#ifndef RLQR_H_
#define RLQR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t, declared here so that this header does not
 * need the CUDA headers. */
typedef struct CUstream_st *rlqr_stream_t;

typedef enum {
  RLQR_OK = 0,
  RLQR_NOT_PD = 1,             /* solved; at least one pivot is not PD (informational) */
  RLQR_ERR_ARG = 2,            /* invalid argument (dimensions, null pointer, option) */
  RLQR_ERR_SINGULAR = 3,       /* zero or non-finite pivot: recursion undefined */
  RLQR_ERR_NOT_CONVERGED = 4,  /* refinement stopped above the residual tolerance */
  RLQR_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
  RLQR_ERR_WORKSPACE = 6,      /* workspace too small or misaligned */
  RLQR_ERR_CUDA = 7            /* a CUDA launch or runtime call failed */
} rlqr_status;

/* Algorithm of a single-instance factor / solve.  SCAN (Section "Parallel
 * Algorithm": interval elements of eq. lqr-gpu-init-running, combination
 * rule eq. lqr-gpu-combo, chunked reverse scan, p-recurrence and composed
 * affine x maps) has kernels for (nx, nu) in {(4,2), (6,2), (12,4), (32,8)},
 * needs delta > 0 and every R_i invertible, and applies to rlqr_factor /
 * rlqr_solve only (RLQR_ERR_ARG elsewhere or for other sizes).  AUTO takes
 * SCAN for N >= 4096 where it applies, SEQ otherwise; batches always run SEQ.
 * An R_i with a zero or non-finite pivot in the scan's elimination makes the
 * device status RLQR_ERR_SINGULAR (the host return stays RLQR_OK, as for
 * every pivot decision); AUTO does not re-run such an instance with SEQ,
 * which needs only the G_i invertible -- the caller can. */
typedef enum {
  RLQR_ALGO_AUTO = 0,
  RLQR_ALGO_SEQ = 1,  /* sequential Riccati recursion, O(N) depth (Section "Sequential Algorithm") */
  RLQR_ALGO_SCAN = 2  /* associative-scan recursion, O(log N) depth (Section "Parallel Algorithm") */
} rlqr_algo;

typedef enum {
  RLQR_FP64 = 0, /* every step in FP64 */
  RLQR_MIXED = 1 /* FP32 recursion; FP64 pivot certificate, FP64 residual, FP64 correction */
} rlqr_prec;

/* One dual-regularized LQR instance (all pointers device, see above). */
typedef struct {
  int32_t N;  /* number of stages, >= 1 */
  int32_t nx; /* state dimension n, >= 1 */
  int32_t nu; /* control dimension m, >= 1 */
  const double *Q, *M, *R, *q, *r, *A, *B, *c;
  double delta; /* Delta_i = delta * I, delta >= 0 (0 = standard LQR, SEQ only) */
} rlqr_problem;

/* Option bits (rlqr_opts.flags). */
#define RLQR_OPT_SYNC 1 /* single-instance calls wait for their stream and return the
                           instance's status (see rlqr_factor / rlqr_solve) */

typedef struct {
  int32_t max_refine; /* iterative-refinement passes after the first solve (MIXED); >= 0 */
  double tol;         /* target normwise backward error ||Kz+b|| / (||K|| ||z|| + ||b||) */
  rlqr_algo algo;
  rlqr_prec prec;
  int32_t flags;      /* RLQR_OPT_* bits; 0 = stream-ordered, no host wait */
} rlqr_opts;

/* Default options: SEQ-or-SCAN automatic, FP64, tol 1e-9, max_refine 3. */
rlqr_opts rlqr_default_opts(void);

/* Version string of the library build. */
const char *rlqr_version(void);

/* Human-readable name of a status code (static storage). */
const char *rlqr_status_string(rlqr_status s);

/* ------------------------------------------------------------------ *
 * Single instance: factor / solve / residual, the split of the factor, *
 * solve and residual callbacks (Section "Software"), with factor reuse  *
 * across right-hand sides by Corollary p-recurrence.                    *
 * ------------------------------------------------------------------ */

/* Bytes of workspace rlqr_factor needs for these dimensions and options.
 * Returns 0 for invalid dimensions. */
size_t rlqr_workspace_bytes(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts);

/* Backward Riccati sweep (Theorem main-seq-theorem, eq. value-fn-formulas;
 * or the associative-scan form of Section "Parallel Algorithm") for the
 * matrices of `prob`: writes into `ws` the per-stage factors (W_i = P_i
 * (I + delta P_i)^{-1}, K_i, G_i^{-1}) and writes the certificate to
 * pivot_pd (device, N+1 bytes).  `ws` (device, >= rlqr_workspace_bytes,
 * 256-byte aligned) stays valid for rlqr_solve until the next rlqr_factor on
 * it.  The right-hand side (q, r, c) of `prob` is not read.  status (device
 * int32[1], may be NULL) receives the instance status.  The host return
 * covers argument and launch errors only, unless opts->flags has
 * RLQR_OPT_SYNC: then the call waits for `stream` and returns the instance
 * status (RLQR_NOT_PD, RLQR_ERR_SINGULAR) as well. */
rlqr_status rlqr_factor(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                        size_t ws_bytes, uint8_t *pivot_pd, int32_t *status,
                        rlqr_stream_t stream);

/* Solve with the factor in `ws` for the right-hand side (q, r, c) of `prob`
 * (the matrices of `prob` must be those given to rlqr_factor): the
 * p-recurrence of Corollary p-recurrence backward, then the forward rollout
 * of eq. recover-x0 / control-law / recover-x with y_k = P_k x_k + p_k.
 * Writes x, u, y (device).  In RLQR_MIXED mode it then refines against the
 * FP64 residual up to opts->max_refine times (Section "Residual
 * Computation").  rel_resid (device double[1], may be NULL in FP64 mode)
 * receives the final normwise backward error; iters (device int32[1], may be
 * NULL) the refinement passes taken.  `ws` is also used as solve scratch.
 * With RLQR_OPT_SYNC in opts->flags the call waits for `stream` and returns
 * the instance status (RLQR_NOT_PD, RLQR_ERR_SINGULAR,
 * RLQR_ERR_NOT_CONVERGED) instead of RLQR_OK. */
rlqr_status rlqr_solve(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                       size_t ws_bytes, double *x, double *u, double *y, double *rel_resid,
                       int32_t *iters, int32_t *status, rlqr_stream_t stream);

/* FP64 KKT residual of Section "Residual Computation":
 *   res_q[i] = Q_i x_i + M_i u_i + A_i^T y_{i+1} + q_i - y_i   (i < N)
 *   res_r[i] = M_i^T x_i + R_i u_i + B_i^T y_{i+1} + r_i       (i < N)
 *   res_q[N] = Q_N x_N + q_N - y_N
 *   res_c[0] = c_0 - delta y_0 - x_0
 *   res_c[i+1] = A_i x_i + B_i u_i + c_{i+1} - delta y_{i+1} - x_{i+1}
 * res (device, (N+1)*nx + N*nu + (N+1)*nx doubles, laid out res_q | res_r |
 * res_c) may be NULL.  norms (device double[5]) receives
 * [||Kz+b||_inf, ||K||_inf, ||z||_inf, ||b||_inf, rel] with
 * rel = ||Kz+b|| / (||K|| ||z|| + ||b||). */
rlqr_status rlqr_residual(const rlqr_problem *prob, const double *x, const double *u,
                          const double *y, double *res, double *norms, rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Batches of independent instances, possibly of different N, nx, nu.  *
 * ------------------------------------------------------------------ */

/* Instance b's arrays start at the given element offsets into the pooled
 * buffers.  All arrays below are DEVICE arrays of length `count`; h_N, h_nx,
 * h_nu are HOST copies of N, nx, nu used for validation, workspace sizing
 * and scheduling. */
typedef struct {
  int32_t count;
  const int32_t *h_N, *h_nx, *h_nu;             /* host [count] */
  const int32_t *N, *nx, *nu;                   /* device [count] */
  const int64_t *off_Q, *off_M, *off_R, *off_q, *off_r, *off_A, *off_B, *off_c; /* device */
  const int64_t *off_x, *off_u, *off_y, *off_flag;                               /* device */
  const double *delta;                                                            /* device */
  const double *Q, *M, *R, *q, *r, *A, *B, *c; /* pooled device inputs */
  double *x, *u, *y;                           /* pooled device outputs */
  uint8_t *pivot_pd;                           /* pooled device certificate */
} rlqr_batch;

/* Workspace bytes for rlqr_solve_batched (reads only the host dims). */
size_t rlqr_batched_workspace_bytes(const rlqr_batch *batch, const rlqr_opts *opts);

/* Factor + solve (+ refinement in RLQR_MIXED mode) for every instance of the
 * batch, stream-ordered, no host synchronisation.  Per instance (device
 * arrays [count], each may be NULL): status, rel_resid (final normwise
 * backward error; computed when non-NULL or in MIXED mode), iters
 * (refinement passes). */
rlqr_status rlqr_solve_batched(const rlqr_batch *batch, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, int32_t *status, double *rel_resid,
                               int32_t *iters, rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Autotuning: the scan's chunk length and the batched residual route.  *
 * ------------------------------------------------------------------ */

/* The scan path (RLQR_ALGO_SCAN, or AUTO from N = 4096) folds the horizon in
 * chunks of L stages, one CTA per chunk; by default about 444 chunks (three
 * CTAs per SM of a 148-SM part), L >= 8.  rlqr_autotune_scan times
 * rlqr_factor + rlqr_solve of `prob` (three timed runs after a warm-up,
 * CUDA events, host-synchronising) for 148, 296, 444, 592 and 888 chunks
 * and records the fastest for (nx, nu, opts->prec, floor(log2 N)) in a
 * process-wide table (mutex-protected) that later factorizations of that
 * shape use; best_chunks / best_ms (host, may be NULL) receive the choice
 * and its time.  x, u, y, pivot_pd are scratch outputs of the timed solves;
 * ws as for rlqr_factor (rlqr_workspace_bytes sizes every scan workspace
 * for the largest candidate count).  RLQR_ERR_ARG if the problem does not
 * take the scan path.  A factorization and the solves that use it must run
 * with the same table entry: re-factor after tuning.
 * rlqr_tune_scan_set records a chunk count explicitly (1..888; 0 removes
 * the entry) and rlqr_tune_reset clears the table. */
rlqr_status rlqr_autotune_scan(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, double *x, double *u, double *y,
                               uint8_t *pivot_pd, int32_t *best_chunks, double *best_ms,
                               rlqr_stream_t stream);
rlqr_status rlqr_tune_scan_set(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts,
                               int32_t chunks);

/* Routes of rlqr_solve_batched that the tuner chooses between.
 * Uniform batches of the FP32 warp-sweep sizes ((4,1), (4,2), (6,1), (6,2),
 * (12,3), (12,4)): the residual route, 1 = one warp per instance
 * (float-float in mixed mode), 2 = the stage-parallel grid over all stages
 * of the batch, 5 = (mixed precision, max_refine >= 1) no separate first
 * residual: the control pivots are certified by a grid kernel and the first
 * refinement pass computes the residual (float-float) stage by stage ahead
 * of its backward chain; 6 and 7 = routes 1 and 5 with every refinement
 * pass on two warps per instance (one runs the recursion, the other the
 * copies, right-hand sides, the rows of K dz and, route 7, the residual),
 * which shortens each instance's chain at more instructions in all.
 * Without a recorded route the refinement takes one warp per instance.  Ragged mixed-precision
 * batches whose size classes are all
 * among (4,2), (6,2), (12,4), (24,8), (32,8), (48,16): the sweep route,
 * 3 = one launch per size class on the library's concurrent streams (the
 * default), 4 = one persistent launch for every class (CTAs take work items
 * -- 8 instances of a warp size or one of a CTA size, longest chain first --
 * from an atomic counter).
 * rlqr_autotune_batched times rlqr_solve_batched on `batch` with each of
 * its routes (a warm-up and three timed runs, CUDA events,
 * host-synchronising) and records the fastest for (nx, nu, opts->prec,
 * floor(log2 max N), floor(log2 count)), or for ragged batches (the set of
 * size classes, floor(log2 max N), floor(log2 count)), in the process-wide
 * table; status (device [count], may be NULL) is scratch for the timed
 * solves; best_route / best_ms (host, may be NULL) receive the choice and
 * its time.  RLQR_ERR_ARG for other batches.  rlqr_tune_batched_set records
 * a route explicitly (0 removes the entry).  rlqr_tune_reset clears both
 * tables.  rlqr_solve_batched creates its class streams and events once
 * per device on first use of a ragged batch and keeps them. */
rlqr_status rlqr_autotune_batched(const rlqr_batch *batch, const rlqr_opts *opts, void *ws,
                                  size_t ws_bytes, int32_t *status, int32_t *best_route,
                                  double *best_ms, rlqr_stream_t stream);
rlqr_status rlqr_tune_batched_set(const rlqr_batch *batch, const rlqr_opts *opts, int32_t route);
rlqr_status rlqr_tune_reset(void);

/* ------------------------------------------------------------------ *
 * General diagonal dual regularization Delta_i = diag(d_i).            *
 * ------------------------------------------------------------------ */

/* Workspace bytes of rlqr_solve_diag (0 for invalid dimensions). */
size_t rlqr_diag_workspace_bytes(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts);

/* Factor + solve one instance whose dual regularization is Delta_i =
 * diag(delta_diag[i]) (device (N+1)*nx doubles, every entry > 0) instead of
 * prob->delta * I (prob->delta is ignored): the problem statement of Section
 * "Dual-Regularized LQR" allows any SPD Delta_i, and the certificate of
 * Section "Inertia Certification" then tests S_i = I + Delta_i^{1/2} P_i
 * Delta_i^{1/2}.  Method: with D_i = Delta_i^{1/2}, the congruence
 * x_i = D_i x~_i, y_i = D_i^{-1} y~_i maps the system to one with Delta = I
 * (Q~ = D Q D, M~ = D M, q~ = D q, A~_i = D_{i+1}^{-1} A_i D_i,
 * B~_i = D_{i+1}^{-1} B_i, c~ = D^{-1} c), whose pivots are exactly S_i and
 * G_i; the scaled copy lives in `ws` and is solved with rlqr_factor /
 * rlqr_solve (opts as there), then x, y are mapped back.  In RLQR_MIXED
 * mode one more refinement pass follows against the FP64 residual of the
 * ORIGINAL system (the refinement inside rlqr_solve measures the scaled
 * system).  pivot_pd (N+1 bytes), x, u, y as for rlqr_solve; rel_resid (may
 * be NULL) receives the normwise backward error of the original system;
 * status (device int32[1], may be NULL) the instance status.  A d_i entry
 * that is not positive and finite makes the pivots non-finite:
 * RLQR_ERR_SINGULAR.  RLQR_OPT_SYNC in opts->flags returns the status. */
rlqr_status rlqr_solve_diag(const rlqr_problem *prob, const double *delta_diag,
                            const rlqr_opts *opts, void *ws, size_t ws_bytes, double *x, double *u,
                            double *y, uint8_t *pivot_pd, double *rel_resid, int32_t *status,
                            rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Allocation-free solve (no counterpart in the paper).                 *
 * ------------------------------------------------------------------ */

/* Largest scratch the allocation-free entry point can use, in bytes.  The
 * scratch is a file-scope __device__ array of this size inside the library:
 * every GPU that loads the library holds it until the process exits. */
#define RLQR_NOALLOC_SCRATCH_BYTES (8u << 20)

/* Factor + solve one instance with the sequential recursion (the kernels
 * rlqr_factor and rlqr_solve run with algo RLQR_ALGO_SEQ, the solve fused
 * with the factorization) without any workspace argument and without
 * allocating: for callers that cannot call cudaMalloc -- e.g. a control loop
 * with a fixed memory budget that forbids allocation after start-up, or code
 * running inside another runtime that owns the device allocator.  AUTO runs
 * the sequential recursion; RLQR_ALGO_SCAN is refused with RLQR_ERR_ARG.
 * Scratch is the library's static device array (RLQR_NOALLOC_SCRATCH_BYTES);
 * an instance whose sequential workspace (rlqr_workspace_bytes(N, nx, nu,
 * opts) with opts->algo = RLQR_ALGO_SEQ) exceeds it is rejected with
 * RLQR_ERR_WORKSPACE before anything runs.  The caller passes inputs (prob)
 * and device outputs x, u, y, pivot_pd (N+1 bytes) and optional device
 * rel_resid / status (1 element each), exactly as for rlqr_solve.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents; the per-instance state at its start is cleared by each
 *     call.  Calls whose executions overlap on the GPU (different streams,
 *     or host threads) race on the array: serialise them.
 *   - RLQR_OPT_SYNC in opts->flags works as for rlqr_solve. */
rlqr_status rlqr_solve_noalloc(const rlqr_problem *prob, const rlqr_opts *opts, double *x,
                               double *u, double *y, uint8_t *pivot_pd, double *rel_resid,
                               int32_t *status, rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Cross-stage variables (Section "Cross-Stage Variables").            *
 * ------------------------------------------------------------------ */

/* Scratch bytes of rlqr_solve_cross (0 for invalid dimensions, options or
 * p outside 1..31): p + 1 solution columns, the Schur complement's partial
 * sums and p + 1 copies of the instance's workspace (the solves run
 * concurrently). */
size_t rlqr_cross_scratch_bytes(int32_t N, int32_t nx, int32_t nu, int32_t p,
                                const rlqr_opts *opts);

/* The bordered system of eq. cross-stage-kkt for p cross-stage variables
 * theta shared by every stage:
 *   [K    J ] [dw    ]     [b      ]
 *   [J^T  H ] [dtheta] = - [r_theta],
 * K the instance's KKT matrix factored in `ws` by rlqr_factor, b its
 * right-hand side (q, r, c of prob).  J (device, p columns of length
 * L = (N+1) nx + N nu + (N+1) nx, column j at J + j L): each column in the
 * layout of the right-hand side, q-part (pairs with x), r-part (with u),
 * c-part (with y).  H (device, p x p row-major), r_theta (device, p).
 * Steps (eq. cross-stage-schur): p + 1 solves with the factor (the columns
 * of J and b, each as rlqr_solve on its own copy of the factored workspace
 * and its own stream, forked from and joined back to `stream`, refined in
 * RLQR_MIXED mode), the Schur
 * complement S = H - J^T K^{-1} J and g = r_theta - J^T K^{-1} b from FP64
 * dot products in a fixed order, S dtheta = -g by Gaussian elimination with
 * partial pivoting (FP64, one warp), and dw = -K^{-1}(b + J dtheta) written
 * to x, u, y (device) with dtheta (device, p).  scratch (device, >=
 * rlqr_cross_scratch_bytes, 256-byte aligned).  status (device int32[1], may
 * be NULL): the worst status of the p + 1 solves, or RLQR_ERR_SINGULAR for a
 * zero or non-finite pivot of S (dtheta = 0 then).  RLQR_OPT_SYNC works as
 * for rlqr_solve.  p must be 1..31. */
rlqr_status rlqr_solve_cross(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                             size_t ws_bytes, int32_t p, const double *J, const double *H,
                             const double *r_theta, void *scratch, size_t scratch_bytes,
                             double *x, double *u, double *y, double *dtheta, int32_t *status,
                             rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Horizon shards of one long instance (one GPU per shard).            *
 * ------------------------------------------------------------------ */

/* The horizon [0, N] of one instance is split into G contiguous shards
 * [s_g, e_g] (s_0 = 0, e_g = s_{g+1}, e_{G-1} = N).  Shard g is solved as an
 * ordinary rlqr_problem with N_g = e_g - s_g stages whose arrays hold stages
 * s_g .. e_g of Q, q, c and s_g .. e_g - 1 of M, R, r, A, B, except three
 * boundary entries that the caller overwrites (dynamic-programming cut):
 *   Q[N_g] = P_{e_g}, q[N_g] = p_{e_g}   (the cost-to-go after the shard;
 *                                          the true Q_N, q_N for the last),
 *   c[0]   = the initial term whose first state is x_{s_g} (the true c_0
 *            for shard 0; rlqr_shard_entry for the others).
 * The boundary values come from summaries the shards exchange (Section
 * "Parallel Algorithm": interval elements compose with the associative rule
 * of eq. lqr-gpu-combo; Corollary p-recurrence and Section "Composing Affine
 * Functions" for the vector maps):
 *   1. rlqr_shard_element on every shard, gathered -> rlqr_shard_boundary;
 *   2. after rlqr_factor (with Q[N_g] = P_{e_g}) and a solve with
 *      q[N_g] = 0: rlqr_shard_pmap, gathered -> rlqr_shard_p_end;
 *   3. after a solve with the true q[N_g] and c[0] = 0: rlqr_shard_x_offset,
 *      gathered -> rlqr_shard_x_start -> rlqr_shard_entry -> the final solve.
 * Every call below is FP64 and stream-ordered; the shard calls need the
 * scan sizes (nx, nu) in {(4,2), (6,2), (12,4), (32,8)}, delta > 0,
 * opts->prec == RLQR_FP64 and opts->algo == RLQR_ALGO_SCAN; all pointers
 * are device pointers to row-major FP64 arrays owned by the caller.  Host
 * return: RLQR_ERR_ARG for invalid arguments, RLQR_ERR_WORKSPACE for a
 * missing or small workspace, RLQR_ERR_CUDA for a launch error. */

/* Interval element (P, A, C) of the shard's stages 0 .. N_g - 1 (its
 * terminal entry is not used): elem = 3 n^2 doubles, P then A then C.
 * Uses ws (rlqr_workspace_bytes of the shard) as scratch. */
rlqr_status rlqr_shard_element(const rlqr_problem *shard, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, double *elem, rlqr_stream_t stream);

/* From the G gathered elements (G x 3 n^2, shard order) and Q_N (n^2):
 * P_end = P_{e_g} (the composition of the elements of shards g+1 .. G-1 and
 * the terminal element (Q_N, 0, 0)) and, when P_start is not NULL,
 * P_start = P_{s_g} (shard g's element in front of that). */
rlqr_status rlqr_shard_boundary(int32_t G, int32_t g, int32_t nx, int32_t nu,
                                const double *elems, const double *QN, double *P_end,
                                double *P_start, rlqr_stream_t stream);

/* After rlqr_factor and rlqr_solve of the shard (SCAN, FP64) in ws: the p map
 * p_0 = Phi p_{N_g} + phi of its p-recurrence, Phi = n^2 (the product of the
 * chunk maps F_s ... F_{e-1}), phi = n (p_0 of that solve, which is the
 * offset when q[N_g] was 0). */
rlqr_status rlqr_shard_pmap(const rlqr_problem *shard, const rlqr_opts *opts, const void *ws,
                            size_t ws_bytes, double *Phi, double *phi, rlqr_stream_t stream);

/* p_{e_g} from the gathered maps (Phis G x n^2, phis G x n) and q_N (n):
 * v = q_N, then v <- Phi_h v + phi_h for h = G-1 down to g+1. */
rlqr_status rlqr_shard_p_end(int32_t G, int32_t g, int32_t nx, const double *Phis,
                             const double *phis, const double *qN, double *p_end,
                             rlqr_stream_t stream);

/* psi = x_last - Phi^T x_first: the offset of the shard's x map
 * x_{N_g} = Phi^T x_0 + psi from any of its solved trajectories (shard 0
 * passes x_first = 0 so that psi is its true last state). */
rlqr_status rlqr_shard_x_offset(int32_t nx, const double *Phi, const double *x_first,
                                const double *x_last, double *psi, rlqr_stream_t stream);

/* x_{s_g} for g >= 1 from the gathered maps (Phis G x n^2, psis G x n):
 * v = psi_0, then v <- Phi_h^T v + psi_h for h = 1 .. g-1. */
rlqr_status rlqr_shard_x_start(int32_t g, int32_t nx, const double *Phis, const double *psis,
                               double *x_start, rlqr_stream_t stream);

/* c0 = (I + delta P_start)(x_start - x_first): the initial term that gives
 * the shard the first state x_start, where x_first is its first state with
 * c[0] = 0 (eq. recover-x0: x_0 = (I + delta P_0)^{-1} (c_0 - delta p_0)). */
rlqr_status rlqr_shard_entry(int32_t nx, double delta, const double *P_start,
                             const double *x_start, const double *x_first, double *c0,
                             rlqr_stream_t stream);

/* ------------------------------------------------------------------ *
 * Instrumentation (no counterpart in the paper): per-kernel timing.    *
 * ------------------------------------------------------------------ */

/* enable != 0: from now on every kernel the library launches is bracketed by
 * a pair of CUDA events recorded on the launch stream (at most 8192 launches
 * are kept; later ones are counted but not timed).  enable == 0 stops it.
 * Either call discards the launches recorded so far.  Events are created on
 * first use (no device memory is allocated).  Not thread-safe. */
rlqr_status rlqr_instrument(int enable);

/* Waits for the recorded events and reports, per kernel name, the number of
 * launches and their summed device time in milliseconds.  names[i] receives
 * a pointer to a static string.  Returns the number of distinct kernels
 * (entries beyond max are dropped), or -1 on a CUDA error. */
int rlqr_instrument_report(int max, const char **names, int64_t *launches, double *ms);

/* Device bytes of the sink buffer rlqr_measure_pipes needs on the current
 * device (one double per thread of 4 CTAs of 256 threads per SM; 0 on a
 * CUDA error). */
size_t rlqr_measure_pipes_bytes(void);

/* Microbenchmarks of the arithmetic pipes on the current device, for the
 * roofline denominators: FP64 FMA, FP32 FMA and packed f32x2 FMA rates in
 * TFLOP/s (2 flops per FMA lane-operation; independent chains over 4 CTAs
 * of 256 threads per SM; best of 5 CUDA-event-timed launches).  scratch
 * (device, >= rlqr_measure_pipes_bytes(), caller-owned, 8-byte aligned)
 * receives the chains' results so that they are not optimised away; like the
 * solver calls, this call allocates nothing.  Synchronous on the default
 * stream.  RLQR_ERR_WORKSPACE for a missing or small buffer, RLQR_ERR_CUDA
 * on any CUDA error. */
rlqr_status rlqr_measure_pipes(void *scratch, size_t scratch_bytes, double *fp64_tflops,
                               double *fp32_tflops, double *fp32x2_tflops);

/* Microbenchmark of the tensor pipe on the current device: the rate of
 * mma.sync.m16n8k8 with TF32 operands and FP32 accumulation (2 * 16 * 8 * 8
 * flops per instruction; 8 independent accumulator tiles per warp over 4
 * CTAs of 256 threads per SM; best of 5 CUDA-event-timed launches), in
 * TFLOP/s.  The scan's 3xTF32 products issue three such instructions per
 * product tile, so their effective peak is a third of this rate.  scratch:
 * as for rlqr_measure_pipes (the same buffer size suffices; 4-byte aligned);
 * allocates nothing; synchronous on the default stream; RLQR_ERR_WORKSPACE
 * for a missing or small buffer, RLQR_ERR_CUDA on any CUDA error. */
rlqr_status rlqr_measure_tf32(void *scratch, size_t scratch_bytes, double *tf32_tflops);

#ifdef __cplusplus
}
#endif

#endif /* RLQR_H_ */

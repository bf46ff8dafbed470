/*
 * rlqr_ipm.h -- C ABI of the batched regularized interior-point method on a
 * nonlinear multiple-shooting problem: the cart with a double pendulum.
 *
 * What it computes (Section "The Regularized Interior Point Method" and
 * Section "Applying the regularized IPM to optimal control"): for every
 * instance b, a local solution of
 *
 *   min  sum_{i<N} 1/2 (x_i-x_g)^T Wx (x_i-x_g) + 1/2 wu u_i^2
 *        + 1/2 (x_N-x_g)^T Wf (x_N-x_g)
 *   s.t. x_0 = x0_b,  x_{i+1} = phi(x_i, u_i)   (RK4 step of the dynamics)
 *        |u_i| <= u_max (i < N),  |p_i| <= p_max (i = 0..N)
 *
 * by the regularized primal-dual IPM: barrier-Lagrangian
 * L = f - mu sum log s + y^T c + z^T (g + s), Newton-KKT system eq.
 * ipm-3x3-newton-kkt with Delta_C = Delta_G = eta I and the exact Hessian
 * of L (or its FP32 evaluation, or the Gauss-Newton approximation), Delta z
 * and Delta s eliminated so that the (x, y) system is a dual-regularized LQR
 * with delta = 1/eta, solved for all running instances by one
 * rlqr_solve_batched call per iteration.  The LQR pivot-PD certificate
 * decides the inertia correction rho I (Theorem inertia-al-descent: with
 * correct inertia the primal step descends the augmented barrier-Lagrangian
 * merit), and an Armijo backtracking line search on that merit, with (y, z)
 * fixed, takes the step.
 *
 * State x = (p, th1, th2, dp, dth1, dth2) (cart position, link angles from
 * the upright, rates), control u = horizontal force on the cart; point masses
 * m1, m2 on massless links l1, l2, cart mass m0, no friction.  Inequality
 * rows per stage: 0: u - u_max, 1: -u - u_max (absent at i = N),
 * 2: p - p_max, 3: -p - p_max.
 *
 * Layouts (all DEVICE, FP64 unless stated, instance-major, row-major):
 *   x0, xg  [count][6]            initial states, goal states
 *   X [count][N+1][6]  U [count][N]  Y [count][N+1][6]
 *   S, Z [count][N+1][4]          slacks and bound duals (rows 0, 1 at
 *                                 i = N are unused: S = 1, Z = 0)
 *   mu, rho, kkt [count]          barrier parameter, last inertia shift,
 *                                 last KKT error max(|grad L|, |c|, |g+s|, |s z|)
 *   iters, factorizations, status [count] (int32)
 *                                 status: 0 running, 1 converged (kkt <= tol),
 *                                 2 iteration limit, 3 shift above rho_max
 * The caller owns every buffer; scratch lives in a caller-provided
 * workspace (rlqr_ipm_workspace_bytes), which holds the LQR data of the
 * last iteration between calls.
 *
 * Synchronisation: rlqr_ipm_iterate and rlqr_ipm_solve read the number of
 * running instances back to the host once per iteration and once per
 * inertia-correction round (a stream synchronisation each); everything else
 * is stream-ordered on `stream`.
 */
#ifndef RLQR_IPM_H_
#define RLQR_IPM_H_

#include "rlqr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t N;          /* stages, 1 <= N <= 4096 */
  double dt;          /* RK4 step */
  double m0, m1, m2;  /* cart and point masses */
  double l1, l2;      /* link lengths */
  double grav;
  double u_max, p_max;
  double wx[6];       /* diagonal stage weight of x - x_g */
  double wu;          /* stage weight of u */
  double wf[6];       /* diagonal terminal weight */
} rlqr_cdp_model;

typedef enum {
  RLQR_IPM_HESS_EXACT_FP64 = 0, /* second derivatives of the RK4 map in FP64 */
  RLQR_IPM_HESS_EXACT_FP32 = 1, /* the same term evaluated in FP32 */
  RLQR_IPM_HESS_GAUSS_NEWTON = 2 /* without the dynamics' second derivatives */
} rlqr_ipm_hessian;

typedef struct {
  int32_t max_iter;   /* Newton systems per instance */
  double tol;         /* on max(|grad_x L|, |c|, |g + s|, |s z|) */
  double eta;         /* Delta_C = Delta_G = eta I (LQR delta = 1/eta) */
  double mu0, mu_min, kappa_mu; /* mu <- max(mu_min, min(mu/5, mu^1.5)) once E_mu <= kappa_mu mu */
  double tau;         /* fraction to the boundary */
  double armijo;      /* sufficient-decrease constant */
  int32_t ls_steps;   /* step halvings (1..30); the last trial is taken if none passes */
  double rho_first, rho_grow, rho_shrink, rho_min, rho_max; /* inertia correction */
  double kappa_sigma; /* z kept in [mu/(kappa s), kappa mu/s] */
  double s_min;       /* initial slack floor */
  int32_t hessian;    /* rlqr_ipm_hessian */
  int32_t lqr_prec;   /* rlqr_prec of the LQR solves */
  int32_t lqr_max_refine;
  double lqr_tol;
} rlqr_ipm_opts;

typedef struct {
  double *X, *U, *Y, *S, *Z;
  double *mu, *rho, *kkt;
  int32_t *iters, *factorizations, *status;
} rlqr_ipm_state;

/* Device pointers into the workspace: the LQR data and solution of the last
 * Newton system (same layouts as rlqr_problem, instance-major with stride
 * of one instance, nx = 6, nu = 1), for inspection. */
typedef struct {
  double *Q, *M, *R, *q, *r, *A, *B, *c, *dx, *du, *dy;
  uint8_t *pivot_pd;
} rlqr_ipm_lqr;

/* Workspace bytes for `count` instances (0 on invalid arguments). */
size_t rlqr_ipm_workspace_bytes(int32_t count, const rlqr_cdp_model *model,
                                const rlqr_ipm_opts *opts);

/* Initial point: X = the RK4 rollout of U0 from x0 (U0 NULL: zeros) or a copy
 * of X0 when it is not NULL; y = 0, s = max(-g, s_min), z = mu0 / s,
 * mu = mu0, rho = 0, counters 0, status 0, kkt = +inf. */
rlqr_status rlqr_ipm_init(int32_t count, const rlqr_cdp_model *model, const rlqr_ipm_opts *opts,
                          const double *x0, const double *U0, const double *X0,
                          rlqr_ipm_state *state, rlqr_stream_t stream);

/* Linearization of every running instance at its current point: the LQR data
 * of the Newton system (rho = 0) in the workspace, the KKT errors, the
 * convergence / iteration-limit decision and the mu update (the first part of
 * one iteration; rlqr_ipm_iterate calls it). */
rlqr_status rlqr_ipm_linearize(int32_t count, const rlqr_cdp_model *model,
                               const rlqr_ipm_opts *opts, const double *x0, const double *xg,
                               rlqr_ipm_state *state, void *ws, size_t ws_bytes,
                               rlqr_stream_t stream);

/* One iteration for every running instance: linearize, one batched LQR solve
 * per inertia-correction round, line search and update.  *n_running (host,
 * may be NULL) receives the number of instances that took this iteration. */
rlqr_status rlqr_ipm_iterate(int32_t count, const rlqr_cdp_model *model,
                             const rlqr_ipm_opts *opts, const double *x0, const double *xg,
                             rlqr_ipm_state *state, void *ws, size_t ws_bytes,
                             int32_t *n_running, rlqr_stream_t stream);

/* Iterations until no instance is running (at most max_iter + 1 calls of
 * rlqr_ipm_iterate).  *n_iterations (host, may be NULL) receives the number
 * of iterations run. */
rlqr_status rlqr_ipm_solve(int32_t count, const rlqr_cdp_model *model, const rlqr_ipm_opts *opts,
                           const double *x0, const double *xg, rlqr_ipm_state *state, void *ws,
                           size_t ws_bytes, int32_t *n_iterations, rlqr_stream_t stream);

/* Pointers to the LQR data inside the workspace. */
rlqr_status rlqr_ipm_lqr_view(int32_t count, const rlqr_cdp_model *model,
                              const rlqr_ipm_opts *opts, void *ws, rlqr_ipm_lqr *out);

#ifdef __cplusplus
}
#endif

#endif /* RLQR_IPM_H_ */

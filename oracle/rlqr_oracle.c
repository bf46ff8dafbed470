/*
 * rlqr_oracle.c -- plain FP64 CPU oracle for the dual-regularized LQR solve.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may call this code.  It shares nothing with the CUDA
 * library (no header, helper, table or constant), and the CUDA library never
 * calls it.  It is deliberately slow and written for reading: no blocking,
 * no fusion, no reordering beyond what the cited passage states.
 *
 * Problem (Section "Dual-Regularized LQR", eq. min-max-with-ys and
 * eq. primal-dual-linear-system / optimal-control-specialization):
 *   stage data Q_i (n x n, i=0..N), M_i (n x m), R_i (m x m), q_i (n, i=0..N),
 *   r_i (m), A_i (n x n), B_i (n x m), c_i (n, i=0..N), Delta_i = delta*I.
 *   All matrices row-major, stage-major contiguous, FP64.
 *
 * Parts
 *   1. rlqr_orc_riccati    -- the sequential recursion (Theorem main-seq-theorem,
 *                             eq. value-fn-formulas, control-law, recover-x0,
 *                             recover-x, and the y_k = P_k x_k + p_k rewrite),
 *                             with unpivoted LDL^T of each state pivot
 *                             I + delta P_i and control pivot G_i; their D signs
 *                             give the pivot-PD certificate (Section
 *                             "Inertia Certification", Theorem
 *                             riccati-inertia-certification-theorem).
 *   2. rlqr_orc_bk_*       -- dense Bunch-Kaufman LDL^T of an assembled symmetric
 *                             matrix (Bunch & Kaufman, Math. Comp. 1977), solve,
 *                             and inertia from the 1x1 / 2x2 blocks of D.
 *   3. rlqr_orc_jacobi_inertia -- cyclic Jacobi eigenvalues (textbook), counted
 *                             by sign with a threshold.
 *   4. rlqr_orc_band_solve -- the KKT system of eq. primal-dual-linear-system in
 *                             the interleaved order (y_0,x_0,u_0,y_1,...,y_N,x_N),
 *                             which is banded, solved by banded LU with partial
 *                             pivoting (the textbook gbtrf algorithm).
 *   5. rlqr_orc_residual   -- the stagewise KKT residual of Section "Residual
 *                             Computation" and the normwise backward error.
 *
 * Status codes: 0 ok, 1 some pivot not positive-definite (solution still
 * returned), 3 zero or non-finite pivot (recursion undefined), 2 bad argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_PD 1
#define ORC_ERR_ARG 2
#define ORC_SINGULAR 3

/* ---------------------------------------------------------------- helpers */

/* C (r x s) = A (r x t) * B (t x s), all row-major. */
static void mm(int r, int t, int s, const double *A, const double *B, double *C) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int k = 0; k < t; ++k) acc += A[i * t + k] * B[k * s + j];
      C[i * s + j] = acc;
    }
}

/* C (r x s) = A^T * B with A (t x r), B (t x s). */
static void mtm(int r, int t, int s, const double *A, const double *B, double *C) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int k = 0; k < t; ++k) acc += A[k * r + i] * B[k * s + j];
      C[i * s + j] = acc;
    }
}

/* y (r) = A (r x t) x (t). */
static void mv(int r, int t, const double *A, const double *x, double *y) {
  for (int i = 0; i < r; ++i) {
    double acc = 0.0;
    for (int k = 0; k < t; ++k) acc += A[i * t + k] * x[k];
    y[i] = acc;
  }
}

/* y (r) = A^T x with A (t x r). */
static void mtv(int r, int t, const double *A, const double *x, double *y) {
  for (int i = 0; i < r; ++i) {
    double acc = 0.0;
    for (int k = 0; k < t; ++k) acc += A[k * r + i] * x[k];
    y[i] = acc;
  }
}

/* Out = (X + X^T) / 2 for an n x n matrix (in place allowed). */
static void symmetrize(int n, double *X) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double v = 0.5 * (X[i * n + j] + X[j * n + i]);
      X[i * n + j] = v;
      X[j * n + i] = v;
    }
}

/* Unpivoted LDL^T of a symmetric n x n matrix (lower triangle read).
 * On exit the strict lower triangle holds the unit-lower L and the diagonal
 * holds D.  Returns -1 on a zero or non-finite D_jj, else the number of
 * negative D_jj (which, by Sylvester's law of inertia, is the number of
 * negative eigenvalues). */
static int ldlt(int n, double *a) {
  int nneg = 0;
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k] * a[k * n + k];
    if (!isfinite(d) || d == 0.0) return -1;
    a[j * n + j] = d;
    if (d < 0.0) ++nneg;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * n + j];
      for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k] * a[k * n + k];
      a[i * n + j] = s / d;
    }
  }
  return nneg;
}

/* Solve (L D L^T) X = B in place for B (n x r), factor from ldlt(). */
static void ldlt_solve(int n, const double *f, int r, double *B) {
  for (int col = 0; col < r; ++col) {
    for (int i = 0; i < n; ++i) { /* L z = b */
      double s = B[i * r + col];
      for (int k = 0; k < i; ++k) s -= f[i * n + k] * B[k * r + col];
      B[i * r + col] = s;
    }
    for (int i = 0; i < n; ++i) B[i * r + col] /= f[i * n + i]; /* D w = z */
    for (int i = n - 1; i >= 0; --i) { /* L^T x = w */
      double s = B[i * r + col];
      for (int k = i + 1; k < n; ++k) s -= f[k * n + i] * B[k * r + col];
      B[i * r + col] = s;
    }
  }
}

/* ------------------------------------------- 1. sequential recursion */

/*
 * The sequential dual-regularized Riccati recursion, in the paper's order.
 *
 * Backward (proof of Theorem main-seq-theorem):
 *   P_N = Q_N, p_N = q_N;
 *   for k = N-1 .. 0:
 *     W_{k+1} = P_{k+1} (I + Delta P_{k+1})^{-1}   (symmetric, Corollary
 *               inverse-helper-corollary; computed as (I+delta P)^{-1} P)
 *     G_k = R_k + B_k^T W_{k+1} B_k
 *     g_{k+1} = p_{k+1} + W_{k+1} (c_{k+1} - Delta p_{k+1})
 *     H_k = B_k^T W_{k+1} A_k + M_k^T,   h_k = r_k + B_k^T g_{k+1}
 *     K_k = -G_k^{-1} H_k,               k_k = -G_k^{-1} h_k
 *     P_k = A_k^T W_{k+1} A_k + Q_k + H_k^T K_k      (eq. value-fn-formulas)
 *     p_k = q_k + A_k^T g_{k+1} + H_k^T k_k
 * Forward:
 *   x_0 = (I + Delta P_0)^{-1} (c_0 - Delta p_0)                (eq. recover-x0)
 *   u_k = K_k x_k + k_k                                          (eq. control-law)
 *   x_{k+1} = (I + Delta P_{k+1})^{-1}(A_k x_k + B_k u_k + c_{k+1} - Delta p_{k+1})
 *                                                                 (eq. recover-x)
 *   y_k = P_k x_k + p_k                                 (end of that proof)
 * Certificate (Section "Inertia Certification"): the state pivot is
 * Shat_i = I + Delta^{1/2} P_i Delta^{1/2} = I + delta P_i for Delta = delta I;
 * the control pivot is G_i.  flags[i] bit0 = Shat_i PD, bit1 = G_i PD
 * (bit1 is set for i = N, which has no control pivot).  PD is decided by the
 * signs of D in an unpivoted LDL^T (strictly positive = PD).
 *
 * Q and R are symmetrized as (X + X^T)/2 before use; P_k and W_k are kept
 * exactly symmetric the same way.
 *
 * Outputs x ((N+1) n), u (N m), y ((N+1) n), flags (N+1).  Optional (may be
 * NULL): neg_S (N+1) / neg_G (N) negative-eigenvalue counts of the pivots,
 * P_out ((N+1) n n), p_out ((N+1) n), K_out (N m n), k_out (N m), and the
 * pivots before factorization: S_out ((N+1) n n, I + delta P_i) and
 * G_out (N m m).
 */
int rlqr_orc_riccati(int N, int n, int m, const double *Q, const double *M, const double *R,
                     const double *q, const double *r, const double *A, const double *B,
                     const double *c, double delta, double *x, double *u, double *y,
                     uint8_t *flags, int32_t *neg_S, int32_t *neg_G, double *P_out,
                     double *p_out, double *K_out, double *k_out, double *S_out,
                     double *G_out) {
  if (N < 1 || n < 1 || m < 1 || !(delta >= 0.0)) return ORC_ERR_ARG;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
  double *P = (double *)malloc(sizeof(double) * nn * (N + 1));
  double *p = (double *)malloc(sizeof(double) * n * (size_t)(N + 1));
  double *K = (double *)malloc(sizeof(double) * nm * N);
  double *kk = (double *)malloc(sizeof(double) * m * (size_t)N);
  double *F = (double *)malloc(sizeof(double) * nn * (N + 1)); /* LDL^T of I + delta P_i */
  double *W = (double *)malloc(sizeof(double) * nn);
  double *WA = (double *)malloc(sizeof(double) * nn);
  double *WB = (double *)malloc(sizeof(double) * nm);
  double *G = (double *)malloc(sizeof(double) * mm_);
  double *H = (double *)malloc(sizeof(double) * nm);
  double *T = (double *)malloc(sizeof(double) * nn);
  double *g = (double *)malloc(sizeof(double) * n);
  double *h = (double *)malloc(sizeof(double) * m);
  double *v = (double *)malloc(sizeof(double) * n);
  double *t = (double *)malloc(sizeof(double) * n);
  int status = ORC_OK;
  if (!P || !p || !K || !kk || !F || !W || !WA || !WB || !G || !H || !T || !g || !h || !v || !t) {
    status = ORC_ERR_ARG;
    goto done;
  }

  /* P_N = Q_N, p_N = q_N */
  memcpy(P + nn * N, Q + nn * N, sizeof(double) * nn);
  symmetrize(n, P + nn * N);
  memcpy(p + (size_t)n * N, q + (size_t)n * N, sizeof(double) * n);
  flags[N] = 2; /* no control pivot at the terminal stage */

  for (int k = N - 1; k >= 0; --k) {
    const double *Pn = P + nn * (k + 1), *pn = p + (size_t)n * (k + 1);
    const double *Ak = A + nn * k, *Bk = B + nm * k, *Mk = M + nm * k, *Rk = R + mm_ * k;
    const double *cn = c + (size_t)n * (k + 1);
    /* state pivot I + delta P_{k+1} */
    double *Fk = F + nn * (k + 1);
    for (size_t i = 0; i < nn; ++i) Fk[i] = delta * Pn[i];
    for (int i = 0; i < n; ++i) Fk[i * n + i] += 1.0;
    if (S_out) memcpy(S_out + nn * (k + 1), Fk, sizeof(double) * nn);
    int ns = ldlt(n, Fk);
    if (ns < 0) { status = ORC_SINGULAR; goto done; }
    if (neg_S) neg_S[k + 1] = ns;
    if (ns == 0) flags[k + 1] |= 1;
    /* W_{k+1} = (I + delta P_{k+1})^{-1} P_{k+1} */
    memcpy(W, Pn, sizeof(double) * nn);
    ldlt_solve(n, Fk, n, W);
    symmetrize(n, W);
    /* G_k = R_k + B_k^T W B_k */
    mm(n, n, m, W, Bk, WB);
    mtm(m, n, m, Bk, WB, G);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) G[i * m + j] += 0.5 * (Rk[i * m + j] + Rk[j * m + i]);
    /* g_{k+1} = p_{k+1} + W (c_{k+1} - delta p_{k+1}) */
    for (int i = 0; i < n; ++i) v[i] = cn[i] - delta * pn[i];
    mv(n, n, W, v, g);
    for (int i = 0; i < n; ++i) g[i] += pn[i];
    /* H_k = B^T W A + M^T ; h_k = r_k + B^T g */
    mm(n, n, n, W, Ak, WA);
    mtm(m, n, n, Bk, WA, H);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) H[i * n + j] += Mk[j * m + i];
    mtv(m, n, Bk, g, h);
    for (int i = 0; i < m; ++i) h[i] += r[(size_t)m * k + i];
    /* control pivot G_k */
    if (G_out) memcpy(G_out + mm_ * k, G, sizeof(double) * mm_);
    int ng = ldlt(m, G);
    if (ng < 0) { status = ORC_SINGULAR; goto done; }
    if (neg_G) neg_G[k] = ng;
    flags[k] = (ng == 0) ? 2 : 0;
    /* K_k = -G^{-1} H ; k_k = -G^{-1} h */
    double *Kk = K + nm * k, *kv = kk + (size_t)m * k;
    for (size_t i = 0; i < nm; ++i) Kk[i] = -H[i];
    ldlt_solve(m, G, n, Kk);
    for (int i = 0; i < m; ++i) kv[i] = -h[i];
    ldlt_solve(m, G, 1, kv);
    /* P_k = A^T W A + Q_k + H^T K */
    double *Pk = P + nn * k;
    mtm(n, n, n, Ak, WA, Pk);
    mtm(n, m, n, H, Kk, T);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        Pk[i * n + j] += T[i * n + j] + 0.5 * (Q[nn * k + i * n + j] + Q[nn * k + j * n + i]);
    symmetrize(n, Pk);
    /* p_k = q_k + A^T g + H^T k_k */
    double *pk = p + (size_t)n * k;
    mtv(n, n, Ak, g, pk);
    mtv(n, m, H, kv, t);
    for (int i = 0; i < n; ++i) pk[i] += t[i] + q[(size_t)n * k + i];
  }
  /* initial-state pivot I + delta P_0 */
  {
    double *F0 = F;
    for (size_t i = 0; i < nn; ++i) F0[i] = delta * P[i];
    for (int i = 0; i < n; ++i) F0[i * n + i] += 1.0;
    if (S_out) memcpy(S_out, F0, sizeof(double) * nn);
    int ns = ldlt(n, F0);
    if (ns < 0) { status = ORC_SINGULAR; goto done; }
    if (neg_S) neg_S[0] = ns;
    if (ns == 0) flags[0] |= 1;
  }
  /* forward pass */
  for (int i = 0; i < n; ++i) x[i] = c[i] - delta * p[i];
  ldlt_solve(n, F, 1, x);
  for (int k = 0; k < N; ++k) {
    const double *xk = x + (size_t)n * k;
    double *uk = u + (size_t)m * k, *xn = x + (size_t)n * (k + 1);
    mv(m, n, K + nm * k, xk, uk);
    for (int i = 0; i < m; ++i) uk[i] += kk[(size_t)m * k + i];
    mv(n, n, A + nn * k, xk, xn);
    mv(n, m, B + nm * k, uk, t);
    for (int i = 0; i < n; ++i)
      xn[i] += t[i] + c[(size_t)n * (k + 1) + i] - delta * p[(size_t)n * (k + 1) + i];
    ldlt_solve(n, F + nn * (k + 1), 1, xn);
  }
  for (int k = 0; k <= N; ++k) {
    mv(n, n, P + nn * k, x + (size_t)n * k, y + (size_t)n * k);
    for (int i = 0; i < n; ++i) y[(size_t)n * k + i] += p[(size_t)n * k + i];
  }
  for (int k = 0; k <= N; ++k)
    if (flags[k] != 3) status = ORC_NOT_PD;
  if (P_out) memcpy(P_out, P, sizeof(double) * nn * (N + 1));
  if (p_out) memcpy(p_out, p, sizeof(double) * n * (size_t)(N + 1));
  if (K_out) memcpy(K_out, K, sizeof(double) * nm * N);
  if (k_out) memcpy(k_out, kk, sizeof(double) * m * (size_t)N);
done:
  free(P); free(p); free(K); free(kk); free(F); free(W); free(WA); free(WB);
  free(G); free(H); free(T); free(g); free(h); free(v); free(t);
  return status;
}

/* Many independent instances with the same (N, n, m), stacked along a leading
 * batch axis; delta per instance.  Instances run in parallel with OpenMP
 * (this is the CPU baseline's only concession to speed). status[b] per
 * instance. */
void rlqr_orc_riccati_batch(int count, int N, int n, int m, const double *Q, const double *M,
                            const double *R, const double *q, const double *r, const double *A,
                            const double *B, const double *c, const double *delta, double *x,
                            double *u, double *y, uint8_t *flags, int32_t *status) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < count; ++b) {
    status[b] = rlqr_orc_riccati(
        N, n, m, Q + nn * (N + 1) * b, M + nm * N * b, R + mm_ * N * b, q + (size_t)n * (N + 1) * b,
        r + (size_t)m * N * b, A + nn * N * b, B + nm * N * b, c + (size_t)n * (N + 1) * b,
        delta[b], x + (size_t)n * (N + 1) * b, u + (size_t)m * N * b, y + (size_t)n * (N + 1) * b,
        flags + (size_t)(N + 1) * b, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
  }
}

/* --------------------------------------- 2. dense Bunch-Kaufman LDL^T */

/*
 * In-place Bunch-Kaufman factorization P K P^T = L D L^T of a dense symmetric
 * dim x dim matrix K (full storage, both triangles kept symmetric).  Partial
 * pivoting with alpha = (1 + sqrt(17)) / 8 (Bunch & Kaufman 1977; Golub & Van
 * Loan, Matrix Computations, Section 4.4).
 *   perm[k]  : row/column swapped with the pivot row at step k (k itself if none)
 *   bsize[k] : 1 for a 1x1 pivot at k, 2 for the first index of a 2x2 pivot,
 *              0 for the second index of a 2x2 pivot.
 * On exit: strict lower triangle = L (the (k+1, k) entry of a 2x2 block holds
 * D's off-diagonal), diagonal = D's diagonal.  Returns the number of exactly
 * zero 1x1 pivots (0 for a nonsingular matrix in exact arithmetic).
 */
int rlqr_orc_bk_factor(int dim, double *K, int32_t *perm, int32_t *bsize) {
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int zero = 0;
  int k = 0;
  while (k < dim) {
    double absakk = fabs(K[(size_t)k * dim + k]);
    int imax = k;
    double colmax = 0.0;
    for (int i = k + 1; i < dim; ++i) {
      double a = fabs(K[(size_t)i * dim + k]);
      if (a > colmax) { colmax = a; imax = i; }
    }
    int kstep = 1, kp = k;
    if (fmax(absakk, colmax) == 0.0) {
      ++zero; /* zero column: D_kk = 0, nothing to eliminate */
      perm[k] = k;
      bsize[k] = 1;
      ++k;
      continue;
    }
    if (absakk >= alpha * colmax) {
      kp = k;
    } else {
      double rowmax = 0.0; /* largest off-diagonal in row/column imax of the trailing block */
      for (int j = k; j < dim; ++j)
        if (j != imax) rowmax = fmax(rowmax, fabs(K[(size_t)imax * dim + j]));
      if (absakk * rowmax >= alpha * colmax * colmax) {
        kp = k;
      } else if (fabs(K[(size_t)imax * dim + imax]) >= alpha * rowmax) {
        kp = imax;
      } else {
        kp = imax;
        kstep = 2;
      }
    }
    int kk = k + kstep - 1;
    if (kp != kk) {
      /* symmetric interchange of kk and kp: rows over all columns (this also
       * permutes the rows of the L computed so far), then columns over the
       * trailing rows */
      for (int j = 0; j < dim; ++j) {
        double tmp = K[(size_t)kk * dim + j];
        K[(size_t)kk * dim + j] = K[(size_t)kp * dim + j];
        K[(size_t)kp * dim + j] = tmp;
      }
      for (int i = k; i < dim; ++i) {
        double tmp = K[(size_t)i * dim + kk];
        K[(size_t)i * dim + kk] = K[(size_t)i * dim + kp];
        K[(size_t)i * dim + kp] = tmp;
      }
    }
    if (kstep == 1) {
      perm[k] = kp;
      bsize[k] = 1;
      double d = K[(size_t)k * dim + k];
      for (int i = k + 1; i < dim; ++i) {
        double lik = K[(size_t)i * dim + k] / d;
        for (int j = k + 1; j < dim; ++j) K[(size_t)i * dim + j] -= lik * K[(size_t)k * dim + j];
      }
      for (int i = k + 1; i < dim; ++i) {
        K[(size_t)i * dim + k] /= d;
        K[(size_t)k * dim + i] = K[(size_t)i * dim + k] * d; /* keep row k consistent (unused) */
      }
    } else {
      perm[k] = k;
      perm[k + 1] = kp;
      bsize[k] = 2;
      bsize[k + 1] = 0;
      double d11 = K[(size_t)k * dim + k], d21 = K[(size_t)(k + 1) * dim + k];
      double d22 = K[(size_t)(k + 1) * dim + k + 1];
      double det = d11 * d22 - d21 * d21;
      /* rows i > k+1: [l_i1 l_i2] = [a_i1 a_i2] D^{-1} */
      for (int i = k + 2; i < dim; ++i) {
        double a1 = K[(size_t)i * dim + k], a2 = K[(size_t)i * dim + k + 1];
        double l1 = (a1 * d22 - a2 * d21) / det;
        double l2 = (a2 * d11 - a1 * d21) / det;
        for (int j = k + 2; j < dim; ++j)
          K[(size_t)i * dim + j] -= l1 * K[(size_t)k * dim + j] + l2 * K[(size_t)(k + 1) * dim + j];
        /* stash the multipliers; row k / k+1 entries for j > i are still
         * needed by later rows, so write L after the loop */
        K[(size_t)i * dim + k] = l1;
        K[(size_t)i * dim + k + 1] = l2;
      }
    }
    k += kstep;
  }
  return zero;
}

/* Solve K z = rhs with the factor from rlqr_orc_bk_factor (in place on rhs). */
void rlqr_orc_bk_solve(int dim, const double *F, const int32_t *perm, const int32_t *bsize,
                       double *b) {
  /* P b: apply the interchanges in order */
  for (int k = 0; k < dim; ++k) {
    if (bsize[k] == 1 || bsize[k] == 0) {
      int kk = k, kp = perm[k];
      if (kp != kk) { double t = b[kk]; b[kk] = b[kp]; b[kp] = t; }
    }
  }
  /* L z = P b (unit lower, the 2x2 blocks' off-diagonal is D's, not L's) */
  for (int i = 0; i < dim; ++i) {
    double s = b[i];
    int lim = (bsize[i] == 0) ? i - 1 : i; /* skip D's off-diagonal inside a 2x2 block */
    for (int j = 0; j < lim; ++j) s -= F[(size_t)i * dim + j] * b[j];
    b[i] = s;
  }
  /* D w = z */
  for (int k = 0; k < dim;) {
    if (bsize[k] == 1) {
      double d = F[(size_t)k * dim + k];
      b[k] = (d != 0.0) ? b[k] / d : 0.0;
      k += 1;
    } else {
      double d11 = F[(size_t)k * dim + k], d21 = F[(size_t)(k + 1) * dim + k];
      double d22 = F[(size_t)(k + 1) * dim + k + 1];
      double det = d11 * d22 - d21 * d21;
      double b1 = b[k], b2 = b[k + 1];
      b[k] = (d22 * b1 - d21 * b2) / det;
      b[k + 1] = (d11 * b2 - d21 * b1) / det;
      k += 2;
    }
  }
  /* L^T x = w */
  for (int i = dim - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < dim; ++j) {
      if (bsize[j] == 0 && j == i + 1) continue; /* D's off-diagonal */
      s -= F[(size_t)j * dim + i] * b[j];
    }
    b[i] = s;
  }
  /* P^T: undo the interchanges in reverse order */
  for (int k = dim - 1; k >= 0; --k) {
    if (bsize[k] == 1 || bsize[k] == 0) {
      int kk = k, kp = perm[k];
      if (kp != kk) { double t = b[kk]; b[kk] = b[kp]; b[kp] = t; }
    }
  }
}

/* Inertia (n_plus, n_minus, n_zero) from the D of rlqr_orc_bk_factor. */
void rlqr_orc_bk_inertia(int dim, const double *F, const int32_t *bsize, int32_t *inertia) {
  int pos = 0, neg = 0, zer = 0;
  for (int k = 0; k < dim;) {
    if (bsize[k] == 1) {
      double d = F[(size_t)k * dim + k];
      if (d > 0) ++pos; else if (d < 0) ++neg; else ++zer;
      k += 1;
    } else {
      double d11 = F[(size_t)k * dim + k], d21 = F[(size_t)(k + 1) * dim + k];
      double d22 = F[(size_t)(k + 1) * dim + k + 1];
      double det = d11 * d22 - d21 * d21, tr = d11 + d22;
      if (det < 0) { ++pos; ++neg; }
      else if (det > 0) { if (tr > 0) pos += 2; else neg += 2; }
      else { ++zer; if (tr > 0) ++pos; else if (tr < 0) ++neg; else ++zer; }
      k += 2;
    }
  }
  inertia[0] = pos; inertia[1] = neg; inertia[2] = zer;
}

/* ------------------------------------------- 3. cyclic Jacobi inertia */

/* Eigenvalues of a dense symmetric matrix by the cyclic Jacobi method
 * (Golub & Van Loan, Section 8.5), destroying K.  Counts eigenvalues > tau,
 * < -tau and in [-tau, tau].  Returns the number of sweeps used. */
int rlqr_orc_jacobi_inertia(int dim, double *K, double tau, int max_sweeps, int32_t *inertia,
                            double *eig) {
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) {
        double v = K[(size_t)i * dim + j] * K[(size_t)i * dim + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < dim - 1; ++p)
      for (int qq = p + 1; qq < dim; ++qq) {
        double apq = K[(size_t)p * dim + qq];
        if (apq == 0.0) continue;
        double app = K[(size_t)p * dim + p], aqq = K[(size_t)qq * dim + qq];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int kx = 0; kx < dim; ++kx) { /* columns p, q */
          double akp = K[(size_t)kx * dim + p], akq = K[(size_t)kx * dim + qq];
          K[(size_t)kx * dim + p] = cs * akp - sn * akq;
          K[(size_t)kx * dim + qq] = sn * akp + cs * akq;
        }
        for (int kx = 0; kx < dim; ++kx) { /* rows p, q */
          double apk = K[(size_t)p * dim + kx], aqk = K[(size_t)qq * dim + kx];
          K[(size_t)p * dim + kx] = cs * apk - sn * aqk;
          K[(size_t)qq * dim + kx] = sn * apk + cs * aqk;
        }
      }
  }
  int pos = 0, neg = 0, zer = 0;
  for (int i = 0; i < dim; ++i) {
    double d = K[(size_t)i * dim + i];
    if (eig) eig[i] = d;
    if (d > tau) ++pos; else if (d < -tau) ++neg; else ++zer;
  }
  inertia[0] = pos; inertia[1] = neg; inertia[2] = zer;
  return sweep;
}

/* ------------------------------------------------ 4. banded LU solve */

/*
 * Solve the KKT system of eq. primal-dual-linear-system by banded LU with
 * partial pivoting.  Unknowns are ordered per stage as (y_i, x_i, u_i) for
 * i < N and (y_N, x_N) last, so every coupling (the -I, A_i, B_i and Delta
 * blocks of C and Delta, and the Q, M, R blocks of P) lies within
 * kl = ku = 2n + m - 1 of the diagonal.  Returns 0, or 3 on a zero pivot.
 */
typedef struct {
  double *ab;
  int dim, kl, ku, width;
} band_t;

static double *bref(band_t *b, int i, int j) {
  int off = j - i + b->kl; /* row i stores columns [i - kl, i - kl + width) */
  if (off < 0 || off >= b->width) return NULL;
  return b->ab + (size_t)i * b->width + off;
}

static void bset(band_t *b, int i, int j, double v) {
  double *p = bref(b, i, j);
  if (p) *p += v;
}

int rlqr_orc_band_solve(int N, int n, int m, const double *Q, const double *M, const double *R,
                        const double *q, const double *r, const double *A, const double *B,
                        const double *c, double delta, double *x, double *u, double *y) {
  const int blk = 2 * n + m;
  const int dim = N * blk + 2 * n;
  band_t bd;
  bd.dim = dim;
  bd.kl = bd.ku = 2 * n + m - 1;
  bd.width = 2 * bd.kl + bd.ku + 1;
  bd.ab = (double *)calloc((size_t)dim * bd.width, sizeof(double));
  double *rhs = (double *)calloc((size_t)dim, sizeof(double));
  if (!bd.ab || !rhs) { free(bd.ab); free(rhs); return ORC_ERR_ARG; }
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
#define YI(i) ((i) * blk)
#define XI(i) ((i) * blk + n)
#define UI(i) ((i) * blk + 2 * n)
  for (int i = 0; i <= N; ++i) {
    /* P block: Q_i (and M_i, R_i for i < N), symmetrized */
    for (int a = 0; a < n; ++a)
      for (int b2 = 0; b2 < n; ++b2)
        bset(&bd, XI(i) + a, XI(i) + b2, 0.5 * (Q[nn * i + a * n + b2] + Q[nn * i + b2 * n + a]));
    if (i < N) {
      for (int a = 0; a < n; ++a)
        for (int b2 = 0; b2 < m; ++b2) {
          bset(&bd, XI(i) + a, UI(i) + b2, M[nm * i + a * m + b2]);
          bset(&bd, UI(i) + b2, XI(i) + a, M[nm * i + a * m + b2]);
        }
      for (int a = 0; a < m; ++a)
        for (int b2 = 0; b2 < m; ++b2)
          bset(&bd, UI(i) + a, UI(i) + b2, 0.5 * (R[mm_ * i + a * m + b2] + R[mm_ * i + b2 * m + a]));
    }
    /* C and -Delta: row y_i has -I on x_i and -delta on y_i; row y_{i+1} has
     * A_i on x_i and B_i on u_i.  The matrix is symmetric: mirror C^T. */
    for (int a = 0; a < n; ++a) {
      bset(&bd, YI(i) + a, XI(i) + a, -1.0);
      bset(&bd, XI(i) + a, YI(i) + a, -1.0);
      bset(&bd, YI(i) + a, YI(i) + a, -delta);
    }
    if (i < N) {
      for (int a = 0; a < n; ++a) {
        for (int b2 = 0; b2 < n; ++b2) {
          bset(&bd, YI(i + 1) + a, XI(i) + b2, A[nn * i + a * n + b2]);
          bset(&bd, XI(i) + b2, YI(i + 1) + a, A[nn * i + a * n + b2]);
        }
        for (int b2 = 0; b2 < m; ++b2) {
          bset(&bd, YI(i + 1) + a, UI(i) + b2, B[nm * i + a * m + b2]);
          bset(&bd, UI(i) + b2, YI(i + 1) + a, B[nm * i + a * m + b2]);
        }
      }
    }
    /* right-hand side: K z = -[s; c] */
    for (int a = 0; a < n; ++a) {
      rhs[XI(i) + a] = -q[(size_t)n * i + a];
      rhs[YI(i) + a] = -c[(size_t)n * i + a];
    }
    if (i < N)
      for (int a = 0; a < m; ++a) rhs[UI(i) + a] = -r[(size_t)m * i + a];
  }
  /* LU with partial pivoting; the multipliers overwrite the eliminated entries */
  int *piv = (int *)malloc(sizeof(int) * dim);
  int status = ORC_OK;
  for (int k = 0; k < dim; ++k) {
    int last = k + bd.kl < dim - 1 ? k + bd.kl : dim - 1;
    int p = k;
    double best = fabs(*bref(&bd, k, k));
    for (int i = k + 1; i <= last; ++i) {
      double *e = bref(&bd, i, k);
      if (e && fabs(*e) > best) { best = fabs(*e); p = i; }
    }
    piv[k] = p;
    if (best == 0.0 || !isfinite(best)) { status = ORC_SINGULAR; break; }
    int jend = k + bd.kl + bd.ku < dim - 1 ? k + bd.kl + bd.ku : dim - 1;
    if (p != k) {
      for (int j = k; j <= jend; ++j) {
        double *e1 = bref(&bd, k, j), *e2 = bref(&bd, p, j);
        double v1 = e1 ? *e1 : 0.0, v2 = e2 ? *e2 : 0.0;
        if (e1) *e1 = v2;
        if (e2) *e2 = v1;
      }
      double t = rhs[k]; rhs[k] = rhs[p]; rhs[p] = t;
    }
    double d = *bref(&bd, k, k);
    for (int i = k + 1; i <= last; ++i) {
      double *e = bref(&bd, i, k);
      if (!e || *e == 0.0) continue;
      double l = *e / d;
      *e = 0.0;
      for (int j = k + 1; j <= jend; ++j) {
        double *ukj = bref(&bd, k, j);
        if (!ukj || *ukj == 0.0) continue;
        double *eij = bref(&bd, i, j);
        if (eij) *eij -= l * *ukj;
      }
      rhs[i] -= l * rhs[k];
    }
  }
  if (status == ORC_OK) {
    for (int k = dim - 1; k >= 0; --k) {
      int jend = k + bd.kl + bd.ku < dim - 1 ? k + bd.kl + bd.ku : dim - 1;
      double s = rhs[k];
      for (int j = k + 1; j <= jend; ++j) {
        double *e = bref(&bd, k, j);
        if (e) s -= *e * rhs[j];
      }
      rhs[k] = s / *bref(&bd, k, k);
    }
    for (int i = 0; i <= N; ++i) {
      for (int a = 0; a < n; ++a) {
        x[(size_t)n * i + a] = rhs[XI(i) + a];
        y[(size_t)n * i + a] = rhs[YI(i) + a];
      }
      if (i < N)
        for (int a = 0; a < m; ++a) u[(size_t)m * i + a] = rhs[UI(i) + a];
    }
  }
#undef YI
#undef XI
#undef UI
  free(piv);
  free(bd.ab);
  free(rhs);
  return status;
}

/* ----------------------------------------------------- 5. residual */

/*
 * KKT residual of Section "Residual Computation":
 *   res_q[i] = Q_i x_i + M_i u_i + A_i^T y_{i+1} + q_i - y_i   (i < N)
 *   res_r[i] = M_i^T x_i + R_i u_i + B_i^T y_{i+1} + r_i       (i < N)
 *   res_q[N] = Q_N x_N + q_N - y_N
 *   res_c[0] = c_0 - delta y_0 - x_0
 *   res_c[i+1] = A_i x_i + B_i u_i + c_{i+1} - delta y_{i+1} - x_{i+1}
 * This is K z + [s; c] with K the matrix of eq. primal-dual-linear-system.
 * Any of res_q / res_r / res_c may be NULL.  norms (may be NULL) receives
 * [ ||K z + b||_inf, ||K||_inf, ||z||_inf, ||b||_inf, rel ] with
 * rel = ||K z + b||_inf / (||K||_inf ||z||_inf + ||b||_inf), the normwise
 * backward error (Rigal-Gaches; Higham, Accuracy and Stability, Thm 7.1).
 * Q and R are symmetrized as in part 1.
 */
void rlqr_orc_residual(int N, int n, int m, const double *Q, const double *M, const double *R,
                       const double *q, const double *r, const double *A, const double *B,
                       const double *c, double delta, const double *x, const double *u,
                       const double *y, double *res_q, double *res_r, double *res_c,
                       double *norms) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
  double rmax = 0.0, kmax = 0.0, zmax = 0.0, bmax = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double *Qi = Q + nn * i, *xi = x + (size_t)n * i, *yi = y + (size_t)n * i;
    /* stationarity in x_i */
    for (int a = 0; a < n; ++a) {
      double s = q[(size_t)n * i + a] - yi[a];
      double rowabs = 1.0; /* the -I on y_i */
      for (int b2 = 0; b2 < n; ++b2) {
        double qab = 0.5 * (Qi[a * n + b2] + Qi[b2 * n + a]);
        s += qab * xi[b2];
        rowabs += fabs(qab);
      }
      if (i < N) {
        const double *Mi = M + nm * i, *Ai = A + nn * i, *ui = u + (size_t)m * i;
        const double *yn = y + (size_t)n * (i + 1);
        for (int b2 = 0; b2 < m; ++b2) { s += Mi[a * m + b2] * ui[b2]; rowabs += fabs(Mi[a * m + b2]); }
        for (int b2 = 0; b2 < n; ++b2) { s += Ai[b2 * n + a] * yn[b2]; rowabs += fabs(Ai[b2 * n + a]); }
      }
      if (res_q) res_q[(size_t)n * i + a] = s;
      rmax = fmax(rmax, fabs(s));
      kmax = fmax(kmax, rowabs);
      bmax = fmax(bmax, fabs(q[(size_t)n * i + a]));
    }
    /* stationarity in u_i */
    if (i < N) {
      const double *Mi = M + nm * i, *Ri = R + mm_ * i, *Bi = B + nm * i, *ui = u + (size_t)m * i;
      const double *yn = y + (size_t)n * (i + 1);
      for (int a = 0; a < m; ++a) {
        double s = r[(size_t)m * i + a], rowabs = 0.0;
        for (int b2 = 0; b2 < n; ++b2) { s += Mi[b2 * m + a] * xi[b2]; rowabs += fabs(Mi[b2 * m + a]); }
        for (int b2 = 0; b2 < m; ++b2) {
          double rab = 0.5 * (Ri[a * m + b2] + Ri[b2 * m + a]);
          s += rab * ui[b2];
          rowabs += fabs(rab);
        }
        for (int b2 = 0; b2 < n; ++b2) { s += Bi[b2 * m + a] * yn[b2]; rowabs += fabs(Bi[b2 * m + a]); }
        if (res_r) res_r[(size_t)m * i + a] = s;
        rmax = fmax(rmax, fabs(s));
        kmax = fmax(kmax, rowabs);
        bmax = fmax(bmax, fabs(r[(size_t)m * i + a]));
        zmax = fmax(zmax, fabs(ui[a]));
      }
    }
    /* primal feasibility rows (y_i) */
    for (int a = 0; a < n; ++a) {
      double s = c[(size_t)n * i + a] - delta * yi[a] - xi[a];
      double rowabs = 1.0 + delta;
      if (i > 0) {
        const double *Ap = A + nn * (i - 1), *Bp = B + nm * (i - 1);
        const double *xp = x + (size_t)n * (i - 1), *up = u + (size_t)m * (i - 1);
        for (int b2 = 0; b2 < n; ++b2) { s += Ap[a * n + b2] * xp[b2]; rowabs += fabs(Ap[a * n + b2]); }
        for (int b2 = 0; b2 < m; ++b2) { s += Bp[a * m + b2] * up[b2]; rowabs += fabs(Bp[a * m + b2]); }
      }
      if (res_c) res_c[(size_t)n * i + a] = s;
      rmax = fmax(rmax, fabs(s));
      kmax = fmax(kmax, rowabs);
      bmax = fmax(bmax, fabs(c[(size_t)n * i + a]));
      zmax = fmax(zmax, fmax(fabs(xi[a]), fabs(yi[a])));
    }
  }
  if (norms) {
    norms[0] = rmax;
    norms[1] = kmax;
    norms[2] = zmax;
    norms[3] = bmax;
    double den = kmax * zmax + bmax;
    norms[4] = den > 0.0 ? rmax / den : rmax;
  }
}

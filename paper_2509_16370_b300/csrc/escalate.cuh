// escalate.cuh -- FP64 re-decision of the pivot certificate for instances
// whose FP32-computed pivot matrices fell inside the decision margin.
//
// The mixed-precision path keeps a certificate decision only when it holds
// with a margin (kMarginTau, relative to the Jacobi-scaled pivot matrix:
// X - tau D provably PD, or X + tau D provably not PD).  A decision that
// does not, or a non-finite pivot, marks the instance (InstState::escalated).
// k_escalate then runs the backward recursion of Theorem main-seq-theorem
// once more in FP64 with the formulas of the plain path -- W_{k+1} = (I +
// delta P_{k+1})^{-1} P_{k+1} by LDL^T solves, G_k = R_k + B_k^T W B_k, H_k =
// B_k^T W A_k + M_k^T, K_k = -G_k^{-1} H_k, P_k = A_k^T W A_k + Q_k + H_k^T
// K_k, with Q, R, P and W symmetrized -- and takes every flag of the
// instance from the signs of the unpivoted LDL^T of I + delta P_i and G_i
// (Section "Inertia Certification").  A zero or non-finite pivot stops the
// recursion with RLQR_ERR_SINGULAR.  Only the flags, the pivot status and
// the status output change: the solution has already been refined against
// the FP64 residual.  One CTA per instance; unmarked instances return at
// once.
#pragma once

#include "common.cuh"

namespace rlqr {

constexpr int kEscThreads = 128;

__host__ __device__ inline size_t escalate_smem_bytes(int n, int m) {
  return sizeof(double) * (4 * (size_t)n * n + 3 * (size_t)n * m + (size_t)m * m) + 64;
}

// In-place unpivoted LDL^T of the symmetric k x k matrix F (row-major, lower
// triangle used; strict lower triangle <- L, diagonal <- D).  Returns the
// number of negative pivots, or -1 on a zero or non-finite pivot.  All
// threads of the block call it.
__device__ int esc_ldlt(double *F, int k) {
  const int tid = threadIdx.x;
  int neg = 0;
  for (int j = 0; j < k; ++j) {
    __syncthreads();
    const double d = F[j * k + j];
    if (!isfinite(d) || d == 0.0) return -1;  // uniform: every thread read the same d
    if (d < 0.0) ++neg;
    const int r = k - 1 - j;
    for (int idx = tid; idx < r * (r + 1) / 2; idx += blockDim.x) {
      int i, c;
      tri_decode(idx, i, c);
      i += j + 1;
      c += j + 1;
      F[i * k + c] -= F[i * k + j] * F[c * k + j] / d;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += blockDim.x) F[i * k + j] /= d;
  }
  __syncthreads();
  return neg;
}

// X (k x cols, row-major) <- (L D L^T)^{-1} X with the factor of esc_ldlt.
__device__ void esc_ldlt_solve(const double *F, int k, double *X, int cols) {
  const int tid = threadIdx.x;
  for (int j = 0; j < k; ++j) {  // L z = x
    __syncthreads();
    for (int e = tid; e < (k - 1 - j) * cols; e += blockDim.x) {
      const int i = j + 1 + e / cols, c = e % cols;
      X[i * cols + c] -= F[i * k + j] * X[j * cols + c];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * cols; e += blockDim.x) X[e] /= F[(e / cols) * k + e / cols];
  for (int j = k - 1; j >= 0; --j) {  // L^T x = w
    __syncthreads();
    for (int e = tid; e < j * cols; e += blockDim.x) {
      const int i = e / cols, c = e % cols;
      X[i * cols + c] -= F[j * k + i] * X[j * cols + c];
    }
  }
  __syncthreads();
}

__device__ void esc_symmetrize(double *X, int k) {
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    if (j < i) {
      const double v = 0.5 * (X[i * k + j] + X[j * k + i]);
      X[i * k + j] = v;
      X[j * k + i] = v;
    }
  }
  __syncthreads();
}

// solved: 1 = the call produced a solution (the status output then also
// reflects convergence); 0 = the status is the pivot status; 2 = the flags
// and the pivot status only (the call's refinement runs concurrently on
// another stream, and k_escalate_status writes the status afterwards).  scan:
// the factor came from the associative scan, whose singular-R marker
// (InstState::r_singular) is then valid; the sequential paths never write
// that field, so it is not read for them.
__global__ void __launch_bounds__(kEscThreads) k_escalate(BatchArgs a, int solved, int scan) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= a.count) return;
  const Inst I = get_inst(a, b);
  if (!I.st->escalated) return;
  const int N = I.N, n = I.n, m = I.m, nn = n * n, nm = n * m, mmm = m * m;
  const int tid = threadIdx.x;
  const double delta = I.delta;
  double *P = reinterpret_cast<double *>(smem_raw);
  double *F = P + nn, *W = F + nn, *WA = W + nn, *WB = WA + nn, *H = WB + nm, *K = H + nm,
         *G = K + nm;
  int status = RLQR_OK;
  // P_N = Q_N (symmetrized)
  for (int e = tid; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    P[e] = 0.5 * (I.Q[(size_t)N * nn + i * n + j] + I.Q[(size_t)N * nn + j * n + i]);
  }
  uint8_t bits_next = 2;  // flags[k + 1] under construction (bit1 of stage N is set)
  for (int k = N - 1; k >= -1; --k) {
    // state pivot I + delta P_{k+1}
    __syncthreads();
    for (int e = tid; e < nn; e += blockDim.x) F[e] = delta * P[e] + ((e / n == e % n) ? 1.0 : 0.0);
    const int ns = esc_ldlt(F, n);
    if (ns < 0) {
      status = RLQR_ERR_SINGULAR;
      break;
    }
    if (ns == 0) bits_next |= 1;
    if (tid == 0) I.flags[k + 1] = bits_next;
    if (ns != 0) status = RLQR_NOT_PD;
    if (k < 0) break;
    const double *Ak = I.A + (size_t)k * nn, *Bk = I.B + (size_t)k * nm, *Mk = I.M + (size_t)k * nm;
    const double *Rk = I.R + (size_t)k * mmm, *Qk = I.Q + (size_t)k * nn;
    // W = (I + delta P)^{-1} P, symmetrized
    for (int e = tid; e < nn; e += blockDim.x) W[e] = P[e];
    esc_ldlt_solve(F, n, W, n);
    esc_symmetrize(W, n);
    // WB = W B, WA = W A
    for (int e = tid; e < nn + nm; e += blockDim.x) {
      if (e < nm) {
        const int i = e / m, t = e % m;
        double v = 0.0;
        for (int l = 0; l < n; ++l) v = fma(W[i * n + l], Bk[l * m + t], v);
        WB[e] = v;
      } else {
        const int f = e - nm, i = f / n, j = f % n;
        double v = 0.0;
        for (int l = 0; l < n; ++l) v = fma(W[i * n + l], Ak[l * n + j], v);
        WA[f] = v;
      }
    }
    __syncthreads();
    // G = B^T W B + R (R symmetrized), H = B^T W A + M^T
    for (int e = tid; e < mmm + nm; e += blockDim.x) {
      if (e < mmm) {
        const int i = e / m, j = e % m;
        double v = 0.0;
        for (int l = 0; l < n; ++l) v = fma(Bk[l * m + i], WB[l * m + j], v);
        G[e] = v + 0.5 * (Rk[i * m + j] + Rk[j * m + i]);
      } else {
        const int f = e - mmm, t = f / n, j = f % n;
        double v = 0.0;
        for (int l = 0; l < n; ++l) v = fma(Bk[l * m + t], WA[l * n + j], v);
        H[f] = v + Mk[j * m + t];
      }
    }
    // control pivot G_k
    const int ng = esc_ldlt(G, m);
    if (ng < 0) {
      status = RLQR_ERR_SINGULAR;
      break;
    }
    bits_next = ng == 0 ? 2 : 0;
    if (ng != 0) status = RLQR_NOT_PD;
    // K = -G^{-1} H
    for (int e = tid; e < nm; e += blockDim.x) K[e] = -H[e];
    esc_ldlt_solve(G, m, K, n);
    // P_k = A^T W A + Q_k + H^T K (Q symmetrized), then symmetrized
    for (int e = tid; e < nn; e += blockDim.x) {
      const int i = e / n, j = e % n;
      double v = 0.0;
      for (int l = 0; l < n; ++l) v = fma(Ak[l * n + i], WA[l * n + j], v);
      double t = 0.0;
      for (int l = 0; l < m; ++l) t = fma(H[l * n + i], K[l * n + j], t);
      P[e] = v + t + 0.5 * (Qk[i * n + j] + Qk[j * n + i]);
    }
    esc_symmetrize(P, n);
  }
  // the scan path's factor needs every R_i invertible: a singular R_i keeps
  // the instance singular whatever the recursion's pivots
  if (scan && I.st->r_singular) status = RLQR_ERR_SINGULAR;
  if (tid == 0) {
    I.st->pivot_status = status;
    if (a.status && solved != 2) {
      const int conv = I.st->converged;
      a.status[b] = !solved ? status
                            : (status == RLQR_ERR_SINGULAR ? RLQR_ERR_SINGULAR
                                                           : (conv ? status : RLQR_ERR_NOT_CONVERGED));
    }
  }
}

// The status output of the escalated instances after a concurrent
// escalation (k_escalate with solved = 2) and refinement have both finished:
// the FP64 pivot status, or RLQR_ERR_NOT_CONVERGED if the refinement did not
// converge.  One thread per instance.
__global__ void k_escalate_status(BatchArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.count || !a.status) return;
  const Inst I = get_inst(a, b);
  if (!I.st->escalated) return;
  const int32_t ps = I.st->pivot_status;
  a.status[b] = ps == RLQR_ERR_SINGULAR ? RLQR_ERR_SINGULAR
                                        : (I.st->converged ? ps : RLQR_ERR_NOT_CONVERGED);
}

}  // namespace rlqr

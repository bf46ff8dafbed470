// ipm.cu -- batched regularized interior-point method on the cart with a
// double pendulum (include/rlqr_ipm.h): Section "The Regularized Interior
// Point Method" and Section "Applying the regularized IPM to optimal
// control".  One CTA per instance for the per-stage work; the Newton system
// of every running instance is one dual-regularized LQR, solved for all of
// them together by rlqr_solve_batched over a compacted instance list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/rlqr.h"
#include "../../include/rlqr_ipm.h"
#include "ipm_model.cuh"

namespace rlqr {
namespace ipm {

constexpr int kThreads = 128;  // CTA size of the per-instance kernels
// Control dimension of the LQR data: the cart force (the batched solve takes
// the FP32 tableau sweep and the float-float warp residual at (6, 1)).
constexpr int kNu = 1;
constexpr int kMaxN = 4096;
constexpr size_t kAlignB = 256;

inline size_t up(size_t v) { return (v + kAlignB - 1) / kAlignB * kAlignB; }

// Everything a kernel needs about the batch: the model, the options, the
// caller's state and the workspace sections.
struct Args {
  int count, N;
  rlqr_cdp_model md;
  rlqr_ipm_opts op;
  const double *x0, *xg;
  double *X, *U, *Y, *S, *Z, *mu, *rho, *kkt;
  int32_t *iters, *facts, *status;
  // LQR pooled buffers (rlqr_batch layout, one instance per stride)
  double *Q, *M, *R, *q, *r, *A, *B, *c, *dx, *du, *dy;
  uint8_t *flags;
  // per-instance scratch
  double *rho_try, *merit0, *alpha;
  int32_t *lqr_status, *counter;
  double *dS, *dZ;  // [count][N+1][4]
};

// ---- workspace layout
struct Layout {
  size_t Q, M, R, q, r, A, B, c, dx, du, dy, flags;
  size_t dimN, dimn, dimm, oQ, oM, oR, oq, or_, oA, oB, oc, ox, ou, oy, of, delta;
  size_t rho_try, merit0, alpha, lqr_status, list, list2, list3, counter, dS, dZ;
  size_t lqr_ws, total;
};

inline Layout layout(int count, int N, size_t lqr_ws_bytes) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = up(o + bytes);
    return at;
  };
  const size_t C = (size_t)count, n1 = (size_t)N + 1, n0 = (size_t)N;
  L.Q = take(C * n1 * 36 * 8);
  L.M = take(C * n0 * 6 * kNu * 8);
  L.R = take(C * n0 * kNu * kNu * 8);
  L.q = take(C * n1 * 6 * 8);
  L.r = take(C * n0 * kNu * 8);
  L.A = take(C * n0 * 36 * 8);
  L.B = take(C * n0 * 6 * kNu * 8);
  L.c = take(C * n1 * 6 * 8);
  L.dx = take(C * n1 * 6 * 8);
  L.du = take(C * n0 * kNu * 8);
  L.dy = take(C * n1 * 6 * 8);
  L.flags = take(C * n1);
  L.dimN = take(C * 4);
  L.dimn = take(C * 4);
  L.dimm = take(C * 4);
  L.oQ = take(C * 8);
  L.oM = take(C * 8);
  L.oR = take(C * 8);
  L.oq = take(C * 8);
  L.or_ = take(C * 8);
  L.oA = take(C * 8);
  L.oB = take(C * 8);
  L.oc = take(C * 8);
  L.ox = take(C * 8);
  L.ou = take(C * 8);
  L.oy = take(C * 8);
  L.of = take(C * 8);
  L.delta = take(C * 8);
  L.rho_try = take(C * 8);
  L.merit0 = take(C * 8);
  L.alpha = take(C * 8);
  L.lqr_status = take(C * 4);
  L.list = take(C * 4);
  L.list2 = take(C * 4);
  L.list3 = take(C * 4);
  L.counter = take(16);
  L.dS = take(C * n1 * 4 * 8);
  L.dZ = take(C * n1 * 4 * 8);
  L.lqr_ws = take(lqr_ws_bytes);
  L.total = o;
  return L;
}

// ---- block reductions (kThreads threads, deterministic order)
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kThreads / 32; ++i) t += sh[i];
  return t;
}

__device__ __forceinline__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = sh[0];
  for (int i = 1; i < kThreads / 32; ++i) t = fmax(t, sh[i]);
  return t;
}

__device__ __forceinline__ double block_min(double v, double *sh) {
  return -block_max(-v, sh);
}

// Inequality values of stage i: rows 0, 1 (control, i < N) and 2, 3 (cart).
__device__ __forceinline__ void ineq(const rlqr_cdp_model &md, int i, int N, double p, double u,
                                     double g[4]) {
  g[0] = i < N ? u - md.u_max : 0.0;
  g[1] = i < N ? -u - md.u_max : 0.0;
  g[2] = p - md.p_max;
  g[3] = -p - md.p_max;
}

// Variables of (x_i, u_i) that the right-hand side depends on, and the 15
// pairs (j <= k) among them.
__constant__ int kDirs[5] = {1, 2, 4, 5, 6};
__constant__ int kPairs[15][2] = {{1, 1}, {1, 2}, {1, 4}, {1, 5}, {1, 6}, {2, 2}, {2, 4},
                                  {2, 5}, {2, 6}, {4, 4}, {4, 5}, {4, 6}, {5, 5}, {5, 6},
                                  {6, 6}};

// ---- initial point
__global__ void k_ipm_init(Args a, const double *U0, const double *X0, CdpConst<double> kd) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.count) return;
  const int N = a.N;
  double *X = a.X + (size_t)b * (N + 1) * 6, *U = a.U + (size_t)b * N;
  double *Y = a.Y + (size_t)b * (N + 1) * 6, *S = a.S + (size_t)b * (N + 1) * 4;
  double *Z = a.Z + (size_t)b * (N + 1) * 4;
  for (int i = 0; i < N; ++i) U[i] = U0 ? U0[(size_t)b * N + i] : 0.0;
  if (X0) {
    for (int e = 0; e < (N + 1) * 6; ++e) X[e] = X0[(size_t)b * (N + 1) * 6 + e];
  } else {
    double x[6];
    for (int j = 0; j < 6; ++j) X[j] = x[j] = a.x0[(size_t)b * 6 + j];
    for (int i = 0; i < N; ++i) {
      double nx[6];
      const double u = U[i];
      cdp_rk4<double, double>(kd, x, u, nx);
      for (int j = 0; j < 6; ++j) X[(i + 1) * 6 + j] = x[j] = nx[j];
    }
  }
  for (int e = 0; e < (N + 1) * 6; ++e) Y[e] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double g[4];
    ineq(a.md, i, N, X[i * 6], i < N ? U[i] : 0.0, g);
    for (int k = 0; k < 4; ++k) {
      const bool on = i < N || k >= 2;
      const double s = on ? fmax(-g[k], a.op.s_min) : 1.0;
      S[i * 4 + k] = s;
      Z[i * 4 + k] = on ? a.op.mu0 / s : 0.0;
    }
  }
  a.mu[b] = a.op.mu0;
  a.rho[b] = 0.0;
  a.kkt[b] = INFINITY;
  a.iters[b] = 0;
  a.facts[b] = 0;
  a.status[b] = 0;
}

// ---- linearization: the Newton system of eq. ipm-3x3-newton-kkt reduced to
// a dual-regularized LQR, the KKT errors and the barrier update.
//   pass 1 (task = stage i, direction j of (x_i, u_i), FP64 forward mode):
//     phi_i, column j of [A_i B_i], (y_{i+1}^T d phi / d w_j) -> grad_w L
//   pass 2 (task = stage i, pair (j, k), hyper-dual numbers in HT):
//     d^2 (y_{i+1}^T phi) / d w_j d w_k -> the Hessian blocks Q, M, R
//   then E_0 / E_mu, the convergence and mu decisions, the barrier terms
//   (W + Delta_G^{-1})^{-1} on Q_i[0][0] and R_i, and the merit A at the
//   current point.
template <class HT, bool EXACT>
__global__ void __launch_bounds__(kThreads)
    k_ipm_lin(Args a, CdpConst<double> kd, CdpConst<HT> kh) {
  __shared__ double sh[kThreads / 32];
  __shared__ int go;
  __shared__ double mu_s, rho_s;
  const int b = blockIdx.x;
  if (a.status[b] != 0) return;
  const int N = a.N;
  const size_t n1 = (size_t)N + 1;
  const double *X = a.X + b * n1 * 6, *U = a.U + (size_t)b * N, *Y = a.Y + b * n1 * 6;
  const double *S = a.S + b * n1 * 4, *Z = a.Z + b * n1 * 4;
  const double *x0 = a.x0 + (size_t)b * 6, *xg = a.xg + (size_t)b * 6;
  double *Q = a.Q + b * n1 * 36, *Mx = a.M + (size_t)b * N * 6 * kNu;
  double *R = a.R + (size_t)b * N * kNu * kNu;
  double *q = a.q + b * n1 * 6, *r = a.r + (size_t)b * N * kNu, *A = a.A + (size_t)b * N * 36;
  double *B = a.B + (size_t)b * N * 6 * kNu, *c = a.c + b * n1 * 6;
  const rlqr_cdp_model &md = a.md;

  // The right-hand side depends on neither p (w_0) nor dp (w_3), so the RK4
  // map is affine in them with constant coefficients: d phi / d p = e_0,
  // d phi / d dp = dt e_0 + e_3, and every second derivative involving them
  // vanishes.  Those columns are written directly; forward mode runs over
  // the other five directions (kDirs) and the 15 pairs among them (kPairs).
  for (int t = threadIdx.x; t < 2 * N; t += kThreads) {
    const int i = t >> 1, j = (t & 1) ? 3 : 0;
    const double y0 = Y[(i + 1) * 6], gj = j == 0 ? y0 : md.dt * y0 + Y[(i + 1) * 6 + 3];
#pragma unroll
    for (int l = 0; l < 6; ++l)
      A[i * 36 + l * 6 + j] = j == 0 ? (l == 0 ? 1.0 : 0.0) : (l == 0 ? md.dt : (l == 3 ? 1.0 : 0.0));
    double g = md.wx[j] * (X[i * 6 + j] - xg[j]) + gj - Y[i * 6 + j];
    if (j == 0) g += Z[i * 4 + 2] - Z[i * 4 + 3];
    q[i * 6 + j] = g;
  }
  // Stages in chunks of kThreads: one plain FP64 RK4 per stage gives phi_i
  // (the defect c_{i+1}) and records the 12 sines / cosines of its four
  // right-hand sides; the five forward-mode directions of the stage replay
  // them (their value path is the same RK4) instead of evaluating them again.
  __shared__ double trig_rec[kThreads][24];
  for (int c0 = 0; c0 < N; c0 += kThreads) {
    const int nc = min(kThreads, N - c0);
    if (threadIdx.x < nc) {
      const int i = c0 + threadIdx.x;
      double xv[6], ov[6];
#pragma unroll
      for (int l = 0; l < 6; ++l) xv[l] = X[i * 6 + l];
      const double uv = U[i];
      cdp_rk4<double, double>(kd, xv, uv, ov, TrigRecord{trig_rec[threadIdx.x]});
#pragma unroll
      for (int l = 0; l < 6; ++l) c[(i + 1) * 6 + l] = ov[l] - X[(i + 1) * 6 + l];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 5 * nc; t += kThreads) {
      const int il = t / 5, i = c0 + il, j = kDirs[t - 5 * il];
      D1<double> x[6], u, o[6];
#pragma unroll
      for (int l = 0; l < 6; ++l) x[l] = {X[i * 6 + l], l == j ? 1.0 : 0.0};
      u = {U[i], j == 6 ? 1.0 : 0.0};
      cdp_rk4<D1<double>, double>(kd, x, u, o, TrigReplay{trig_rec[il]});
      double gj = 0.0;
#pragma unroll
      for (int l = 0; l < 6; ++l) gj += Y[(i + 1) * 6 + l] * o[l].d;
      if (j < 6) {
#pragma unroll
        for (int l = 0; l < 6; ++l) A[i * 36 + l * 6 + j] = o[l].d;
        q[i * 6 + j] = md.wx[j] * (X[i * 6 + j] - xg[j]) + gj - Y[i * 6 + j];
      } else {
#pragma unroll
        for (int l = 0; l < 6; ++l) B[(i * 6 + l) * kNu] = o[l].d;
        r[i * kNu] = md.wu * U[i] + gj + Z[i * 4 + 0] - Z[i * 4 + 1];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) {
    const int j = threadIdx.x;
    double g = md.wf[j] * (X[N * 6 + j] - xg[j]) - Y[N * 6 + j];
    if (j == 0) g += Z[N * 4 + 2] - Z[N * 4 + 3];
    q[N * 6 + j] = g;
    c[j] = x0[j] - X[j];
  }
  for (int e = threadIdx.x; e < 36; e += kThreads) Q[(size_t)N * 36 + e] = 0.0;
  if (EXACT) {
    for (int t = threadIdx.x; t < 13 * N; t += kThreads) {  // the zero entries
      const int i = t / 13, e = t - 13 * i;
      if (e < 11) {                       // rows/columns 0 and 3 of Q_i
        const int r = e < 6 ? 0 : 3, cc = e < 6 ? e : e - 5;   // row 3: columns 1..5
        Q[i * 36 + r * 6 + cc] = 0.0;
        Q[i * 36 + cc * 6 + r] = 0.0;
      } else {
        Mx[(i * 6 + (e == 11 ? 0 : 3)) * kNu] = 0.0;
      }
    }
    for (int t = threadIdx.x; t < 15 * N; t += kThreads) {
      const int i = t / 15;
      const int j = kPairs[t - 15 * i][0], k = kPairs[t - 15 * i][1];
      HD<HT> x[6], u, o[6];
#pragma unroll
      for (int l = 0; l < 6; ++l)
        x[l] = {HT(X[i * 6 + l]), HT(l == j ? 1 : 0), HT(l == k ? 1 : 0), HT(0)};
      u = {HT(U[i]), HT(j == 6 ? 1 : 0), HT(k == 6 ? 1 : 0), HT(0)};
      cdp_rk4<HD<HT>, HT>(kh, x, u, o);
      double h = 0.0;
#pragma unroll
      for (int l = 0; l < 6; ++l) h += Y[(i + 1) * 6 + l] * (double)o[l].ab;
      if (k < 6) {
        Q[i * 36 + j * 6 + k] = h;
        Q[i * 36 + k * 6 + j] = h;
      } else if (j < 6) {
        Mx[(i * 6 + j) * kNu] = h;
      } else {
        R[i * kNu * kNu] = h;
      }
    }
  } else {
    for (int e = threadIdx.x; e < 36 * N; e += kThreads) Q[e] = 0.0;
    for (int e = threadIdx.x; e < 6 * N; e += kThreads) Mx[e * kNu] = 0.0;
    for (int e = threadIdx.x; e < N; e += kThreads) R[e * kNu * kNu] = 0.0;
  }
  __syncthreads();

  // KKT errors at the current point (mu before its update)
  const double mu = a.mu[b];
  double m_base = 0.0, m_sz = 0.0, m_szmu = 0.0;
  for (int i = threadIdx.x; i <= N; i += kThreads) {
#pragma unroll
    for (int j = 0; j < 6; ++j) m_base = fmax(m_base, fmax(fabs(q[i * 6 + j]), fabs(c[i * 6 + j])));
    if (i < N) m_base = fmax(m_base, fabs(r[i * kNu]));
    double g[4];
    ineq(md, i, N, X[i * 6], i < N ? U[i] : 0.0, g);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i == N && k < 2) continue;
      const double s = S[i * 4 + k], sz = s * Z[i * 4 + k];
      m_base = fmax(m_base, fabs(g[k] + s));
      m_sz = fmax(m_sz, fabs(sz));
      m_szmu = fmax(m_szmu, fabs(sz - mu));
    }
  }
  m_base = block_max(m_base, sh);
  m_sz = block_max(m_sz, sh);
  m_szmu = block_max(m_szmu, sh);
  if (threadIdx.x == 0) {
    const double err0 = fmax(m_base, m_sz), errmu = fmax(m_base, m_szmu);
    a.kkt[b] = err0;
    double mun = mu, rho0 = 0.0;
    int g = 0;
    if (err0 <= a.op.tol) {
      a.status[b] = 1;
    } else if (a.iters[b] >= a.op.max_iter) {
      a.status[b] = 2;
    } else {
      if (errmu <= a.op.kappa_mu * mu) mun = fmax(a.op.mu_min, fmin(0.2 * mu, pow(mu, 1.5)));
      a.mu[b] = mun;
      a.iters[b] += 1;
      // first inertia shift: a third of the last one that gave the correct
      // inertia, 0 if that was 0 or the third is below rho_min
      const double r3 = a.rho[b] / a.op.rho_shrink;
      rho0 = r3 > a.op.rho_min ? r3 : 0.0;
      a.rho_try[b] = rho0;
      g = 1;
    }
    go = g;
    mu_s = mun;
    rho_s = rho0;
  }
  __syncthreads();
  if (!go) return;
  const double mun = mu_s, eta = a.op.eta, ieta = 1.0 / a.op.eta, rho0 = rho_s;

  // barrier terms of the reduced system and the merit at the current point
  double macc = 0.0;
  for (int i = threadIdx.x; i <= N; i += kThreads) {
    double g[4], Dg[4], rz[4];
    const double u = i < N ? U[i] : 0.0;
    ineq(md, i, N, X[i * 6], u, g);
    double sprod = 1.0;  // the stage's barrier term as one log of the slack product
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool on = i < N || k >= 2;
      const double s = S[i * 4 + k], z = Z[i * 4 + k];
      Dg[k] = on ? 1.0 / (s / z + ieta) : 0.0;
      rz[k] = on ? g[k] + mun / z : 0.0;
      if (on) {
        const double gs = g[k] + s;
        sprod *= s;
        macc += z * gs + 0.5 * eta * gs * gs;
      }
    }
    macc -= mun * log(sprod);
    double cst = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double w = i < N ? md.wx[j] : md.wf[j];
      const double d = X[i * 6 + j] - xg[j];
      cst += w * d * d;
      Q[i * 36 + j * 6 + j] += w + rho0;
      const double cj = c[i * 6 + j];
      macc += Y[i * 6 + j] * cj + 0.5 * eta * cj * cj;
    }
    Q[i * 36] += Dg[2] + Dg[3];
    q[i * 6] += Dg[2] * rz[2] - Dg[3] * rz[3];
    if (i < N) {
      cst += md.wu * u * u;
      R[i * kNu * kNu] += md.wu + rho0 + Dg[0] + Dg[1];
      r[i * kNu] += Dg[0] * rz[0] - Dg[1] * rz[1];
    }
    macc += 0.5 * cst;
  }
  macc = block_sum(macc, sh);
  if (threadIdx.x == 0) a.merit0[b] = macc;
}

// The running instances (status 0) in index order, and their count.
__global__ void k_ipm_compact(Args a, int32_t *list, int32_t *count_out) {
  __shared__ int32_t part[1024];
  const int per = (a.count + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(a.count, b0 + per);
  int n = 0;
  for (int b = b0; b < b1; ++b) n += a.status[b] == 0;
  part[threadIdx.x] = n;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int at = part[threadIdx.x] - n;
  for (int b = b0; b < b1; ++b)
    if (a.status[b] == 0) list[at++] = b;
  if (threadIdx.x == blockDim.x - 1) *count_out = part[threadIdx.x];
}

// Offsets of the listed instances into the pooled LQR buffers (the batch
// descriptor of the compacted solve).
__global__ void k_ipm_offsets(Args a, const int32_t *list, int n, int64_t *oQ, int64_t *oM,
                              int64_t *oR, int64_t *oq, int64_t *or_, int64_t *oA, int64_t *oB,
                              int64_t *oc, int64_t *ox, int64_t *ou, int64_t *oy, int64_t *of) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t b = list[t], N = a.N, n1 = N + 1;
  oQ[t] = b * n1 * 36;
  oM[t] = b * N * 6 * kNu;
  oR[t] = b * N * kNu * kNu;
  oq[t] = b * n1 * 6;
  or_[t] = b * N * kNu;
  oA[t] = b * N * 36;
  oB[t] = b * N * 6 * kNu;
  oc[t] = b * n1 * 6;
  ox[t] = b * n1 * 6;
  ou[t] = b * N * kNu;
  oy[t] = b * n1 * 6;
  of[t] = b * n1;
}

// Inertia certificate of the last solve of the listed instances (warp per
// instance): every pivot flag 3 and a solved status -> keep the step;
// otherwise the shift rho restarts from a third of the last successful one
// (rho_first if none) or grows by rho_grow, is added to the diagonals of
// Q_i and R_i, and the instance joins the retry list (or fails above rho_max).
__global__ void k_ipm_cert(Args a, const int32_t *list, int n, int32_t *retry, int32_t *nretry) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= n) return;
  const int b = list[t], N = a.N;
  const uint8_t *fl = a.flags + (size_t)b * (N + 1);
  int bad = 0;
  for (int i = lane; i <= N; i += 32) bad |= fl[i] != 3;
  bad = __any_sync(0xffffffffu, bad);
  const int st = a.lqr_status[t];
  if (st != RLQR_OK && st != RLQR_NOT_PD && st != RLQR_ERR_NOT_CONVERGED) bad = 1;
  if (lane == 0) a.facts[b] += 1;
  if (!bad) return;
  const double old = a.rho_try[b];
  double nr;
  if (old == 0.0) {
    const double last = a.rho[b];
    nr = last == 0.0 ? a.op.rho_first : fmax(a.op.rho_min, last / a.op.rho_shrink);
  } else {
    nr = old * a.op.rho_grow;
  }
  if (nr > a.op.rho_max) {
    if (lane == 0) a.status[b] = 3;
    return;
  }
  const double add = nr - old;
  double *Q = a.Q + (size_t)b * (N + 1) * 36, *R = a.R + (size_t)b * N * kNu * kNu;
  for (int e = lane; e < (N + 1) * 6; e += 32) Q[(e / 6) * 36 + (e % 6) * 7] += add;
  for (int i = lane; i < N; i += 32) R[i * kNu * kNu] += add;
  if (lane == 0) {
    a.rho_try[b] = nr;
    retry[atomicAdd(nretry, 1)] = b;
  }
}

// Step recovery (Delta z = (W + Delta_G^{-1})^{-1} (G Delta x + r_z),
// Delta s = -W (Delta z - mu S^{-1} e + z)), fractions to the boundary,
// the merit slope (grad f.dx + (y + eta c)^T C dx + (z + eta (g+s))^T
// (G dx + ds) - mu sum ds/s), Armijo backtracking on the augmented
// barrier-Lagrangian with (y, z) fixed, and the update.
__global__ void __launch_bounds__(kThreads)
    k_ipm_step(Args a, const int32_t *list, CdpConst<double> kd) {
  __shared__ double sh[kThreads / 32];
  const int b = list[blockIdx.x];
  if (a.status[b] != 0) return;
  const int N = a.N;
  const size_t n1 = (size_t)N + 1;
  double *X = a.X + b * n1 * 6, *U = a.U + (size_t)b * N, *Y = a.Y + b * n1 * 6;
  double *S = a.S + b * n1 * 4, *Z = a.Z + b * n1 * 4;
  const double *x0 = a.x0 + (size_t)b * 6, *xg = a.xg + (size_t)b * 6;
  const double *A = a.A + (size_t)b * N * 36, *B = a.B + (size_t)b * N * 6 * kNu;
  const double *c = a.c + b * n1 * 6;
  const double *dX = a.dx + b * n1 * 6, *dU = a.du + (size_t)b * N * kNu, *dY = a.dy + b * n1 * 6;
  double *dS = a.dS + b * n1 * 4, *dZ = a.dZ + b * n1 * 4;
  const rlqr_cdp_model &md = a.md;
  const double mu = a.mu[b], eta = a.op.eta, ieta = 1.0 / eta, tau = a.op.tau;

  double as = 1.0, az = 1.0, slope = 0.0;
  for (int i = threadIdx.x; i <= N; i += kThreads) {
    const double du = i < N ? dU[i * kNu] : 0.0, u = i < N ? U[i] : 0.0;
    double g[4];
    ineq(md, i, N, X[i * 6], u, g);
    const double Gdx[4] = {du, -du, dX[i * 6], -dX[i * 6]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool on = i < N || k >= 2;
      double ds = 0.0, dz = 0.0;
      if (on) {
        const double s = S[i * 4 + k], z = Z[i * 4 + k];
        const double Dg = 1.0 / (s / z + ieta), rz = g[k] + mu / z;
        dz = Dg * (Gdx[k] + rz);
        ds = -(s / z) * dz + mu / z - s;
        if (ds < 0.0) as = fmin(as, -tau * s / ds);
        if (dz < 0.0) az = fmin(az, -tau * z / dz);
        slope += (z + eta * (g[k] + s)) * (Gdx[k] + ds) - mu * (ds / s);
      }
      dS[i * 4 + k] = ds;
      dZ[i * 4 + k] = dz;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double w = i < N ? md.wx[j] : md.wf[j];
      slope += w * (X[i * 6 + j] - xg[j]) * dX[i * 6 + j];
      double cd;
      if (i == 0) {
        cd = -dX[j];
      } else {
        cd = B[((i - 1) * 6 + j) * kNu] * dU[(i - 1) * kNu] - dX[i * 6 + j];
#pragma unroll
        for (int l = 0; l < 6; ++l) cd += A[(i - 1) * 36 + j * 6 + l] * dX[(i - 1) * 6 + l];
      }
      slope += (Y[i * 6 + j] + eta * c[i * 6 + j]) * cd;
    }
    if (i < N) slope += md.wu * u * du;
  }
  as = block_min(as, sh);
  az = block_min(az, sh);
  slope = block_sum(slope, sh);
  const double A0 = a.merit0[b];
  const double allow = 10.0 * 2.220446049250313e-16 * fabs(A0);
  double alpha = as;
  for (int k = 0; k < a.op.ls_steps; ++k) {
    alpha = as * ldexp(1.0, -k);
    double acc = 0.0;
    for (int i = threadIdx.x; i <= N; i += kThreads) {
      double xt[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) xt[j] = X[i * 6 + j] + alpha * dX[i * 6 + j];
      const double ut = i < N ? U[i] + alpha * dU[i * kNu] : 0.0;
      double ct[6];
      if (i == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) ct[j] = x0[j] - xt[j];
      } else {
        double xp[6], ph[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) xp[j] = X[(i - 1) * 6 + j] + alpha * dX[(i - 1) * 6 + j];
        const double up_ = U[i - 1] + alpha * dU[(i - 1) * kNu];
        cdp_rk4<double, double>(kd, xp, up_, ph);
#pragma unroll
        for (int j = 0; j < 6; ++j) ct[j] = ph[j] - xt[j];
      }
      double cst = 0.0;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const double w = i < N ? md.wx[j] : md.wf[j];
        const double d = xt[j] - xg[j];
        cst += w * d * d;
        acc += Y[i * 6 + j] * ct[j] + 0.5 * eta * ct[j] * ct[j];
      }
      if (i < N) cst += md.wu * ut * ut;
      acc += 0.5 * cst;
      double g[4];
      ineq(md, i, N, xt[0], ut, g);
      double sprod = 1.0;  // one log of the slack product per stage
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (i == N && kk < 2) continue;
        const double st = S[i * 4 + kk] + alpha * dS[i * 4 + kk], gs = g[kk] + st;
        sprod *= st;
        acc += Z[i * 4 + kk] * gs + 0.5 * eta * gs * gs;
      }
      acc -= mu * log(sprod);
    }
    acc = block_sum(acc, sh);
    if (acc <= A0 + a.op.armijo * alpha * slope + allow) break;
  }
  __syncthreads();  // every thread has read the old point
  const double azz = fmin(az, alpha), ks = a.op.kappa_sigma;
  for (int i = threadIdx.x; i <= N; i += kThreads) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      X[i * 6 + j] += alpha * dX[i * 6 + j];
      Y[i * 6 + j] += alpha * dY[i * 6 + j];
    }
    if (i < N) U[i] += alpha * dU[i * kNu];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i == N && k < 2) continue;
      const double s = S[i * 4 + k] + alpha * dS[i * 4 + k];
      const double z = Z[i * 4 + k] + azz * dZ[i * 4 + k];
      S[i * 4 + k] = s;
      Z[i * 4 + k] = fmin(fmax(z, mu / (ks * s)), ks * mu / s);
    }
  }
  if (threadIdx.x == 0) {
    a.alpha[b] = alpha;
    a.rho[b] = a.rho_try[b];  // the shift that gave the correct inertia (may be 0)
  }
}

__global__ void k_ipm_dims(int count, int N, double delta, int32_t *dN, int32_t *dn, int32_t *dm,
                           double *dd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  dN[t] = N;
  dn[t] = 6;
  dm[t] = kNu;
  dd[t] = delta;
}

// ---- host side
bool valid(int count, const rlqr_cdp_model *md, const rlqr_ipm_opts *op) {
  if (count < 1 || !md || !op) return false;
  if (md->N < 1 || md->N > kMaxN) return false;
  if (!(md->dt > 0) || !(md->m0 > 0) || !(md->m1 > 0) || !(md->m2 > 0) || !(md->l1 > 0) ||
      !(md->l2 > 0) || !std::isfinite(md->grav) || !(md->u_max > 0) || !(md->p_max > 0) ||
      !(md->wu >= 0))
    return false;
  for (int j = 0; j < 6; ++j)
    if (!(md->wx[j] >= 0) || !(md->wf[j] >= 0)) return false;
  if (op->max_iter < 0 || !(op->tol > 0) || !(op->eta > 0) || !(op->mu0 > 0) ||
      !(op->mu_min > 0) || !(op->kappa_mu > 0) || !(op->tau > 0 && op->tau < 1) ||
      !(op->armijo > 0 && op->armijo < 1) || op->ls_steps < 1 || op->ls_steps > 30 ||
      !(op->rho_first > 0) || !(op->rho_grow > 1) || !(op->rho_shrink > 1) ||
      !(op->rho_min > 0) || !(op->rho_max > op->rho_first) || !(op->kappa_sigma >= 1) ||
      !(op->s_min > 0) || op->hessian < 0 || op->hessian > 2 ||
      (op->lqr_prec != RLQR_FP64 && op->lqr_prec != RLQR_MIXED) || op->lqr_max_refine < 0 ||
      !(op->lqr_tol > 0))
    return false;
  return true;
}

rlqr_opts lqr_opts(const rlqr_ipm_opts *op) {
  rlqr_opts o{};
  o.max_refine = op->lqr_max_refine;
  o.tol = op->lqr_tol;
  o.algo = RLQR_ALGO_SEQ;
  o.prec = (rlqr_prec)op->lqr_prec;
  o.flags = 0;
  return o;
}

struct HostDims {
  std::vector<int32_t> N, n, m;
  HostDims(int count, int NN) : N(count, NN), n(count, 6), m(count, kNu) {}
};

size_t lqr_ws_bytes(int count, const rlqr_cdp_model *md, const rlqr_ipm_opts *op) {
  HostDims h(count, md->N);
  rlqr_batch bt{};
  bt.count = count;
  bt.h_N = h.N.data();
  bt.h_nx = h.n.data();
  bt.h_nu = h.m.data();
  const rlqr_opts o = lqr_opts(op);
  return rlqr_batched_workspace_bytes(&bt, &o);
}

Args make_args(int count, const rlqr_cdp_model *md, const rlqr_ipm_opts *op, const double *x0,
               const double *xg, rlqr_ipm_state *st, char *ws, const Layout &L) {
  Args a{};
  a.count = count;
  a.N = md->N;
  a.md = *md;
  a.op = *op;
  a.x0 = x0;
  a.xg = xg;
  a.X = st->X;
  a.U = st->U;
  a.Y = st->Y;
  a.S = st->S;
  a.Z = st->Z;
  a.mu = st->mu;
  a.rho = st->rho;
  a.kkt = st->kkt;
  a.iters = st->iters;
  a.facts = st->factorizations;
  a.status = st->status;
  if (ws) {
    a.Q = reinterpret_cast<double *>(ws + L.Q);
    a.M = reinterpret_cast<double *>(ws + L.M);
    a.R = reinterpret_cast<double *>(ws + L.R);
    a.q = reinterpret_cast<double *>(ws + L.q);
    a.r = reinterpret_cast<double *>(ws + L.r);
    a.A = reinterpret_cast<double *>(ws + L.A);
    a.B = reinterpret_cast<double *>(ws + L.B);
    a.c = reinterpret_cast<double *>(ws + L.c);
    a.dx = reinterpret_cast<double *>(ws + L.dx);
    a.du = reinterpret_cast<double *>(ws + L.du);
    a.dy = reinterpret_cast<double *>(ws + L.dy);
    a.flags = reinterpret_cast<uint8_t *>(ws + L.flags);
    a.rho_try = reinterpret_cast<double *>(ws + L.rho_try);
    a.merit0 = reinterpret_cast<double *>(ws + L.merit0);
    a.alpha = reinterpret_cast<double *>(ws + L.alpha);
    a.lqr_status = reinterpret_cast<int32_t *>(ws + L.lqr_status);
    a.counter = reinterpret_cast<int32_t *>(ws + L.counter);
    a.dS = reinterpret_cast<double *>(ws + L.dS);
    a.dZ = reinterpret_cast<double *>(ws + L.dZ);
  }
  return a;
}

bool state_ok(const rlqr_ipm_state *st) {
  return st && st->X && st->U && st->Y && st->S && st->Z && st->mu && st->rho && st->kkt &&
         st->iters && st->factorizations && st->status;
}

rlqr_status read_count(const int32_t *d, int32_t *h, cudaStream_t s) {
  if (cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RLQR_ERR_CUDA;
  return RLQR_OK;
}

// The batched LQR solve of the listed instances (positions 0..n-1).
rlqr_status solve_list(const Args &a, char *ws, const Layout &L, const int32_t *list, int n,
                       const HostDims &h, const rlqr_ipm_opts *op, cudaStream_t s) {
  auto I64 = [&](size_t off) { return reinterpret_cast<int64_t *>(ws + off); };
  k_ipm_offsets<<<(n + 255) / 256, 256, 0, s>>>(a, list, n, I64(L.oQ), I64(L.oM), I64(L.oR),
                                                 I64(L.oq), I64(L.or_), I64(L.oA), I64(L.oB),
                                                 I64(L.oc), I64(L.ox), I64(L.ou), I64(L.oy),
                                                 I64(L.of));
  if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  rlqr_batch bt{};
  bt.count = n;
  bt.h_N = h.N.data();
  bt.h_nx = h.n.data();
  bt.h_nu = h.m.data();
  bt.N = reinterpret_cast<const int32_t *>(ws + L.dimN);
  bt.nx = reinterpret_cast<const int32_t *>(ws + L.dimn);
  bt.nu = reinterpret_cast<const int32_t *>(ws + L.dimm);
  bt.off_Q = I64(L.oQ);
  bt.off_M = I64(L.oM);
  bt.off_R = I64(L.oR);
  bt.off_q = I64(L.oq);
  bt.off_r = I64(L.or_);
  bt.off_A = I64(L.oA);
  bt.off_B = I64(L.oB);
  bt.off_c = I64(L.oc);
  bt.off_x = I64(L.ox);
  bt.off_u = I64(L.ou);
  bt.off_y = I64(L.oy);
  bt.off_flag = I64(L.of);
  bt.delta = reinterpret_cast<const double *>(ws + L.delta);
  bt.Q = a.Q;
  bt.M = a.M;
  bt.R = a.R;
  bt.q = a.q;
  bt.r = a.r;
  bt.A = a.A;
  bt.B = a.B;
  bt.c = a.c;
  bt.x = a.dx;
  bt.u = a.du;
  bt.y = a.dy;
  bt.pivot_pd = a.flags;
  const rlqr_opts o = lqr_opts(op);
  const size_t need = rlqr_batched_workspace_bytes(&bt, &o);
  return rlqr_solve_batched(&bt, &o, ws + L.lqr_ws, need, a.lqr_status, nullptr, nullptr,
                            reinterpret_cast<rlqr_stream_t>(s));
}

}  // namespace ipm
}  // namespace rlqr

using namespace rlqr::ipm;

extern "C" {

size_t rlqr_ipm_workspace_bytes(int32_t count, const rlqr_cdp_model *model,
                                const rlqr_ipm_opts *opts) {
  if (!valid(count, model, opts)) return 0;
  const size_t lw = lqr_ws_bytes(count, model, opts);
  if (lw == 0) return 0;
  return layout(count, model->N, lw).total;
}

rlqr_status rlqr_ipm_init(int32_t count, const rlqr_cdp_model *model, const rlqr_ipm_opts *opts,
                          const double *x0, const double *U0, const double *X0,
                          rlqr_ipm_state *state, rlqr_stream_t stream) {
  if (!valid(count, model, opts) || !state_ok(state) || (!x0 && !X0)) return RLQR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Layout L{};
  Args a = make_args(count, model, opts, x0, nullptr, state, nullptr, L);
  k_ipm_init<<<(count + 127) / 128, 128, 0, s>>>(a, U0, X0, cdp_const<double>(*model));
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

static rlqr_status prepare(int32_t count, const rlqr_cdp_model *model, const rlqr_ipm_opts *opts,
                           const double *x0, const double *xg, rlqr_ipm_state *state, void *ws,
                           size_t ws_bytes, Layout &L) {
  if (!valid(count, model, opts) || !state_ok(state) || !x0 || !xg) return RLQR_ERR_ARG;
  const size_t lw = lqr_ws_bytes(count, model, opts);
  if (lw == 0) return RLQR_ERR_ARG;
  L = layout(count, model->N, lw);
  if (!ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) % kAlignB) != 0)
    return RLQR_ERR_WORKSPACE;
  return RLQR_OK;
}

static rlqr_status launch_lin(const Args &a, const rlqr_cdp_model *model,
                              const rlqr_ipm_opts *opts, cudaStream_t s) {
  const CdpConst<double> kd = cdp_const<double>(*model);
  switch (opts->hessian) {
    case RLQR_IPM_HESS_EXACT_FP64:
      k_ipm_lin<double, true><<<a.count, kThreads, 0, s>>>(a, kd, kd);
      break;
    case RLQR_IPM_HESS_EXACT_FP32:
      k_ipm_lin<float, true><<<a.count, kThreads, 0, s>>>(a, kd, cdp_const<float>(*model));
      break;
    default:
      k_ipm_lin<float, false><<<a.count, kThreads, 0, s>>>(a, kd, cdp_const<float>(*model));
  }
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

rlqr_status rlqr_ipm_linearize(int32_t count, const rlqr_cdp_model *model,
                               const rlqr_ipm_opts *opts, const double *x0, const double *xg,
                               rlqr_ipm_state *state, void *ws, size_t ws_bytes,
                               rlqr_stream_t stream) {
  Layout L{};
  rlqr_status e = prepare(count, model, opts, x0, xg, state, ws, ws_bytes, L);
  if (e != RLQR_OK) return e;
  const Args a = make_args(count, model, opts, x0, xg, state, static_cast<char *>(ws), L);
  return launch_lin(a, model, opts, reinterpret_cast<cudaStream_t>(stream));
}

rlqr_status rlqr_ipm_iterate(int32_t count, const rlqr_cdp_model *model,
                             const rlqr_ipm_opts *opts, const double *x0, const double *xg,
                             rlqr_ipm_state *state, void *ws, size_t ws_bytes,
                             int32_t *n_running, rlqr_stream_t stream) {
  Layout L{};
  rlqr_status e = prepare(count, model, opts, x0, xg, state, ws, ws_bytes, L);
  if (e != RLQR_OK) return e;
  if (n_running) *n_running = 0;
  char *w = static_cast<char *>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Args a = make_args(count, model, opts, x0, xg, state, w, L);
  int32_t *list = reinterpret_cast<int32_t *>(w + L.list);
  int32_t *rbuf[2] = {reinterpret_cast<int32_t *>(w + L.list2),
                      reinterpret_cast<int32_t *>(w + L.list3)};
  if ((e = launch_lin(a, model, opts, s)) != RLQR_OK) return e;
  k_ipm_compact<<<1, 1024, 0, s>>>(a, list, a.counter);
  k_ipm_dims<<<(count + 255) / 256, 256, 0, s>>>(
      count, model->N, 1.0 / opts->eta, reinterpret_cast<int32_t *>(w + L.dimN),
      reinterpret_cast<int32_t *>(w + L.dimn), reinterpret_cast<int32_t *>(w + L.dimm),
      reinterpret_cast<double *>(w + L.delta));
  if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  int32_t n = 0;
  if ((e = read_count(a.counter, &n, s)) != RLQR_OK) return e;
  if (n == 0) return RLQR_OK;
  const HostDims h(count, model->N);
  // inertia-correction rounds: the first solves every running instance, each
  // later one only those whose certificate failed (at most ~log_8(rho_max /
  // rho_min) + 2 rounds; the bound below is a safeguard)
  const int32_t *cur = list;
  int ncur = n;
  for (int round = 0; ncur > 0; ++round) {
    if (round >= 64) return RLQR_ERR_NOT_CONVERGED;
    if ((e = solve_list(a, w, L, cur, ncur, h, opts, s)) != RLQR_OK) return e;
    int32_t *next = rbuf[round & 1];
    if (cudaMemsetAsync(a.counter, 0, sizeof(int32_t), s) != cudaSuccess) return RLQR_ERR_CUDA;
    k_ipm_cert<<<(ncur + 3) / 4, 128, 0, s>>>(a, cur, ncur, next, a.counter);
    if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
    int32_t nr = 0;
    if ((e = read_count(a.counter, &nr, s)) != RLQR_OK) return e;
    cur = next;
    ncur = nr;
  }
  k_ipm_step<<<n, kThreads, 0, s>>>(a, list, cdp_const<double>(*model));
  if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  if (n_running) *n_running = n;
  return RLQR_OK;
}

rlqr_status rlqr_ipm_solve(int32_t count, const rlqr_cdp_model *model, const rlqr_ipm_opts *opts,
                           const double *x0, const double *xg, rlqr_ipm_state *state, void *ws,
                           size_t ws_bytes, int32_t *n_iterations, rlqr_stream_t stream) {
  if (n_iterations) *n_iterations = 0;
  if (!opts) return RLQR_ERR_ARG;
  for (int it = 0; it <= opts->max_iter + 1; ++it) {
    int32_t n = 0;
    const rlqr_status e =
        rlqr_ipm_iterate(count, model, opts, x0, xg, state, ws, ws_bytes, &n, stream);
    if (e != RLQR_OK) return e;
    if (n == 0) break;
    if (n_iterations) *n_iterations = it + 1;
  }
  return RLQR_OK;
}

rlqr_status rlqr_ipm_lqr_view(int32_t count, const rlqr_cdp_model *model,
                              const rlqr_ipm_opts *opts, void *ws, rlqr_ipm_lqr *out) {
  if (!valid(count, model, opts) || !ws || !out) return RLQR_ERR_ARG;
  const size_t lw = lqr_ws_bytes(count, model, opts);
  if (lw == 0) return RLQR_ERR_ARG;
  const Layout L = layout(count, model->N, lw);
  char *w = static_cast<char *>(ws);
  out->Q = reinterpret_cast<double *>(w + L.Q);
  out->M = reinterpret_cast<double *>(w + L.M);
  out->R = reinterpret_cast<double *>(w + L.R);
  out->q = reinterpret_cast<double *>(w + L.q);
  out->r = reinterpret_cast<double *>(w + L.r);
  out->A = reinterpret_cast<double *>(w + L.A);
  out->B = reinterpret_cast<double *>(w + L.B);
  out->c = reinterpret_cast<double *>(w + L.c);
  out->dx = reinterpret_cast<double *>(w + L.dx);
  out->du = reinterpret_cast<double *>(w + L.du);
  out->dy = reinterpret_cast<double *>(w + L.dy);
  out->pivot_pd = reinterpret_cast<uint8_t *>(w + L.flags);
  return RLQR_OK;
}

}  // extern "C"

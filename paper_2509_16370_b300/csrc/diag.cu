// diag.cu -- dual regularization with a general diagonal Delta_i = diag(d_i)
// (the problem statement of Section "Dual-Regularized LQR" allows any SPD
// Delta_i; the certificate of Section "Inertia Certification" then tests
// S_i = I + Delta_i^{1/2} P_i Delta_i^{1/2}).
//
// With D_i = Delta_i^{1/2}, the substitution x_i = D_i x~_i, y_i = D_i^{-1} y~_i
// and the scaling of stationarity row i by D_i and of constraint row i by
// D_i^{-1} is a congruence of the KKT matrix that maps the problem to one
// with Delta = I:
//   Q~_i = D_i Q_i D_i, M~_i = D_i M_i, q~_i = D_i q_i, R, r unchanged,
//   A~_i = D_{i+1}^{-1} A_i D_i, B~_i = D_{i+1}^{-1} B_i, c~_i = D_i^{-1} c_i.
// Its value functions are P~_i = D_i P_i D_i, so its state pivot I + P~_i is
// exactly S_i and its control pivots G_i are unchanged: the flags of the
// scaled solve are the certificate of the original problem.  The scaled copy
// is solved by rlqr_factor / rlqr_solve with delta = 1 and mapped back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rlqr {
namespace {

struct ScaledLayout {
  size_t Q, M, q, A, B, c, rq, ru, rc, dx, du, dy, norms, lqr, total;
};

ScaledLayout scaled_layout(int N, int n, int m, size_t lqr_bytes) {
  ScaledLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = align_up(o + b);
    return at;
  };
  L.Q = take((size_t)(N + 1) * n * n * 8);
  L.M = take((size_t)N * n * m * 8);
  L.q = take((size_t)(N + 1) * n * 8);
  L.A = take((size_t)N * n * n * 8);
  L.B = take((size_t)N * n * m * 8);
  L.c = take((size_t)(N + 1) * n * 8);
  L.rq = take((size_t)(N + 1) * n * 8);
  L.ru = take((size_t)N * m * 8);
  L.rc = take((size_t)(N + 1) * n * 8);
  L.dx = take((size_t)(N + 1) * n * 8);
  L.du = take((size_t)N * m * 8);
  L.dy = take((size_t)(N + 1) * n * 8);
  L.norms = take(4 * 8);
  L.lqr = take(lqr_bytes);
  L.total = o;
  return L;
}

__global__ void k_diag_scale(int N, int n, int m, const double *d, const double *Q,
                             const double *M, const double *q, const double *A, const double *B,
                             const double *c, double *Qs, double *Ms, double *qs, double *As,
                             double *Bs, double *cs) {
  const int64_t nn = (int64_t)n * n, nm = (int64_t)n * m;
  const int64_t nQ = (N + 1) * nn, nM = N * nm, nq = (int64_t)(N + 1) * n, nA = N * nn;
  const int64_t total = nQ + nM + nq + nA + nM + nq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e;
    if (f < nQ) {
      const int64_t i = f / nn, rc = f - i * nn, r = rc / n, cc = rc - r * n;
      Qs[f] = sqrt(d[i * n + r]) * Q[f] * sqrt(d[i * n + cc]);
      continue;
    }
    f -= nQ;
    if (f < nM) {
      const int64_t i = f / nm, r = (f - i * nm) / m;
      Ms[f] = sqrt(d[i * n + r]) * M[f];
      continue;
    }
    f -= nM;
    if (f < nq) {
      qs[f] = sqrt(d[f]) * q[f];
      continue;
    }
    f -= nq;
    if (f < nA) {
      const int64_t i = f / nn, rc = f - i * nn, r = rc / n, cc = rc - r * n;
      As[f] = A[f] * sqrt(d[i * n + cc]) / sqrt(d[(i + 1) * n + r]);
      continue;
    }
    f -= nA;
    if (f < nM) {
      const int64_t i = f / nm, r = (f - i * nm) / m;
      Bs[f] = B[f] / sqrt(d[(i + 1) * n + r]);
      continue;
    }
    f -= nM;
    cs[f] = c[f] / sqrt(d[f]);
  }
}

// x = D x~, y = D^{-1} y~ in place.
__global__ void k_diag_unscale(int64_t len, const double *d, double *x, double *y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double s = sqrt(d[e]);
    x[e] *= s;
    y[e] /= s;
  }
}

// Non-negative doubles order like their bit patterns: a deterministic max.
__device__ __forceinline__ void atomic_max_pos(double *a, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(a), __double_as_longlong(v));
}

// FP64 residual of the ORIGINAL system (Section "Residual Computation" with
// Delta_i = diag(d_i)), one thread per stage, written as the right-hand side
// of the correction in the scaled variables (rq~ = D r_x, ru, rc~ = D^{-1} r_c)
// and the norms of the backward error: norms = (||r||, ||K|| stagewise,
// ||z||, ||b||) (infinity norms, bit-pattern max).
__global__ void k_diag_residual(int N, int n, int m, const double *d, const double *Q,
                                const double *M, const double *R, const double *q,
                                const double *r, const double *A, const double *B,
                                const double *c, const double *x, const double *u,
                                const double *y, double *rq, double *ru, double *rc,
                                double *norms) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= N; i += gridDim.x * blockDim.x) {
    double mr = 0.0, mk = 0.0, mz = 0.0, mb = 0.0;
    const double *xi = x + (size_t)i * n, *yi = y + (size_t)i * n;
    const double *y1 = i < N ? y + (size_t)(i + 1) * n : nullptr;
    for (int j = 0; j < n; ++j) {
      // stationarity row of x_i[j]
      double t = q[(size_t)i * n + j] - yi[j], rs = 1.0;
      for (int k = 0; k < n; ++k) {
        const double qv = Q[((size_t)i * n + j) * n + k];
        t += qv * xi[k];
        rs += fabs(qv);
      }
      if (i < N) {
        for (int k = 0; k < m; ++k) {
          const double mv = M[((size_t)i * n + j) * m + k];
          t += mv * u[(size_t)i * m + k];
          rs += fabs(mv);
        }
        for (int k = 0; k < n; ++k) {
          const double av = A[((size_t)i * n + k) * n + j];
          t += av * y1[k];
          rs += fabs(av);
        }
      }
      const double sd = sqrt(d[(size_t)i * n + j]);
      rq[(size_t)i * n + j] = sd * t;
      mr = fmax(mr, fabs(t));
      mk = fmax(mk, rs);
      mz = fmax(mz, fmax(fabs(xi[j]), fabs(yi[j])));
      mb = fmax(mb, fmax(fabs(q[(size_t)i * n + j]), fabs(c[(size_t)i * n + j])));
      // constraint row i, component j: (A x + B u)_{i-1} - x_i - Delta_i y_i + c_i
      const double dj = d[(size_t)i * n + j];
      double tc = c[(size_t)i * n + j] - xi[j] - dj * yi[j], cs = 1.0 + dj;
      if (i > 0) {
        for (int k = 0; k < n; ++k) {
          const double av = A[((size_t)(i - 1) * n + j) * n + k];
          tc += av * x[(size_t)(i - 1) * n + k];
          cs += fabs(av);
        }
        for (int k = 0; k < m; ++k) {
          const double bv = B[((size_t)(i - 1) * n + j) * m + k];
          tc += bv * u[(size_t)(i - 1) * m + k];
          cs += fabs(bv);
        }
      }
      rc[(size_t)i * n + j] = tc / sd;
      mr = fmax(mr, fabs(tc));
      mk = fmax(mk, cs);
    }
    if (i < N) {
      for (int j = 0; j < m; ++j) {
        double t = r[(size_t)i * m + j], rs = 0.0;
        for (int k = 0; k < n; ++k) {
          const double mv = M[((size_t)i * n + k) * m + j];
          t += mv * xi[k];
          rs += fabs(mv);
        }
        for (int k = 0; k < m; ++k) {
          const double rv = R[((size_t)i * m + j) * m + k];
          t += rv * u[(size_t)i * m + k];
          rs += fabs(rv);
        }
        for (int k = 0; k < n; ++k) {
          const double bv = B[((size_t)i * n + k) * m + j];
          t += bv * y1[k];
          rs += fabs(bv);
        }
        ru[(size_t)i * m + j] = t;
        mr = fmax(mr, fabs(t));
        mk = fmax(mk, rs);
        mz = fmax(mz, fabs(u[(size_t)i * m + j]));
        mb = fmax(mb, fabs(r[(size_t)i * m + j]));
      }
    }
    atomic_max_pos(norms + 0, mr);
    atomic_max_pos(norms + 1, mk);
    atomic_max_pos(norms + 2, mz);
    atomic_max_pos(norms + 3, mb);
  }
}

__global__ void k_diag_rel(const double *norms, double *rel) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *rel = norms[0] / (norms[1] * norms[2] + norms[3]);
}

// x += D dx~, u += du, y += D^{-1} dy~ (the correction mapped back).
__global__ void k_diag_update(int N, int n, int m, const double *d, const double *dx,
                              const double *du, const double *dy, double *x, double *u,
                              double *y) {
  const int64_t len = (int64_t)(N + 1) * n, lu = (int64_t)N * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len + lu;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < len) {
      const double s = sqrt(d[e]);
      x[e] += s * dx[e];
      y[e] += dy[e] / s;
    } else {
      u[e - len] += du[e - len];
    }
  }
}

}  // namespace
}  // namespace rlqr

using namespace rlqr;

extern "C" {

size_t rlqr_diag_workspace_bytes(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts) {
  const size_t lw = rlqr_workspace_bytes(N, nx, nu, opts);
  if (lw == 0) return 0;
  return scaled_layout(N, nx, nu, lw).total;
}

rlqr_status rlqr_solve_diag(const rlqr_problem *prob, const double *delta_diag,
                            const rlqr_opts *opts, void *ws, size_t ws_bytes, double *x, double *u,
                            double *y, uint8_t *pivot_pd, double *rel_resid, int32_t *status,
                            rlqr_stream_t stream) {
  if (!prob || !delta_diag || !opts || !x || !u || !y || !pivot_pd) return RLQR_ERR_ARG;
  const int N = prob->N, n = prob->nx, m = prob->nu;
  const size_t lw = rlqr_workspace_bytes(N, n, m, opts);
  if (lw == 0 || !prob->Q || !prob->M || !prob->R || !prob->q || !prob->r || !prob->A ||
      !prob->B || !prob->c)
    return RLQR_ERR_ARG;
  const ScaledLayout L = scaled_layout(N, n, m, lw);
  if (!ws || ws_bytes < L.total || reinterpret_cast<uintptr_t>(ws) % kAlign) return RLQR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char *w = static_cast<char *>(ws);
  double *Qs = reinterpret_cast<double *>(w + L.Q), *Ms = reinterpret_cast<double *>(w + L.M);
  double *qs = reinterpret_cast<double *>(w + L.q), *As = reinterpret_cast<double *>(w + L.A);
  double *Bs = reinterpret_cast<double *>(w + L.B), *cs = reinterpret_cast<double *>(w + L.c);
  k_diag_scale<<<1184, 256, 0, s>>>(N, n, m, delta_diag, prob->Q, prob->M, prob->q, prob->A,
                                     prob->B, prob->c, Qs, Ms, qs, As, Bs, cs);
  if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  rlqr_problem sp = *prob;
  sp.Q = Qs;
  sp.M = Ms;
  sp.q = qs;
  sp.A = As;
  sp.B = Bs;
  sp.c = cs;
  sp.delta = 1.0;
  rlqr_opts o = *opts;
  o.flags = 0;
  rlqr_status e = rlqr_factor(&sp, &o, w + L.lqr, lw, pivot_pd, status, stream);
  if (e != RLQR_OK) return e;
  e = rlqr_solve(&sp, &o, w + L.lqr, lw, x, u, y, rel_resid, nullptr, status, stream);
  if (e != RLQR_OK) return e;
  const int64_t len = (int64_t)(N + 1) * n;
  const int gb = (int)std::min<int64_t>(1184, (len + 255) / 256);
  k_diag_unscale<<<gb, 256, 0, s>>>(len, delta_diag, x, y);
  if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  double *rq = reinterpret_cast<double *>(w + L.rq), *ru = reinterpret_cast<double *>(w + L.ru);
  double *rc = reinterpret_cast<double *>(w + L.rc), *dx = reinterpret_cast<double *>(w + L.dx);
  double *du = reinterpret_cast<double *>(w + L.du), *dy = reinterpret_cast<double *>(w + L.dy);
  double *norms = reinterpret_cast<double *>(w + L.norms);
  const int rb = (N + 1 + 127) / 128;
  auto residual = [&]() -> bool {
    if (cudaMemsetAsync(norms, 0, 4 * sizeof(double), s) != cudaSuccess) return false;
    k_diag_residual<<<rb, 128, 0, s>>>(N, n, m, delta_diag, prob->Q, prob->M, prob->R, prob->q,
                                       prob->r, prob->A, prob->B, prob->c, x, u, y, rq, ru, rc,
                                       norms);
    return cudaGetLastError() == cudaSuccess;
  };
  if (opts->prec == RLQR_MIXED) {
    // one refinement pass against the ORIGINAL system: the refinement inside
    // rlqr_solve measures the scaled system, whose backward error differs
    // from the original one by the condition of the diagonal scaling
    if (!residual()) return RLQR_ERR_CUDA;
    rlqr_problem cp = sp;
    cp.q = rq;
    cp.r = ru;
    cp.c = rc;
    e = rlqr_solve(&cp, &o, w + L.lqr, lw, dx, du, dy, nullptr, nullptr, nullptr, stream);
    if (e != RLQR_OK) return e;
    k_diag_update<<<gb, 256, 0, s>>>(N, n, m, delta_diag, dx, du, dy, x, u, y);
    if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (rel_resid) {
    if (!residual()) return RLQR_ERR_CUDA;
    k_diag_rel<<<1, 32, 0, s>>>(norms, rel_resid);
    if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (opts->flags & RLQR_OPT_SYNC) {
    int32_t st = RLQR_OK;
    if (status &&
        (cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
      return RLQR_ERR_CUDA;
    return (rlqr_status)st;
  }
  return RLQR_OK;
}

}  // extern "C"

// cross.cuh -- cross-stage variables theta in R^p (Section "Cross-Stage
// Variables", eq. cross-stage-kkt / cross-stage-schur): after the p + 1
// solves with the instance's factor (the right-hand side b, giving z_b, and
// the p columns of J, giving V = -K^{-1} J), the bordered system reduces to
//   S dtheta = -g,   S = H + J^T V = H - J^T K^{-1} J,   g = r_theta + J^T z_b,
//   dw = z_b + V dtheta.
// J and V columns share the layout of the right-hand side (q | r | c, paired
// with x | u | y).  Included by one translation unit (rlqr_api.cu).
#pragma once

#include "common.cuh"

namespace rlqr {

constexpr int kCrossBlocks = 296;  // partial-sum blocks of the dot products
constexpr int kCrossMaxP = 31;     // one warp solves the p x p system (p + 1 columns)

// Element e of z_b (x | u | y order, lengths nX, nU, nX).
__device__ __forceinline__ double zb_at(const double *x, const double *u, const double *y,
                                        int64_t nX, int64_t nU, int64_t e) {
  return e < nX ? x[e] : (e < nX + nU ? u[e - nX] : y[e - nX - nU]);
}

// Partial sums of J_i . V_j (j < p) and J_i . z_b (j = p) over this block's
// contiguous segment of the L entries: part[blk][i][j], (p+1) p per block.
// Fixed segments and in-block reduction order: the sums are deterministic.
__global__ void __launch_bounds__(256) k_cross_dots(int p, int64_t L, int64_t nX, int64_t nU,
                                                    const double *J, const double *V,
                                                    const double *x, const double *u,
                                                    const double *y, double *part) {
  __shared__ double red[8][kCrossMaxP + 1];
  const int64_t seg = (L + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * seg, e1 = min(L, e0 + seg);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = 0; i < p; ++i) {
    const double *Ji = J + (size_t)i * L;
    for (int j = 0; j <= p; ++j) {
      double acc = 0.0;
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double v = j < p ? V[(size_t)j * L + e] : zb_at(x, u, y, nX, nU, e);
        acc = fma(Ji[e], v, acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) red[w][j] = acc;
    }
    __syncthreads();
    if (threadIdx.x <= p) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
      part[((size_t)blockIdx.x * p + i) * (p + 1) + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// S and g from H, r_theta and the partials (each entry summed by one warp in
// a fixed order), then S dtheta = -g by Gaussian elimination with partial
// pivoting (warp 0, lane = row).  status: the worst of the factor's pivot
// status and the p + 1 solve statuses (slots cleared before the solves), or
// RLQR_ERR_SINGULAR for a zero or non-finite pivot of S.  One block of 1024
// threads.
__global__ void __launch_bounds__(1024) k_cross_theta(int p, int nblk, const double *H,
                                                      const double *rt, const double *part,
                                                      const InstState *inst,
                                                      const int32_t *solve_st, double *dtheta,
                                                      int32_t *status) {
  __shared__ double S[kCrossMaxP + 1][kCrossMaxP + 2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pr = w; pr < p * (p + 1); pr += nw) {
    const int i = pr / (p + 1), j = pr - i * (p + 1);
    double t = 0.0;
    for (int b = lane; b < nblk; b += 32) t += part[((size_t)b * p + i) * (p + 1) + j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      t += j < p ? H[i * p + j] : rt[i];
      S[i][j] = j < p ? t : -t;  // column p: the right-hand side -g
    }
  }
  __syncthreads();
  if (w != 0) return;
  int sing = 0;
  for (int k = 0; k < p; ++k) {
    // pivot: the largest |S[i][k]|, i >= k
    double best = (lane >= k && lane < p) ? fabs(S[lane][k]) : -1.0;
    int arg = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    if (!(best > 0.0) || !isfinite(best)) sing = 1;
    if (arg != k && lane <= p) {  // swap rows k and arg, lane = column
      const double a = S[k][lane];
      S[k][lane] = S[arg][lane];
      S[arg][lane] = a;
    }
    __syncwarp();
    if (lane > k && lane < p && !sing) {
      const double f = S[lane][k] / S[k][k];
      for (int c = k + 1; c <= p; ++c) S[lane][c] = fma(-f, S[k][c], S[lane][c]);
    }
    __syncwarp();
  }
  if (lane == 0) {
    for (int k = p - 1; k >= 0; --k) {
      double t = S[k][p];
      for (int c = k + 1; c < p; ++c) t = fma(-S[k][c], dtheta[c], t);
      dtheta[k] = sing ? 0.0 : t / S[k][k];
    }
    int32_t st = inst->pivot_status;
    for (int j = 0; j <= p; ++j) st = max(st, solve_st[j]);
    if (sing) st = RLQR_ERR_SINGULAR;
    status[0] = st;
  }
}

// dw = z_b + V dtheta into x | u | y (z_b is column p of V).
__global__ void k_cross_combine(int p, int64_t L, int64_t nX, int64_t nU, const double *V,
                                const double *dtheta, double *x, double *u, double *y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x) {
    double t = V[(size_t)p * L + e];
    for (int j = 0; j < p; ++j) t = fma(V[(size_t)j * L + e], __ldg(dtheta + j), t);
    if (e < nX) x[e] = t;
    else if (e < nX + nU) u[e - nX] = t;
    else y[e - nX - nU] = t;
  }
}

}  // namespace rlqr

// residual_grid.cuh -- the first residual of a ragged batch (Section
// "Residual Computation"), stage-parallel over all instances: one warp per
// (instance, stage) work item, FP64 products straight from global memory, the
// maxima of each instance by atomicMax on order-preserving bit patterns and
// a per-instance finalize of the normwise backward error.  Work item g of the
// flattened index belongs to instance b with spre[b] <= g < spre[b+1]
// (spre: exclusive prefix sum of N_b + 1, from k_plan; null for a single
// instance); item N_b of an instance holds its rows x_N and c_0.  Included by rlqr_api.cu only.
#pragma once

#include "common.cuh"
#include "refine.cuh"

namespace rlqr {

__device__ __forceinline__ int instance_of_item(const int64_t *spre, int count, int64_t g) {
  if (!spre) return 0;  // one instance: items 0..N
  int lo = 0, hi = count;  // spre[lo] <= g < spre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (spre[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_resb_reset(BatchArgs a) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.count; b += gridDim.x * blockDim.x) {
    InstState *st = get_inst(a, b).st;
    if (a.recheck && (st->converged || st->pivot_status == RLQR_ERR_SINGULAR)) continue;
    st->rmax = 0.0;
    st->zmax = 0.0;
    st->kmax = 0.0;
    st->bmax = 0.0;
  }
}

// FP64 certificate with margin of the stored FP32 control pivots G_s (mixed
// path), one stage per thread (pd_margin_f32): bit1 of flags[s], the worst
// status, and the escalation mark for a decision without its margin.
__global__ void k_certb(BatchArgs a, const int64_t *spre, int64_t total) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int b = instance_of_item(spre, a.count, g);
    const Inst I = get_inst(a, b);
    const int s = (int)(g - (spre ? spre[b] : 0));
    if (s >= I.N) continue;
    const int m = I.m;
    const float *G = reinterpret_cast<const float *>(I.ws + I.L.G) + (size_t)s * m * m;
    const int dec = pd_margin_f32<16>(G, m, (double)kMarginTau);
    I.flags[s] = (uint8_t)((I.flags[s] & 1) | (dec == kPdYes ? 2 : 0));
    if (dec == kPdNo) atomicMax(&I.st->pivot_status, (int32_t)RLQR_NOT_PD);
    if (dec == kPdAmbiguous) I.st->escalated = 1;
  }
}

// Residual rows of work item g (warp per item); store: write res for the
// refinement.  Maxima of |res|, |z|, |b| and the row sums of |K| per instance.
__global__ void __launch_bounds__(256) k_resb(BatchArgs a, const int64_t *spre, int64_t total,
                                              int store) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w0; g < total; g += nw) {
    const int b = instance_of_item(spre, a.count, g);
    const Inst I = get_inst(a, b);
    if (a.recheck && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) continue;
    const int N = I.N, n = I.n, m = I.m, s = (int)(g - (spre ? spre[b] : 0));
    const int nn = n * n, nm = n * m, mmm = m * m;
    const double delta = I.delta;
    double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
    double *rr = rq + (size_t)(N + 1) * n;
    double *rc = rr + (size_t)N * m;
    unsigned long long rbits = 0, zbits = 0, bbits = 0;
    float kmaxf = 0.f;
    if (s < N) {
      const double *Q = I.Q + (size_t)s * nn, *M = I.M + (size_t)s * nm, *R = I.R + (size_t)s * mmm;
      const double *A = I.A + (size_t)s * nn, *B = I.B + (size_t)s * nm;
      const double *x = I.x + (size_t)s * n, *u = I.u + (size_t)s * m;
      const double *yn = I.y + (size_t)(s + 1) * n, *xn = I.x + (size_t)(s + 1) * n;
      for (int r = lane; r < 2 * n + m; r += 32) {
        double v;
        float ra;
        if (r < n) {  // x row: Q x + M u + A^T y_{s+1} + q - y_s
          const double qv = __ldg(I.q + (size_t)s * n + r);
          v = qv - __ldg(I.y + (size_t)s * n + r);
          ra = 1.f;
          for (int l = 0; l < n; ++l) {
            const double qq = __ldg(Q + (r <= l ? r * n + l : l * n + r)), aa = __ldg(A + l * n + r);
            v = fma(qq, __ldg(x + l), fma(aa, __ldg(yn + l), v));
            ra += abs_f32_trunc(qq) + abs_f32_trunc(aa);
          }
          for (int l = 0; l < m; ++l) {
            const double mv = __ldg(M + r * m + l);
            v = fma(mv, __ldg(u + l), v);
            ra += abs_f32_trunc(mv);
          }
          bbits = max(bbits, abs_bits(qv));
          if (store) rq[(size_t)s * n + r] = v;
          zbits = max(zbits, abs_bits(__ldg(x + r)));
        } else if (r < n + m) {  // u row: M^T x + R u + B^T y_{s+1} + r
          const int t = r - n;
          const double rv = __ldg(I.r + (size_t)s * m + t);
          v = rv;
          ra = 0.f;
          for (int l = 0; l < n; ++l) {
            const double mv = __ldg(M + l * m + t), bv = __ldg(B + l * m + t);
            v = fma(mv, __ldg(x + l), fma(bv, __ldg(yn + l), v));
            ra += abs_f32_trunc(mv) + abs_f32_trunc(bv);
          }
          for (int l = 0; l < m; ++l) {
            const double rr2 = __ldg(R + (t <= l ? t * m + l : l * m + t));
            v = fma(rr2, __ldg(u + l), v);
            ra += abs_f32_trunc(rr2);
          }
          bbits = max(bbits, abs_bits(rv));
          if (store) rr[(size_t)s * m + t] = v;
          zbits = max(zbits, abs_bits(__ldg(u + t)));
        } else {  // c row of stage s+1: A x + B u + c_{s+1} - x_{s+1} - delta y_{s+1}
          const int i = r - n - m;
          const double cv = __ldg(I.c + (size_t)(s + 1) * n + i);
          v = cv - __ldg(xn + i) - delta * __ldg(yn + i);
          ra = 1.f + abs_f32_trunc(delta);
          for (int l = 0; l < n; ++l) {
            const double av = __ldg(A + i * n + l);
            v = fma(av, __ldg(x + l), v);
            ra += abs_f32_trunc(av);
          }
          for (int l = 0; l < m; ++l) {
            const double bv = __ldg(B + i * m + l);
            v = fma(bv, __ldg(u + l), v);
            ra += abs_f32_trunc(bv);
          }
          bbits = max(bbits, abs_bits(cv));
          if (store) rc[(size_t)(s + 1) * n + i] = v;
          zbits = max(zbits, abs_bits(__ldg(yn + i)));
        }
        rbits = max(rbits, abs_bits(v));
        kmaxf = fmaxf(kmaxf, ra);
      }
    } else {  // rows x_N (Q_N x_N + q_N - y_N) and c_0 (c_0 - delta y_0 - x_0)
      for (int r = lane; r < 2 * n; r += 32) {
        double v;
        if (r < n) {
          const double qv = __ldg(I.q + (size_t)N * n + r), yv = __ldg(I.y + (size_t)N * n + r);
          v = qv - yv;
          float ra = 1.f;
          for (int l = 0; l < n; ++l) {
            const double q = __ldg(I.Q + (size_t)N * nn + (r <= l ? r * n + l : l * n + r));
            v = fma(q, __ldg(I.x + (size_t)N * n + l), v);
            ra += abs_f32_trunc(q);
          }
          kmaxf = fmaxf(kmaxf, ra);
          bbits = max(bbits, abs_bits(qv));
          zbits = max(zbits, max(abs_bits(__ldg(I.x + (size_t)N * n + r)), abs_bits(yv)));
          if (store) rq[(size_t)N * n + r] = v;
        } else {
          const int i = r - n;
          const double cv = __ldg(I.c + i), yv = __ldg(I.y + i);
          v = cv - delta * yv - __ldg(I.x + i);
          kmaxf = fmaxf(kmaxf, 1.f + abs_f32_trunc(delta));
          bbits = max(bbits, abs_bits(cv));
          zbits = max(zbits, abs_bits(yv));
          if (store) rc[i] = v;
        }
        rbits = max(rbits, abs_bits(v));
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
      zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
      bbits = max(bbits, __shfl_xor_sync(0xffffffffu, bbits, o));
      kmaxf = fmaxf(kmaxf, __shfl_xor_sync(0xffffffffu, kmaxf, o));
    }
    if (lane == 0) {
      InstState *st = I.st;
      atomicMax(reinterpret_cast<unsigned long long *>(&st->rmax), rbits);
      atomicMax(reinterpret_cast<unsigned long long *>(&st->zmax), zbits);
      atomicMax(reinterpret_cast<unsigned long long *>(&st->bmax), bbits);
      atomicMax(reinterpret_cast<unsigned long long *>(&st->kmax), abs_bits(widen(kmaxf)));
    }
  }
}

// Backward error, convergence and the per-instance outputs.
__global__ void k_resb_final(BatchArgs a) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.count; b += gridDim.x * blockDim.x) {
    InstState *st = get_inst(a, b).st;
    if (a.recheck && (st->converged || st->pivot_status == RLQR_ERR_SINGULAR)) continue;
    const double den = st->kmax * st->zmax + st->bmax;
    const double rel = den > 0.0 ? st->rmax / den : st->rmax;
    st->rel = rel;
    st->upd = 0.0;  // a residual computed from scratch
    const int32_t conv = (rel <= a.tol) ? 1 : 0;
    st->converged = conv;
    if (a.rel) a.rel[b] = rel;
    if (a.iters) a.iters[b] = st->iters;
    write_status(a, b, st, conv);
  }
}

}  // namespace rlqr

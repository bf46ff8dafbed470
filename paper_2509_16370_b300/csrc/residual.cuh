// residual.cuh -- the FP64 KKT residual kernel (and the FP64 certificate of
// the control pivots of the mixed-precision sweep).  Included by exactly one
// translation unit (rlqr_api.cu).
#pragma once

#include "common.cuh"
#include "refine.cuh"

namespace rlqr {

// FP64 residual of the current (x, u, y), its infinity norm, ||z||, and the
// normwise backward error; one CTA per instance, one warp per stage.
//
// For stage s < N the rows [x_s; u_s; c_{s+1}] of K z + b are one dense
// (2n+m) x (2n+m) block times z_s = [x_s; u_s; y_{s+1}] plus a per-row base:
//   x rows  [Q_s  M_s  A_s^T] z_s + q_s - y_s
//   u rows  [M_s^T R_s B_s^T] z_s + r_s
//   c rows  [A_s  B_s  0    ] z_s + c_{s+1} - delta y_{s+1} - x_{s+1}
// The warp assembles the block in shared memory from coalesced loads, then
// each lane takes one row: all lanes run the same FP64 dot product (no
// divergence, which on B300 would cost FP64 issue slots on idle lanes).  The
// rows x_N and c_0 are a short epilogue.
//
// `store` writes res into the workspace for a following correction solve.
// `res_out` (single-instance API) is an optional caller buffer in the same
// res_q | res_r | res_c layout, and `norms_out` receives
// [rmax, kmax, zmax, bmax, rel].  `standalone`: no workspace (rlqr_residual);
// the instance state is local.  `recompute_norms`: take ||K|| and ||b|| here
// instead of from the sweep.
__global__ void k_residual(BatchArgs a, int store, double *res_out, double *norms_out,
                           int recompute_norms, int standalone, int rs_max, int cert_g,
                           int do_residual) {
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  const int N = I.N, n = I.n, m = I.m;
  const double delta = I.delta;
  const int nn = n * n, nm = n * m, mmm = m * m;
  const int rs = 2 * n + m, ld = rs + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *Kb = reinterpret_cast<double *>(smem_raw + residual_warp_bytes(rs_max) * warp);
  double *zb = Kb + (size_t)rs_max * (rs_max + 1);
  double *base = zb + rs_max;
  __shared__ double s_red[32];
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;
  double *oq = res_out, *orr = res_out ? res_out + (size_t)(N + 1) * n : nullptr;
  double *oc = res_out ? orr + (size_t)N * m : nullptr;
  // ||K|| row sums in FP32 (they only scale the backward error); the maxima
  // of |res|, |z| and |b| as order-preserving bit patterns (INT pipe)
  float kmaxf = 0.f;
  unsigned long long rbits = 0, zbits = 0, bbits = 0;

  if (cert_g) {
    // Control-pivot certificate with margin (mixed path), one stage per
    // thread (pd_margin_f32): bit1 of flags[s]; a decision without its
    // margin escalates the instance to the FP64 recursion.
    const float *gG = reinterpret_cast<const float *>(I.ws + I.L.G);
    int bad = 0, esc = 0;
    for (int s = threadIdx.x; s < N; s += blockDim.x) {
      const int dec = pd_margin_f32<16>(gG + (size_t)s * m * m, m, (double)kMarginTau);
      const uint8_t old = I.flags[s];
      I.flags[s] = (uint8_t)((old & 1) | (dec == kPdYes ? 2 : 0));
      bad |= dec == kPdNo;
      esc |= dec == kPdAmbiguous;
    }
    const int any_bad = __syncthreads_or(bad);
    const int any_esc = __syncthreads_or(esc);
    if (threadIdx.x == 0 && !standalone) {
      int32_t ps = I.st->pivot_status;
      if (any_bad && ps == RLQR_OK) ps = RLQR_NOT_PD;
      I.st->pivot_status = ps;
      if (any_esc) I.st->escalated = 1;
      if (!do_residual && a.status) a.status[b] = ps;
    }
    __syncthreads();
  }
  if (!do_residual) return;

  // the c-row x y-column block is identically zero
  for (int e = lane; e < n * n; e += 32) Kb[(n + m + e / n) * ld + n + m + e % n] = 0.0;

  for (int s = warp; s < N; s += nwarps) {
    const double *Qs = I.Q + (size_t)s * nn, *Ms = I.M + (size_t)s * nm;
    const double *Rs = I.R + (size_t)s * mmm, *As = I.A + (size_t)s * nn;
    const double *Bs = I.B + (size_t)s * nm;
    __syncwarp();
    for (int e = lane; e < nn; e += 32) {
      const int i = e / n, j = e % n;
      const double q = __ldg(Qs + e), av = __ldg(As + e);
      if (i <= j) {
        Kb[i * ld + j] = q;
        Kb[j * ld + i] = q;
      }
      Kb[(n + m + i) * ld + j] = av;      // c rows: A_s
      Kb[j * ld + n + m + i] = av;        // x rows: A_s^T
    }
    for (int e = lane; e < nm; e += 32) {
      const int i = e / m, j = e % m;
      const double mv = __ldg(Ms + e), bv = __ldg(Bs + e);
      Kb[i * ld + n + j] = mv;            // x rows: M_s
      Kb[(n + j) * ld + i] = mv;          // u rows: M_s^T
      Kb[(n + m + i) * ld + n + j] = bv;  // c rows: B_s
      Kb[(n + j) * ld + n + m + i] = bv;  // u rows: B_s^T
    }
    for (int e = lane; e < mmm; e += 32) {
      const int i = e / m, j = e % m;
      if (i <= j) {
        const double rv = __ldg(Rs + e);
        Kb[(n + i) * ld + n + j] = rv;
        Kb[(n + j) * ld + n + i] = rv;
      }
    }
    for (int r = lane; r < rs; r += 32) {
      double zv, bv;
      if (r < n) {
        zv = __ldg(I.x + (size_t)s * n + r);
        bv = __ldg(I.q + (size_t)s * n + r) - __ldg(I.y + (size_t)s * n + r);
        if (recompute_norms) bbits = max(bbits, abs_bits(__ldg(I.q + (size_t)s * n + r)));
      } else if (r < n + m) {
        zv = __ldg(I.u + (size_t)s * m + r - n);
        bv = __ldg(I.r + (size_t)s * m + r - n);
        if (recompute_norms) bbits = max(bbits, abs_bits(bv));
      } else {
        const size_t o = (size_t)(s + 1) * n + r - n - m;
        zv = __ldg(I.y + o);
        const double cv = __ldg(I.c + o);
        bv = cv - delta * zv - __ldg(I.x + o);
        if (recompute_norms) bbits = max(bbits, abs_bits(cv));
      }
      zb[r] = zv;
      base[r] = bv;
      zbits = max(zbits, abs_bits(zv));
    }
    __syncwarp();
    for (int r = lane; r < rs; r += 32) {
      double v = base[r];
      const double *row = Kb + r * ld;
      for (int j = 0; j < rs; ++j) v = fma(row[j], zb[j], v);
      if (recompute_norms) {
        float ra = (r < n) ? 1.f : ((r < n + m) ? 0.f : 1.f + abs_f32_trunc(delta));
        for (int j = 0; j < rs; ++j) ra += abs_f32_trunc(row[j]);
        kmaxf = fmaxf(kmaxf, ra);
      }
      rbits = max(rbits, abs_bits(v));
      if (r < n) {
        if (store) rq[(size_t)s * n + r] = v;
        if (oq) oq[(size_t)s * n + r] = v;
      } else if (r < n + m) {
        if (store) rr[(size_t)s * m + r - n] = v;
        if (orr) orr[(size_t)s * m + r - n] = v;
      } else {
        if (store) rc[(size_t)(s + 1) * n + r - n - m] = v;
        if (oc) oc[(size_t)(s + 1) * n + r - n - m] = v;
      }
    }
  }
  // epilogue: rows x_N (Q_N x_N + q_N - y_N) and c_0 (c_0 - delta y_0 - x_0)
  for (int r = threadIdx.x; r < 2 * n; r += blockDim.x) {
    double v;
    if (r < n) {
      const double *QN = I.Q + (size_t)N * nn, *xN = I.x + (size_t)N * n;
      const double qv = __ldg(I.q + (size_t)N * n + r), yv = __ldg(I.y + (size_t)N * n + r);
      v = qv - yv;
      float ra = 1.f;
      for (int j = 0; j < n; ++j) {
        const double q = (r <= j) ? __ldg(QN + r * n + j) : __ldg(QN + j * n + r);
        v = fma(q, __ldg(xN + j), v);
        ra += abs_f32_trunc(q);
      }
      zbits = max(zbits, max(abs_bits(__ldg(xN + r)), abs_bits(yv)));
      if (recompute_norms) {
        kmaxf = fmaxf(kmaxf, ra);
        bbits = max(bbits, abs_bits(qv));
      }
      if (store) rq[(size_t)N * n + r] = v;
      if (oq) oq[(size_t)N * n + r] = v;
    } else {
      const int i = r - n;
      const double xv = __ldg(I.x + i), yv = __ldg(I.y + i), cv = __ldg(I.c + i);
      v = cv - delta * yv - xv;
      zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
      if (recompute_norms) {
        kmaxf = fmaxf(kmaxf, 1.f + abs_f32_trunc(delta));
        bbits = max(bbits, abs_bits(cv));
      }
      if (store) rc[i] = v;
      if (oc) oc[i] = v;
    }
    rbits = max(rbits, abs_bits(v));
  }
  const double rmax = block_max_dyn(bits_to_double(rbits), s_red);
  const double zmax = block_max_dyn(bits_to_double(zbits), s_red);
  double kmax = 0.0, bmax = 0.0;
  if (recompute_norms) {
    kmax = block_max_dyn((double)kmaxf, s_red);
    bmax = block_max_dyn(bits_to_double(bbits), s_red);
  }
  if (threadIdx.x == 0) {
    InstState local{};
    InstState *st = standalone ? &local : I.st;
    if (recompute_norms) {
      st->kmax = kmax;
      st->bmax = bmax;
    }
    const double den = st->kmax * zmax + st->bmax;
    const double rel = den > 0.0 ? rmax / den : rmax;
    st->rmax = rmax;
    st->zmax = zmax;
    st->rel = rel;
    st->upd = 0.0;  // a residual computed from scratch
    const int32_t conv = (rel <= a.tol) ? 1 : 0;
    st->converged = conv;
    if (a.rel) a.rel[b] = rel;
    if (a.iters) a.iters[b] = st->iters;
    write_status(a, b, st, conv);
    if (norms_out) {
      norms_out[0] = rmax;
      norms_out[1] = st->kmax;
      norms_out[2] = zmax;
      norms_out[3] = st->bmax;
      norms_out[4] = rel;
    }
  }
}

}  // namespace rlqr

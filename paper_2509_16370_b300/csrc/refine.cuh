// refine.cuh -- FP64 KKT residual, right-hand-side solves with a stored
// factor, and iterative refinement.
//
// Residual (Section "Residual Computation"), per stage s = 0..N:
//   res_q[s] = Q_s x_s + M_s u_s + A_s^T y_{s+1} + q_s - y_s   (last two terms
//              only for s < N)
//   res_r[s] = M_s^T x_s + R_s u_s + B_s^T y_{s+1} + r_s       (s < N)
//   res_c[s] = c_s - delta y_s - x_s + A_{s-1} x_{s-1} + B_{s-1} u_{s-1} (s > 0)
// It equals K z + b for the matrix of eq. primal-dual-linear-system.
//
// Solve with a stored factor (Corollary p-recurrence): with W_i, K_i, G_i^{-1}
// from the sweep, for a right-hand side (q', r', c'):
//   p_N = q'_N;  g = p_{k+1} + W_{k+1}(c'_{k+1} - delta p_{k+1})
//   h = r'_k + B_k^T g,  k_k = -G_k^{-1} h,  p_k = q'_k + A_k^T g + K_k^T h
// (K^T h = H^T k because H = -G K), then the forward rollout of seq.cuh.
//
// Refinement: the correction dz solves K dz = -res, z <- z + dz in FP64, and
// the residual is updated as res <- res + K dz with the products in the
// working precision and the accumulation in FP64.  Since |dz| ~ u_w |z|, the
// updated residual is accurate to ~u_w^2 |K||z|, far below the 1e-9 target,
// so only the first residual of a solve needs full FP64 products.
#pragma once

#include "common.cuh"

namespace rlqr {

__device__ __forceinline__ void write_status(const BatchArgs &a, int b, const InstState *st,
                                             int32_t conv) {
  if (!a.status) return;
  int32_t ps = st->pivot_status;
  a.status[b] = (ps == RLQR_ERR_SINGULAR) ? RLQR_ERR_SINGULAR
                                          : (conv ? ps : RLQR_ERR_NOT_CONVERGED);
}

// Block-wide max of non-negative doubles for any blockDim (multiple of 32).
__device__ __forceinline__ double block_max_dyn(double v, double *scratch /* >= 32 */) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < nw; ++i) r = fmax(r, scratch[i]);
  __syncthreads();
  return r;
}

// Shared memory of k_residual per warp: the dense stage block (rs x (rs+1)),
// the stage vector z and the row bases.
__host__ __device__ inline size_t residual_warp_bytes(int rs_max) {
  return sizeof(double) * ((size_t)rs_max * (rs_max + 1) + 2 * (size_t)rs_max);
}

template <typename T, int NM, int MM>
struct SolveSmem {
  static constexpr int kT = 3 * NM * NM /*W A Q*/ + 3 * NM * MM /*B M K*/ + 2 * MM * MM /*R Gi*/ +
                            10 * NM + 6 * MM;
  static constexpr int kD = 4 * NM + 2 * MM;  // FP64 x, y, u, res_q, res_r, res_c of a stage
  static constexpr size_t bytes() { return align_up(sizeof(T) * kT, 16) + sizeof(double) * kD + 64; }
};

// Right-hand-side solve with the factor stored in the workspace; one CTA per
// instance.  FROM_RES = false: the right-hand side is the problem's (q, r, c)
// and x, u, y are overwritten with the solution.  FROM_RES = true: it is the
// stored FP64 residual; the correction is added to x, u, y in FP64 and the
// residual, ||z|| and the backward error are updated.
template <typename T, class D, int THREADS, bool FROM_RES>
__global__ void __launch_bounds__(THREADS) k_solve(BatchArgs a) {
  constexpr int NM = D::NM, MM = D::MM;
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  InstState *stp = I.st;
  if (FROM_RES) {
    if (stp->converged || stp->pivot_status == RLQR_ERR_SINGULAR) return;
  } else if (threadIdx.x == 0) {
    stp->iters = 0;
    stp->converged = 0;
  }
  const D dims(I.n, I.m);
  const int N = I.N, n = dims.n, m = dims.m;
  const T delta = (T)I.delta;
  const double delta64 = I.delta;
  const int tid = threadIdx.x;
  const int nn = n * n, nm = n * m, mmm = m * m;
  using S = SolveSmem<T, NM, MM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *sW = sm;  sm += NM * NM;
  T *sA = sm;  sm += NM * NM;
  T *sQ = sm;  sm += NM * NM;
  T *sB = sm;  sm += NM * MM;
  T *sM = sm;  sm += NM * MM;
  T *sK = sm;  sm += NM * MM;
  T *sR = sm;  sm += MM * MM;
  T *sGi = sm; sm += MM * MM;
  T *sp = sm;  sm += NM;   // p_{k+1}
  T *sq = sm;  sm += NM;   // rhs q_k
  T *sc = sm;  sm += NM;   // rhs c_{k+1}
  T *sv = sm;  sm += NM;
  T *sg = sm;  sm += NM;
  T *sdx = sm; sm += NM;   // dx_k
  T *sdxn = sm; sm += NM;  // dx_{k+1}
  T *sdy = sm; sm += NM;   // dy_k
  T *sdyn = sm; sm += NM;  // dy_{k+1}
  T *st = sm;  sm += NM;
  T *sr = sm;  sm += MM;
  T *sh = sm;  sm += MM;
  T *skk = sm; sm += MM;
  T *sdu = sm; sm += MM;
  (void)S::kT;
  __shared__ double s_red[THREADS / 32 + 1];

  const T *gW = reinterpret_cast<const T *>(I.ws + I.L.W);
  const T *gK = reinterpret_cast<const T *>(I.ws + I.L.K);
  const T *gGi = reinterpret_cast<const T *>(I.ws + I.L.Gi);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;
  const double *Rq = FROM_RES ? rq : I.q;
  const double *Rr = FROM_RES ? rr : I.r;
  const double *Rc = FROM_RES ? rc : I.c;

  constexpr int CP = (NM * NM + THREADS - 1) / THREADS;
  constexpr int CB = (NM * MM + THREADS - 1) / THREADS;
  constexpr int CR = (MM * MM + THREADS - 1) / THREADS;
  constexpr int CV = (NM + THREADS - 1) / THREADS;
  constexpr int CM = (MM + THREADS - 1) / THREADS;

  // ---------------- backward: p-recurrence
  for (int i = tid; i < n; i += THREADS) {
    T v = to_work<T>(__ldcg(Rq + (size_t)N * n + i));
    sp[i] = v;
    gpv[(size_t)N * n + i] = v;
  }
  RegSeg<T, THREADS, CP> bW;
  RegSeg<double, THREADS, CP> bA;
  RegSeg<double, THREADS, CB> bB;
  RegSeg<T, THREADS, CB> bK;
  RegSeg<T, THREADS, CR> bG;
  RegSeg<double, THREADS, CV> bq, bc;
  RegSeg<double, THREADS, CM> br;
  auto bprefetch = [&](int k) {
    bW.load_cg(gW + (size_t)(k + 1) * nn, nn);
    bA.load(I.A + (size_t)k * nn, nn);
    bB.load(I.B + (size_t)k * nm, nm);
    bK.load_cg(gK + (size_t)k * nm, nm);
    bG.load_cg(gGi + (size_t)k * mmm, mmm);
    bq.load_cg(Rq + (size_t)k * n, n);
    bc.load_cg(Rc + (size_t)(k + 1) * n, n);
    br.load_cg(Rr + (size_t)k * m, m);
  };
  bprefetch(N - 1);
  __syncthreads();
  for (int k = N - 1; k >= 0; --k) {
    bW.store(sW, nn);
    bA.store(sA, nn);
    bB.store(sB, nm);
    bK.store(sK, nm);
    bG.store(sGi, mmm);
    bq.store(sq, n);
    bc.store(sc, n);
    br.store(sr, m);
    if (k > 0) bprefetch(k - 1);
    __syncthreads();
    // g = p + W (c' - delta p)
    for (int i = tid; i < n; i += THREADS) {
      T s = sp[i];
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sW[i * n + l] * (sc[l] - delta * sp[l]);
      sg[i] = s;
    }
    __syncthreads();
    for (int i = tid; i < m; i += THREADS) {
      T s = sr[i];
      for (int l = 0; l < n; ++l) s += sB[l * m + i] * sg[l];
      sh[i] = s;
    }
    __syncthreads();
    for (int i = tid; i < n + m; i += THREADS) {
      if (i < n) {
        T s = sq[i];
        for (int l = 0; l < n; ++l) s += sA[l * n + i] * sg[l];
        for (int l = 0; l < m; ++l) s += sK[l * n + i] * sh[l];
        sp[i] = s;
        gpv[(size_t)k * n + i] = s;
      } else {
        int j = i - n;
        T s = 0;
        for (int l = 0; l < m; ++l) s += sGi[j * m + l] * sh[l];
        gkv[(size_t)k * m + j] = -s;
      }
    }
    __syncthreads();
  }

  // ---------------- forward rollout (+ z update and residual update)
  // The FP64 iterate and residual rows of the next stage are prefetched with
  // the stage data, so their read-modify-writes never wait on HBM.
  unsigned long long rbits = 0, zbits = 0, dzbits = 0;  // max |.| as order-preserving bit patterns
  double *dsm = reinterpret_cast<double *>(smem_raw + align_up(sizeof(T) * S::kT, 16));
  double *zx = dsm, *zy = dsm + NM, *zq = dsm + 2 * NM, *zc = dsm + 3 * NM;
  double *zu = dsm + 4 * NM, *zr = zu + MM;
  T *dx = sdx, *dxn = sdxn, *dy = sdy, *dyn = sdyn;
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0, v0 = c'_0 - delta p_0
  for (int idx = tid; idx < nn; idx += THREADS) sW[idx] = __ldcg(gW + idx);
  for (int i = tid; i < n; i += THREADS) sv[i] = to_work<T>(__ldcg(Rc + i)) - delta * sp[i];
  __syncthreads();
  for (int i = tid; i < n; i += THREADS) {
    T t = 0;
#pragma unroll
    for (int l = 0; l < NM; ++l)
      if (l < n) t += sW[i * n + l] * sv[l];
    T dxv = sv[i] - delta * t, dyv = t + sp[i];
    dx[i] = dxv;
    dy[i] = dyv;
    if (FROM_RES) {
      double xv = I.x[i] + widen(dxv), yv = I.y[i] + widen(dyv);
      I.x[i] = xv;
      I.y[i] = yv;
      zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
      dzbits = max(dzbits, max(abs_bits(widen(dxv)), abs_bits(widen(dyv))));
      double r0 = __ldcg(rc + i) - widen(dxv) - delta64 * widen(dyv);  // (K dz) rows of y_0
      rc[i] = r0;
      rbits = max(rbits, abs_bits(r0));
    } else {
      I.x[i] = widen(dxv);
      I.y[i] = widen(dyv);
    }
  }
  RegSeg<T, THREADS, CP> fW;
  RegSeg<double, THREADS, CP> fA, fQ;
  RegSeg<double, THREADS, CB> fB, fM;
  RegSeg<T, THREADS, CB> fK;
  RegSeg<double, THREADS, CR> fR;
  RegSeg<T, THREADS, CM> fk;
  RegSeg<T, THREADS, CV> fp;
  RegSeg<double, THREADS, CV> fc, fzx, fzy, fzq, fzc;
  RegSeg<double, THREADS, CM> fzu, fzr;
  auto fprefetch = [&](int k) {
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn);
    fA.load(I.A + (size_t)k * nn, nn);
    fB.load(I.B + (size_t)k * nm, nm);
    fK.load_cg(gK + (size_t)k * nm, nm);
    fk.load_cg(gkv + (size_t)k * m, m);
    fp.load_cg(gpv + (size_t)(k + 1) * n, n);
    fc.load_cg(Rc + (size_t)(k + 1) * n, n);
    if (FROM_RES) {
      fQ.load(I.Q + (size_t)k * nn, nn);
      fM.load(I.M + (size_t)k * nm, nm);
      fR.load(I.R + (size_t)k * mmm, mmm);
      fzx.load_cg(I.x + (size_t)(k + 1) * n, n);
      fzy.load_cg(I.y + (size_t)(k + 1) * n, n);
      fzu.load_cg(I.u + (size_t)k * m, m);
      fzq.load_cg(rq + (size_t)k * n, n);
      fzr.load_cg(rr + (size_t)k * m, m);
      fzc.load_cg(rc + (size_t)(k + 1) * n, n);
    }
  };
  __syncthreads();
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
    fW.store(sW, nn);
    fA.store(sA, nn);
    fB.store(sB, nm);
    fK.store(sK, nm);
    fk.store(skk, m);
    fp.store(sp, n);
    fc.store(sc, n);
    if (FROM_RES) {
      fQ.store_sym(sQ, n);
      fM.store(sM, nm);
      fR.store_sym(sR, m);
      fzx.store(zx, n);
      fzy.store(zy, n);
      fzu.store(zu, m);
      fzq.store(zq, n);
      fzr.store(zr, m);
      fzc.store(zc, n);
    }
    if (k + 1 < N) fprefetch(k + 1);
    __syncthreads();
    // du_k = K_k dx_k + k_k
    for (int i = tid; i < m; i += THREADS) {
      T s = skk[i];
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sK[i * n + l] * dx[l];
      sdu[i] = s;
      if (FROM_RES) {
        const double uv = zu[i] + widen(s);
        I.u[(size_t)k * m + i] = uv;
        zbits = max(zbits, abs_bits(uv));
        dzbits = max(dzbits, abs_bits(widen(s)));
      } else {
        I.u[(size_t)k * m + i] = widen(s);
      }
    }
    __syncthreads();
    // v = A dx + B du + c'_{k+1} - delta p_{k+1}
    for (int i = tid; i < n; i += THREADS) {
      T s = sc[i] - delta * sp[i];
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sA[i * n + l] * dx[l];
#pragma unroll
      for (int l = 0; l < MM; ++l)
        if (l < m) s += sB[i * m + l] * sdu[l];
      sv[i] = s;
    }
    __syncthreads();
    // dx_{k+1} = v - delta W v, dy_{k+1} = W v + p_{k+1}
    for (int i = tid; i < n; i += THREADS) {
      T t = 0;
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) t += sW[i * n + l] * sv[l];
      const T dxv = sv[i] - delta * t, dyv = t + sp[i];
      dxn[i] = dxv;
      dyn[i] = dyv;
      const size_t o = (size_t)(k + 1) * n + i;
      if (FROM_RES) {
        const double xv = zx[i] + widen(dxv), yv = zy[i] + widen(dyv);
        I.x[o] = xv;
        I.y[o] = yv;
        zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
        dzbits = max(dzbits, max(abs_bits(widen(dxv)), abs_bits(widen(dyv))));
      } else {
        I.x[o] = widen(dxv);
        I.y[o] = widen(dyv);
      }
    }
    __syncthreads();
    if (FROM_RES) {
      // res += K dz for the rows of stage k (x_k, u_k) and of c_{k+1}
      for (int i = tid; i < 2 * n + m; i += THREADS) {
        T s = 0;
        double old, *dst;
        if (i < n) {
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sQ[i * n + l] * dx[l] + sA[l * n + i] * dyn[l];
#pragma unroll
          for (int l = 0; l < MM; ++l)
            if (l < m) s += sM[i * m + l] * sdu[l];
          s -= dy[i];
          old = zq[i];
          dst = rq + (size_t)k * n + i;
        } else if (i < n + m) {
          const int j = i - n;
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sM[l * m + j] * dx[l] + sB[l * m + j] * dyn[l];
#pragma unroll
          for (int l = 0; l < MM; ++l)
            if (l < m) s += sR[j * m + l] * sdu[l];
          old = zr[j];
          dst = rr + (size_t)k * m + j;
        } else {
          const int j = i - n - m;
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sA[j * n + l] * dx[l];
#pragma unroll
          for (int l = 0; l < MM; ++l)
            if (l < m) s += sB[j * m + l] * sdu[l];
          s -= dxn[j] + delta * dyn[j];
          old = zc[j];
          dst = rc + (size_t)(k + 1) * n + j;
        }
        const double nv = old + widen(s);
        *dst = nv;
        rbits = max(rbits, abs_bits(nv));
      }
      __syncthreads();
    }
    T *t1 = dx; dx = dxn; dxn = t1;
    T *t2 = dy; dy = dyn; dyn = t2;
  }
  if (!FROM_RES) return;
  // terminal rows x_N: res += Q_N dx_N - dy_N
  for (int idx = tid; idx < nn; idx += THREADS) {
    const int i = idx / n, j = idx - i * n;
    if (i <= j) {
      const T v = to_work<T>(__ldg(I.Q + (size_t)N * nn + idx));
      sQ[i * n + j] = v;
      sQ[j * n + i] = v;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += THREADS) {
    T s = -dy[i];
    for (int l = 0; l < n; ++l) s += sQ[i * n + l] * dx[l];
    double *dst = rq + (size_t)N * n + i;
    double nv = __ldcg(dst) + widen(s);
    *dst = nv;
    rbits = max(rbits, abs_bits(nv));
  }
  const double rmax = block_max<THREADS>(bits_to_double(rbits), s_red);
  const double zmax = block_max<THREADS>(bits_to_double(zbits), s_red);
  const double dzmax = block_max<THREADS>(bits_to_double(dzbits), s_red);
  if (tid == 0) {
    // the working-precision products of this pass's residual update err by
    // at most 2 gamma_L ||K||_inf max|dz| per entry (L = 2n + m); the bound
    // accumulates over passes and is part of the reported backward error
    const double uw = sizeof(T) == 4 ? 0x1p-24 : 0x1p-53;
    stp->upd += 2.0 * (2 * n + m) * uw * stp->kmax * dzmax;
    double den = stp->kmax * zmax + stp->bmax;
    double rel = den > 0.0 ? (rmax + stp->upd) / den : rmax + stp->upd;
    stp->rmax = rmax;
    stp->zmax = zmax;
    stp->rel = rel;
    stp->iters += 1;
    int32_t conv = (rel <= a.tol) ? 1 : 0;
    stp->converged = conv;
    if (a.rel) a.rel[b] = rel;
    if (a.iters) a.iters[b] = stp->iters;
    write_status(a, b, stp, conv);
  }
}

}  // namespace rlqr

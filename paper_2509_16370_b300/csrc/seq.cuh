// seq.cuh -- sequential dual-regularized Riccati sweep on B300.
//
// One CTA per LQR instance walks the horizon (Section "Sequential Algorithm",
// Theorem main-seq-theorem).  Per stage k = N-1 .. 0, with P = P_{k+1} and
// p = p_{k+1} resident in shared memory:
//
//   Gauss-Jordan on [I + delta P | P]   -> W_{k+1} = (I + delta P)^{-1} P
//                                          = P (I + delta P)^{-1}
//                                          (Corollary inverse-helper-corollary)
//   WA = W A_k, WB = W B_k, g = p + W (c_{k+1} - delta p)
//   G = R_k + B^T WB, H = B^T WA + M_k^T, h = r_k + B^T g
//   Gauss-Jordan on [G | H | h | I]     -> K_k = -G^{-1}H, k_k = -G^{-1}h, G^{-1}
//   P_k = Q_k + A^T WA + H^T K_k,  p_k = q_k + A^T g + H^T k_k
//                                          (eq. value-fn-formulas)
//
// Certificate (Section "Inertia Certification"): flags[i] bit0 says that the
// state pivot I + delta P_i is PD, bit1 that the control pivot G_i is PD.
//  * FP64 sweep: Gauss-Jordan without pivoting meets the pivots of an LDL^T
//    of the symmetric pivot matrix, so their signs are the certificate.
//  * FP32 sweep: every decision is still taken in FP64.  For the state pivot
//    an FP64 Gershgorin test proves I + delta P PD in O(n^2) work (each row's
//    1 + delta P_ii - delta sum_{j!=i} |P_ij| > 0, with a rigorous bound on the
//    FP32 row sum); only a stage that fails the test runs an FP64 LDL^T of
//    I + delta P (under the same barriers as the FP32 elimination).  The
//    control pivot G_i is stored and factored in FP64 by k_residual,
//    one stage per thread.  On B300 a warp FP64 instruction costs the same
//    whatever its active lanes, so FP64 work is kept lane-packed.
//
// The forward rollout (eq. recover-x0, control-law, recover-x) uses only W:
// with v = A_k x_k + B_k u_k + c_{k+1} - delta p_{k+1},
//   x_{k+1} = (I + delta P_{k+1})^{-1} v = v - delta W_{k+1} v
//   y_{k+1} = P_{k+1} x_{k+1} + p_{k+1} = W_{k+1} v + p_{k+1}
// because (I + delta P)^{-1} = I - delta P (I + delta P)^{-1}.
//
// Each pivot reciprocal is computed once (by the thread that finalises the
// pivot entry).  The next stage's data is prefetched into registers while the
// current stage computes, so the HBM latency is off the per-stage critical
// path.  The common (n, m) get compile-time dimensions (FixDims): all loop
// bounds and index divisions fold.
#pragma once

#include "common.cuh"

namespace rlqr {

template <typename T, int NM, int MM>
struct SeqSmem {
  static constexpr int kP = NM * NM, kAug = NM * 2 * NM, kB = NM * MM, kR = MM * MM;
  static constexpr int kGaug = MM * (2 * MM + NM + 1);
  static constexpr int kT = kP /*P*/ + kAug + kP /*W*/ + kP /*A*/ + kB /*B*/ + kP /*Q*/ +
                            kB /*M*/ + kR /*R*/ + kP /*WA*/ + kB /*WB*/ + kB /*H*/ + kGaug +
                            kB /*K*/ + 8 * NM + 3 * MM;
  static constexpr int kD = NM * NM;  // FP64 shadow of I + delta P (FP32 sweep)
  static constexpr size_t bytes(bool shadow) {
    return align_up(sizeof(T) * kT, 16) + (shadow ? sizeof(double) * kD : 0) + 64;
  }
};

// Pivot bookkeeping shared by the CTA.
template <typename T, int NM, int MM>
struct PivotShared {
  T rinv[NM];          // reciprocals of the Gauss-Jordan pivots of [I + delta P | P]
  T ginv[MM];          // ... of [G | H | h | I]
  double rinv64[NM];   // ... of the FP64 LDL^T of I + delta P (FP32 sweep fallback)
  int bit0, bit1, singular, status;
};

// Records the decision on pivot value d (FP64) into the shared flags.
__device__ __forceinline__ void decide(double d, int *bit, int *singular) {
  if (!(d > 0.0)) *bit = 0;
  if (!finite_nonzero(d)) *singular = 1;
}

// Gauss-Jordan elimination (no pivoting, rows left unscaled) of the `rows` x
// `w` matrix X in shared memory on its leading rows x rows block.  After it,
// X = [D | D X_0^{-1} X_right] with D the pivots; rinv[j] = 1 / D_j.  The
// entry (j+1, j+1) is final after step j, so its reciprocal is taken there.
// DECIDE: the Gauss-Jordan pivots decide the certificate bit (FP64 sweep).
// With `shadow` (CTA-uniform) an FP64 LDL^T of the symmetric S (rows x rows,
// lower triangle) runs under the same barriers and decides it instead.
// rinv[0] / rinv64[0] must be set by the caller.  RMAX bounds `rows`; with
// FixDims everything below unrolls to constant index math.
template <typename T, int THREADS, int RMAX, bool DECIDE, bool HAS_SHADOW>
__device__ __forceinline__ void gauss_jordan(const int rows, const int w, T *X, T *rinv,
                                             bool shadow, double *S, double *rinv64, int *bit,
                                             int *singular) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int j = 0; j < RMAX; ++j) {
    if (j >= rows) break;
    if (tid == 0) {
      if (HAS_SHADOW && shadow) decide(S[j * rows + j], bit, singular);
      else if (DECIDE) decide((double)X[j * w + j], bit, singular);
    }
    const T inv = rinv[j];
    const int cols = w - j - 1;
    for (int idx = tid; idx < (rows - 1) * cols; idx += THREADS) {
      const int ii = idx / cols, cc = j + 1 + (idx - ii * cols);
      const int i = ii < j ? ii : ii + 1;
      const T v = X[i * w + cc] - X[i * w + j] * (X[j * w + cc] * inv);
      X[i * w + cc] = v;
      if (i == j + 1 && cc == j + 1) rinv[j + 1] = (T)1 / v;
    }
    if (HAS_SHADOW && shadow) {
      const double rd = rinv64[j];
      const int r = rows - j - 1;
      for (int idx = tid; idx < r * (r + 1) / 2; idx += THREADS) {
        int i, cc;
        tri_decode(idx, i, cc);
        i += j + 1;
        cc += j + 1;
        const double v = S[i * rows + cc] - S[i * rows + j] * (S[cc * rows + j] * rd);
        S[i * rows + cc] = v;
        if (i == j + 1 && cc == j + 1) rinv64[j + 1] = 1.0 / v;
      }
    }
    __syncthreads();
  }
}

// State pivot of a stage: [I + delta P | P] -> W = (I + delta P)^{-1} P,
// symmetrized, into sW and gW (global), and the certificate bit of
// I + delta P into ps.bit0.  Ends with a barrier.
template <typename T, int NM, int MM, int THREADS, bool FP32SWEEP>
__device__ __forceinline__ void state_pivot(const int n, T delta, double delta64, const T *sP,
                                            T *sAug, T *sW, T *gW, double *sS64,
                                            PivotShared<T, NM, MM> &ps) {
  const int tid = threadIdx.x, w2 = 2 * n, nn = n * n;
  for (int idx = tid; idx < n * w2; idx += THREADS) {
    const int i = idx / w2, j = idx - i * w2;
    const T v = (j < n) ? (T)(i == j) + delta * sP[i * n + j] : sP[i * n + (j - n)];
    sAug[idx] = v;
    if (idx == 0) ps.rinv[0] = (T)1 / v;
  }
  bool shadow = false;
  if (FP32SWEEP) {
    // Gershgorin certificate of I + delta P: sum_{j != i} |P_ij| is taken in
    // FP32 (non-negative terms: relative error <= (n-1) 2^-24), the test in FP64.
    int pass = 1;
    if (tid < n) {
      float off = 0.f;
      for (int j = 0; j < n; ++j)
        if (j != tid) off += fabsf((float)sP[tid * n + j]);
      const double bound = (double)off * (1.0 + 2.0 * n * 5.960464477539063e-08);
      const double g = 1.0 + delta64 * ((double)sP[tid * n + tid] - bound);
      pass = g > 1e-12;
    }
    shadow = !__syncthreads_and(pass);
    if (shadow) {
      for (int idx = tid; idx < nn; idx += THREADS) {
        const int i = idx / n, j = idx - i * n;
        const double v = (double)(i == j) + delta64 * (double)sP[idx];
        sS64[idx] = v;
        if (idx == 0) ps.rinv64[0] = 1.0 / v;
      }
      __syncthreads();
    }
  } else {
    __syncthreads();
  }
  gauss_jordan<T, THREADS, NM, !FP32SWEEP, FP32SWEEP>(n, w2, sAug, ps.rinv, shadow, sS64,
                                                     ps.rinv64, &ps.bit0, &ps.singular);
  for (int idx = tid; idx < nn; idx += THREADS) {
    const int i = idx / n, j = idx - i * n;
    const T w = (T)0.5 * (sAug[i * w2 + n + j] * ps.rinv[i] + sAug[j * w2 + n + i] * ps.rinv[j]);
    sW[idx] = w;
    gW[idx] = w;
  }
  __syncthreads();
}

// Sweep kernel.  SOLVE: also run the vector recursion on (q, r, c) and the
// forward rollout, writing x, u, y.  T = float is the mixed-precision sweep
// (certificate as described above).  D: DynDims or FixDims.
template <typename T, class D, int THREADS, bool SOLVE>
__global__ void __launch_bounds__(THREADS) k_seq(BatchArgs a) {
  constexpr bool FP32SWEEP = sizeof(T) == 4;
  constexpr int NM = D::NM, MM = D::MM;
  const int b = blockIdx.x;
  if (b >= a.count) return;
  const Inst I = get_inst(a, b);
  const D dims(I.n, I.m);
  const int N = I.N, n = dims.n, m = dims.m;
  const T delta = (T)I.delta;
  const int tid = threadIdx.x;
  using S = SeqSmem<T, NM, MM>;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *sP = sm;   sm += S::kP;
  T *sAug = sm; sm += S::kAug;
  T *sW = sm;   sm += S::kP;
  T *sA = sm;   sm += S::kP;
  T *sB = sm;   sm += S::kB;
  T *sQ = sm;   sm += S::kP;
  T *sM = sm;   sm += S::kB;
  T *sR = sm;   sm += S::kR;
  T *sWA = sm;  sm += S::kP;
  T *sWB = sm;  sm += S::kB;
  T *sH = sm;   sm += S::kB;
  T *sG = sm;   sm += S::kGaug;
  T *sK = sm;   sm += S::kB;
  T *sp = sm;   sm += NM;
  T *sq = sm;   sm += NM;
  T *sc = sm;   sm += NM;
  T *sv = sm;   sm += NM;
  T *sg = sm;   sm += NM;
  T *sx = sm;   sm += NM;
  T *sr = sm;   sm += MM;
  T *skk = sm;  sm += MM;
  T *su = sm;   sm += MM;
  double *sS64 = reinterpret_cast<double *>(smem_raw + align_up(sizeof(T) * S::kT, 16));
  __shared__ PivotShared<T, NM, MM> ps;
  __shared__ double s_red[THREADS / 32 + 1];

  T *gW = reinterpret_cast<T *>(I.ws + I.L.W);
  T *gK = reinterpret_cast<T *>(I.ws + I.L.K);
  T *gGi = reinterpret_cast<T *>(I.ws + I.L.Gi);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  T *gG = reinterpret_cast<T *>(I.ws + I.L.G);

  const int nn = n * n, nm = n * m, mmm = m * m;
  const int wg = 2 * m + n + 1;  // row length of [G | H | h | I]
  constexpr int CP = (NM * NM + THREADS - 1) / THREADS;
  constexpr int CB = (NM * MM + THREADS - 1) / THREADS;
  constexpr int CR = (MM * MM + THREADS - 1) / THREADS;
  constexpr int CV = (NM + THREADS - 1) / THREADS;
  constexpr int CM = (MM + THREADS - 1) / THREADS;

  bool notpd = false;
  T kmax_loc = 0, bmax_loc = 0;  // norms of the data, working precision (they only scale rel)

  // ---- terminal stage: P_N = Q_N (upper triangle), p_N = q_N
  for (int idx = tid; idx < nn; idx += THREADS) {
    const int i = idx / n, j = idx - i * n;
    sP[idx] = (T)((i <= j) ? I.Q[(size_t)N * nn + idx] : I.Q[(size_t)N * nn + j * n + i]);
  }
  if (SOLVE)
    for (int i = tid; i < n; i += THREADS) {
      sp[i] = (T)I.q[(size_t)N * n + i];
      gpv[(size_t)N * n + i] = sp[i];
    }
  if (a.want_norms) {
    // x_N rows: |Q_N| + 1 (the -y_N); y_0 rows: 1 + delta; entries q_N and c_0 of b
    for (int i = tid; i < n; i += THREADS) {
      T s = 1;
      for (int j = 0; j < n; ++j)
        s += (T)fabs(i <= j ? I.Q[(size_t)N * nn + i * n + j] : I.Q[(size_t)N * nn + j * n + i]);
      kmax_loc = fmax(kmax_loc, fmax(s, (T)1 + delta));
      bmax_loc = fmax(bmax_loc, (T)fmax(fabs(I.q[(size_t)N * n + i]), fabs(I.c[i])));
    }
  }
  if (tid == 0) {
    ps.bit0 = 1;
    ps.bit1 = 1;
    ps.singular = 0;
  }
  int bit1_next = 1;  // stage N has no control pivot

  RegSeg<double, THREADS, CP> pfA, pfQ;
  RegSeg<double, THREADS, CB> pfB, pfM;
  RegSeg<double, THREADS, CR> pfR;
  RegSeg<double, THREADS, CV> pfq, pfc;
  RegSeg<double, THREADS, CM> pfr;
  auto prefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn);
    pfQ.load(I.Q + (size_t)k * nn, nn);
    pfB.load(I.B + (size_t)k * nm, nm);
    pfM.load(I.M + (size_t)k * nm, nm);
    pfR.load(I.R + (size_t)k * mmm, mmm);
    if (SOLVE) {
      pfq.load(I.q + (size_t)k * n, n);
      pfc.load(I.c + (size_t)(k + 1) * n, n);
      pfr.load(I.r + (size_t)k * m, m);
    }
  };
  prefetch(N - 1);
  __syncthreads();

  for (int k = N - 1; k >= 0; --k) {
    // ---- (1) commit stage k's data to shared memory, start fetching stage k-1
    pfA.store(sA, nn);
    pfQ.store_sym(sQ, n);
    pfB.store(sB, nm);
    pfM.store(sM, nm);
    pfR.store_sym(sR, m);
    if (SOLVE) {
      pfq.store(sq, n);
      pfc.store(sc, n);
      pfr.store(sr, m);
    }
    if (k > 0) prefetch(k - 1);
    __syncthreads();
    if (SOLVE)
      for (int i = tid; i < n; i += THREADS) sv[i] = sc[i] - delta * sp[i];
    if (a.want_norms) {
      // row sums of |K| (working precision: they only scale the backward error):
      // x_k rows |Q_k| + |M_k| + |A_k^T| + 1, u_k rows |M_k^T| + |R_k| + |B_k^T|,
      // y_{k+1} rows |A_k| + |B_k| + 1 + delta
      for (int i = tid; i < 2 * n + m; i += THREADS) {
        T s = 0;
        if (i < n) {
          s = 1;
          for (int j = 0; j < n; ++j) s += fabs(sQ[i * n + j]);
          for (int j = 0; j < m; ++j) s += fabs(sM[i * m + j]);
          for (int j = 0; j < n; ++j) s += fabs(sA[j * n + i]);
          bmax_loc = fmax(bmax_loc, fmax(fabs(sq[i]), fabs(sc[i])));
        } else if (i < n + m) {
          const int a2 = i - n;
          for (int j = 0; j < n; ++j) s += fabs(sM[j * m + a2]);
          for (int j = 0; j < m; ++j) s += fabs(sR[a2 * m + j]);
          for (int j = 0; j < n; ++j) s += fabs(sB[j * m + a2]);
          bmax_loc = fmax(bmax_loc, fabs(sr[a2]));
        } else {
          const int a2 = i - n - m;
          s = (T)1 + delta;
          for (int j = 0; j < n; ++j) s += fabs(sA[a2 * n + j]);
          for (int j = 0; j < m; ++j) s += fabs(sB[a2 * m + j]);
        }
        kmax_loc = fmax(kmax_loc, s);
      }
    }

    // ---- (2)-(4) state pivot of stage k+1: W_{k+1}
    state_pivot<T, NM, MM, THREADS, FP32SWEEP>(n, delta, I.delta, sP, sAug, sW,
                                              gW + (size_t)(k + 1) * nn, sS64, ps);

    // ---- (5) WA = W A, WB = W B, g = p + W v
    {
      const int tot = nn + nm + (SOLVE ? n : 0);
      for (int idx = tid; idx < tot; idx += THREADS) {
        if (idx < nn) {
          const int i = idx / n, j = idx - i * n;
          T s = 0;
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * sA[l * n + j];
          sWA[idx] = s;
        } else if (idx < nn + nm) {
          const int e = idx - nn, i = e / m, j = e - i * m;
          T s = 0;
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * sB[l * m + j];
          sWB[e] = s;
        } else {
          const int i = idx - nn - nm;
          T s = sp[i];
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * sv[l];
          sg[i] = s;
        }
      }
    }
    __syncthreads();

    // ---- (6) [G | H | h | I], H copy, P_k <- Q_k + A^T WA (lower), p_k <- q_k + A^T g
    {
      const int nlo = n * (n + 1) / 2;
      const int tot = m * wg + nlo + (SOLVE ? n : 0);
      for (int idx = tid; idx < tot; idx += THREADS) {
        if (idx < m * wg) {
          const int i = idx / wg, j = idx - i * wg;
          T s;
          if (j < m) {
            s = sR[i * m + j];
#pragma unroll
            for (int l = 0; l < NM; ++l)
              if (l < n) s += sB[l * m + i] * sWB[l * m + j];
            if (FP32SWEEP) gG[(size_t)k * mmm + i * m + j] = s;
          } else if (j < m + n) {
            const int jj = j - m;
            s = sM[jj * m + i];
#pragma unroll
            for (int l = 0; l < NM; ++l)
              if (l < n) s += sB[l * m + i] * sWA[l * n + jj];
            sH[i * n + jj] = s;
          } else if (j == m + n) {
            s = 0;
            if (SOLVE) {
              s = sr[i];
#pragma unroll
              for (int l = 0; l < NM; ++l)
                if (l < n) s += sB[l * m + i] * sg[l];
            }
          } else {
            s = (T)((j - m - n - 1) == i);
          }
          sG[idx] = s;
          if (idx == 0) ps.ginv[0] = (T)1 / s;
        } else if (idx < m * wg + nlo) {
          int i, j;
          tri_decode(idx - m * wg, i, j);
          T s = sQ[i * n + j];
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sA[l * n + i] * sWA[l * n + j];
          sP[i * n + j] = s;
          sP[j * n + i] = s;
        } else {
          const int i = idx - m * wg - nlo;
          T s = sq[i];
#pragma unroll
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sA[l * n + i] * sg[l];
          sp[i] = s;
        }
      }
    }
    __syncthreads();

    // ---- (7) Gauss-Jordan on [G | H | h | I] (FP64 sweep: its pivots decide bit1)
    gauss_jordan<T, THREADS, MM, !FP32SWEEP, false>(m, wg, sG, ps.ginv, false, nullptr, nullptr,
                                                     &ps.bit1, &ps.singular);

    // ---- (8) K_k = -G^{-1} H, k_k = -G^{-1} h, G^{-1}; store
    for (int idx = tid; idx < nm + mmm + (SOLVE ? m : 0); idx += THREADS) {
      if (idx < nm) {
        const int i = idx / n, j = idx - i * n;
        const T kv = -sG[i * wg + m + j] * ps.ginv[i];
        sK[idx] = kv;
        gK[(size_t)k * nm + idx] = kv;
      } else if (idx < nm + mmm) {
        const int e = idx - nm, i = e / m, j = e - i * m;
        gGi[(size_t)k * mmm + e] = sG[i * wg + m + n + 1 + j] * ps.ginv[i];
      } else {
        const int i = idx - nm - mmm;
        const T kv = -sG[i * wg + m + n] * ps.ginv[i];
        skk[i] = kv;
        gkv[(size_t)k * m + i] = kv;
      }
    }
    __syncthreads();

    // ---- (9) P_k += H^T K_k (symmetric), p_k += H^T k_k; store p_k; flags
    {
      const int nlo = n * (n + 1) / 2;
      for (int idx = tid; idx < nlo + (SOLVE ? n : 0); idx += THREADS) {
        if (idx < nlo) {
          int i, j;
          tri_decode(idx, i, j);
          T s = 0;
#pragma unroll
          for (int l = 0; l < MM; ++l)
            if (l < m) s += sH[l * n + i] * sK[l * n + j];
          const T v = sP[i * n + j] + s;
          sP[i * n + j] = v;
          sP[j * n + i] = v;
        } else {
          const int i = idx - nlo;
          T s = sp[i];
#pragma unroll
          for (int l = 0; l < MM; ++l)
            if (l < m) s += sH[l * n + i] * skk[l];
          sp[i] = s;
          gpv[(size_t)k * n + i] = s;
        }
      }
    }
    if (tid == 0) {
      // FP32 sweep: bit1 of stages < N is added by the FP64 control-pivot pass
      const int b1 = FP32SWEEP ? (k + 1 == N) : bit1_next;
      I.flags[k + 1] = (uint8_t)(ps.bit0 | (b1 << 1));
      if (!ps.bit0 || (!FP32SWEEP && !b1)) notpd = true;
      bit1_next = ps.bit1;
      ps.bit0 = 1;
      ps.bit1 = 1;
    }
    __syncthreads();
  }

  // ---- initial-state pivot I + delta P_0: W_0 and bit0 of stage 0
  state_pivot<T, NM, MM, THREADS, FP32SWEEP>(n, delta, I.delta, sP, sAug, sW, gW, sS64, ps);
  if (tid == 0) {
    const int b1 = FP32SWEEP ? (N == 0) : bit1_next;
    I.flags[0] = (uint8_t)(ps.bit0 | (b1 << 1));
    if (!ps.bit0 || (!FP32SWEEP && !b1)) notpd = true;
    ps.status = ps.singular ? RLQR_ERR_SINGULAR : (notpd ? RLQR_NOT_PD : RLQR_OK);
  }
  if (a.want_norms) {
    const double km = block_max<THREADS>((double)kmax_loc, s_red);
    const double bm = block_max<THREADS>((double)bmax_loc, s_red);
    if (tid == 0) {
      I.st->kmax = km;
      I.st->bmax = bm;
    }
  }
  __syncthreads();
  if (tid == 0) {
    I.st->pivot_status = ps.status;
    I.st->iters = 0;
    I.st->converged = 0;
    I.st->rel = 0.0;
    if (a.status) a.status[b] = ps.status;
  }
  if (!SOLVE) return;

  // ---- forward rollout
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  for (int i = tid; i < n; i += THREADS) {
    sp[i] = __ldcg(gpv + i);
    sv[i] = (T)I.c[i] - delta * sp[i];
  }
  __syncthreads();
  for (int i = tid; i < n; i += THREADS) {
    T t = 0;
#pragma unroll
    for (int l = 0; l < NM; ++l)
      if (l < n) t += sW[i * n + l] * sv[l];
    const T xv = sv[i] - delta * t, yv = t + sp[i];
    sx[i] = xv;
    I.x[i] = (double)xv;
    I.y[i] = (double)yv;
  }
  RegSeg<T, THREADS, CP> fW;
  RegSeg<T, THREADS, CB> fK;
  RegSeg<T, THREADS, CM> fk;
  RegSeg<T, THREADS, CV> fp;
  auto fprefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn);
    pfB.load(I.B + (size_t)k * nm, nm);
    pfc.load(I.c + (size_t)(k + 1) * n, n);
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn);
    fK.load_cg(gK + (size_t)k * nm, nm);
    fk.load_cg(gkv + (size_t)k * m, m);
    fp.load_cg(gpv + (size_t)(k + 1) * n, n);
  };
  __syncthreads();
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
    pfA.store(sA, nn);
    pfB.store(sB, nm);
    pfc.store(sc, n);
    fW.store(sW, nn);
    fK.store(sK, nm);
    fk.store(skk, m);
    fp.store(sp, n);
    if (k + 1 < N) fprefetch(k + 1);
    __syncthreads();
    // u_k = K_k x_k + k_k
    for (int i = tid; i < m; i += THREADS) {
      T s = skk[i];
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sK[i * n + l] * sx[l];
      su[i] = s;
      I.u[(size_t)k * m + i] = (double)s;
    }
    __syncthreads();
    // v = A x + B u + c_{k+1} - delta p_{k+1}
    for (int i = tid; i < n; i += THREADS) {
      T s = sc[i] - delta * sp[i];
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sA[i * n + l] * sx[l];
#pragma unroll
      for (int l = 0; l < MM; ++l)
        if (l < m) s += sB[i * m + l] * su[l];
      sv[i] = s;
    }
    __syncthreads();
    // x_{k+1} = v - delta W v, y_{k+1} = W v + p_{k+1}
    for (int i = tid; i < n; i += THREADS) {
      T t = 0;
#pragma unroll
      for (int l = 0; l < NM; ++l)
        if (l < n) t += sW[i * n + l] * sv[l];
      const T xv = sv[i] - delta * t, yv = t + sp[i];
      sx[i] = xv;
      I.x[(size_t)(k + 1) * n + i] = (double)xv;
      I.y[(size_t)(k + 1) * n + i] = (double)yv;
    }
    __syncthreads();
  }
}

}  // namespace rlqr

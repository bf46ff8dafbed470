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
// Both eliminations are register-resident: each thread owns a fixed column
// and a fixed block of rows of the augmented matrix, and only the pivot row
// and pivot column of each step go through shared memory (double-buffered,
// one barrier per step).  There is no index arithmetic inside the steps.
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
// Each pivot reciprocal is computed once, by the thread that owns the pivot
// entry.  The next stage's data is prefetched into registers while the
// current stage computes, so the HBM latency is off the per-stage critical
// path.  The common (n, m) get compile-time dimensions (FixDims).
#pragma once

#include "common.cuh"

namespace rlqr {

// Records the decision on pivot value d (FP64) into shared flags.
__device__ __forceinline__ void decide(double d, int *bit, int *singular) {
  if (!(d > 0.0)) *bit = 0;
  if (!finite_nonzero(d)) *singular = 1;
}

// Shared state of one register-resident Gauss-Jordan elimination.
template <typename T, int RMAX, int WMAX>
struct GJShared {
  T col[2][RMAX];   // pivot column of the current / next step
  T row[2][WMAX];   // pivot row of the current / next step
  T rinv[RMAX];     // reciprocals of the pivots
  int bit, singular;
};

// Gauss-Jordan (no pivoting, rows left unscaled) of an R x W matrix spread
// over the CTA: thread t owns column c = t % WMAX and rows r0 .. r0+RPT-1 with
// r0 = (t / WMAX) * RPT.  After the R steps the leading block is diag(D) (D the
// pivots, which are those of an LDL^T of a symmetric leading block) and the
// trailing columns hold D X_0^{-1} X_right.
template <typename T, int THREADS, int RMAX, int WMAX>
struct RegGJ {
  static constexpr int G = THREADS / WMAX;
  static constexpr int RPT = (RMAX + (G > 0 ? G : 1) - 1) / (G > 0 ? G : 1);
  static_assert(G >= 1, "the CTA must have at least one thread per column");
  using Sh = GJShared<T, RMAX, WMAX>;
  T v[RPT];
  int c, r0;
  bool own;

  __device__ __forceinline__ RegGJ() {
    c = threadIdx.x % WMAX;
    const int g = threadIdx.x / WMAX;
    r0 = g * RPT;
    own = g < G;
  }

  // Publish the pivot row / column of step 0 (after v has been filled).
  template <bool DECIDE>
  __device__ __forceinline__ void publish0(int rows, int w, Sh &sh) {
    if (!own || c >= w) return;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i = r0 + r;
      if (i < rows && c == 0) sh.col[0][i] = v[r];
      if (i == 0) {
        sh.row[0][c] = v[r];
        if (c == 0) {
          sh.rinv[0] = recip_pivot(v[r]);
          if (DECIDE) decide((double)v[r], &sh.bit, &sh.singular);
        }
      }
    }
  }

  // Step j: eliminate column j from every row but j, then publish the pivot
  // row / column of step j + 1.  The caller puts a barrier after it.
  template <bool DECIDE>
  __device__ __forceinline__ void step(int j, int rows, int w, Sh &sh) {
    if (!own || c >= w) return;
    const int cur = j & 1, nxt = cur ^ 1;
    if (c > j) {
      const T f = sh.row[cur][c] * sh.rinv[j];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = r0 + r;
        if (i < rows && i != j) v[r] -= sh.col[cur][i] * f;
      }
    }
    if (j + 1 < rows) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = r0 + r;
        if (i < rows && c == j + 1) sh.col[nxt][i] = v[r];
        if (i == j + 1) {
          sh.row[nxt][c] = v[r];
          if (c == j + 1) {
            sh.rinv[j + 1] = recip_pivot(v[r]);
            if (DECIDE) decide((double)v[r], &sh.bit, &sh.singular);
          }
        }
      }
    }
  }
};

// FP64 LDL^T step j of the symmetric rows x rows matrix S (lower triangle),
// flat over the CTA (fallback certificate of the FP32 sweep).
template <int THREADS>
__device__ __forceinline__ void ldlt64_step(int j, int rows, double *S, double *rinv64, int *bit,
                                            int *singular) {
  const int tid = threadIdx.x;
  if (tid == 0) decide(S[j * rows + j], bit, singular);
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

template <typename T, int NM, int MM>
struct SeqSmem {
  static constexpr int kP = NM * NM, kB = NM * MM, kR = MM * MM;
  static constexpr int kT = 5 * kP /*P W A Q WA*/ + 5 * kB /*B M WB H K*/ + kR /*R*/ +
                            6 * NM + 3 * MM;
  static constexpr int kD = NM * NM;  // FP64 shadow of I + delta P (FP32 sweep fallback)
  static constexpr size_t bytes(bool shadow) {
    return align_up(sizeof(T) * kT, 16) + (shadow ? sizeof(double) * kD : 0) + 64;
  }
};

// Sweep kernel.  SOLVE: also run the vector recursion on (q, r, c) and the
// forward rollout, writing x, u, y.  T = float is the mixed-precision sweep
// (certificate as described above).  D: DynDims or FixDims.
template <typename T, class D, int THREADS, bool SOLVE>
__global__ void __launch_bounds__(THREADS) k_seq(BatchArgs a) {
  constexpr bool FP32SWEEP = sizeof(T) == 4;
  constexpr bool DECIDE = !FP32SWEEP;
  constexpr int NM = D::NM, MM = D::MM;
  constexpr int WS = 2 * NM;           // columns of [I + delta P | P]
  constexpr int WC = 2 * MM + NM + 1;  // columns of [G | H | h | I]
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  const D dims(I.n, I.m);
  const int N = I.N, n = dims.n, m = dims.m;
  const T delta = (T)I.delta;
  const float delta_up = __double2float_ru(I.delta);  // Gershgorin test (FP32 sweep)
  const float delta_dn = __double2float_rd(I.delta);
  const int tid = threadIdx.x;
  using S = SeqSmem<T, NM, MM>;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *sP = sm;   sm += S::kP;
  T *sW = sm;   sm += S::kP;
  T *sA = sm;   sm += S::kP;
  T *sQ = sm;   sm += S::kP;
  T *sWA = sm;  sm += S::kP;
  T *sB = sm;   sm += S::kB;
  T *sM = sm;   sm += S::kB;
  T *sWB = sm;  sm += S::kB;
  T *sH = sm;   sm += S::kB;
  T *sK = sm;   sm += S::kB;
  T *sR = sm;   sm += S::kR;
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
  __shared__ GJShared<T, NM, WS> shs;   // state pivot elimination
  __shared__ GJShared<T, MM, WC> shc;   // control pivot elimination
  __shared__ double rinv64[NM];

  T *gW = reinterpret_cast<T *>(I.ws + I.L.W);
  T *gK = reinterpret_cast<T *>(I.ws + I.L.K);
  T *gGi = reinterpret_cast<T *>(I.ws + I.L.Gi);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  T *gG = reinterpret_cast<T *>(I.ws + I.L.G);

  const int nn = n * n, nm = n * m, mmm = m * m;
  const int w2 = 2 * n, wg = 2 * m + n + 1;
  constexpr int CP = (NM * NM + THREADS - 1) / THREADS;
  constexpr int CB = (NM * MM + THREADS - 1) / THREADS;
  constexpr int CR = (MM * MM + THREADS - 1) / THREADS;
  constexpr int CV = (NM + THREADS - 1) / THREADS;
  constexpr int CM = (MM + THREADS - 1) / THREADS;

  RegGJ<T, THREADS, NM, WS> gs;  // owner of entries of [I + delta P | P]
  RegGJ<T, THREADS, MM, WC> gc;  // owner of entries of [G | H | h | I]
  bool notpd = false, singular = false, escal = false;
  int bit1_next = 1;  // stage N has no control pivot

  // ---- terminal stage: P_N = Q_N (upper triangle), p_N = q_N
  for (int idx = tid; idx < nn; idx += THREADS) {
    const int i = idx / n, j = idx - i * n;
    sP[idx] = to_work<T>((i <= j) ? I.Q[(size_t)N * nn + idx] : I.Q[(size_t)N * nn + j * n + i]);
  }
  if (SOLVE)
    for (int i = tid; i < n; i += THREADS) {
      sp[i] = to_work<T>(I.q[(size_t)N * n + i]);
      gpv[(size_t)N * n + i] = sp[i];
    }

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
  auto commit = [&]() {
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
  };
  prefetch(N - 1);
  commit();
  if (N > 1) prefetch(N - 2);
  __syncthreads();

  // State pivot elimination of P (in sP): [I + delta P | P] -> W into sW and
  // gWk; the certificate bit into shs.bit.  Ends with a barrier.
  auto state_pivot = [&](T *gWk) {
    if (tid == 0) {
      shs.bit = 1;
      shs.singular = 0;
    }
    if (gs.own && gs.c < w2) {
#pragma unroll
      for (int r = 0; r < gs.RPT; ++r) {
        const int i = gs.r0 + r;
        if (i < n) {
          const int cc = gs.c;
          gs.v[r] = (cc < n) ? (i == cc ? (T)1 : (T)0) + delta * sP[i * n + cc] : sP[i * n + (cc - n)];
        }
      }
    }
    bool shadow = false;
    if constexpr (FP32SWEEP) {
      // Gershgorin proof, with the certificate's margin, that I + delta P
      // is PD, in FP32 with directed rounding; otherwise the FP64 LDL^T of
      // I + delta P - tau D (D its diagonal) proves it, or the instance is
      // escalated to the FP64 recursion.
      int pass = 1;
      if (tid < n) {
        float off = 0.f;
        for (int j = 0; j < n; ++j)
          if (j != tid) off = __fadd_ru(off, fabsf(sP[tid * n + j]));
        pass = gershgorin_row_margin(sP[tid * n + tid], off, delta_dn, delta_up, kMarginTau);
      }
      __syncthreads();  // the flag reset by thread 0 precedes every later write
      gs.template publish0<DECIDE>(n, w2, shs);
      shadow = !__syncthreads_and(pass);
      if (shadow) {
        for (int idx = tid; idx < nn; idx += THREADS) {
          const int i = idx / n, j = idx - i * n;
          double v = (i == j ? 1.0 : 0.0) + I.delta * widen(sP[idx]);
          if (i == j) v -= (double)kMarginTau * fabs(v);
          sS64[idx] = v;
          if (idx == 0) rinv64[0] = 1.0 / v;
        }
        __syncthreads();
      }
    } else {
      __syncthreads();
      gs.template publish0<DECIDE>(n, w2, shs);
      __syncthreads();
    }
#pragma unroll(NM <= 16 ? NM : 1)
    for (int j = 0; j < NM; ++j) {
      if (j >= n) break;
      gs.template step<DECIDE>(j, n, w2, shs);
      if (FP32SWEEP && shadow) ldlt64_step<THREADS>(j, n, sS64, rinv64, &shs.bit, &shs.singular);
      if (j == n - 1 && gs.own && gs.c >= n && gs.c < w2) {
        // final right block: W[i][c - n] = v / D_i
#pragma unroll
        for (int r = 0; r < gs.RPT; ++r) {
          const int i = gs.r0 + r;
          if (i < n) {
            const T w = gs.v[r] * shs.rinv[i];
            sW[i * n + gs.c - n] = w;
            gWk[i * n + gs.c - n] = w;
          }
        }
      }
      __syncthreads();
    }
  };

  for (int k = N - 1; k >= 0; --k) {
    // ---- state pivot of stage k+1: W_{k+1}
    state_pivot(gW + (size_t)(k + 1) * nn);

    // ---- WA = W A, WB = W B, g = p + W (c_{k+1} - delta p)
    {
      const int tot = nn + nm + (SOLVE ? n : 0);
      for (int idx = tid; idx < tot; idx += THREADS) {
        if (idx < nn) {
          const int i = idx / n, j = idx - i * n;
          T s = 0;
#pragma unroll(NM <= 16 ? NM : 8)
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * sA[l * n + j];
          sWA[idx] = s;
        } else if (idx < nn + nm) {
          const int e = idx - nn, i = e / m, j = e - i * m;
          T s = 0;
#pragma unroll(NM <= 16 ? NM : 8)
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * sB[l * m + j];
          sWB[e] = s;
        } else {
          const int i = idx - nn - nm;
          T s = sp[i];
#pragma unroll(NM <= 16 ? NM : 8)
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sW[i * n + l] * (sc[l] - delta * sp[l]);
          sg[i] = s;
        }
      }
    }
    if (tid == 0) {
      shc.bit = 1;
      shc.singular = 0;
    }
    __syncthreads();

    // ---- [G | H | h | I] built directly into its owners' registers;
    //      P_k <- Q_k + A^T WA (lower triangle, mirrored), p_k <- q_k + A^T g
    if (gc.own && gc.c < wg) {
      const int j = gc.c;
#pragma unroll
      for (int r = 0; r < gc.RPT; ++r) {
        const int i = gc.r0 + r;
        if (i < m) {
          T s;
          if (j < m) {
            s = sR[i * m + j];
#pragma unroll(NM <= 16 ? NM : 8)
            for (int l = 0; l < NM; ++l)
              if (l < n) s += sB[l * m + i] * sWB[l * m + j];
            if (FP32SWEEP) gG[(size_t)k * mmm + i * m + j] = s;
          } else if (j < m + n) {
            const int jj = j - m;
            s = sM[jj * m + i];
#pragma unroll(NM <= 16 ? NM : 8)
            for (int l = 0; l < NM; ++l)
              if (l < n) s += sB[l * m + i] * sWA[l * n + jj];
            sH[i * n + jj] = s;
          } else if (j == m + n) {
            s = 0;
            if (SOLVE) {
              s = sr[i];
#pragma unroll(NM <= 16 ? NM : 8)
              for (int l = 0; l < NM; ++l)
                if (l < n) s += sB[l * m + i] * sg[l];
            }
          } else {
            s = ((j - m - n - 1) == i) ? (T)1 : (T)0;
          }
          gc.v[r] = s;
        }
      }
    }
    {
      const int nlo = n * (n + 1) / 2;
      for (int idx = tid; idx < nlo + (SOLVE ? n : 0); idx += THREADS) {
        if (idx < nlo) {
          int i, j;
          tri_decode(idx, i, j);
          T s = sQ[i * n + j];
#pragma unroll(NM <= 16 ? NM : 8)
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sA[l * n + i] * sWA[l * n + j];
          sP[i * n + j] = s;
          sP[j * n + i] = s;
        } else {
          const int i = idx - nlo;
          T s = sq[i];
#pragma unroll(NM <= 16 ? NM : 8)
          for (int l = 0; l < NM; ++l)
            if (l < n) s += sA[l * n + i] * sg[l];
          sp[i] = s;
        }
      }
    }
    gc.template publish0<DECIDE>(m, wg, shc);
    __syncthreads();

    // ---- control pivot elimination; K_k = -G^{-1} H, k_k = -G^{-1} h, G^{-1}
#pragma unroll(MM <= 16 ? MM : 1)
    for (int j = 0; j < MM; ++j) {
      if (j >= m) break;
      gc.template step<DECIDE>(j, m, wg, shc);
      if (j == m - 1 && gc.own && gc.c >= m && gc.c < wg) {
#pragma unroll
        for (int r = 0; r < gc.RPT; ++r) {
          const int i = gc.r0 + r;
          if (i < m) {
            const T x = gc.v[r] * shc.rinv[i];
            const int cc = gc.c;
            if (cc < m + n) {
              sK[i * n + cc - m] = -x;
              gK[(size_t)k * nm + i * n + cc - m] = -x;
            } else if (cc == m + n) {
              if (SOLVE) {
                skk[i] = -x;
                gkv[(size_t)k * m + i] = -x;
              }
            } else {
              gGi[(size_t)k * mmm + i * m + cc - m - n - 1] = x;
            }
          }
        }
      }
      __syncthreads();
    }

    // ---- P_k += H^T K_k (symmetric), p_k += H^T k_k; store p_k; flags;
    //      commit stage k-1's data and start fetching stage k-2
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
    if (k > 0) {
      commit();
      if (k > 1) prefetch(k - 2);
    }
    if (tid == 0) {
      // FP32 sweep: bit1 of stages < N is added by the FP64 control-pivot pass
      const int b1 = FP32SWEEP ? (k + 1 == N) : bit1_next;
      if (FP32SWEEP) {
        // the shifted FP64 LDL^T failed: no decision with margin
        if (!shs.bit || shs.singular) escal = true;
        I.flags[k + 1] = (uint8_t)(1 | (b1 << 1));
      } else {
        I.flags[k + 1] = (uint8_t)(shs.bit | (b1 << 1));
        if (!shs.bit || !b1) notpd = true;
        if (shs.singular || shc.singular) singular = true;
      }
      bit1_next = shc.bit;
    }
    __syncthreads();
  }

  // ---- initial-state pivot I + delta P_0: W_0 and bit0 of stage 0
  state_pivot(gW);
  if (tid == 0) {
    const int b1 = FP32SWEEP ? (N == 0) : bit1_next;
    if (FP32SWEEP) {
      if (!shs.bit || shs.singular) escal = true;
      I.flags[0] = (uint8_t)(1 | (b1 << 1));
    } else {
      I.flags[0] = (uint8_t)(shs.bit | (b1 << 1));
      if (!shs.bit || !b1) notpd = true;
      if (shs.singular) singular = true;
    }
    const int32_t st = singular ? RLQR_ERR_SINGULAR : (notpd ? RLQR_NOT_PD : RLQR_OK);
    I.st->pivot_status = st;
    I.st->escalated = escal ? 1 : 0;
    I.st->iters = 0;
    I.st->converged = 0;
    I.st->rel = 0.0;
    if (a.status) a.status[b] = st;
  }
  if (!SOLVE) return;

  // ---- forward rollout
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  for (int i = tid; i < n; i += THREADS) {
    sp[i] = __ldcg(gpv + i);
    sv[i] = to_work<T>(I.c[i]) - delta * sp[i];
  }
  __syncthreads();
  for (int i = tid; i < n; i += THREADS) {
    T t = 0;
#pragma unroll(NM <= 16 ? NM : 8)
    for (int l = 0; l < NM; ++l)
      if (l < n) t += sW[i * n + l] * sv[l];
    const T xv = sv[i] - delta * t, yv = t + sp[i];
    sx[i] = xv;
    I.x[i] = widen(xv);
    I.y[i] = widen(yv);
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
#pragma unroll(NM <= 16 ? NM : 8)
      for (int l = 0; l < NM; ++l)
        if (l < n) s += sK[i * n + l] * sx[l];
      su[i] = s;
      I.u[(size_t)k * m + i] = widen(s);
    }
    __syncthreads();
    // v = A x + B u + c_{k+1} - delta p_{k+1}
    for (int i = tid; i < n; i += THREADS) {
      T s = sc[i] - delta * sp[i];
#pragma unroll(NM <= 16 ? NM : 8)
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
#pragma unroll(NM <= 16 ? NM : 8)
      for (int l = 0; l < NM; ++l)
        if (l < n) t += sW[i * n + l] * sv[l];
      const T xv = sv[i] - delta * t, yv = t + sp[i];
      sx[i] = xv;
      I.x[(size_t)(k + 1) * n + i] = widen(xv);
      I.y[(size_t)(k + 1) * n + i] = widen(yv);
    }
    __syncthreads();
  }
}

}  // namespace rlqr

// seq_warp.cuh -- warp-per-instance sequential Riccati sweep for small
// dimensions (2 n <= 32 and 2 m + n + 1 <= 32), the shape of batched
// trajectory-optimization subproblems.
//
// Same recursion as seq.cuh (Theorem main-seq-theorem, eq. value-fn-formulas,
// Corollary p-recurrence, eq. recover-x0 / control-law / recover-x), organised
// for one warp:
//  * Gauss-Jordan on [I + delta P | P] and on [G | H | h | I]: lane c owns
//    column c in registers; the pivot column of each step is broadcast with
//    warp shuffles, so a step is n shuffles + n FMAs per lane and needs no
//    barrier at all.
//  * Every product of a stage is of the form out = init + X^T Y with X, Y
//    row-major in shared memory (W is symmetric, so W Y = W^T Y).  A lane
//    computes one full output column: per inner index l it loads the row
//    X[l, :] (vector loads, broadcast to all lanes) and one Y[l, c], then does
//    n FMAs.  All products of a phase share one instruction stream; only the
//    per-lane pointers differ, so lanes working on different products do
//    not diverge.
//  * Shared memory is per warp; phases are separated by __syncwarp only.
// A CTA holds WPC warps = WPC instances.  The certificate follows seq.cuh:
// FP64 sweep -> the Gauss-Jordan pivots; FP32 sweep -> FP64 Gershgorin proof
// for I + delta P (FP64 LDL^T fallback) and G_i stored for the FP64 pass.
#pragma once

#include "common.cuh"

namespace rlqr {

template <typename T, int NX, int NU>
struct WarpSmem {
  static constexpr int n = NX, m = NU, WG = 2 * NU + NX + 1, LG = NU + NX + 1;
  static constexpr int AL = 16 / sizeof(T) > 0 ? 16 / sizeof(T) : 1;  // vector width
  static constexpr int pad(int v) { return (v + AL - 1) / AL * AL; }
  // stage data (committed)
  alignas(16) T A[pad(n * n)];
  alignas(16) T Q[pad(n * n)];
  alignas(16) T B[pad(n * m)];
  alignas(16) T M[pad(n * m)];
  alignas(16) T R[pad(m * m)];
  alignas(16) T q[pad(n)];
  alignas(16) T c[pad(n)];
  alignas(16) T r[pad(m)];
  // value function and products
  alignas(16) T P[pad(n * n)];
  alignas(16) T p[pad(n)];
  alignas(16) T W[pad(n * n)];
  alignas(16) T WA[pad(n * n)];
  alignas(16) T WB[pad(n * m)];
  alignas(16) T g[pad(n)];
  alignas(16) T v[pad(n)];
  alignas(16) T Ga[pad(m * LG)];   // [G | H | h] row-major, row length LG
  alignas(16) T K[pad(m * n)];
  alignas(16) T kk[pad(m)];
  alignas(16) T x[pad(n)];
  alignas(16) T u[pad(m)];
  double S64[n * n];               // FP64 LDL^T of I + delta P (FP32-sweep fallback)
  double rinv64[n];
  // one row (padded length L) of X[l, :], vector-loaded
};

// out[:, col] (TR values, rows 0..TR-1) = sum_{l < L} X[l * ldx + i] * Y[l * ldy]
// X rows are vector-loaded (aligned when ldx and the base are multiples of
// the vector width).
template <typename T, int TR, int L, bool VEC>
__device__ __forceinline__ void xty_col(const T *X, int ldx, const T *Y, int ldy, T (&acc)[TR]) {
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const T y = Y[l * ldy];
    const T *xr = X + l * ldx;
    if (VEC && sizeof(T) == 4 && TR % 4 == 0) {
#pragma unroll
      for (int i = 0; i < TR; i += 4) {
        const float4 xv = *reinterpret_cast<const float4 *>(xr + i);
        acc[i] += (T)xv.x * y;
        acc[i + 1] += (T)xv.y * y;
        acc[i + 2] += (T)xv.z * y;
        acc[i + 3] += (T)xv.w * y;
      }
    } else if (VEC && sizeof(T) == 8 && TR % 2 == 0) {
#pragma unroll
      for (int i = 0; i < TR; i += 2) {
        const double2 xv = *reinterpret_cast<const double2 *>(xr + i);
        acc[i] += (T)xv.x * y;
        acc[i + 1] += (T)xv.y * y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < TR; ++i) acc[i] += xr[i] * y;
    }
  }
}

// Warp-level Gauss-Jordan step j on a matrix whose column `lane` lives in
// v[0..R-1]: every lane with lane > j eliminates column j from its rows i != j
// using the pivot column broadcast from lane j.  Returns the pivot d_j.
template <typename T, int R>
__device__ __forceinline__ T warp_gj_step(int j, int lane, bool active, T (&v)[R], T &rinv_j) {
  T colj[R];
#pragma unroll
  for (int i = 0; i < R; ++i) colj[i] = __shfl_sync(0xffffffffu, v[i], j);
  const T d = colj[j];
  rinv_j = recip_pivot(d);
  if (active && lane > j) {
    const T f = v[j] * rinv_j;
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (i != j) v[i] -= colj[i] * f;
  }
  return d;
}

template <typename T, int NX, int NU>
constexpr bool warp_fits() {
  return 2 * NX <= 32 && 2 * NU + NX + 1 <= 32;
}

// Sweep kernel, one warp per instance, WPC instances per CTA.
template <typename T, int NX, int NU, int WPC, bool SOLVE>
__global__ void __launch_bounds__(32 * WPC) k_seq_warp(BatchArgs a) {
  static_assert(warp_fits<T, NX, NU>(), "dimensions too large for one warp");
  constexpr bool FP32SWEEP = sizeof(T) == 4;
  constexpr int n = NX, m = NU, LG = NU + NX + 1, WG = 2 * NU + NX + 1;
  constexpr int nn = n * n, nm = n * m, mmm = m * m;
  constexpr int AL = WarpSmem<T, NX, NU>::AL;
  constexpr bool VN = (n % AL == 0);  // rows of length n are vector-aligned
  constexpr bool VM = (m % AL == 0);
  using SM = WarpSmem<T, NX, NU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = blockIdx.x * WPC + wid;
  if (slot >= a.count) return;  // whole warp exits together
  const int b = inst_of(a, slot);
  SM &s = reinterpret_cast<SM *>(smem_raw)[wid];
  const Inst I = get_inst(a, b);
  const int N = I.N;
  const T delta = (T)I.delta;
  const float delta_up = __double2float_ru(I.delta);  // Gershgorin test (FP32 sweep)
  T *gW = reinterpret_cast<T *>(I.ws + I.L.W);
  T *gK = reinterpret_cast<T *>(I.ws + I.L.K);
  T *gGi = reinterpret_cast<T *>(I.ws + I.L.Gi);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  T *gG = reinterpret_cast<T *>(I.ws + I.L.G);

  // prefetch registers for one stage's data (lane-strided)
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  constexpr int CV = (n + 31) / 32, CM = (m + 31) / 32;
  LaneSeg<double, CP> pfA, pfQ;
  LaneSeg<double, CB> pfB, pfM;
  LaneSeg<double, CR> pfR;
  LaneSeg<double, CV> pfq, pfc;
  LaneSeg<double, CM> pfr;
  auto prefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn, lane);
    pfQ.load(I.Q + (size_t)k * nn, nn, lane);
    pfB.load(I.B + (size_t)k * nm, nm, lane);
    pfM.load(I.M + (size_t)k * nm, nm, lane);
    pfR.load(I.R + (size_t)k * mmm, mmm, lane);
    if (SOLVE) {
      pfq.load(I.q + (size_t)k * n, n, lane);
      pfc.load(I.c + (size_t)(k + 1) * n, n, lane);
      pfr.load(I.r + (size_t)k * m, m, lane);
    }
  };
  auto commit = [&]() {
    pfA.store(s.A, nn, lane);
    pfQ.store_sym(s.Q, n, lane);
    pfB.store(s.B, nm, lane);
    pfM.store(s.M, nm, lane);
    pfR.store_sym(s.R, m, lane);
    if (SOLVE) {
      pfq.store(s.q, n, lane);
      pfc.store(s.c, n, lane);
      pfr.store(s.r, m, lane);
    }
  };

  // ---- terminal stage: P_N = Q_N (upper triangle), p_N = q_N
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, j = e - i * n;
    s.P[e] = to_work<T>((i <= j) ? I.Q[(size_t)N * nn + e] : I.Q[(size_t)N * nn + j * n + i]);
  }
  if (SOLVE)
    for (int i = lane; i < n; i += 32) {
      s.p[i] = to_work<T>(I.q[(size_t)N * n + i]);
      gpv[(size_t)N * n + i] = s.p[i];
    }
  prefetch(N - 1);
  commit();
  if (N > 1) prefetch(N - 2);
  __syncwarp();

  bool notpd = false, singular = false;
  int bit1_next = 1;
  T vs[n];          // column `lane` of [I + delta P | P]
  T rinv[n];        // reciprocals of its pivots (identical in every lane)

  // State pivot elimination of P (in s.P) -> W into s.W and gWk; returns the
  // certificate bit (and sets `sing` on a zero / non-finite pivot).
  auto state_pivot = [&](T *gWk, bool &sing) -> int {
    const bool act = lane < 2 * n;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      T val = 0;
      if (act) val = (lane < n) ? (i == lane ? (T)1 : (T)0) + delta * s.P[lane * n + i]
                                : s.P[(lane - n) * n + i];
      vs[i] = val;
    }
    int bit = 1;
    bool shadow = false;
    if constexpr (FP32SWEEP) {
      // Gershgorin proof that I + delta P is PD, in FP32 with directed
      // rounding; otherwise an FP64 LDL^T decides.
      bool pass = true;
      if (lane < n) {
        float off = 0.f;
#pragma unroll
        for (int j = 0; j < n; ++j)
          if (j != lane) off = __fadd_ru(off, fabsf(s.P[lane * n + j]));
        pass = gershgorin_row_pd(s.P[lane * n + lane], off, delta_up);
      }
      shadow = !__all_sync(0xffffffffu, pass);
      if (shadow) {
        for (int e = lane; e < nn; e += 32) {
          const int i = e / n, j = e - i * n;
          s.S64[e] = (i == j ? 1.0 : 0.0) + I.delta * widen(s.P[e]);
        }
        __syncwarp();
        for (int j = 0; j < n; ++j) {
          const double d = s.S64[j * n + j];
          if (!(d > 0.0)) bit = 0;
          if (!finite_nonzero(d)) sing = true;
          const double rd = 1.0 / d;
          const int r = n - j - 1;
          for (int idx = lane; idx < r * (r + 1) / 2; idx += 32) {
            int i, cc;
            tri_decode(idx, i, cc);
            i += j + 1;
            cc += j + 1;
            s.S64[i * n + cc] -= s.S64[i * n + j] * (s.S64[cc * n + j] * rd);
          }
          __syncwarp();
        }
      }
    }
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const T d = warp_gj_step<T, n>(j, lane, act, vs, rinv[j]);
      if (!FP32SWEEP) {
        if (!((double)d > 0.0)) bit = 0;
        if (!finite_nonzero((double)d)) sing = true;
      }
    }
    // W = right block scaled by 1 / D_i; lane n + cc holds column cc.  The
    // stored W is exactly symmetric: rows i >= cc of column cc, mirrored.
    if (lane >= n && lane < 2 * n) {
      const int cc = lane - n;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        if (i >= cc) {
          const T w = vs[i] * rinv[i];
          s.W[cc * n + i] = w;
          s.W[i * n + cc] = w;
          gWk[cc * n + i] = w;
          gWk[i * n + cc] = w;
        }
      }
    }
    __syncwarp();
    return bit;
  };

  for (int k = N - 1; k >= 0; --k) {
    bool sing = false;
    const int bit0 = state_pivot(gW + (size_t)(k + 1) * nn, sing);

    // ---- WA = W A (n columns), WB = W B (m columns), g = p + W (c - delta p)
    if (SOLVE && lane < n) s.v[lane] = s.c[lane] - delta * s.p[lane];
    __syncwarp();
    if (lane < n + m + (SOLVE ? 1 : 0)) {
      const T *Y;
      int ldy;
      T *out;
      if (lane < n) {
        Y = s.A + lane; ldy = n; out = s.WA;
      } else if (lane < n + m) {
        Y = s.B + (lane - n); ldy = m; out = s.WB;
      } else {
        Y = s.v; ldy = 1; out = s.g;
      }
      T acc[n];
#pragma unroll
      for (int i = 0; i < n; ++i) acc[i] = 0;
      xty_col<T, n, n, VN>(s.W, n, Y, ldy, acc);
      if (lane < n) {
#pragma unroll
        for (int i = 0; i < n; ++i) out[i * n + lane] = acc[i];
      } else if (lane < n + m) {
#pragma unroll
        for (int i = 0; i < n; ++i) out[i * m + lane - n] = acc[i];
      } else {
#pragma unroll
        for (int i = 0; i < n; ++i) out[i] = acc[i] + s.p[i];
      }
    }
    __syncwarp();

    // ---- G = R + B^T WB, H = M^T + B^T WA, h = r + B^T g (into Ga);
    //      P_k = Q + A^T WA, p_k = q + A^T g
    {
      // items: lanes 0..n-1 -> P column, n -> p, n+1..n+m -> G column,
      // n+m+1..2n+m -> H column, 2n+m+1 -> h
      const int L = lane;
      const bool act = L < 2 * n + m + 1 + (SOLVE ? 1 : 0);
      if (act) {
        // one instruction stream for every item: X = A (row length n) for the
        // P / p items, X = B (row length m) for the G / H / h items; with
        // X = B only acc[0..m-1] are used (the rest reads neighbouring
        // shared memory and is discarded)
        const bool xa = L <= n;
        const T *X = xa ? s.A : s.B;
        const int ldx = xa ? n : m;
        const T *Y;
        int ldy;
        if (L < n) {
          Y = s.WA + L; ldy = n;
        } else if (L == n || L > 2 * n + m) {
          Y = s.g; ldy = 1;
        } else if (L <= n + m) {
          Y = s.WB + (L - n - 1); ldy = m;
        } else {
          Y = s.WA + (L - n - m - 1); ldy = n;
        }
        T acc[n];
#pragma unroll
        for (int i = 0; i < n; ++i) acc[i] = 0;
        xty_col<T, n, n, VN && VM>(X, ldx, Y, ldy, acc);
        if (L < n) {
          // lower triangle of column L, mirrored: P stays exactly symmetric
#pragma unroll
          for (int i = 0; i < n; ++i)
            if (i >= L) {
              const T pv = acc[i] + s.Q[i * n + L];
              s.P[i * n + L] = pv;
              s.P[L * n + i] = pv;
            }
        } else if (L == n) {
          if (SOLVE) {
#pragma unroll
            for (int i = 0; i < n; ++i) s.p[i] = acc[i] + s.q[i];
          }
        } else if (L <= n + m) {
          const int cc = L - n - 1;
#pragma unroll
          for (int i = 0; i < m; ++i) {
            const T gv = acc[i] + s.R[i * m + cc];
            s.Ga[i * LG + cc] = gv;
            if (FP32SWEEP) gG[(size_t)k * mmm + i * m + cc] = gv;
          }
        } else if (L <= 2 * n + m) {
          const int cc = L - n - m - 1;
#pragma unroll
          for (int i = 0; i < m; ++i) s.Ga[i * LG + m + cc] = acc[i] + s.M[cc * m + i];
        } else {
#pragma unroll
          for (int i = 0; i < m; ++i) s.Ga[i * LG + m + n] = SOLVE ? acc[i] + s.r[i] : (T)0;
        }
      }
    }
    __syncwarp();

    // ---- control pivot: Gauss-Jordan on [G | H | h | I], lane = column
    int bit1 = 1;
    {
      T vc[m];
      const bool act = lane < WG;
#pragma unroll
      for (int i = 0; i < m; ++i) {
        T val = 0;
        if (act) val = (lane < LG) ? s.Ga[i * LG + lane] : (lane - LG == i ? (T)1 : (T)0);
        vc[i] = val;
      }
      T ginv[m];
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const T d = warp_gj_step<T, m>(j, lane, act, vc, ginv[j]);
        if (!FP32SWEEP) {
          if (!((double)d > 0.0)) bit1 = 0;
          if (!finite_nonzero((double)d)) sing = true;
        }
      }
      if (lane >= m && lane < WG) {
#pragma unroll
        for (int i = 0; i < m; ++i) {
          const T xv = vc[i] * ginv[i];
          if (lane < m + n) {
            s.K[i * n + lane - m] = -xv;
            gK[(size_t)k * nm + i * n + lane - m] = -xv;
          } else if (lane == m + n) {
            s.kk[i] = -xv;
            if (SOLVE) gkv[(size_t)k * m + i] = -xv;
          } else {
            gGi[(size_t)k * mmm + i * m + lane - m - n - 1] = xv;
          }
        }
      }
    }
    __syncwarp();

    // ---- P_k += H^T K (column per lane), p_k += H^T k; commit stage k-1
    if (lane < n + (SOLVE ? 1 : 0)) {
      T acc[n];
#pragma unroll
      for (int i = 0; i < n; ++i) acc[i] = 0;
      const T *Y = (lane < n) ? s.K + lane : s.kk;
      const int ldy = (lane < n) ? n : 1;
      // X = H with row l = Ga[l, m .. m+n-1] (row stride LG)
      xty_col<T, n, m, false>(s.Ga + m, LG, Y, ldy, acc);
      if (lane < n) {
#pragma unroll
        for (int i = 0; i < n; ++i)
          if (i >= lane) {
            const T pv = s.P[i * n + lane] + acc[i];
            s.P[i * n + lane] = pv;
            s.P[lane * n + i] = pv;
          }
      } else {
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const T pv = s.p[i] + acc[i];
          s.p[i] = pv;
          gpv[(size_t)k * n + i] = pv;
        }
      }
    }
    if (k > 0) {
      commit();
      if (k > 1) prefetch(k - 2);
    }
    if (lane == 0) {
      const int b1 = FP32SWEEP ? (k + 1 == N) : bit1_next;
      I.flags[k + 1] = (uint8_t)(bit0 | (b1 << 1));
      if (!bit0 || (!FP32SWEEP && !b1)) notpd = true;
    }
    if (sing) singular = true;
    bit1_next = bit1;
    __syncwarp();
  }

  // ---- initial-state pivot
  {
    bool sing = false;
    const int bit0 = state_pivot(gW, sing);
    if (sing) singular = true;
    if (lane == 0) {
      const int b1 = FP32SWEEP ? 0 : bit1_next;
      I.flags[0] = (uint8_t)(bit0 | (b1 << 1));
      if (!bit0 || (!FP32SWEEP && !b1)) notpd = true;
      const int32_t st = singular ? RLQR_ERR_SINGULAR : (notpd ? RLQR_NOT_PD : RLQR_OK);
      I.st->pivot_status = st;
      I.st->iters = 0;
      I.st->converged = 0;
      I.st->rel = 0.0;
      if (a.status) a.status[b] = st;
    }
  }
  if (!SOLVE) return;

  // ---- forward rollout (lane = row)
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  if (lane < n) {
    s.p[lane] = __ldcg(gpv + lane);
    s.v[lane] = to_work<T>(I.c[lane]) - delta * s.p[lane];
  }
  __syncwarp();
  if (lane < n) {
    T t = 0;
#pragma unroll
    for (int l = 0; l < n; ++l) t += s.W[lane * n + l] * s.v[l];
    const T xv = s.v[lane] - delta * t, yv = t + s.p[lane];
    s.x[lane] = xv;
    I.x[lane] = widen(xv);
    I.y[lane] = widen(yv);
  }
  LaneSeg<T, CP> fW;
  LaneSeg<T, CB> fK;
  LaneSeg<T, CM> fk;
  LaneSeg<T, CV> fp;
  auto fprefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn, lane);
    pfB.load(I.B + (size_t)k * nm, nm, lane);
    pfc.load(I.c + (size_t)(k + 1) * n, n, lane);
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    fK.load_cg(gK + (size_t)k * nm, nm, lane);
    fk.load_cg(gkv + (size_t)k * m, m, lane);
    fp.load_cg(gpv + (size_t)(k + 1) * n, n, lane);
  };
  __syncwarp();
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
    pfA.store(s.A, nn, lane);
    pfB.store(s.B, nm, lane);
    pfc.store(s.c, n, lane);
    fW.store(s.W, nn, lane);
    fK.store(s.K, nm, lane);
    fk.store(s.kk, m, lane);
    fp.store(s.p, n, lane);
    if (k + 1 < N) fprefetch(k + 1);
    __syncwarp();
    if (lane < m) {
      T t = s.kk[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.K[lane * n + l] * s.x[l];
      s.u[lane] = t;
      I.u[(size_t)k * m + lane] = widen(t);
    }
    __syncwarp();
    if (lane < n) {
      T t = s.c[lane] - delta * s.p[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.A[lane * n + l] * s.x[l];
#pragma unroll
      for (int l = 0; l < m; ++l) t += s.B[lane * m + l] * s.u[l];
      s.v[lane] = t;
    }
    __syncwarp();
    if (lane < n) {
      T t = 0;
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.W[lane * n + l] * s.v[l];
      const T xv = s.v[lane] - delta * t, yv = t + s.p[lane];
      s.x[lane] = xv;
      I.x[(size_t)(k + 1) * n + lane] = widen(xv);
      I.y[(size_t)(k + 1) * n + lane] = widen(yv);
    }
    __syncwarp();
  }
}

}  // namespace rlqr

namespace rlqr {

// Right-hand-side solve with a stored factor, one warp per instance (lane =
// row); same arithmetic as k_solve in refine.cuh: the p-recurrence of
// Corollary p-recurrence backward, the forward rollout, and with FROM_RES the
// FP64 update of z and of the residual (res += K dz, FP32 products).
template <typename T, int NX, int NU, int WPC, bool FROM_RES>
__global__ void __launch_bounds__(32 * WPC) k_solve_warp(BatchArgs a) {
  static_assert(warp_fits<T, NX, NU>(), "dimensions too large for one warp");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  using SM = WarpSmem<T, NX, NU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = blockIdx.x * WPC + wid;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  SM &s = reinterpret_cast<SM *>(smem_raw)[wid];
  // FP64 staging of the iterate and residual rows of a stage (after the
  // T-typed arrays of the warp's block)
  __shared__ double zbuf[WPC][6][32];
  double *zx = zbuf[wid][0], *zy = zbuf[wid][1], *zq = zbuf[wid][2], *zc = zbuf[wid][3];
  double *zu = zbuf[wid][4], *zr = zbuf[wid][5];
  const Inst I = get_inst(a, b);
  InstState *stp = I.st;
  if (FROM_RES) {
    if (stp->converged || stp->pivot_status == RLQR_ERR_SINGULAR) return;
  } else if (lane == 0) {
    stp->iters = 0;
    stp->converged = 0;
  }
  const int N = I.N;
  const T delta = (T)I.delta;
  const double delta64 = I.delta;
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
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  constexpr int CV = (n + 31) / 32, CM = (m + 31) / 32;
  T *sGi = s.R;  // G^{-1} of the stage (the R slot is free in this kernel)

  // ---------------- backward: p-recurrence
  if (lane < n) {
    const T v = to_work<T>(__ldcg(Rq + (size_t)N * n + lane));
    s.p[lane] = v;
    gpv[(size_t)N * n + lane] = v;
  }
  LaneSeg<T, CP> bW;
  LaneSeg<double, CP> bA;
  LaneSeg<double, CB> bB;
  LaneSeg<T, CB> bK;
  LaneSeg<T, CR> bG;
  LaneSeg<double, CV> bq, bc;
  LaneSeg<double, CM> br;
  auto bprefetch = [&](int k) {
    bW.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    bA.load(I.A + (size_t)k * nn, nn, lane);
    bB.load(I.B + (size_t)k * nm, nm, lane);
    bK.load_cg(gK + (size_t)k * nm, nm, lane);
    bG.load_cg(gGi + (size_t)k * mmm, mmm, lane);
    bq.load_cg(Rq + (size_t)k * n, n, lane);
    bc.load_cg(Rc + (size_t)(k + 1) * n, n, lane);
    br.load_cg(Rr + (size_t)k * m, m, lane);
  };
  bprefetch(N - 1);
  __syncwarp();
  for (int k = N - 1; k >= 0; --k) {
    bW.store(s.W, nn, lane);
    bA.store(s.A, nn, lane);
    bB.store(s.B, nm, lane);
    bK.store(s.K, nm, lane);
    bG.store(sGi, mmm, lane);
    bq.store(s.q, n, lane);
    bc.store(s.c, n, lane);
    br.store(s.r, m, lane);
    if (k > 0) bprefetch(k - 1);
    __syncwarp();
    // g = p + W (c' - delta p)
    if (lane < n) {
      T t = s.p[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.W[lane * n + l] * (s.c[l] - delta * s.p[l]);
      s.g[lane] = t;
    }
    __syncwarp();
    // h = r' + B^T g
    if (lane < m) {
      T t = s.r[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.B[l * m + lane] * s.g[l];
      s.u[lane] = t;
    }
    __syncwarp();
    // p_k = q' + A^T g + K^T h ; k_k = -G^{-1} h
    if (lane < n) {
      T t = s.q[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.A[l * n + lane] * s.g[l];
#pragma unroll
      for (int l = 0; l < m; ++l) t += s.K[l * n + lane] * s.u[l];
      s.p[lane] = t;
      gpv[(size_t)k * n + lane] = t;
    } else if (lane < n + m) {
      const int i = lane - n;
      T t = 0;
#pragma unroll
      for (int l = 0; l < m; ++l) t += sGi[i * m + l] * s.u[l];
      gkv[(size_t)k * m + i] = -t;
    }
    __syncwarp();
  }

  // ---------------- forward rollout (+ z update and residual update)
  unsigned long long rbits = 0, zbits = 0;
  T *dx = s.x, *du = s.u, *dy = s.v;  // dx_k, du_k, dy_k
  T *dxn = s.g, *dyn = s.WA;          // dx_{k+1}, dy_{k+1}
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0, v0 = c'_0 - delta p_0
  for (int e = lane; e < nn; e += 32) s.W[e] = __ldcg(gW + e);
  if (lane < n) s.c[lane] = to_work<T>(__ldcg(Rc + lane)) - delta * s.p[lane];
  __syncwarp();
  if (lane < n) {
    T t = 0;
#pragma unroll
    for (int l = 0; l < n; ++l) t += s.W[lane * n + l] * s.c[l];
    const T dxv = s.c[lane] - delta * t, dyv = t + s.p[lane];
    dx[lane] = dxv;
    dy[lane] = dyv;
    if (FROM_RES) {
      const double xv = I.x[lane] + widen(dxv), yv = I.y[lane] + widen(dyv);
      I.x[lane] = xv;
      I.y[lane] = yv;
      zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
      const double r0 = __ldcg(rc + lane) - widen(dxv) - delta64 * widen(dyv);
      rc[lane] = r0;
      rbits = max(rbits, abs_bits(r0));
    } else {
      I.x[lane] = widen(dxv);
      I.y[lane] = widen(dyv);
    }
  }
  LaneSeg<T, CP> fW;
  LaneSeg<double, CP> fA, fQ;
  LaneSeg<double, CB> fB, fM;
  LaneSeg<T, CB> fK;
  LaneSeg<double, CR> fR;
  LaneSeg<T, CM> fk;
  LaneSeg<T, CV> fp;
  LaneSeg<double, CV> fc;
  double zv[6];
  auto fprefetch = [&](int k) {
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    fA.load(I.A + (size_t)k * nn, nn, lane);
    fB.load(I.B + (size_t)k * nm, nm, lane);
    fK.load_cg(gK + (size_t)k * nm, nm, lane);
    fk.load_cg(gkv + (size_t)k * m, m, lane);
    fp.load_cg(gpv + (size_t)(k + 1) * n, n, lane);
    fc.load_cg(Rc + (size_t)(k + 1) * n, n, lane);
    if (FROM_RES) {
      fQ.load(I.Q + (size_t)k * nn, nn, lane);
      fM.load(I.M + (size_t)k * nm, nm, lane);
      fR.load(I.R + (size_t)k * mmm, mmm, lane);
      zv[0] = lane < n ? __ldcg(I.x + (size_t)(k + 1) * n + lane) : 0.0;
      zv[1] = lane < n ? __ldcg(I.y + (size_t)(k + 1) * n + lane) : 0.0;
      zv[2] = lane < n ? __ldcg(rq + (size_t)k * n + lane) : 0.0;
      zv[3] = lane < n ? __ldcg(rc + (size_t)(k + 1) * n + lane) : 0.0;
      zv[4] = lane < m ? __ldcg(I.u + (size_t)k * m + lane) : 0.0;
      zv[5] = lane < m ? __ldcg(rr + (size_t)k * m + lane) : 0.0;
    }
  };
  __syncwarp();
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
    fW.store(s.W, nn, lane);
    fA.store(s.A, nn, lane);
    fB.store(s.B, nm, lane);
    fK.store(s.K, nm, lane);
    fk.store(s.kk, m, lane);
    fp.store(s.p, n, lane);
    fc.store(s.c, n, lane);
    if (FROM_RES) {
      fQ.store_sym(s.Q, n, lane);
      fM.store(s.M, nm, lane);
      fR.store_sym(s.R, m, lane);
      zx[lane] = zv[0];
      zy[lane] = zv[1];
      zq[lane] = zv[2];
      zc[lane] = zv[3];
      zu[lane] = zv[4];
      zr[lane] = zv[5];
    }
    if (k + 1 < N) fprefetch(k + 1);
    __syncwarp();
    // du_k = K_k dx_k + k_k
    if (lane < m) {
      T t = s.kk[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.K[lane * n + l] * dx[l];
      du[lane] = t;
      if (FROM_RES) {
        const double uv = zu[lane] + widen(t);
        I.u[(size_t)k * m + lane] = uv;
        zbits = max(zbits, abs_bits(uv));
      } else {
        I.u[(size_t)k * m + lane] = widen(t);
      }
    }
    __syncwarp();
    // w = A dx + B du + c'_{k+1} - delta p_{k+1}   (into s.WB: n slots)
    T *w = s.WB;
    if (lane < n) {
      T t = s.c[lane] - delta * s.p[lane];
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.A[lane * n + l] * dx[l];
#pragma unroll
      for (int l = 0; l < m; ++l) t += s.B[lane * m + l] * du[l];
      w[lane] = t;
    }
    __syncwarp();
    // dx_{k+1} = w - delta W w, dy_{k+1} = W w + p_{k+1}
    if (lane < n) {
      T t = 0;
#pragma unroll
      for (int l = 0; l < n; ++l) t += s.W[lane * n + l] * w[l];
      const T dxv = w[lane] - delta * t, dyv = t + s.p[lane];
      dxn[lane] = dxv;
      dyn[lane] = dyv;
      const size_t o = (size_t)(k + 1) * n + lane;
      if (FROM_RES) {
        const double xv = zx[lane] + widen(dxv), yv = zy[lane] + widen(dyv);
        I.x[o] = xv;
        I.y[o] = yv;
        zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
      } else {
        I.x[o] = widen(dxv);
        I.y[o] = widen(dyv);
      }
    }
    __syncwarp();
    if (FROM_RES) {
      // res += K dz for the rows of stage k (x_k, u_k) and of c_{k+1}
      if (lane < 2 * n + m) {
        T t = 0;
        double old, *dst;
        if (lane < n) {
#pragma unroll
          for (int l = 0; l < n; ++l) t += s.Q[lane * n + l] * dx[l] + s.A[l * n + lane] * dyn[l];
#pragma unroll
          for (int l = 0; l < m; ++l) t += s.M[lane * m + l] * du[l];
          t -= dy[lane];
          old = zq[lane];
          dst = rq + (size_t)k * n + lane;
        } else if (lane < n + m) {
          const int j = lane - n;
#pragma unroll
          for (int l = 0; l < n; ++l) t += s.M[l * m + j] * dx[l] + s.B[l * m + j] * dyn[l];
#pragma unroll
          for (int l = 0; l < m; ++l) t += s.R[j * m + l] * du[l];
          old = zr[j];
          dst = rr + (size_t)k * m + j;
        } else {
          const int j = lane - n - m;
#pragma unroll
          for (int l = 0; l < n; ++l) t += s.A[j * n + l] * dx[l];
#pragma unroll
          for (int l = 0; l < m; ++l) t += s.B[j * m + l] * du[l];
          t -= dxn[j] + delta * dyn[j];
          old = zc[j];
          dst = rc + (size_t)(k + 1) * n + j;
        }
        const double nv = old + widen(t);
        *dst = nv;
        rbits = max(rbits, abs_bits(nv));
      }
      __syncwarp();
    }
    T *t1 = dx; dx = dxn; dxn = t1;
    T *t2 = dy; dy = dyn; dyn = t2;
  }
  if (!FROM_RES) return;
  // terminal rows x_N: res += Q_N dx_N - dy_N
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, j = e - i * n;
    if (i <= j) {
      const T v = to_work<T>(__ldg(I.Q + (size_t)N * nn + e));
      s.Q[i * n + j] = v;
      s.Q[j * n + i] = v;
    }
  }
  __syncwarp();
  if (lane < n) {
    T t = -dy[lane];
#pragma unroll
    for (int l = 0; l < n; ++l) t += s.Q[lane * n + l] * dx[l];
    double *dst = rq + (size_t)N * n + lane;
    const double nv = __ldcg(dst) + widen(t);
    *dst = nv;
    rbits = max(rbits, abs_bits(nv));
  }
  // warp max of the bit patterns
  for (int o = 16; o > 0; o >>= 1) {
    rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
    zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
  }
  if (lane == 0) {
    const double rmax = bits_to_double(rbits), zmax = bits_to_double(zbits);
    const double den = stp->kmax * zmax + stp->bmax;
    const double rel = den > 0.0 ? rmax / den : rmax;
    stp->rmax = rmax;
    stp->zmax = zmax;
    stp->rel = rel;
    stp->iters += 1;
    const int32_t conv = (rel <= a.tol) ? 1 : 0;
    stp->converged = conv;
    if (a.rel) a.rel[b] = rel;
    if (a.iters) a.iters[b] = stp->iters;
    if (a.status) {
      const int32_t ps = stp->pivot_status;
      a.status[b] = (ps == RLQR_ERR_SINGULAR) ? RLQR_ERR_SINGULAR
                                              : (conv ? ps : RLQR_ERR_NOT_CONVERGED);
    }
  }
}

}  // namespace rlqr

// scan_vec.cuh -- vector passes of the associative-scan path (rows a8 / a9
// of the path: the p-recurrence and the forward affine maps), one warp per
// chunk, lane = row (n <= 32), and the residual kernels of a long horizon.
//
// p (Corollary p-recurrence): p_i = F_i p_{i+1} + f_i.  Per chunk c with stages
// [s, e): p_s = Phi_c p_e + phi_c (Phi_c from k_scan_finalize).
//   k_scan_pvec<MODE 0>  phi_c: the recursion over the chunk from p_e = 0;
//   k_scan_pbound        p at every chunk start, from p_N = q_N backwards:
//                        pb[c] = Phi_c pb[c+1] + phi_c (one warp, C steps);
//   k_scan_pvec<MODE 1>  from p_e = pb[c+1]: p_i and k_i of the chunk.
// x (eq. recover-x0 / control-law / recover-x, Section "Composing Affine
// Functions"): x_{i+1} = E_i x_i + e_i with E_i = F_i^T, so x_e = Phi_c^T x_s + psi_c.
//   k_scan_xvec<MODE 0>  psi_c: the forward recursion over the chunk from x_s = 0;
//   k_scan_xbound        x_0, y_0, then xb[c+1] = Phi_c^T xb[c] + psi_c;
//   k_scan_xvec<MODE 1>  from x_s = xb[c]: x, u, y of the chunk.
// FROM_RES (refinement): the right-hand side is the FP64 residual; MODE 1 of
// the x pass adds dz to z in FP64 and updates the residual rows of the
// chunk's stages with K dz (see refine.cuh).  The x rows of a chunk's first
// stage need dy_s, computed in the chunk as P_s dx_s + dp_s (y = P x + p,
// Theorem main-seq-theorem) from the chunk's finalized P_s, so that no
// residual entry is written by two chunks.
#pragma once

#include "common.cuh"
#include "scan.cuh"

namespace rlqr {
namespace scan {

// Data element: the FP32 copy in the mixed path, the FP64 array otherwise.
template <typename T>
__device__ __forceinline__ T data_at(const double *g64, const float *g32, size_t idx) {
  if constexpr (sizeof(T) == 4) {
    return __ldcg(g32 + idx);
  } else {
    return __ldg(g64 + idx);
  }
}

template <typename T, int NX, int NU>
struct VecSmem {
  alignas(16) T W[NX * NX];
  alignas(16) T A[NX * NX];
  alignas(16) T B[NX * NU];
  alignas(16) T K[NU * NX];
  alignas(16) T G[NU * NU];
  alignas(16) T Q[NX * NX];
  alignas(16) T M[NX * NU];
  alignas(16) T R[NU * NU];
  alignas(16) T p[NX];
  alignas(16) T pn[NX];
  alignas(16) T g[NX];
  alignas(16) T h[NU];
  alignas(16) T v[NX];
  alignas(16) T x[NX];
  alignas(16) T u[NU];
  alignas(16) T dy[NX];
  alignas(16) T dyn[NX];
  alignas(16) T dxn[NX];
};

// The data array the vector passes read: the FP32 copy (mixed) or FP64 array.
template <typename T>
__device__ __forceinline__ const T *data_ptr(const double *g64, const float *g32) {
  if constexpr (sizeof(T) == 4) {
    return g32;
  } else {
    return g64;
  }
}

// sum_l a[l] b[l] over contiguous rows (two accumulators)
template <typename T, int L>
__device__ __forceinline__ T dotc(const T *a, const T *b) {
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int l = 0; l + 1 < L; l += 2) {
    s0 = fma(a[l], b[l], s0);
    s1 = fma(a[l + 1], b[l + 1], s1);
  }
  if (L & 1) s0 = fma(a[L - 1], b[L - 1], s0);
  return s0 + s1;
}

// sum_l a[l * stride] b[l] (a column of a row-major matrix; two accumulators)
template <typename T, int L>
__device__ __forceinline__ T dots(const T *a, int stride, const T *b) {
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int l = 0; l + 1 < L; l += 2) {
    s0 = fma(a[l * stride], b[l], s0);
    s1 = fma(a[(l + 1) * stride], b[l + 1], s1);
  }
  if (L & 1) s0 = fma(a[(L - 1) * stride], b[L - 1], s0);
  return s0 + s1;
}

}  // namespace scan

// Right-hand side entries (q', r', c') as T: the problem's or the residual.
struct ScanRhs {
  const double *q, *r, *c;
};

__device__ __forceinline__ ScanRhs scan_rhs(const Inst &I, bool from_res) {
  ScanRhs R;
  if (from_res) {
    const double *rq = reinterpret_cast<const double *>(I.ws + I.L.res);
    R.q = rq;
    R.r = rq + (size_t)(I.N + 1) * I.n;
    R.c = R.r + (size_t)I.N * I.m;
  } else {
    R.q = I.q;
    R.r = I.r;
    R.c = I.c;
  }
  return R;
}

// Backward p recursion over chunk c.  MODE 0: from p_e = 0, writes phi_c.
// MODE 1: from p_e = pb[c+1], writes p_i (i in [s, e)) and k_i.  The next
// stage's matrices are prefetched into registers while a stage computes.
template <typename T, int NX, int NU, int MODE, bool FROM_RES>
__global__ void __launch_bounds__(32) k_scan_pvec(BatchArgs a, ScanLayout SL, size_t sbase) {
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  using SM = scan::VecSmem<T, NX, NU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int lane = threadIdx.x, c = blockIdx.x;
  const int lm = lane < m ? lane : 0;  // row of the m-row rounds (0 past m)
  const Inst I = get_inst(a, 0);
  if (FROM_RES && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) return;
  const int N = I.N, s0 = c * SL.L, e0 = min(s0 + SL.L, N);
  const T delta = (T)I.delta;
  const ScanRhs rhs = scan_rhs(I, FROM_RES);
  const T *gW = reinterpret_cast<const T *>(I.ws + I.L.W);
  const T *gK = reinterpret_cast<const T *>(I.ws + I.L.K);
  const T *gGi = reinterpret_cast<const T *>(I.ws + I.L.Gi);
  const T *dA = scan::data_ptr<T>(I.A, reinterpret_cast<const float *>(I.ws + I.L.Af));
  const T *dB = scan::data_ptr<T>(I.B, reinterpret_cast<const float *>(I.ws + I.L.Bf));
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *pb = reinterpret_cast<T *>(I.ws + sbase + SL.pb);
  T *phi = reinterpret_cast<T *>(I.ws + sbase + SL.phi);
  LaneSeg<T, CP> fW, fA;
  LaneSeg<T, CB> fB, fK;
  LaneSeg<T, CR> fG;
  double vc = 0.0, vr = 0.0, vq = 0.0;
  auto prefetch = [&](int i) {
    fW.load(gW + (size_t)(i + 1) * nn, nn, lane);
    fA.load(dA + (size_t)i * nn, nn, lane);
    fB.load(dB + (size_t)i * nm, nm, lane);
    fK.load(gK + (size_t)i * nm, nm, lane);
    if (MODE == 1) fG.load(gGi + (size_t)i * mmm, mmm, lane);
    if (lane < n) {
      vc = __ldg(rhs.c + (size_t)(i + 1) * n + lane);
      vq = __ldg(rhs.q + (size_t)i * n + lane);
    }
    if (lane < m) vr = __ldg(rhs.r + (size_t)i * m + lane);
  };
  if (lane < n) s.p[lane] = (MODE == 0) ? (T)0 : pb[(size_t)(c + 1) * n + lane];
  prefetch(e0 - 1);
  for (int i = e0 - 1; i >= s0; --i) {
    __syncwarp();
    fW.store(s.W, nn, lane);
    fA.store(s.A, nn, lane);
    fB.store(s.B, nm, lane);
    fK.store(s.K, nm, lane);
    if (MODE == 1) fG.store(s.G, mmm, lane);
    const T cq = to_work<T>(vq), cr = to_work<T>(vr);
    if (lane < n) s.v[lane] = to_work<T>(vc) - delta * s.p[lane];
    if (i > s0) prefetch(i - 1);
    __syncwarp();
    // g = p + W (c' - delta p)
    if (lane < n) s.g[lane] = s.p[lane] + scan::dotc<T, NX>(s.W + lane * n, s.v);
    __syncwarp();
    // h = r' + B^T g (every lane on a clamped column; lanes < m store)
    {
      const T hv = cr + scan::dots<T, NX>(s.B + lm, m, s.g);
      if (lane < m) s.h[lane] = hv;
    }
    __syncwarp();
    // p_i = q' + A^T g + K^T h;  k_i = -G^{-1} h
    T pnew = 0;
    if (lane < n) {
      pnew = cq + scan::dots<T, NX>(s.A + lane, n, s.g) + scan::dots<T, NU>(s.K + lane, n, s.h);
      if (MODE == 1) gpv[(size_t)i * n + lane] = pnew;
    }
    if (MODE == 1) {
      const T kv = -scan::dotc<T, NU>(s.G + lm * m, s.h);
      if (lane < m) gkv[(size_t)i * m + lane] = kv;
    }
    __syncwarp();
    if (lane < n) s.p[lane] = pnew;
  }
  if (MODE == 0 && lane < n) phi[(size_t)c * n + lane] = s.p[lane];
}

// Depth of the register rings of the boundary passes (chunks in flight).
template <typename T>
__host__ __device__ constexpr int bound_ring_depth() {
  return sizeof(T) == 4 ? 4 : 2;
}

// dst[0..NX) = src[0..NX) (one row, __ldcg), in 16- or 8-byte pieces when the
// row's size and the address allow.
template <typename T, int NX>
__device__ __forceinline__ void ld_vec_row(const T *src, T (&dst)[NX]) {
  constexpr int BYTES = NX * (int)sizeof(T);
  const uintptr_t ad = reinterpret_cast<uintptr_t>(src);
  if constexpr (BYTES % 16 == 0) {
    if (ad % 16 == 0) {
      constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
      for (int q = 0; q < NX / V; ++q) {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(src) + q);
        const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int e = 0; e < V; ++e) dst[q * V + e] = pv[e];
      }
      return;
    }
  }
  if constexpr (BYTES % 8 == 0 && sizeof(T) == 4) {
    if (ad % 8 == 0) {
#pragma unroll
      for (int q = 0; q < NX / 2; ++q) {
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(src) + q);
        dst[2 * q] = v.x;
        dst[2 * q + 1] = v.y;
      }
      return;
    }
  }
#pragma unroll
  for (int l = 0; l < NX; ++l) dst[l] = __ldcg(src + l);
}

// p at the chunk starts: pb[C] = q'_N, pb[c] = Phi_c pb[c+1] + phi_c.  One warp.
template <typename T, int NX, bool FROM_RES>
__global__ void __launch_bounds__(32) k_scan_pbound(BatchArgs a, ScanLayout SL, size_t sbase) {
  constexpr int n = NX, nn = n * n;
  __shared__ T pv[NX];
  const int lane = threadIdx.x;
  const Inst I = get_inst(a, 0);
  if (FROM_RES && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) return;
  const ScanRhs rhs = scan_rhs(I, FROM_RES);
  const T *Phi = reinterpret_cast<const T *>(I.ws + sbase + SL.Phi);
  const T *phi = reinterpret_cast<const T *>(I.ws + sbase + SL.phi);
  T *pb = reinterpret_cast<T *>(I.ws + sbase + SL.pb);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  const int C = SL.C;
  if (lane < n) {
    const T q = to_work<T>(__ldcg(rhs.q + (size_t)I.N * n + lane));
    pv[lane] = q;
    pb[(size_t)C * n + lane] = q;
    gpv[(size_t)I.N * n + lane] = q;
  }
  // row `lane` of Phi_c and phi_c[lane] in a register ring D chunks deep:
  // the chain over the chunks is one n-term dot product per chunk, far
  // shorter than a load, so D chunks are in flight
  constexpr int D = bound_ring_depth<T>();
  T row[D][NX], off[D];
  auto fetch = [&](int j, int cc) {
    if (cc >= 0 && lane < n) {
      ld_vec_row<T, NX>(Phi + (size_t)cc * nn + lane * n, row[j]);
      off[j] = __ldcg(phi + (size_t)cc * n + lane);
    }
  };
#pragma unroll
  for (int j = 0; j < D; ++j) fetch(j, C - 1 - j);
  for (int c0 = C - 1; c0 >= 0; c0 -= D) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int c = c0 - j;
      if (c < 0) break;  // uniform over the warp
      __syncwarp();
      T t = 0;
      if (lane < n) {
        t = off[j];
#pragma unroll
        for (int l = 0; l < NX; ++l) t = fma(row[j][l], pv[l], t);
      }
      __syncwarp();
      if (lane < n) {
        pv[lane] = t;
        pb[(size_t)c * n + lane] = t;
      }
      fetch(j, c - D);
    }
  }
}

// Forward pass over chunk c.  MODE 0: from x_s = 0, writes psi_c = x_e.
// MODE 1: from x_s = xb[c], writes x_{i+1}, u_i, y_{i+1} (FP64); FROM_RES adds
// them to z and updates the residual rows of the chunk's stages.  The next
// stage's operands are prefetched into registers.
template <typename T, int NX, int NU, int MODE, bool FROM_RES>
__global__ void __launch_bounds__(32) k_scan_xvec(BatchArgs a, ScanLayout SL, size_t sbase,
                                                  int sfin1) {
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  constexpr bool RES = FROM_RES && MODE == 1;
  using SM = scan::VecSmem<T, NX, NU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int lane = threadIdx.x, c = blockIdx.x;
  const int lm = lane < m ? lane : 0;  // row of the m-row rounds (0 past m)
  const Inst I = get_inst(a, 0);
  if (FROM_RES && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) return;
  const int N = I.N, s0 = c * SL.L, e0 = min(s0 + SL.L, N);
  const T delta = (T)I.delta;
  const ScanRhs rhs = scan_rhs(I, FROM_RES);
  const T *gW = reinterpret_cast<const T *>(I.ws + I.L.W);
  const T *gK = reinterpret_cast<const T *>(I.ws + I.L.K);
  const T *gkv = reinterpret_cast<const T *>(I.ws + I.L.kv);
  const T *gpv = reinterpret_cast<const T *>(I.ws + I.L.pv);
  const T *dA = scan::data_ptr<T>(I.A, reinterpret_cast<const float *>(I.ws + I.L.Af));
  const T *dB = scan::data_ptr<T>(I.B, reinterpret_cast<const float *>(I.ws + I.L.Bf));
  const T *dQ = scan::data_ptr<T>(I.Q, reinterpret_cast<const float *>(I.ws + I.L.Qf));
  const T *dM = scan::data_ptr<T>(I.M, reinterpret_cast<const float *>(I.ws + I.L.Mf));
  const T *dR = scan::data_ptr<T>(I.R, reinterpret_cast<const float *>(I.ws + I.L.Rf));
  unsigned long long dzb = 0;  // max |dz| applied by this lane (refinement)
  const T *xb = reinterpret_cast<const T *>(I.ws + sbase + SL.xb);
  const T *pb = reinterpret_cast<const T *>(I.ws + sbase + SL.pb);
  T *psi = reinterpret_cast<T *>(I.ws + sbase + SL.psi);
  (void)sfin1;
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;
  LaneSeg<T, CP> fW, fA, fQ;
  LaneSeg<T, CB> fB, fK, fM;
  LaneSeg<T, CR> fR;
  double vc = 0.0, zx = 0.0, zy = 0.0, zu = 0.0, rxq = 0.0, rxc = 0.0, rur = 0.0;
  T vk = 0, vp = 0;
  auto prefetch = [&](int i) {
    fW.load(gW + (size_t)(i + 1) * nn, nn, lane);
    fA.load(dA + (size_t)i * nn, nn, lane);
    fB.load(dB + (size_t)i * nm, nm, lane);
    fK.load(gK + (size_t)i * nm, nm, lane);
    if (lane < n) {
      vc = __ldg(rhs.c + (size_t)(i + 1) * n + lane);
      vp = __ldg(gpv + (size_t)(i + 1) * n + lane);
    }
    if (lane < m) vk = __ldg(gkv + (size_t)i * m + lane);
    if (RES) {
      fQ.load(dQ + (size_t)i * nn, nn, lane);
      fM.load(dM + (size_t)i * nm, nm, lane);
      fR.load(dR + (size_t)i * mmm, mmm, lane);
      if (lane < n) {
        const size_t o = (size_t)(i + 1) * n + lane;
        zx = __ldcg(I.x + o);
        zy = __ldcg(I.y + o);
        rxq = __ldcg(rq + (size_t)i * n + lane);
        rxc = __ldcg(rc + o);
      }
      if (lane < m) {
        zu = __ldcg(I.u + (size_t)i * m + lane);
        rur = __ldcg(rr + (size_t)i * m + lane);
      }
    }
  };
  if (lane < n) s.x[lane] = (MODE == 0) ? (T)0 : xb[(size_t)c * n + lane];
  __syncwarp();
  if (RES) {
    // dy at the chunk's first stage: P_s dx_s + dp_s (P_s of the finalize)
    if (lane < n) {
      const T *Ps = reinterpret_cast<const T *>(I.ws + sbase + SL.PstB) + (size_t)c * nn;
      s.dy[lane] = pb[(size_t)c * n + lane] + scan::dotc<T, NX>(Ps + lane * n, s.x);
    }
  }
  prefetch(s0);
  for (int i = s0; i < e0; ++i) {
    __syncwarp();
    fW.store(s.W, nn, lane);
    fA.store(s.A, nn, lane);
    fB.store(s.B, nm, lane);
    fK.store(s.K, nm, lane);
    if (RES) {
      fQ.store_sym(s.Q, n, lane);
      fM.store(s.M, nm, lane);
      fR.store_sym(s.R, m, lane);
    }
    const double zx0 = zx, zy0 = zy, zu0 = zu, rxq0 = rxq, rxc0 = rxc, rur0 = rur;
    const T cvc = to_work<T>(vc), cvp = vp, cvk = vk;
    if (lane < n) s.pn[lane] = cvp;
    if (i + 1 < e0) prefetch(i + 1);
    __syncwarp();
    // u_i = K x_i + k_i (every lane on a clamped row; lanes < m store)
    {
      const T uv = cvk + scan::dotc<T, NX>(s.K + lm * n, s.x);
      if (lane < m) s.u[lane] = uv;
    }
    __syncwarp();
    // v = A x + B u + c'_{i+1} - delta p_{i+1}
    if (lane < n)
      s.v[lane] = (cvc - delta * cvp) + scan::dotc<T, NX>(s.A + lane * n, s.x) +
                  scan::dotc<T, NU>(s.B + lane * m, s.u);
    __syncwarp();
    // x_{i+1} = v - delta W v, y_{i+1} = W v + p_{i+1}
    T xn = 0, yn = 0;
    if (lane < n) {
      const T t = scan::dotc<T, NX>(s.W + lane * n, s.v);
      xn = s.v[lane] - delta * t;
      yn = t + cvp;
      s.dxn[lane] = xn;
      s.dyn[lane] = yn;
    }
    __syncwarp();
    if (MODE == 1) {
      if (!FROM_RES) {
        if (lane < n) {
          I.x[(size_t)(i + 1) * n + lane] = widen(xn);
          I.y[(size_t)(i + 1) * n + lane] = widen(yn);
        }
        if (lane < m) I.u[(size_t)i * m + lane] = widen(s.u[lane]);
      } else {
        if (lane < n) {
          const size_t o = (size_t)(i + 1) * n + lane;
          I.x[o] = zx0 + widen(xn);
          I.y[o] = zy0 + widen(yn);
          dzb = max(dzb, max(abs_bits(widen(xn)), abs_bits(widen(yn))));
          // x rows of stage i: Q dx + M du + A^T dy_{i+1} - dy_i
          const T t = scan::dotc<T, NX>(s.Q + lane * n, s.x) + scan::dots<T, NX>(s.A + lane, n, s.dyn) +
                      scan::dotc<T, NU>(s.M + lane * m, s.u) - s.dy[lane];
          rq[(size_t)i * n + lane] = rxq0 + widen(t);
          // c rows of stage i+1: A dx + B du - dx_{i+1} - delta dy_{i+1}
          const T tc = scan::dotc<T, NX>(s.A + lane * n, s.x) + scan::dotc<T, NU>(s.B + lane * m, s.u) -
                       (xn + delta * yn);
          rc[o] = rxc0 + widen(tc);
        }
        if (lane < m) {
          const size_t o = (size_t)i * m + lane;
          I.u[o] = zu0 + widen(s.u[lane]);
          dzb = max(dzb, abs_bits(widen(s.u[lane])));
          // u rows of stage i: M^T dx + R du + B^T dy_{i+1}
          const T t = scan::dots<T, NX>(s.M + lane, m, s.x) + scan::dots<T, NX>(s.B + lane, m, s.dyn) +
                      scan::dotc<T, NU>(s.R + lane * m, s.u);
          rr[o] = rur0 + widen(t);
        }
      }
    }
    __syncwarp();
    if (lane < n) {
      s.x[lane] = xn;
      s.dy[lane] = yn;
    }
  }
  __syncwarp();
  if (MODE == 0 && lane < n) psi[(size_t)c * n + lane] = s.x[lane];
  if (RES && e0 == N && lane < n) {
    // terminal x rows: Q_N dx_N - dy_N
    T t = -s.dy[lane];
    for (int l = 0; l < n; ++l) {
      const int r = lane, col = l;
      t = fma(to_work<T>(__ldg(I.Q + (size_t)N * nn + (r <= col ? r * n + col : col * n + r))),
              s.x[l], t);
    }
    double *dst = rq + (size_t)N * n + lane;
    *dst = __ldcg(dst) + widen(t);
  }
  if (RES) {
    for (int o = 16; o > 0; o >>= 1) dzb = max(dzb, __shfl_xor_sync(0xffffffffu, dzb, o));
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long *>(&I.st->dzmax), dzb);
  }
}

// x_0, y_0 (eq. recover-x0: v0 = c'_0 - delta p_0, x_0 = v0 - delta W_0 v0,
// y_0 = W_0 v0 + p_0) and x at the chunk starts: xb[c+1] = Phi_c^T xb[c] + psi_c.
template <typename T, int NX, bool FROM_RES>
__global__ void __launch_bounds__(32) k_scan_xbound(BatchArgs a, ScanLayout SL, size_t sbase) {
  constexpr int n = NX, nn = n * n;
  __shared__ T xv[NX], v0[NX];
  const int lane = threadIdx.x;
  const Inst I = get_inst(a, 0);
  if (FROM_RES && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) return;
  const T delta = (T)I.delta;
  const ScanRhs rhs = scan_rhs(I, FROM_RES);
  const T *gW = reinterpret_cast<const T *>(I.ws + I.L.W);
  const T *gpv = reinterpret_cast<const T *>(I.ws + I.L.pv);
  const T *Phi = reinterpret_cast<const T *>(I.ws + sbase + SL.Phi);
  const T *psi = reinterpret_cast<const T *>(I.ws + sbase + SL.psi);
  T *xb = reinterpret_cast<T *>(I.ws + sbase + SL.xb);
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rc = rq + (size_t)(I.N + 1) * n + (size_t)I.N * I.m;
  if (lane < n) v0[lane] = to_work<T>(__ldcg(rhs.c + lane)) - delta * gpv[lane];
  __syncwarp();
  if (lane < n) {
    T t = 0;
    for (int l = 0; l < n; ++l) t = fma(gW[lane * n + l], v0[l], t);
    const T x0 = v0[lane] - delta * t, y0 = t + gpv[lane];
    xv[lane] = x0;
    xb[lane] = x0;
    if (!FROM_RES) {
      I.x[lane] = widen(x0);
      I.y[lane] = widen(y0);
    } else {
      I.x[lane] = __ldcg(I.x + lane) + widen(x0);
      I.y[lane] = __ldcg(I.y + lane) + widen(y0);
      rc[lane] = __ldcg(rc + lane) - widen(x0) - I.delta * widen(y0);
      atomicMax(reinterpret_cast<unsigned long long *>(&I.st->dzmax),
                max(abs_bits(widen(x0)), abs_bits(widen(y0))));
    }
  }
  // column `lane` of Phi_c and psi_c[lane] in a register ring D chunks deep
  constexpr int D = bound_ring_depth<T>();
  const int C = SL.C;
  T col[D][NX], off[D];
  auto fetch = [&](int j, int cc) {
    if (cc < C && lane < n) {
#pragma unroll
      for (int l = 0; l < NX; ++l) col[j][l] = __ldcg(Phi + (size_t)cc * nn + l * n + lane);
      off[j] = __ldcg(psi + (size_t)cc * n + lane);
    }
  };
#pragma unroll
  for (int j = 0; j < D; ++j) fetch(j, j);
  for (int c0 = 0; c0 < C; c0 += D) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int c = c0 + j;
      if (c >= C) break;  // uniform over the warp
      __syncwarp();
      T t = 0;
      if (lane < n) {
        t = off[j];
#pragma unroll
        for (int l = 0; l < NX; ++l) t = fma(col[j][l], xv[l], t);  // (Phi_c^T x)[lane]
      }
      __syncwarp();
      if (lane < n) {
        xv[lane] = t;
        xb[(size_t)(c + 1) * n + lane] = t;
      }
      fetch(j, c + D);
    }
  }
}

// ---- residual of one long instance: one warp per stage, FP64 products
// (Section "Residual Computation"), maxima into the instance state by atomicMax
// of the order-preserving bit patterns; k_res_final forms the backward error.
// cert_g: FP64 LDL^T of the stored G_i (mixed path), one stage per thread.
template <int NX, int NU>
__global__ void __launch_bounds__(128) k_res_grid(BatchArgs a, int cert_g, int do_res) {
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  const Inst I = get_inst(a, 0);
  const int N = I.N;
  const double delta = I.delta;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;
  InstState *st = I.st;
  unsigned long long rbits = 0, zbits = 0, bbits = 0;
  float kmaxf = 0.f;
  if (cert_g) {
    // control pivots with margin (pd_margin_f32); no margin: escalation
    const float *gG = reinterpret_cast<const float *>(I.ws + I.L.G);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
      const int dec = pd_margin_f32<m>(gG + (size_t)s * mmm, m, (double)kMarginTau);
      I.flags[s] = (uint8_t)((I.flags[s] & 1) | (dec == kPdYes ? 2 : 0));
      if (dec == kPdNo) atomicMax(&st->pivot_status, (int32_t)RLQR_NOT_PD);
      if (dec == kPdAmbiguous) st->escalated = 1;
    }
  }
  if (!do_res) return;
  for (int s = gw; s < N; s += nw) {
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
          const double mm = __ldg(M + r * m + l);
          v = fma(mm, __ldg(u + l), v);
          ra += abs_f32_trunc(mm);
        }
        bbits = max(bbits, abs_bits(qv));
        rq[(size_t)s * n + r] = v;
        zbits = max(zbits, abs_bits(__ldg(x + r)));
      } else if (r < n + m) {  // u row: M^T x + R u + B^T y_{s+1} + r
        const int t = r - n;
        const double rv = __ldg(I.r + (size_t)s * m + t);
        v = rv;
        ra = 0.f;
        for (int l = 0; l < n; ++l) {
          const double mm = __ldg(M + l * m + t), bb = __ldg(B + l * m + t);
          v = fma(mm, __ldg(x + l), fma(bb, __ldg(yn + l), v));
          ra += abs_f32_trunc(mm) + abs_f32_trunc(bb);
        }
        for (int l = 0; l < m; ++l) {
          const double rr2 = __ldg(R + (t <= l ? t * m + l : l * m + t));
          v = fma(rr2, __ldg(u + l), v);
          ra += abs_f32_trunc(rr2);
        }
        bbits = max(bbits, abs_bits(rv));
        rr[(size_t)s * m + t] = v;
        zbits = max(zbits, abs_bits(__ldg(u + t)));
      } else {  // c row of stage s+1: A x + B u + c_{s+1} - x_{s+1} - delta y_{s+1}
        const int i = r - n - m;
        const double cv = __ldg(I.c + (size_t)(s + 1) * n + i);
        v = cv - __ldg(xn + i) - delta * __ldg(yn + i);
        ra = 1.f + abs_f32_trunc(delta);
        for (int l = 0; l < n; ++l) {
          const double aa = __ldg(A + i * n + l);
          v = fma(aa, __ldg(x + l), v);
          ra += abs_f32_trunc(aa);
        }
        for (int l = 0; l < m; ++l) {
          const double bb = __ldg(B + i * m + l);
          v = fma(bb, __ldg(u + l), v);
          ra += abs_f32_trunc(bb);
        }
        bbits = max(bbits, abs_bits(cv));
        rc[(size_t)(s + 1) * n + i] = v;
        zbits = max(zbits, abs_bits(__ldg(yn + i)));
      }
      rbits = max(rbits, abs_bits(v));
      kmaxf = fmaxf(kmaxf, ra);
    }
  }
  // rows x_N and c_0 (first warp)
  if (gw == 0) {
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
        rq[(size_t)N * n + r] = v;
      } else {
        const int i = r - n;
        const double cv = __ldg(I.c + i), yv = __ldg(I.y + i);
        v = cv - delta * yv - __ldg(I.x + i);
        kmaxf = fmaxf(kmaxf, 1.f + abs_f32_trunc(delta));
        bbits = max(bbits, abs_bits(cv));
        zbits = max(zbits, abs_bits(yv));
        rc[i] = v;
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
    atomicMax(reinterpret_cast<unsigned long long *>(&st->rmax), rbits);
    atomicMax(reinterpret_cast<unsigned long long *>(&st->zmax), zbits);
    atomicMax(reinterpret_cast<unsigned long long *>(&st->bmax), bbits);
    atomicMax(reinterpret_cast<unsigned long long *>(&st->kmax),
              abs_bits(widen(kmaxf)));
  }
}

// Pivot status of the factor into the caller's status array.
static __global__ void k_scan_status(BatchArgs a) {
  const Inst I = get_inst(a, 0);
  if (a.status) a.status[0] = I.st->pivot_status;
}

// Maxima of |res| and |z| of one instance after a refinement pass.
static __global__ void k_norms_grid(BatchArgs a) {
  const Inst I = get_inst(a, 0);
  if (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR) return;
  const size_t nres = (size_t)(I.N + 1) * I.n * 2 + (size_t)I.N * I.m;
  const size_t nx = (size_t)(I.N + 1) * I.n, nu = (size_t)I.N * I.m;
  const double *res = reinterpret_cast<const double *>(I.ws + I.L.res);
  unsigned long long rbits = 0, zbits = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nres;
       e += (size_t)gridDim.x * blockDim.x) {
    rbits = max(rbits, abs_bits(__ldcg(res + e)));
    if (e < nx) zbits = max(zbits, max(abs_bits(__ldcg(I.x + e)), abs_bits(__ldcg(I.y + e))));
    if (e < nu) zbits = max(zbits, abs_bits(__ldcg(I.u + e)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
    zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long *>(&I.st->rmax), rbits);
    atomicMax(reinterpret_cast<unsigned long long *>(&I.st->zmax), zbits);
  }
}

// rel = rmax / (kmax zmax + bmax), convergence, outputs.  `pass`: 0 after the
// first residual, 1 after a refinement pass (counts the pass).
static __global__ void k_res_final(BatchArgs a, int pass) {
  const Inst I = get_inst(a, 0);
  InstState *st = I.st;
  if (pass && (st->converged || st->pivot_status == RLQR_ERR_SINGULAR)) return;
  if (pass) {
    // rounding bound of the pass's residual update in the working precision
    // (2 gamma_L ||K||_inf max|dz| per entry, L = 2n + m), accumulated
    const double uw = a.tsize == 4 ? 0x1p-24 : 0x1p-53;
    st->upd += 2.0 * (2 * I.n + I.m) * uw * st->kmax * st->dzmax;
    st->dzmax = 0.0;
  } else {
    st->upd = 0.0;  // a residual computed from scratch
    st->dzmax = 0.0;
  }
  const double den = st->kmax * st->zmax + st->bmax;
  const double rel = den > 0.0 ? (st->rmax + st->upd) / den : st->rmax + st->upd;
  st->rel = rel;
  if (pass) st->iters += 1;
  const int32_t conv = (rel <= a.tol) ? 1 : 0;
  st->converged = conv;
  if (a.rel) a.rel[0] = rel;
  if (a.iters) a.iters[0] = st->iters;
  if (a.status) {
    const int32_t ps = st->pivot_status;
    a.status[0] = (ps == RLQR_ERR_SINGULAR) ? RLQR_ERR_SINGULAR : (conv ? ps : RLQR_ERR_NOT_CONVERGED);
  }
}

// Zero the maxima before a residual or norm pass.
static __global__ void k_norms_reset(BatchArgs a, int all) {
  const Inst I = get_inst(a, 0);
  InstState *st = I.st;
  if (!all && (st->converged || st->pivot_status == RLQR_ERR_SINGULAR)) return;
  st->rmax = 0.0;
  st->zmax = 0.0;
  if (all) {  // start of a solve
    st->kmax = 0.0;
    st->bmax = 0.0;
    st->upd = 0.0;
    st->dzmax = 0.0;
    st->iters = 0;
    st->converged = 0;
  }
}

}  // namespace rlqr

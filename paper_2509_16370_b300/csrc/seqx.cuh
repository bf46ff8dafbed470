// seqx.cuh -- the sequential Riccati sweep for the larger compile-time sizes
// ((24,8), (32,8), (48,16)): one CTA of 256 threads per instance, the same
// recursion, certificate and outputs as k_seq in seq.cuh (Theorem
// main-seq-theorem, eq. value-fn-formulas, Corollary p-recurrence, eq.
// recover-x0 / control-law / recover-x), built from the products with 2x2
// register tiles (packed f32x2 FMAs) and the register-resident Gauss-Jordan
// eliminations of scan.cuh (one barrier per elimination step).  The next
// stage's data is prefetched into registers during a stage.  Mixed path:
// bit0 of a stage whose FP32 Gershgorin proof fails is decided afterwards by
// k_seqx_cert / k_seqx_cert64 from the stored FP32 P_i, stage-parallel after
// the sweep; the sweep writes bit0 = 1 there provisionally.
#pragma once

#include "common.cuh"
#include "scan.cuh"

namespace rlqr {

template <int NX, int NU>
constexpr bool seqx_fits() {
  return NX % 2 == 0 && NU % 2 == 0 && NX <= 48 && NU <= 16 && NX >= 16;
}

template <typename T, int NX, int NU>
struct SxSmem {
  static constexpr int LD = NX + 2, LD2 = 2 * NX + 2, LDG = 2 * NU + NX + 2;  // even strides
  static constexpr int WG = 2 * NU + NX + 1;  // columns of [G | H | h | I]
  T P[NX * LD], W[NX * LD], Q[NX * LD], A[NX * LD], WA[NX * LD], T1[NX * LD];
  T S2[NX * LD2];                  // [I + delta P | P]; also the P update's temporary
  T B[NX * NU], M[NX * NU], WB[NX * NU], K[NU * NX], H[NU * NX], R[NU * NU];
  T GH[NU * LDG];                  // [G | H | h | I]
  T rowbuf[2 * (2 * NX + 2 * NU + 2)];
  T p[NX], q[NX], c[NX], v[NX], g[NX], x[NX], r[NU], h[NU], kk[NU], u[NU];
  int bit, sing, pass;
};

// The sweep of instance b by one CTA of scan::kTH threads in the shared
// memory at smem (an SxSmem<T, NX, NU>); the body of k_seqx and of the
// persistent ragged sweep.
template <typename T, int NX, int NU, bool SOLVE>
__device__ __forceinline__ void seqx_body(const BatchArgs &a, int b, unsigned char *smem) {
  static_assert(seqx_fits<NX, NU>(), "size outside the compile-time CTA sweep");
  using SM = SxSmem<T, NX, NU>;
  constexpr bool FP32 = sizeof(T) == 4;
  constexpr int TH = scan::kTH;
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int LD = SM::LD, LD2 = SM::LD2, LDG = SM::LDG, WG = SM::WG;
  SM &s = *reinterpret_cast<SM *>(smem);
  const Inst I = get_inst(a, b);
  const int N = I.N, tid = threadIdx.x;
  const T delta = (T)I.delta;
  const float delta_up = __double2float_ru(I.delta), delta_dn = __double2float_rd(I.delta);
  T *gW = reinterpret_cast<T *>(I.ws + I.L.W);
  T *gK = reinterpret_cast<T *>(I.ws + I.L.K);
  T *gGi = reinterpret_cast<T *>(I.ws + I.L.Gi);
  T *gkv = reinterpret_cast<T *>(I.ws + I.L.kv);
  T *gpv = reinterpret_cast<T *>(I.ws + I.L.pv);
  T *gG = reinterpret_cast<T *>(I.ws + I.L.G);

  constexpr int CP = (nn + TH - 1) / TH, CB = (nm + TH - 1) / TH, CR = (mmm + TH - 1) / TH;
  RegSeg<double, TH, CP> pfA, pfQ;
  RegSeg<double, TH, CB> pfB, pfM;
  RegSeg<double, TH, CR> pfR;
  double vq = 0.0, vc = 0.0, vr = 0.0;
  auto prefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn);
    pfQ.load(I.Q + (size_t)k * nn, nn);
    pfB.load(I.B + (size_t)k * nm, nm);
    pfM.load(I.M + (size_t)k * nm, nm);
    pfR.load(I.R + (size_t)k * mmm, mmm);
    if (SOLVE) {
      if (tid < n) {
        vq = __ldg(I.q + (size_t)k * n + tid);
        vc = __ldg(I.c + (size_t)(k + 1) * n + tid);
      }
      if (tid < m) vr = __ldg(I.r + (size_t)k * m + tid);
    }
  };
  auto commit = [&]() {
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int idx = tid + TH * i;
      if (idx < nn) {
        const int r = idx / n, c = idx - r * n;
        s.A[r * LD + c] = to_work<T>(pfA.v[i]);
        if (r <= c) {
          const T qv = to_work<T>(pfQ.v[i]);
          s.Q[r * LD + c] = qv;
          s.Q[c * LD + r] = qv;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int idx = tid + TH * i;
      if (idx < nm) {
        s.B[idx] = to_work<T>(pfB.v[i]);
        s.M[idx] = to_work<T>(pfM.v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < CR; ++i) {
      const int idx = tid + TH * i;
      if (idx < mmm) {
        const int r = idx / m, c = idx - r * m;
        if (r <= c) {
          const T rv = to_work<T>(pfR.v[i]);
          s.R[r * m + c] = rv;
          s.R[c * m + r] = rv;
        }
      }
    }
    if (SOLVE) {
      if (tid < n) {
        s.q[tid] = to_work<T>(vq);
        s.c[tid] = to_work<T>(vc);
      }
      if (tid < m) s.r[tid] = to_work<T>(vr);
    }
  };

  // ---- terminal stage: P_N = Q_N (upper triangle), p_N = q_N
  for (int e = tid; e < nn; e += TH) {
    const int r = e / n, c = e - r * n;
    s.P[r * LD + c] = to_work<T>(I.Q[(size_t)N * nn + (r <= c ? e : c * n + r)]);
  }
  if (SOLVE && tid < n) {
    s.p[tid] = to_work<T>(I.q[(size_t)N * n + tid]);
    gpv[(size_t)N * n + tid] = s.p[tid];
  }
  prefetch(N - 1);
  commit();
  if (N > 1) prefetch(N - 2);
  bool notpd = false, singular = false;
  int bit1_next = 1;  // stage N has no control pivot

  // state pivot of the P in s.P: W into s.W and gWk; returns bit0
  auto state_pivot = [&](T *gWk) -> int {
    __syncthreads();
    if (tid == 0) {
      s.bit = 1;
      s.sing = 0;
      s.pass = 1;
    }
    for (int e = tid; e < nn; e += TH) {
      const int r = e / n, c = e - r * n;
      const T pv = s.P[r * LD + c];
      s.S2[r * LD2 + c] = (r == c ? (T)1 : (T)0) + delta * pv;
      s.S2[r * LD2 + n + c] = pv;
    }
    __syncthreads();
    if constexpr (FP32) {
      // Gershgorin proof in FP32 with directed rounding, with the
      // certificate's margin; when it fails the stage's P is stored and
      // k_seqx_cert decides bit0 later, off this instance's sequential chain
      if (tid < n) {
        float off = 0.f;
        for (int j = 0; j < n; ++j)
          if (j != tid) off = __fadd_ru(off, fabsf((float)s.P[tid * LD + j]));
        if (!gershgorin_row_margin((float)s.P[tid * LD + tid], off, delta_dn, delta_up, kMarginTau))
          atomicAnd(&s.pass, 0);
      }
      __syncthreads();
      const int stage = (int)((gWk - gW) / nn);
      uint8_t *pend = reinterpret_cast<uint8_t *>(I.ws + I.L.pend);
      if (!s.pass) {
        float *Pc = reinterpret_cast<float *>(I.ws + I.L.Pc) + (size_t)stage * nn;
        for (int e = tid; e < nn; e += TH) {
          const int r = e / n, c = e - r * n;
          Pc[e] = (float)s.P[r * LD + c];
        }
      }
      if (tid == 0) pend[stage] = s.pass ? 0 : 1;
      scan::gjr<T, NX, 2 * NX, TH>(s.S2, LD2, s.rowbuf, nullptr, nullptr);
    } else {
      scan::gjr<T, NX, 2 * NX, TH>(s.S2, LD2, s.rowbuf, &s.bit, &s.sing);
    }
    // W = right block, exactly symmetric (lower triangle mirrored)
    for (int e = tid; e < nn; e += TH) {
      const int r = e / n, c = e - r * n;
      const int lo = r >= c ? r : c, hi = r >= c ? c : r;
      const T w = s.S2[lo * LD2 + n + hi];
      s.W[r * LD + c] = w;
      gWk[e] = w;
    }
    __syncthreads();
    if (s.sing) singular = true;
    return s.bit;
  };

  for (int k = N - 1; k >= 0; --k) {
    const int bit0 = state_pivot(gW + (size_t)(k + 1) * nn);
    // WA = W A, WB = W B, g = p + W (c_{k+1} - delta p)
    scan::mmt<T, NX, NX, NX, false, false>(s.WA, LD, s.W, LD, s.A, LD, nullptr, 0, (T)1);
    scan::mmt<T, NX, NU, NX, false, false>(s.WB, m, s.W, LD, s.B, m, nullptr, 0, (T)1);
    if (SOLVE && tid < n) s.v[tid] = s.c[tid] - delta * s.p[tid];
    __syncthreads();
    if (SOLVE && tid < n) {
      T t = s.p[tid];
      for (int l = 0; l < n; ++l) t = fma(s.W[tid * LD + l], s.v[l], t);
      s.g[tid] = t;
    }
    // G = R + B^T WB (into GH), H = B^T WA
    scan::mmt<T, NU, NU, NX, true, false>(s.GH, LDG, s.B, m, s.WB, m, s.R, m, (T)1);
    scan::mmt<T, NU, NX, NX, true, false>(s.H, n, s.B, m, s.WA, LD, nullptr, 0, (T)1);
    __syncthreads();
    // [G | H | h | I]
    for (int e = tid; e < m * n; e += TH) {
      const int r = e / n, c = e - r * n;
      const T hv = s.H[e] + s.M[c * m + r];
      s.H[e] = hv;
      s.GH[r * LDG + m + c] = hv;
    }
    for (int e = tid; e < mmm; e += TH) {
      const int r = e / m, c = e - r * m;
      s.GH[r * LDG + m + n + 1 + c] = (r == c) ? (T)1 : (T)0;
    }
    if (tid < m) {
      T t = 0;
      if (SOLVE) {
        t = s.r[tid];
        for (int l = 0; l < n; ++l) t = fma(s.B[l * m + tid], s.g[l], t);
      }
      s.GH[tid * LDG + m + n] = t;
    }
    if (tid == 0) {
      s.bit = 1;
      s.sing = 0;
    }
    __syncthreads();
    if (FP32)
      for (int e = tid; e < mmm; e += TH) {
        const int r = e / m, c = e - r * m;
        gG[(size_t)k * mmm + e] = s.GH[r * LDG + c];
      }
    scan::gjr<T, NU, WG, TH>(s.GH, LDG, s.rowbuf, FP32 ? nullptr : &s.bit,
                             FP32 ? nullptr : &s.sing);
    const int bit1 = s.bit;
    if (!FP32 && s.sing) singular = true;
    // K = -G^{-1} H, k = -G^{-1} h, G^{-1}
    for (int e = tid; e < m * n; e += TH) {
      const int r = e / n, c = e - r * n;
      const T kv = -s.GH[r * LDG + m + c];
      s.K[e] = kv;
      gK[(size_t)k * nm + e] = kv;
    }
    for (int e = tid; e < mmm; e += TH) {
      const int r = e / m, c = e - r * m;
      gGi[(size_t)k * mmm + e] = s.GH[r * LDG + m + n + 1 + c];
    }
    if (SOLVE && tid < m) {
      const T kv = -s.GH[tid * LDG + m + n];
      s.kk[tid] = kv;
      gkv[(size_t)k * m + tid] = kv;
    }
    __syncthreads();
    // P_k = Q + A^T WA + H^T K (exactly symmetric), p_k = q + A^T g + H^T k
    scan::mmt<T, NX, NX, NX, true, false>(s.T1, LD, s.A, LD, s.WA, LD, s.Q, LD, (T)1);
    __syncthreads();
    T *T2 = s.S2;  // the elimination buffer is free until the next stage
    scan::mmt<T, NX, NX, NU, true, false>(T2, LD, s.H, n, s.K, n, s.T1, LD, (T)1);
    T pk = 0;
    if (SOLVE && tid < n) {
      pk = s.q[tid];
      for (int l = 0; l < n; ++l) pk = fma(s.A[l * LD + tid], s.g[l], pk);
      for (int l = 0; l < m; ++l) pk = fma(s.H[l * n + tid], s.kk[l], pk);
    }
    __syncthreads();
    for (int e = tid; e < nn; e += TH) {
      const int r = e / n, c = e - r * n;
      const int lo = r >= c ? r : c, hi = r >= c ? c : r;
      s.P[r * LD + c] = T2[lo * LD + hi];
    }
    if (SOLVE && tid < n) {
      s.p[tid] = pk;
      gpv[(size_t)k * n + tid] = pk;
    }
    if (k > 0) {
      commit();
      if (k > 1) prefetch(k - 2);
    }
    if (tid == 0) {
      const int b1 = FP32 ? (k + 1 == N) : bit1_next;
      I.flags[k + 1] = (uint8_t)(bit0 | (b1 << 1));
      if (!bit0 || (!FP32 && !b1)) notpd = true;
    }
    bit1_next = bit1;
  }

  // ---- initial-state pivot
  {
    const int bit0 = state_pivot(gW);
    if (tid == 0) {
      const int b1 = FP32 ? 0 : bit1_next;
      I.flags[0] = (uint8_t)(bit0 | (b1 << 1));
      if (!bit0 || (!FP32 && !b1)) notpd = true;
      const int32_t st = singular ? RLQR_ERR_SINGULAR : (notpd ? RLQR_NOT_PD : RLQR_OK);
      I.st->pivot_status = st;
      I.st->escalated = 0;
      I.st->iters = 0;
      I.st->converged = 0;
      I.st->rel = 0.0;
      if (a.status) a.status[b] = st;
    }
  }
  if constexpr (!SOLVE) return;

  // ---- forward rollout (thread = row)
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  if (tid < n) {
    s.p[tid] = __ldcg(gpv + tid);
    s.v[tid] = to_work<T>(I.c[tid]) - delta * s.p[tid];
  }
  __syncthreads();
  if (tid < n) {
    T t = 0;
    for (int l = 0; l < n; ++l) t = fma(s.W[tid * LD + l], s.v[l], t);
    const T xv = s.v[tid] - delta * t, yv = t + s.p[tid];
    s.x[tid] = xv;
    I.x[tid] = widen(xv);
    I.y[tid] = widen(yv);
  }
  RegSeg<T, TH, CP> fW;
  RegSeg<T, TH, CB> fK;
  T fk = 0, fp = 0;
  auto fprefetch = [&](int k) {
    pfA.load(I.A + (size_t)k * nn, nn);
    pfB.load(I.B + (size_t)k * nm, nm);
    if (tid < n) {
      vc = __ldg(I.c + (size_t)(k + 1) * n + tid);
      fp = __ldcg(gpv + (size_t)(k + 1) * n + tid);
    }
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn);
    fK.load_cg(gK + (size_t)k * nm, nm);
    if (tid < m) fk = __ldcg(gkv + (size_t)k * m + tid);
  };
  __syncthreads();
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int idx = tid + TH * i;
      if (idx < nn) {
        const int r = idx / n, c = idx - r * n;
        s.A[r * LD + c] = to_work<T>(pfA.v[i]);
        s.W[r * LD + c] = fW.v[i];
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int idx = tid + TH * i;
      if (idx < nm) {
        s.B[idx] = to_work<T>(pfB.v[i]);
        s.K[idx] = fK.v[i];
      }
    }
    if (tid < n) {
      s.c[tid] = to_work<T>(vc);
      s.p[tid] = fp;
    }
    if (tid < m) s.kk[tid] = fk;
    if (k + 1 < N) fprefetch(k + 1);
    __syncthreads();
    // u_k = K_k x_k + k_k
    if (tid < m) {
      T t = s.kk[tid];
      for (int l = 0; l < n; ++l) t = fma(s.K[tid * n + l], s.x[l], t);
      s.u[tid] = t;
      I.u[(size_t)k * m + tid] = widen(t);
    }
    __syncthreads();
    // v = A x + B u + c_{k+1} - delta p_{k+1}
    if (tid < n) {
      T t = s.c[tid] - delta * s.p[tid];
      for (int l = 0; l < n; ++l) t = fma(s.A[tid * LD + l], s.x[l], t);
      for (int l = 0; l < m; ++l) t = fma(s.B[tid * m + l], s.u[l], t);
      s.v[tid] = t;
    }
    __syncthreads();
    // x_{k+1} = v - delta W v, y_{k+1} = W v + p_{k+1}
    if (tid < n) {
      T t = 0;
      for (int l = 0; l < n; ++l) t = fma(s.W[tid * LD + l], s.v[l], t);
      const T xv = s.v[tid] - delta * t, yv = t + s.p[tid];
      s.x[tid] = xv;
      I.x[(size_t)(k + 1) * n + tid] = widen(xv);
      I.y[(size_t)(k + 1) * n + tid] = widen(yv);
    }
    __syncthreads();
  }
}

template <typename T, int NX, int NU, bool SOLVE>
__global__ void __launch_bounds__(scan::kTH) k_seqx(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  seqx_body<T, NX, NU, SOLVE>(a, inst_of(a, slot), smem_raw);
}

// Deferred certificate of the state pivots I + delta P_s whose FP32
// Gershgorin proof failed in k_seqx (mixed path), one warp per pending stage
// (pend[s] = 1): the FP32 register proof of warp_pd_proof_f32; a stage it
// does not prove is handed to k_seqx_cert64 (pend[s] = 2).  Grid: x =
// instance slot, y (with the warps of a block) strides over the stages 0..N.
template <int NX>
__global__ void __launch_bounds__(128) k_seqx_cert(BatchArgs a) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const Inst I = get_inst(a, inst_of(a, slot));
  uint8_t *pend = reinterpret_cast<uint8_t *>(I.ws + I.L.pend);
  const float *Pc = reinterpret_cast<const float *>(I.ws + I.L.Pc);
  for (int st = blockIdx.y * nwb + wid; st <= I.N; st += gridDim.y * nwb) {
    if (!__ldcg(pend + st)) continue;
    // proven: bit0 stays as the sweep wrote it (1)
    if (warp_pd_proof_f32<NX>(Pc + (size_t)st * NX * NX, I.delta, kMarginTau)) continue;
    if (lane == 0) pend[st] = 2;
  }
}

// The FP64 decision for the stages the FP32 proof left open (pend[s] = 2),
// with the certificate's margin: unpivoted LDL^T of S - tau D and, when that
// is not PD, of S + tau D (S = I + delta P_s from the stored FP32 P_s, D =
// diag(max(|S_jj|, 2^-24 max |S_jj|))), one warp per stage, the trailing
// triangle's updates spread over the lanes.  S - tau D PD: bit0 stays 1;
// S + tau D not PD: bit0 = 0 and the pivot status (and status output) rise
// to RLQR_NOT_PD; neither, or a non-finite entry: the instance is escalated
// to the FP64 recursion (InstState::escalated).  Same grid as k_seqx_cert.
template <int NX>
__global__ void __launch_bounds__(128) k_seqx_cert64(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = NX, nn = NX * NX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  double *S = reinterpret_cast<double *>(smem_raw) + (size_t)wid * nn;
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  const uint8_t *pend = reinterpret_cast<const uint8_t *>(I.ws + I.L.pend);
  const float *Pc = reinterpret_cast<const float *>(I.ws + I.L.Pc);
  int notpd = 0, esc = 0;
  for (int st = blockIdx.y * nwb + wid; st <= I.N; st += gridDim.y * nwb) {
    if (__ldcg(pend + st) != 2) continue;
    const float *P = Pc + (size_t)st * nn;
    // diagonal scale of the shift
    double dmax = 0.0;
    for (int j = lane; j < n; j += 32)
      dmax = fmax(dmax, fabs(1.0 + I.delta * widen(__ldcg(P + j * n + j))));
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    int dec = kPdAmbiguous;
    for (int pass = 0; pass < 2; ++pass) {
      const double sg = pass == 0 ? -(double)kMarginTau : (double)kMarginTau;
      __syncwarp();
      for (int e = lane; e < nn; e += 32) {
        const int r = e / n, c = e - r * n;
        double v = (r == c ? 1.0 : 0.0) + I.delta * widen(__ldcg(P + e));
        if (r == c) v += sg * fmax(fabs(v), 0x1p-24 * dmax);
        S[e] = v;
      }
      int pos = 1, fin = 1;
      for (int j = 0; j < n; ++j) {
        __syncwarp();
        const double d = S[j * n + j];
        if (!isfinite(d)) fin = 0;
        if (!(d > 0.0)) pos = 0;
        if (!pos || !fin) break;  // uniform over the warp
        const double rd = 1.0 / d;
        const int r = n - 1 - j;
        for (int idx = lane; idx < r * (r + 1) / 2; idx += 32) {
          int i, c;
          tri_decode(idx, i, c);
          i += j + 1;
          c += j + 1;
          S[i * n + c] -= S[i * n + j] * (S[c * n + j] * rd);
        }
      }
      if (!fin) break;
      if (pass == 0 && pos) { dec = kPdYes; break; }
      if (pass == 1 && !pos) { dec = kPdNo; break; }
    }
    if (lane == 0) {
      if (dec == kPdNo) I.flags[st] = (uint8_t)(I.flags[st] & 2);
      notpd |= dec == kPdNo;
      esc |= dec == kPdAmbiguous;
    }
  }
  if (lane == 0 && esc) I.st->escalated = 1;
  if (lane == 0 && notpd) {
    atomicMax(&I.st->pivot_status, (int32_t)RLQR_NOT_PD);
    if (a.status) atomicMax(&a.status[b], (int32_t)RLQR_NOT_PD);
  }
}

}  // namespace rlqr

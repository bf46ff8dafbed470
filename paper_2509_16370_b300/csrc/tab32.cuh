// tab32.cuh -- the FP32 Riccati sweep of the mixed-precision path for small
// state dimensions (n even, m <= n, 2n + m + 1 <= 32): the shape of batched
// trajectory-optimization subproblems.  One CTA of two warps per instance.
//
// Recursion: Theorem main-seq-theorem and eq. value-fn-formulas (backward),
// Corollary p-recurrence (vectors), eq. recover-x0 / control-law / recover-x
// (forward).  Every quantity of a backward stage comes out of ONE Gauss-Jordan
// elimination of a (2n+m)-row tableau whose Schur complements are the
// recursion's formulas.  With L = [A | B] and X = I + delta P_{k+1}:
//
//             cols:  X (lanes < n)   L (lanes n..2n+m-1)        rhs (lane 2n+m)
//   top  n rows   [  I + delta P     P L                        P c_{k+1} + p_{k+1} ]
//   x    n rows   [  -A^T            [Q   M]                     q                  ]
//   u    m rows   [  -B^T            [M^T R]                     r                  ]
//
// (plus P itself as a second column block of the lanes < n, top rows only).
//  * Eliminating the n state pivots (the X block; 2x2 block pivots) leaves
//    X^{-1} P = W in the P block, X^{-1} P L = W L and X^{-1}(P c + p) =
//    p + W (c - delta p) = g in the top rows, and the Schur complement
//    [Q M; M^T R] + L^T W L with right-hand side [q; r] + L^T g below it:
//    the u-u block is G_k = R + B^T W B, the u-x block H_k = B^T W A + M^T.
//  * Eliminating the m control pivots (scalar pivots: G_k may be indefinite)
//    leaves P_k = Q + A^T W A + H^T K in the x rows of the A columns, -K_k in
//    their u rows, p_k and -k_k in the right-hand side, and (with identity
//    columns re-seeded in lanes < m) G_k^{-1} in their u rows.
// Lane c owns column c in registers; the pivot columns reach the other lanes
// through shared memory (one store, a warp sync, broadcast vector loads).
// The first product P [L | c] is the only matrix product on the chain.
//
// Warp 1 (the producer) streams the FP64 stage data: cp.async copies kDP - 1
// stages ahead into a shared-memory ring, then truncation to FP32 into the
// layouts the tableau reads (row-major and transposed) and the FP32 copies
// the refinement reads, handed over through a two-slot ring guarded by named
// barriers (full / empty per slot).
//
// Certificate of I + delta P_{k+1} (bit0): an FP32 Gershgorin proof with
// directed rounding that I + delta P - tau D is positive definite (D its
// diagonal, tau = kMarginTau); a stage it does not prove stores its FP32 P
// and is decided after the sweep, stage-parallel (k_seqx_cert /
// k_seqx_cert64).  G_k is stored for the FP64 certificate pass.
//
// Forward rollout (warp 0, lane = row): u = K x + k, v = A x + B u + c -
// delta p, x' = v - delta W v, y' = W v + p, with the stages' rows of K, A,
// B, W arriving by cp.async kDF - 1 stages ahead.
#pragma once

#include "common.cuh"
#include "sweep32.cuh"

namespace rlqr {

template <int NX, int NU>
constexpr bool tab32_fits() {
  return NX % 2 == 0 && NX >= 2 && NU >= 1 && NU <= NX && 2 * NX + NU + 1 <= 32;
}

template <int NX, int NU>
struct Tb32 {
  static constexpr int n = NX, m = NU;
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4;  // row strides
  static constexpr int RR = 2 * NX + NU;          // tableau rows
  static constexpr int R2 = (RR + 1) / 2;         // float2 per tableau column
  static constexpr int RP = (2 * R2 + 3) / 4 * 4; // broadcast column stride (floats)
  struct Slot {
    alignas(16) float A[NX * N4];
    alignas(16) float At[NX * N4];
    alignas(16) float B[NX * M4];
    alignas(16) float Bt[NU * N4];
    alignas(16) float Q[NX * N4];
    alignas(16) float M[NX * M4];
    alignas(16) float Mt[NU * N4];
    alignas(16) float R[NU * M4];
    alignas(16) float q[N4];
    alignas(16) float r[M4];
    alignas(16) float c[N4];
  };
  Slot slot[2];
  alignas(16) float Ps[NX * N4];   // symmetric P of the stage after the current one
  alignas(16) float Wt[NX * N4];   // row c = computed column c of W (symmetrization)
  alignas(16) float p[N4];         // p of the stage after the current one
  alignas(16) float Id[NX * N4];   // identity rows (the X lanes' product vectors)
  alignas(16) float zero[N4 + M4];
  alignas(16) float bc[2][2][RP];  // state pivot columns (ping-pong)
  alignas(16) float ub[2][RP];     // control pivot column (ping-pong)
  alignas(16) float unit[NU][RP];  // unit tableau columns e_{2n+t} (seeds of G^{-1})
  alignas(16) float x[N4];
  alignas(16) float u[M4];
  alignas(16) float v[N4];
  // backward: FP64 stage data in flight (kDP stages: A | Q | B | M | R | q | r
  // | c_{k+1}, the producer's cp.async ring); forward: the FP32 rows of kDF
  // stages (K | A | B | W_{k+1} padded rows, c_{k+1}, p_{k+1}, k_k)
  static constexpr int S64 = 2 * NX * NX + 2 * NX * NU + NU * NU + 2 * NX + NU;  // doubles
  struct FSlot {
    alignas(16) float K[NU * N4];
    alignas(16) float A[NX * N4];
    alignas(16) float B[NX * M4];
    alignas(16) float W[NX * N4];
    alignas(16) float c[N4];
    alignas(16) float p[N4];
    alignas(16) float k[M4];
  };
  static constexpr int kDP = 4, kDF = 8;
  static constexpr size_t kRing = (kDP * S64 * 8 > kDF * sizeof(FSlot)) ? kDP * S64 * 8
                                                                        : kDF * sizeof(FSlot);
  alignas(16) unsigned char ring[kRing];
};

// K2 packed pairs from 16-byte aligned shared memory into r[OFF .. OFF+K2).
template <int K2, int OFF, int TOT>
__device__ __forceinline__ void ld_seg(const float *p, float2 (&r)[TOT]) {
  static_assert(OFF + K2 <= TOT, "segment outside the register array");
  if constexpr (K2 % 2 == 0) {
#pragma unroll
    for (int q = 0; q < K2 / 2; ++q) {
      const float4 t = reinterpret_cast<const float4 *>(p)[q];
      r[OFF + 2 * q] = make_float2(t.x, t.y);
      r[OFF + 2 * q + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int q = 0; q < K2; ++q) r[OFF + q] = reinterpret_cast<const float2 *>(p)[q];
  }
}

template <int K2>
__device__ __forceinline__ void st_seg(float *p, const float2 (&r)[K2]) {
  if constexpr (K2 % 2 == 0) {
#pragma unroll
    for (int q = 0; q < K2 / 2; ++q)
      reinterpret_cast<float4 *>(p)[q] = make_float4(r[2 * q].x, r[2 * q].y, r[2 * q + 1].x, r[2 * q + 1].y);
  } else {
#pragma unroll
    for (int q = 0; q < K2; ++q) reinterpret_cast<float2 *>(p)[q] = r[q];
  }
}

__device__ __forceinline__ void set_el(float2 &p, int h, float v) {
  if (h) p.y = v; else p.x = v;
}

// Named barriers of the producer / consumer ring (ids 1..4; 0 is
// __syncthreads): full[s] = 1 + s, empty[s] = 3 + s, 64 threads each.  The
// ids are immediates: a register id makes the compiler reserve all 16
// hardware barriers of the CTA, which limits how many CTAs an SM holds.
template <int ID>
__device__ __forceinline__ void nbar_sync_id() {
  asm volatile("bar.sync %0, 64;" ::"n"(ID) : "memory");
}
template <int ID>
__device__ __forceinline__ void nbar_arrive_id() {
  asm volatile("bar.arrive %0, 64;" ::"n"(ID) : "memory");
}
__device__ __forceinline__ void nbar_sync(int id) {
  switch (id) {
    case 1: nbar_sync_id<1>(); break;
    case 2: nbar_sync_id<2>(); break;
    case 3: nbar_sync_id<3>(); break;
    default: nbar_sync_id<4>(); break;
  }
}
__device__ __forceinline__ void nbar_arrive(int id) {
  switch (id) {
    case 1: nbar_arrive_id<1>(); break;
    case 2: nbar_arrive_id<2>(); break;
    case 3: nbar_arrive_id<3>(); break;
    default: nbar_arrive_id<4>(); break;
  }
}

template <int NX, int NU, bool SOLVE>
__global__ void __launch_bounds__(64, 7) k_tab32(BatchArgs a) {
  static_assert(tab32_fits<NX, NU>(), "dimensions outside the FP32 tableau sweep");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  using SM = Tb32<NX, NU>;
  constexpr int N4 = SM::N4, M4 = SM::M4, R2 = SM::R2;
  constexpr int H2 = n / 2;             // float2 of an n-vector
  constexpr int U2 = (m + 1) / 2;       // float2 of an m-vector (padded)
  constexpr int XL = n, BL = 2 * n, RL = 2 * n + m;  // first A lane, first B lane, rhs lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  const int N = I.N;
  float *gAf = reinterpret_cast<float *>(I.ws + I.L.Af);
  float *gBf = reinterpret_cast<float *>(I.ws + I.L.Bf);
  float *gcf = reinterpret_cast<float *>(I.ws + I.L.cf);
  float *gQf = reinterpret_cast<float *>(I.ws + I.L.Qf);
  float *gMf = reinterpret_cast<float *>(I.ws + I.L.Mf);
  float *gRf = reinterpret_cast<float *>(I.ws + I.L.Rf);

  // zero shared memory once (padding entries are read as zeros)
  {
    float4 *z4 = reinterpret_cast<float4 *>(smem_raw);
    for (int i = threadIdx.x; i < (int)(sizeof(SM) / 16); i += 64) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();

  if (warp == 1) {
    // ================= producer: FP64 stage data -> FP32 ring slots.
    // Each lane cp.async-copies its lane-strided elements of stage k - kDP + 1
    // into the FP64 ring while it converts stage k (its own elements, so no
    // barrier is needed between copy and conversion): kDP - 1 stages of loads
    // stay in flight.  The shared-memory offsets of a lane's elements do not
    // depend on the stage and are computed once.
    constexpr int DP = SM::kDP, S64 = SM::S64;
    constexpr int oQ = nn, oB = 2 * nn, oM = 2 * nn + nm, oR = 2 * nn + 2 * nm;
    constexpr int oq = oR + mmm, orr = oq + n, oc = orr + m;
    constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
    double *ring = reinterpret_cast<double *>(s.ring);
    int fA[CP], fAt[CP], fB[CB], fBt[CB], fBm[CB], fR[CR];
    bool upA[CP], upR[CR];
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int idx = lane + 32 * i, row = idx / n, col = idx - row * n;
      fA[i] = row * N4 + col;
      fAt[i] = col * N4 + row;
      upA[i] = row <= col;
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int idx = lane + 32 * i, row = idx / m, col = idx - row * m;
      fB[i] = row * M4 + col;
      fBt[i] = col * N4 + row;
      fBm[i] = row * M4 + col;
    }
#pragma unroll
    for (int i = 0; i < CR; ++i) {
      const int idx = lane + 32 * i, row = idx / m, col = idx - row * m;
      fR[i] = row * M4 + col;
      upR[i] = row <= col;
    }
    auto issue = [&](int k) {
      if (k >= 0) {
        double *d = ring + (size_t)((N - 1 - k) % DP) * S64;
        const double *A = I.A + (size_t)k * nn, *Q = I.Q + (size_t)k * nn;
        const double *B = I.B + (size_t)k * nm, *M = I.M + (size_t)k * nm;
        const double *R = I.R + (size_t)k * mmm;
#pragma unroll
        for (int i = 0; i < CP; ++i) {
          const int e = lane + 32 * i;
          if (e < nn) {
            cp_async8(d + e, A + e);
            cp_async8(d + oQ + e, Q + e);
          }
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const int e = lane + 32 * i;
          if (e < nm) {
            cp_async8(d + oB + e, B + e);
            cp_async8(d + oM + e, M + e);
          }
        }
#pragma unroll
        for (int i = 0; i < CR; ++i) {
          const int e = lane + 32 * i;
          if (e < mmm) cp_async8(d + oR + e, R + e);
        }
        if (SOLVE) {
          if (lane < n) {
            cp_async8(d + oq + lane, I.q + (size_t)k * n + lane);
            cp_async8(d + oc + lane, I.c + (size_t)(k + 1) * n + lane);
          }
          if (lane < m) cp_async8(d + orr + lane, I.r + (size_t)k * m + lane);
        }
      }
      cp_async_commit();  // one group per step, empty past the last stage
    };
#pragma unroll 1
    for (int j = 0; j < DP - 1; ++j) issue(N - 1 - j);
#pragma unroll 1
    for (int k = N - 1; k >= 0; --k) {
      issue(k - (DP - 1));
      cp_async_wait<DP - 1>();  // this lane's copies of stage k have landed
      const double *g = ring + (size_t)((N - 1 - k) % DP) * S64;
      const int sl = k & 1;
      if (k <= N - 3) nbar_sync(3 + sl);  // the consumer released this slot (stage k + 2)
      typename SM::Slot &d = s.slot[sl];
      float *gA = gAf + (size_t)k * nn, *gQ = gQf + (size_t)k * nn;
      float *gB = gBf + (size_t)k * nm, *gM = gMf + (size_t)k * nm, *gR = gRf + (size_t)k * mmm;
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const int idx = lane + 32 * i;
        if (idx < nn) {
          const float fa = f64_to_f32_rz(g[idx]);
          d.A[fA[i]] = fa;
          d.At[fAt[i]] = fa;
          gA[idx] = fa;
          const float fq = f64_to_f32_rz(g[oQ + idx]);
          if (upA[i]) {
            d.Q[fA[i]] = fq;
            d.Q[fAt[i]] = fq;
          }
          gQ[idx] = fq;
        }
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int idx = lane + 32 * i;
        if (idx < nm) {
          const float fb = f64_to_f32_rz(g[oB + idx]);
          d.B[fB[i]] = fb;
          d.Bt[fBt[i]] = fb;
          gB[idx] = fb;
          const float fm = f64_to_f32_rz(g[oM + idx]);
          d.M[fBm[i]] = fm;
          d.Mt[fBt[i]] = fm;
          gM[idx] = fm;
        }
      }
#pragma unroll
      for (int i = 0; i < CR; ++i) {
        const int idx = lane + 32 * i;
        if (idx < mmm) {
          const float fr = f64_to_f32_rz(g[oR + idx]);
          if (upR[i]) {
            const int row = fR[i] / M4, col = fR[i] - row * M4;
            d.R[row * M4 + col] = fr;
            d.R[col * M4 + row] = fr;
          }
          gR[idx] = fr;
        }
      }
      if (SOLVE) {
        if (lane < n) {
          d.q[lane] = f64_to_f32_rz(g[oq + lane]);
          const float fc = f64_to_f32_rz(g[oc + lane]);
          d.c[lane] = fc;
          gcf[(size_t)(k + 1) * n + lane] = fc;
        }
        if (lane < m) d.r[lane] = f64_to_f32_rz(g[orr + lane]);
      }
      nbar_arrive(1 + sl);  // slot full
    }
    cp_async_wait<0>();
    __syncthreads();  // pairs with the consumer's after the backward sweep
    return;
  }

  // ================= consumer (warp 0)
  float *gW = reinterpret_cast<float *>(I.ws + I.L.W);
  float *gK = reinterpret_cast<float *>(I.ws + I.L.K);
  float *gGi = reinterpret_cast<float *>(I.ws + I.L.Gi);
  float *gkv = reinterpret_cast<float *>(I.ws + I.L.kv);
  float *gpv = reinterpret_cast<float *>(I.ws + I.L.pv);
  float *gG = reinterpret_cast<float *>(I.ws + I.L.G);
  float *gPc = reinterpret_cast<float *>(I.ws + I.L.Pc);
  uint8_t *pend = reinterpret_cast<uint8_t *>(I.ws + I.L.pend);
  const float delta = (float)I.delta;
  const float delta_up = __double2float_ru(I.delta), delta_dn = __double2float_rd(I.delta);

  // identity rows, P_N = Q_N (upper triangle mirrored), p_N = q_N
  if (lane < n) s.Id[lane * N4 + lane] = 1.f;
  if (lane < m) s.unit[lane][BL + lane] = 1.f;
  {
    const double *QN = I.Q + (size_t)N * nn;
    for (int e = lane; e < nn; e += 32) {
      const int i = e / n, j = e - i * n;
      s.Ps[i * N4 + j] = f64_to_f32_rz(__ldg(QN + min(i, j) * n + max(i, j)));
    }
    if (SOLVE && lane < n) {
      const float v = f64_to_f32_rz(__ldg(I.q + (size_t)N * n + lane));
      s.p[lane] = v;
      gpv[(size_t)N * n + lane] = v;
    }
  }
  __syncwarp();

  // lane roles
  const bool xlane = lane < n;                        // X column (and P column)
  const bool alane = lane >= XL && lane < BL;         // A column j = lane - n
  const bool blane = lane >= BL && lane < RL;         // B column t = lane - 2n
  const bool rlane = lane == RL;                      // right-hand side
  const float sgn = xlane ? -1.f : 1.f;

  // P_cc of the P column held by lane c (the symmetric P in s.Ps for the
  // stage being certified)
  auto diag_of = [&](const float2 (&)[H2]) { return s.Ps[lane * N4 + lane]; };

  // Certificate bit0 of I + delta P held in pcol (column lane of P, lanes <
  // n); a stage the Gershgorin margin test does not prove stores P and
  // is left pending.  Returns the tentative bit (always 1).
  auto state_cert = [&](const float2 (&pcol)[H2], int st) {
    bool pass = true;
    if (xlane) {
      // off-diagonal sum rounded up: all |P_ic| summed up, then |P_cc| taken
      // off with upward rounding (an upper bound of the exact sum)
      float tot = 0.f;
#pragma unroll
      for (int i = 0; i < n; ++i) tot = __fadd_ru(tot, fabsf(el(pcol[i / 2], i & 1)));
      const float diag = diag_of(pcol);
      pass = gershgorin_row_margin(diag, __fsub_ru(tot, fabsf(diag)), delta_dn, delta_up,
                                   kMarginTau);
    }
    const bool all = __all_sync(0xffffffffu, pass);
    if (!all && xlane) {
      float *dst = gPc + (size_t)st * nn + lane * n;
#pragma unroll
      for (int q = 0; q < H2; ++q) reinterpret_cast<float2 *>(dst)[q] = pcol[q];
    }
    if (lane == 0) pend[st] = all ? 0 : 1;
  };

  // Gauss-Jordan over the state pivots (blocks {2b, 2b+1} of the top rows):
  // col = this lane's tableau column, pcol = its P column (top rows).
  auto state_gj = [&](float2 (&col)[R2], float2 (&pcol)[H2]) {
#pragma unroll
    for (int blk = 0; blk < H2; ++blk) {
      const int j = 2 * blk;
      if (lane == j || lane == j + 1) st_seg<R2>(s.bc[blk & 1][lane - j], col);
      __syncwarp();
      float2 c0[R2], c1[R2];
      ld_seg<R2, 0, R2>(s.bc[blk & 1][0], c0);
      ld_seg<R2, 0, R2>(s.bc[blk & 1][1], c1);
      const float d00 = c0[blk].x, d10 = c0[blk].y, d01 = c1[blk].x, d11 = c1[blk].y;
      const float rd = recip_pivot(fmaf(d00, d11, -d01 * d10));
      {
        const float a0 = col[blk].x, a1 = col[blk].y;
        const float n0 = fmaf(d11, a0, -d01 * a1) * rd;
        const float n1 = fmaf(d00, a1, -d10 * a0) * rd;
        const float2 m0 = bcast2(-n0), m1 = bcast2(-n1);
#pragma unroll
        for (int q = 0; q < R2; ++q)
          if (q != blk) col[q] = fma2(c1[q], m1, fma2(c0[q], m0, col[q]));
        col[blk] = make_float2(n0, n1);
      }
      {
        const float a0 = pcol[blk].x, a1 = pcol[blk].y;
        const float n0 = fmaf(d11, a0, -d01 * a1) * rd;
        const float n1 = fmaf(d00, a1, -d10 * a0) * rd;
        const float2 m0 = bcast2(-n0), m1 = bcast2(-n1);
#pragma unroll
        for (int q = 0; q < H2; ++q)
          if (q != blk) pcol[q] = fma2(c1[q], m1, fma2(c0[q], m0, pcol[q]));
        pcol[blk] = make_float2(n0, n1);
      }
    }
  };

  // W = P (I + delta P)^{-1} from the P columns after the elimination,
  // stored exactly symmetric: W[c][i] = computed entry max(i,c) of column
  // min(i,c) (the symmetric W makes the FP32 solve about as accurate as the
  // FP32 data allow, so that one refinement pass suffices)
  auto store_w = [&](const float2 (&pcol)[H2], float *dst) {
    if (xlane) st_seg<H2>(s.Wt + lane * N4, pcol);
    __syncwarp();
    if (xlane) {
      float2 w[H2];
#pragma unroll
      for (int q = 0; q < H2; ++q) {
        const int i0 = 2 * q, i1 = 2 * q + 1;
        w[q] = make_float2(s.Wt[min(i0, lane) * N4 + max(i0, lane)],
                           s.Wt[min(i1, lane) * N4 + max(i1, lane)]);
      }
#pragma unroll
      for (int q = 0; q < H2; ++q) reinterpret_cast<float2 *>(dst + lane * n)[q] = w[q];
    }
  };

  for (int k = N - 1; k >= 0; --k) {
    const int sl = k & 1;
    nbar_sync(1 + sl);  // stage k's data is in the slot
    const typename SM::Slot &d = s.slot[sl];
    // ---- tableau of stage k
    float2 col[R2], pcol[H2];
    {
      // top rows: P y with y = e_c (X lanes), A[:, j], B[:, t], c_{k+1}
      const float *yp = xlane ? s.Id + lane * N4
                      : alane ? d.At + (lane - XL) * N4
                      : blane ? d.Bt + (lane - BL) * N4
                      : rlane ? d.c : s.zero;
      float2 yv[H2];
      ld_seg<H2, 0, H2>(yp, yv);
      float2 acc[H2];
#pragma unroll
      for (int q = 0; q < H2; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        float2 pr[H2];
        ld_seg<H2, 0, H2>(s.Ps + l * N4, pr);
        const float2 yb = bcast2(el(yv[l / 2], l & 1));
#pragma unroll
        for (int q = 0; q < H2; ++q) acc[q] = fma2(pr[q], yb, acc[q]);
      }
      // this lane's P column (X lanes: P e_c), the rhs adds p_{k+1}
      float2 pv[H2];
      ld_seg<H2, 0, H2>(rlane ? s.p : s.zero, pv);
      const float2 dl2 = bcast2(delta);
      // X lanes: yv is row c of the identity, so col = e_c + delta P[:, c]
#pragma unroll
      for (int q = 0; q < H2; ++q) {
        pcol[q] = acc[q];
        col[q] = xlane ? fma2(dl2, acc[q], yv[q]) : add2(acc[q], pv[q]);
      }
      // lower rows: -[A; B]^T rows (X lanes), [Q M; M^T R] columns, [q; r]
      const float *xp = xlane ? d.A + lane * N4
                      : alane ? d.Q + (lane - XL) * N4
                      : blane ? d.Mt + (lane - BL) * N4
                      : rlane ? d.q : s.zero;
      const float *up = xlane ? d.B + lane * M4
                      : alane ? d.M + (lane - XL) * M4
                      : blane ? d.R + (lane - BL) * M4
                      : rlane ? d.r : s.zero;
      ld_seg<H2, H2, R2>(xp, col);
      ld_seg<U2, n, R2>(up, col);
      const float2 sg = bcast2(sgn);
#pragma unroll
      for (int q = H2; q < R2; ++q) col[q] = mul2(col[q], sg);
    }
    // ---- certificate of I + delta P_{k+1}
    state_cert(pcol, k + 1);
    // ---- state pivots
    state_gj(col, pcol);
    store_w(pcol, gW + (size_t)(k + 1) * nn);
    // G_k (u rows of the B columns), then identity columns for G_k^{-1}
    if (blane) {
      const int t = lane - BL;
#pragma unroll
      for (int i = 0; i < m; ++i) gG[(size_t)k * mmm + t * m + i] = el(col[n + i / 2], i & 1);
    }
    if (lane < m) ld_seg<R2, 0, R2>(s.unit[lane], col);
    // the stage's data has been read: release the slot
    if (k >= 2) nbar_arrive(3 + sl);
    // ---- control pivots (scalar, in order)
#pragma unroll
    for (int t = 0; t < m; ++t) {
      const int pq = n + t / 2, ph = t & 1;
      if (lane == BL + t) st_seg<R2>(s.ub[t & 1], col);
      __syncwarp();
      float2 pc[R2];
      ld_seg<R2, 0, R2>(s.ub[t & 1], pc);
      const float rp = recip_pivot(el(pc[pq], ph));
      const float nv = el(col[pq], ph) * rp;
      const float2 mn = bcast2(-nv);
      // the top rows are no longer needed: only the x and u rows are updated
#pragma unroll
      for (int q = H2; q < R2; ++q) col[q] = fma2(pc[q], mn, col[q]);
      set_el(col[pq], ph, nv);
    }
    // ---- outputs of stage k
    if (alane) {
      const int j = lane - XL;
#pragma unroll
      for (int t = 0; t < m; ++t) gK[(size_t)k * nm + t * n + j] = -el(col[n + t / 2], t & 1);
    } else if (lane < m) {
#pragma unroll
      for (int i = 0; i < m; ++i) gGi[(size_t)k * mmm + lane * m + i] = el(col[n + i / 2], i & 1);
    } else if (SOLVE && rlane) {
      float *pk = gpv + (size_t)k * n;
#pragma unroll
      for (int q = 0; q < H2; ++q) reinterpret_cast<float2 *>(pk)[q] = col[H2 + q];
#pragma unroll
      for (int t = 0; t < m; ++t) gkv[(size_t)k * m + t] = -el(col[n + t / 2], t & 1);
    }
    if (lane == 0) I.flags[k + 1] = (uint8_t)(1 | ((k + 1 == N) ? 2 : 0));
    // P_k (exactly symmetric) and p_k for the next stage
    __syncwarp();
    if (alane) {
      const int j = lane - XL;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        if (i >= j) {
          const float w = el(col[H2 + i / 2], i & 1);
          s.Ps[i * N4 + j] = w;
          s.Ps[j * N4 + i] = w;
        }
      }
    } else if (SOLVE && rlane) {
#pragma unroll
      for (int q = 0; q < H2; ++q) reinterpret_cast<float2 *>(s.p)[q] = col[H2 + q];
    }
    __syncwarp();
  }

  // ---- initial-state pivot: W_0 from [I + delta P_0 | P_0]
  {
    float2 col[R2], pcol[H2];
    float2 pr[H2];
    ld_seg<H2, 0, H2>(xlane ? s.Ps + lane * N4 : s.zero, pr);
#pragma unroll
    for (int q = 0; q < H2; ++q) {
      pcol[q] = pr[q];
      col[q] = xlane ? fma2(bcast2(delta), pr[q], make_float2(2 * q == lane ? 1.f : 0.f, 2 * q + 1 == lane ? 1.f : 0.f))
                     : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = H2; q < R2; ++q) col[q] = make_float2(0.f, 0.f);
    state_cert(pcol, 0);
    state_gj(col, pcol);
    store_w(pcol, gW);
    if (lane == 0) {
      I.flags[0] = 1;
      const int32_t st = RLQR_OK;
      I.st->pivot_status = st;
      I.st->escalated = 0;
      I.st->iters = 0;
      I.st->converged = 0;
      I.st->rel = 0.0;
      if (a.status) a.status[b] = st;
    }
  }
  __syncthreads();  // every global store of the sweep is visible to the forward pass
  if constexpr (!SOLVE) return;

  // ---- forward rollout (lane = row)
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  if (xlane) {
    const float c0 = f64_to_f32_rz(__ldg(I.c + lane));
    gcf[lane] = c0;
    s.v[lane] = fmaf(-delta, s.p[lane], c0);
  }
  __syncwarp();
  if (xlane) {
    float2 wr[H2], vr[H2];
    ld_seg<H2, 0, H2>(gW + lane * n, wr);  // written by this warp above
    ld_seg<H2, 0, H2>(s.v, vr);
    const float t = dot2<n>(wr, vr);
    const float xv = fmaf(-delta, t, s.v[lane]), yv = t + s.p[lane];
    s.x[lane] = xv;
    I.x[lane] = widen(xv);
    I.y[lane] = widen(yv);
  }
  // The factor rows of stage k (K_k, A_k, B_k, W_{k+1}, c_{k+1}, p_{k+1},
  // k_k) travel by cp.async through a ring of kDF stages in shared memory,
  // kDF - 1 stages ahead of the rollout (the ring reuses the producer's
  // staging area, idle since the sweep's end).
  using FS = typename SM::FSlot;
  constexpr int DF = SM::kDF;
  FS *fring = reinterpret_cast<FS *>(s.ring);
  // this lane's elements of a stage (lane-strided) and their padded
  // shared-memory positions, the same for every stage
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32;
  int dK[CB], dA[CP], dB[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int e = lane + 32 * i, t = e / n, c = e - t * n, r = e / m, cc = e - r * m;
    dK[i] = t * N4 + c;
    dB[i] = r * M4 + cc;
  }
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    const int e = lane + 32 * i, r = e / n, c = e - r * n;
    dA[i] = r * N4 + c;
  }
  auto issue = [&](int k) {
    if (k < N) {
      FS &f = fring[k % DF];
      const float *K = gK + (size_t)k * nm, *A = gAf + (size_t)k * nn;
      const float *W = gW + (size_t)(k + 1) * nn, *B = gBf + (size_t)k * nm;
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int e = lane + 32 * i;
        if (e < nm) {
          cp_async4(&f.K[dK[i]], K + e);
          cp_async4(&f.B[dB[i]], B + e);
        }
      }
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const int e = lane + 32 * i;
        if (e < nn) {
          cp_async4(&f.A[dA[i]], A + e);
          cp_async4(&f.W[dA[i]], W + e);
        }
      }
      if (lane < n) {
        cp_async4(&f.c[lane], gcf + (size_t)(k + 1) * n + lane);
        cp_async4(&f.p[lane], gpv + (size_t)(k + 1) * n + lane);
      }
      if (lane < m) cp_async4(&f.k[lane], gkv + (size_t)k * m + lane);
    }
    cp_async_commit();
  };
  // the padding entries of the B rows are read as zeros
  for (int e = lane; e < DF * (int)sizeof(FS) / 4; e += 32) reinterpret_cast<float *>(fring)[e] = 0.f;
  __syncwarp();
  for (int j = 0; j < DF - 1; ++j) issue(j);
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    issue(k + DF - 1);
    cp_async_wait<DF - 1>();
    __syncwarp();  // every lane's copies of stage k are in
    const FS &f = fring[k % DF];
    float2 xr[H2];
    ld_seg<H2, 0, H2>(s.x, xr);
    // u_k = K_k x_k + k_k
    if (lane < m) {
      float2 kr[H2];
      ld_seg<H2, 0, H2>(f.K + lane * N4, kr);
      const float t = dot2<n>(kr, xr) + f.k[lane];
      s.u[lane] = t;
      I.u[(size_t)k * m + lane] = widen(t);
    }
    __syncwarp();
    // v = A x + B u + c_{k+1} - delta p_{k+1}
    float2 ur[U2];
    ld_seg<U2, 0, U2>(s.u, ur);
    float vv = 0.f, pk = 0.f;
    if (xlane) {
      float2 ar[H2], br[U2];
      ld_seg<H2, 0, H2>(f.A + lane * N4, ar);
      ld_seg<U2, 0, U2>(f.B + lane * M4, br);
      float2 acc = mul2(ar[0], xr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], xr[q], acc);
#pragma unroll
      for (int q = 0; q < U2; ++q) acc = fma2(br[q], ur[q], acc);
      pk = f.p[lane];
      vv = acc.x + acc.y + fmaf(-delta, pk, f.c[lane]);
      s.v[lane] = vv;
    }
    __syncwarp();
    // x_{k+1} = v - delta W v, y_{k+1} = W v + p_{k+1}
    float2 vr[H2];
    ld_seg<H2, 0, H2>(s.v, vr);
    if (xlane) {
      float2 wr[H2];
      ld_seg<H2, 0, H2>(f.W + lane * N4, wr);
      const float t = dot2<n>(wr, vr);
      const float xv = fmaf(-delta, t, vv), yv = t + pk;
      s.x[lane] = xv;
      I.x[(size_t)(k + 1) * n + lane] = widen(xv);
      I.y[(size_t)(k + 1) * n + lane] = widen(yv);
    }
    __syncwarp();  // the slot is read: the next issue may refill it
  }
  cp_async_wait<0>();
}

}  // namespace rlqr

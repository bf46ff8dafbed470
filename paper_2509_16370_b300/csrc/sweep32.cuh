// sweep32.cuh -- the FP32 Riccati sweep of the mixed-precision path, one warp
// per instance, for small even dimensions (n, m even, 2n <= 32, n + 2m + 2 <= 32,
// m <= 8): the shape of batched trajectory-optimization subproblems.
//
// Recursion: Theorem main-seq-theorem and eq. value-fn-formulas (backward),
// Corollary p-recurrence (vectors), eq. recover-x0 / control-law / recover-x
// (forward), with the same readings as seq.cuh.  Organisation for B300:
//  * State pivot: Gauss-Jordan on [I + delta P | P] with 2x2 block pivots.
//    Lane c owns column c in registers.  The two pivot columns of a block go
//    through shared memory (vector store, warp sync, vector broadcast
//    loads): n/2 broadcast rounds instead of n rounds of n shuffles (a
//    shuffle issues about once per 4.5 cycles per warp on B300).  The left
//    block ends as I and the right block as W = (I + delta P)^{-1} P.
//  * Products: lane c' forms column c' of W [A | B | v] (v = c - delta p;
//    rows of W broadcast from shared memory), keeps it in registers and then
//    forms column c' of [A | B]^T (W [A | B | v]).  So P' = Q + A^T W A,
//    H = M^T + B^T W A, G = R + B^T W B, p' = q + A^T g and h = r + B^T g
//    (g = p + W v) end up in the lanes that own those columns in the control
//    elimination, with no shared-memory round trip in between.
//  * Control pivot: every lane holds G in registers and runs the scalar
//    Gauss-Jordan elimination of G on its own column of [H | h | I]: lanes
//    c < n get K[:, c] = -G^{-1} H[:, c], lane n+m gets k = -G^{-1} h and
//    lanes n+m+1+t column t of G^{-1} (an elimination per right-hand side,
//    not a product with an explicit inverse).
//  * W and P = P' + H^T K are made exactly symmetric (lower triangle of the
//    computed columns, mirrored) in one shared-memory round trip each; P
//    stays in registers for the next stage's elimination.
//  * Pairs of FP32 values use fma/mul/add .f32x2.  The next stage's data is
//    converted and committed to shared memory while the in-register control
//    elimination runs.
// Certificate: FP32 Gershgorin proof with directed rounding for I + delta P
// (FP64 LDL^T when the proof fails); G_i is stored for the FP64 pass.  The
// sweep also writes FP32 copies of A_i, B_i, Q_i, M_i, R_i (and c_i when it
// solves), which the forward pass and the refinement read instead of
// converting the FP64 data again.
#pragma once

#include "common.cuh"

namespace rlqr {

template <int NX, int NU>
constexpr bool sweep32_fits() {
  return NX % 2 == 0 && NU % 2 == 0 && NX >= 2 && NU >= 2 && 2 * NX <= 32 &&
         NX + 2 * NU + 2 <= 32 && NU <= 8;
}

template <int NX, int NU>
struct Sw32 {
  static constexpr int n = NX, m = NU;
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4;  // row strides
  alignas(16) float A[NX * N4];
  alignas(16) float B[NX * M4];
  alignas(16) float Q[NX * N4];   // full symmetric
  alignas(16) float M[NX * M4];
  alignas(16) float R[NU * M4];   // full symmetric
  alignas(16) float q[N4];
  alignas(16) float c[N4];
  alignas(16) float r[M4];
  alignas(16) float Wc[NX * N4];  // row l = computed column l of W
  alignas(16) float W[NX * N4];   // symmetric W (row l = column l)
  alignas(16) float Pt[NX * N4];  // row l = computed column l of the new P
  alignas(16) float bc[2][2][N4]; // pivot-column broadcast (ping-pong)
  alignas(16) float G[NU * M4];   // row t = column t of G
  alignas(16) float H[NU * N4];   // row t of H
  alignas(16) float K[NU * N4];   // forward pass: K_k rows
  alignas(16) float kk[M4];
  alignas(16) float p[N4];
  alignas(16) float v[N4];
  alignas(16) float x[N4];
  alignas(16) float u[M4];
  double S64[NX * NX];            // FP64 LDL^T of I + delta P (certificate fallback)
  // sizes of chunk16_size: the forward rollout's ring of kFwdSlots stages,
  // each A_k, W_{k+1}, B_k, K_k, c_{k+1}, p_{k+1}, k_k back to back
  static constexpr int kFwdSlot = 2 * NX * NX + 2 * NX * NU + 2 * NX + NU;
  static constexpr int kFwdSlots = 4;
  alignas(16) float fring[chunk16_size(NX, NU) ? kFwdSlots * kFwdSlot : 4];
};

// r[q] = (p[2q], p[2q+1]); 16-byte vector loads when L % 4 == 0 (rows are
// padded to 4 floats), 8-byte ones otherwise.
template <int L>
__device__ __forceinline__ void lds_row2(const float *p, float2 (&r)[L / 2]) {
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int q = 0; q < L / 4; ++q) {
      const float4 t = reinterpret_cast<const float4 *>(p)[q];
      r[2 * q] = make_float2(t.x, t.y);
      r[2 * q + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int q = 0; q < L / 2; ++q) r[q] = reinterpret_cast<const float2 *>(p)[q];
  }
}

template <int L>
__device__ __forceinline__ void st_row2(float *p, const float2 (&r)[L / 2]) {
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int q = 0; q < L / 4; ++q)
      reinterpret_cast<float4 *>(p)[q] = make_float4(r[2 * q].x, r[2 * q].y, r[2 * q + 1].x, r[2 * q + 1].y);
  } else {
#pragma unroll
    for (int q = 0; q < L / 2; ++q) reinterpret_cast<float2 *>(p)[q] = r[q];
  }
}

__device__ __forceinline__ float el(const float2 &p, int h) { return h ? p.y : p.x; }

// Dot product of two packed rows of length L: pairwise FMAs, then one add.
template <int L>
__device__ __forceinline__ float dot2(const float2 (&a)[L / 2], const float2 (&b)[L / 2]) {
  float2 acc = mul2(a[0], b[0]);
#pragma unroll
  for (int q = 1; q < L / 2; ++q) acc = fma2(a[q], b[q], acc);
  return acc.x + acc.y;
}

// Commit a lane-strided FP64 segment of a row-major (len / L) x L matrix to
// shared memory with row stride LD (FP32, truncated), optionally also to a
// contiguous FP32 global copy.
template <int CNT, int L, int LD>
__device__ __forceinline__ void commit_rows(const LaneSeg<double, CNT> &pf, int len, int lane,
                                            float *dst, float *gdst) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < len) {
      const float f = f64_to_f32_rz(pf.v[i]);
      if constexpr (L == LD) {
        dst[idx] = f;
      } else {
        const int row = idx / L;
        dst[row * LD + idx - row * L] = f;
      }
      if (gdst) gdst[idx] = f;
    }
  }
}

// Same for an L x L symmetric matrix given by its upper triangle (mirrored);
// the optional global copy receives every element as given.
template <int CNT, int L, int LD>
__device__ __forceinline__ void commit_sym(const LaneSeg<double, CNT> &pf, int lane, float *dst,
                                           float *gdst) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < L * L) {
      const int row = idx / L, col = idx - row * L;
      const float f = f64_to_f32_rz(pf.v[i]);
      if (row <= col) {
        dst[row * LD + col] = f;
        dst[col * LD + row] = f;
      }
      if (gdst) gdst[idx] = f;
    }
  }
}

// The sweep of instance b by one warp (lane = its lane) in the shared memory
// at smem (a Sw32<NX, NU>); the body of k_sweep32 and of the persistent
// ragged sweep.
template <int NX, int NU, bool SOLVE>
__device__ __forceinline__ void sweep32_body(const BatchArgs &a, int b, unsigned char *smem,
                                             int lane) {
  static_assert(sweep32_fits<NX, NU>(), "dimensions outside the FP32 warp sweep");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int H2 = n / 2, M2 = m / 2;
  using SM = Sw32<NX, NU>;
  constexpr int N4 = SM::N4, M4 = SM::M4;
  constexpr int VL = n + m;  // the lane of the vector recursion (p, g, h, k)
  SM &s = *reinterpret_cast<SM *>(smem);
  const Inst I = get_inst(a, b);
  const int N = I.N;
  const float delta = (float)I.delta;
  const float delta_up = __double2float_ru(I.delta), delta_dn = __double2float_rd(I.delta);
  const float2 delta2 = bcast2(delta);
  float *gW = reinterpret_cast<float *>(I.ws + I.L.W);
  float *gK = reinterpret_cast<float *>(I.ws + I.L.K);
  float *gGi = reinterpret_cast<float *>(I.ws + I.L.Gi);
  float *gkv = reinterpret_cast<float *>(I.ws + I.L.kv);
  float *gpv = reinterpret_cast<float *>(I.ws + I.L.pv);
  float *gG = reinterpret_cast<float *>(I.ws + I.L.G);
  float *gAf = reinterpret_cast<float *>(I.ws + I.L.Af);
  float *gBf = reinterpret_cast<float *>(I.ws + I.L.Bf);
  float *gcf = reinterpret_cast<float *>(I.ws + I.L.cf);
  float *gQf = reinterpret_cast<float *>(I.ws + I.L.Qf);
  float *gMf = reinterpret_cast<float *>(I.ws + I.L.Mf);
  float *gRf = reinterpret_cast<float *>(I.ws + I.L.Rf);

  // ---- one stage's FP64 data, prefetched into registers (lane-strided)
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
  auto commit = [&](int k) {
    commit_rows<CP, n, N4>(pfA, nn, lane, s.A, gAf + (size_t)k * nn);
    commit_sym<CP, n, N4>(pfQ, lane, s.Q, gQf + (size_t)k * nn);
    commit_rows<CB, m, M4>(pfB, nm, lane, s.B, gBf + (size_t)k * nm);
    commit_rows<CB, m, M4>(pfM, nm, lane, s.M, gMf + (size_t)k * nm);
    commit_sym<CR, m, M4>(pfR, lane, s.R, gRf + (size_t)k * mmm);
    if (SOLVE) {
      commit_rows<CV, n, N4>(pfq, n, lane, s.q, nullptr);
      commit_rows<CV, n, N4>(pfc, n, lane, s.c, gcf + (size_t)(k + 1) * n);
      commit_rows<CM, m, M4>(pfr, m, lane, s.r, nullptr);
    }
  };

  // ---- terminal stage: P_N = Q_N (upper triangle), p_N = q_N.  Pc holds
  // column (lane mod n) of the current P, exactly symmetric.
  float2 Pc[H2];
  {
    const int c = lane % n;
    const double *QN = I.Q + (size_t)N * nn;
#pragma unroll
    for (int q = 0; q < H2; ++q) {
      const int i0 = 2 * q, i1 = 2 * q + 1;
      Pc[q] = make_float2(f64_to_f32_rz(__ldg(QN + min(i0, c) * n + max(i0, c))),
                          f64_to_f32_rz(__ldg(QN + min(i1, c) * n + max(i1, c))));
    }
  }
  float2 pv[H2];  // lane VL: p of the stage after the current one
#pragma unroll
  for (int q = 0; q < H2; ++q) pv[q] = make_float2(0.f, 0.f);
  if (SOLVE && lane == VL) {
#pragma unroll
    for (int q = 0; q < H2; ++q)
      pv[q] = make_float2(f64_to_f32_rz(__ldg(I.q + (size_t)N * n + 2 * q)),
                          f64_to_f32_rz(__ldg(I.q + (size_t)N * n + 2 * q + 1)));
    st_row2<n>(gpv + (size_t)N * n, pv);
  }
  prefetch(N - 1);
  commit(N - 1);
  if (N > 1) prefetch(N - 2);
  __syncwarp();

  bool notpd = false, singular = false;

  // State pivot of the P held in Pc: W into s.W (rows = computed columns) and
  // gWk; returns bit0 of the stage's flag.
  auto state_pivot = [&](float *gWk, bool &sing) -> int {
    float2 v2[H2];  // column `lane` of [I + delta P | P]
#pragma unroll
    for (int q = 0; q < H2; ++q) {
      if (lane < n)
        v2[q] = fma2(delta2, Pc[q], make_float2(2 * q == lane ? 1.f : 0.f, 2 * q + 1 == lane ? 1.f : 0.f));
      else
        v2[q] = Pc[q];
    }
    // Gershgorin proof, with the certificate's margin, that I + delta P is PD
    // (lanes n..2n-1 hold column c = row c of P).  Otherwise the FP64 LDL^T
    // of I + delta P - tau D (D = diag, floored at 2^-24 max |D|) proves it;
    // else a non-positive pivot of I + delta P + tau D proves it not PD
    // (bit 0); else the instance is escalated to the FP64 recursion (`sing`;
    // the bit stays 1 until that decides).
    // (every lane runs the test on its column lane mod n of P; only lanes
    // n..2n-1 count, so the warp takes no divergent branch)
    int bit = 1;
    bool pass = true;
    {
      const int c = lane % n;
      float off = 0.f, diag = 0.f;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        const float val = el(Pc[i / 2], i & 1);
        diag = (i == c) ? val : diag;
        off = (i == c) ? off : __fadd_ru(off, fabsf(val));
      }
      const bool g = gershgorin_row_margin(diag, off, delta_dn, delta_up, kMarginTau);
      pass = (lane >= n && lane < 2 * n) ? g : true;
    }
    if (!__all_sync(0xffffffffu, pass)) {
      // largest diagonal magnitude of I + delta P (shift floor)
      double dm = 0.0;
      if (lane >= n && lane < 2 * n)
        dm = fabs(1.0 + I.delta * widen(el(Pc[(lane - n) / 2], (lane - n) & 1)));
      for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
      int decided = 0;
      for (int pass2 = 0; pass2 < 2 && !decided; ++pass2) {
        const double sg = pass2 == 0 ? -(double)kMarginTau : (double)kMarginTau;
        __syncwarp();
        if (lane >= n && lane < 2 * n) {
          const int c = lane - n;
#pragma unroll
          for (int i = 0; i < n; ++i) {
            double v = (i == c ? 1.0 : 0.0) + I.delta * widen(el(Pc[i / 2], i & 1));
            if (i == c) v += sg * fmax(fabs(v), 0x1p-24 * dm);
            s.S64[i * n + c] = v;
          }
        }
        __syncwarp();
        bool pos = true, fin = true;
        for (int j = 0; j < n; ++j) {
          const double d = s.S64[j * n + j];
          if (!isfinite(d)) fin = false;
          if (!(d > 0.0)) pos = false;
          if (!pos || !fin) break;  // uniform over the warp
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
        if (!fin) break;
        if (pass2 == 0 && pos) decided = 1;                // PD with margin
        if (pass2 == 1 && !pos) { decided = 1; bit = 0; }  // not PD with margin
      }
      if (!decided) sing = true;  // escalate
    }
    // block Gauss-Jordan, pivot blocks {j, j+1}
#pragma unroll
    for (int blk = 0; blk < H2; ++blk) {
      const int j = 2 * blk;
      if (lane == j || lane == j + 1) st_row2<n>(s.bc[blk & 1][lane - j], v2);
      __syncwarp();
      float2 c0[H2], c1[H2];
      lds_row2<n>(s.bc[blk & 1][0], c0);
      lds_row2<n>(s.bc[blk & 1][1], c1);
      const float d00 = c0[blk].x, d01 = c1[blk].x, d10 = c0[blk].y, d11 = c1[blk].y;
      const float rd = recip_pivot(fmaf(d00, d11, -d01 * d10));
      const float a0 = v2[blk].x, a1 = v2[blk].y;
      const float nj = fmaf(d11, a0, -d01 * a1) * rd;
      const float nj1 = fmaf(d00, a1, -d10 * a0) * rd;
      const float2 mnj = bcast2(-nj), mnj1 = bcast2(-nj1);
#pragma unroll
      for (int q = 0; q < H2; ++q)
        if (q != blk) v2[q] = fma2(c1[q], mnj1, fma2(c0[q], mnj, v2[q]));
      v2[blk] = make_float2(nj, nj1);
    }
    // exact symmetry: W[i][c] = computed entry max(i,c) of column min(i,c)
    if (lane >= n && lane < 2 * n) st_row2<n>(s.Wc + (lane - n) * N4, v2);
    __syncwarp();
    {  // every lane gathers a column (lane mod n); lanes n..2n-1 store theirs
      const int c = lane % n;
#pragma unroll
      for (int q = 0; q < H2; ++q) {
        const int i0 = 2 * q, i1 = 2 * q + 1;
        v2[q] = make_float2(s.Wc[min(i0, c) * N4 + max(i0, c)], s.Wc[min(i1, c) * N4 + max(i1, c)]);
      }
      if (lane >= n && lane < 2 * n) {
        st_row2<n>(s.W + c * N4, v2);
        st_row2<n>(gWk + c * n, v2);
      }
    }
    __syncwarp();
    return bit;
  };

  for (int k = N - 1; k >= 0; --k) {
    // v = c_{k+1} - delta p_{k+1} (lane VL), read by phase (a); every lane
    // forms it (pv is zero off lane VL), lane VL stores it
    if (SOLVE) {
      float2 cr[H2];
      lds_row2<n>(s.c, cr);
#pragma unroll
      for (int q = 0; q < H2; ++q) cr[q] = fma2(bcast2(-delta), pv[q], cr[q]);
      if (lane == VL) st_row2<n>(s.v, cr);
    }
    bool sing = false;
    const int bit0 = state_pivot(gW + (size_t)(k + 1) * nn, sing);

    // ---- (a) column lane of W [A | B | v]; lane VL then adds p: g
    float2 wz[H2];
    {
      const float *yp = lane < n ? s.A + lane : (lane < n + m ? s.B + (lane - n) : s.v);
      const int ys = lane < n ? N4 : (lane < n + m ? M4 : 1);
#pragma unroll
      for (int q = 0; q < H2; ++q) wz[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        float2 wr[H2];
        lds_row2<n>(s.W + l * N4, wr);
        const float2 y = bcast2(yp[l * ys]);
#pragma unroll
        for (int q = 0; q < H2; ++q) wz[q] = fma2(wr[q], y, wz[q]);
      }
      if (SOLVE) {  // lane VL adds p (pv is zero elsewhere)
#pragma unroll
        for (int q = 0; q < H2; ++q) wz[q] = add2(wz[q], pv[q]);
      }
    }

    // ---- (b) column lane of [A | B]^T (W [A | B | v]) plus the data:
    //      lanes c < n: fa = P'[:, c], fb = H[:, c];  lanes n + t: fb = G[:, t];
    //      lane VL: fa = p', fb = h
    float2 fa[H2], fb[M2];
    {
#pragma unroll
      for (int q = 0; q < H2; ++q) fa[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < M2; ++q) fb[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const float2 w = bcast2(el(wz[l / 2], l & 1));
        float2 ar[H2], br[M2];
        lds_row2<n>(s.A + l * N4, ar);
        lds_row2<m>(s.B + l * M4, br);
#pragma unroll
        for (int q = 0; q < H2; ++q) fa[q] = fma2(ar[q], w, fa[q]);
#pragma unroll
        for (int q = 0; q < M2; ++q) fb[q] = fma2(br[q], w, fb[q]);
      }
      const float *qa = lane < n ? s.Q + lane * N4 : (lane < n + m ? s.Q : s.q);
      const float *qb = lane < n ? s.M + lane * M4 : (lane < n + m ? s.R + (lane - n) * M4 : s.r);
      float2 ta[H2], tb[M2];
      lds_row2<n>(qa, ta);
      lds_row2<m>(qb, tb);
#pragma unroll
      for (int q = 0; q < H2; ++q) fa[q] = add2(fa[q], ta[q]);
#pragma unroll
      for (int q = 0; q < M2; ++q) fb[q] = add2(fb[q], tb[q]);
      if (!SOLVE) {
#pragma unroll
        for (int q = 0; q < M2; ++q) fb[q] = lane == VL ? make_float2(0.f, 0.f) : fb[q];
      }
    }

    // ---- control pivot: G in every lane; each lane eliminates its own
    //      right-hand side: H[:, c] (c < n), h (VL), e_t (VL + 1 + t)
    if (lane >= n && lane < n + m) st_row2<m>(s.G + (lane - n) * M4, fb);
    __syncwarp();
    float g[m][m], rhs[m];
#pragma unroll
    for (int t = 0; t < m; ++t) {
      float2 gr[M2];
      lds_row2<m>(s.G + t * M4, gr);
#pragma unroll
      for (int i = 0; i < m; ++i) g[i][t] = el(gr[i / 2], i & 1);
    }
#pragma unroll
    for (int i = 0; i < m; ++i) rhs[i] = (lane > VL) ? (lane - VL - 1 == i ? 1.f : 0.f) : el(fb[i / 2], i & 1);
    // the stage's data is no longer needed: commit stage k-1, prefetch k-2
    // (independent of the register-only elimination below)
    if (k > 0) {
      commit(k - 1);
      if (k > 1) prefetch(k - 2);
    }
    if (lane == VL + m + 1) {
#pragma unroll
      for (int i = 0; i < m; ++i) {
        float2 r2[M2];
#pragma unroll
        for (int q = 0; q < M2; ++q) r2[q] = make_float2(g[i][2 * q], g[i][2 * q + 1]);
        st_row2<m>(gG + (size_t)k * mmm + i * m, r2);
      }
    }
    // scalar pivots in the order of the recursion: G may be indefinite, and
    // 2x2 blocks of an indefinite G lost up to 10x in backward error on the
    // pivot-indefinite test instances
#pragma unroll
    for (int j = 0; j < m; ++j) {
      const float rp = recip_pivot(g[j][j]);
      float nj[m];
#pragma unroll
      for (int c = j + 1; c < m; ++c) nj[c] = g[j][c] * rp;
      const float r0 = rhs[j] * rp;
#pragma unroll
      for (int i = 0; i < m; ++i) {
        if (i == j) continue;
        const float f = g[i][j];
#pragma unroll
        for (int c = j + 1; c < m; ++c) g[i][c] = fmaf(-f, nj[c], g[i][c]);
        rhs[i] = fmaf(-f, r0, rhs[i]);
      }
#pragma unroll
      for (int c = j + 1; c < m; ++c) g[j][c] = nj[c];
      rhs[j] = r0;
    }
    // K[:, c] = -G^{-1} H[:, c] (lanes c < n), k = -G^{-1} h (lane VL),
    // column t of G^{-1} (lane VL + 1 + t)
    float kc[m];
#pragma unroll
    for (int t = 0; t < m; ++t) kc[t] = -rhs[t];
    // (stores only, each under its own lane predicate)
    {
      float2 k2[M2], r2[M2];
#pragma unroll
      for (int q = 0; q < M2; ++q) {
        k2[q] = make_float2(kc[2 * q], kc[2 * q + 1]);
        r2[q] = make_float2(rhs[2 * q], rhs[2 * q + 1]);
      }
      if (lane < n) {
#pragma unroll
        for (int t = 0; t < m; ++t) {
          gK[(size_t)k * nm + t * n + lane] = kc[t];
          s.H[t * N4 + lane] = el(fb[t / 2], t & 1);
        }
      }
      if (SOLVE && lane == VL) st_row2<m>(gkv + (size_t)k * m, k2);
      // G^{-1} is symmetric up to rounding: column t stored as row t
      if (lane > VL && lane <= VL + m) st_row2<m>(gGi + (size_t)k * mmm + (lane - VL - 1) * m, r2);
    }
    __syncwarp();

    // ---- P_k = P' + H^T K (lanes c < n), p_k = p' + H^T k (lane VL)
#pragma unroll
    for (int t = 0; t < m; ++t) {
      float2 hr[H2];
      lds_row2<n>(s.H + t * N4, hr);
      const float2 kt = bcast2(kc[t]);
#pragma unroll
      for (int q = 0; q < H2; ++q) fa[q] = fma2(hr[q], kt, fa[q]);
    }
    if (SOLVE) {
      if (lane == VL) st_row2<n>(gpv + (size_t)k * n, fa);
#pragma unroll
      for (int q = 0; q < H2; ++q) pv[q] = lane == VL ? fa[q] : pv[q];
    }
    // exact symmetry: P[i][c] = computed entry max(i,c) of column min(i,c)
    if (lane < n) st_row2<n>(s.Pt + lane * N4, fa);
    __syncwarp();
    {
      const int c = lane % n;
#pragma unroll
      for (int q = 0; q < H2; ++q) {
        const int i0 = 2 * q, i1 = 2 * q + 1;
        Pc[q] = make_float2(s.Pt[min(i0, c) * N4 + max(i0, c)], s.Pt[min(i1, c) * N4 + max(i1, c)]);
      }
    }
    if (lane == 0) {
      I.flags[k + 1] = (uint8_t)(bit0 | ((k + 1 == N) ? 2 : 0));
      if (!bit0) notpd = true;
    }
    if (sing) singular = true;
    __syncwarp();
  }

  // ---- initial-state pivot
  {
    bool sing = false;
    const int bit0 = state_pivot(gW, sing);
    if (sing) singular = true;
    if (lane == 0) {
      I.flags[0] = (uint8_t)bit0;
      if (!bit0) notpd = true;
      // `singular` marks a state pivot without a decision with margin
      const int32_t st = notpd ? RLQR_NOT_PD : RLQR_OK;
      I.st->pivot_status = st;
      I.st->escalated = singular ? 1 : 0;
      I.st->iters = 0;
      I.st->converged = 0;
      I.st->rel = 0.0;
      if (a.status) a.status[b] = st;
    }
  }
  if constexpr (!SOLVE) return;

  // ---- forward rollout (lane = row)
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c_0 - delta p_0
  if (lane == VL) st_row2<n>(s.p, pv);
  __syncwarp();
  if (lane < n) {
    const float c0 = f64_to_f32_rz(__ldg(I.c + lane));
    gcf[lane] = c0;
    s.v[lane] = fmaf(-delta, s.p[lane], c0);
  }
  __syncwarp();
  if (lane < n) {
    float2 wr[H2], vr[H2];
    lds_row2<n>(s.W + lane * N4, wr);
    lds_row2<n>(s.v, vr);
    const float t = dot2<n>(wr, vr);
    const float xv = fmaf(-delta, t, s.v[lane]), yv = t + s.p[lane];
    s.x[lane] = xv;
    I.x[lane] = widen(xv);
    I.y[lane] = widen(yv);
  }
  // The stage's FP32 copies and factors, prefetched into registers two
  // stages ahead (two alternating sets): a forward stage is short enough
  // that a one-stage-ahead load of the factor, written by the backward pass
  // and evicted from L2 since, would still be in flight at its commit.
  struct FwdSet {
    LaneSeg<float, CP> A, W;
    LaneSeg<float, CB> B, K;
    LaneSeg<float, CV> c, p;
    LaneSeg<float, CM> k;
  };
  auto fprefetch = [&](FwdSet &f, int k) {
    f.A.load_cg(gAf + (size_t)k * nn, nn, lane);
    f.B.load_cg(gBf + (size_t)k * nm, nm, lane);
    f.c.load_cg(gcf + (size_t)(k + 1) * n, n, lane);
    f.W.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    f.K.load_cg(gK + (size_t)k * nm, nm, lane);
    f.k.load_cg(gkv + (size_t)k * m, m, lane);
    f.p.load_cg(gpv + (size_t)(k + 1) * n, n, lane);
  };
  auto fcommit = [&](const FwdSet &f) {
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int idx = lane + 32 * i;
      if (idx < nn) {
        const int row = idx / n, o = row * N4 + idx - row * n;
        s.A[o] = f.A.v[i];
        s.W[o] = f.W.v[i];
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int idx = lane + 32 * i;
      if (idx < nm) {
        const int rb = idx / m, rk = idx / n;
        s.B[rb * M4 + idx - rb * m] = f.B.v[i];
        s.K[rk * N4 + idx - rk * n] = f.K.v[i];
      }
    }
#pragma unroll
    for (int i = 0; i < CV; ++i) {
      const int idx = lane + 32 * i;
      if (idx < n) {
        s.c[idx] = f.c.v[i];
        s.p[idx] = f.p.v[i];
      }
    }
#pragma unroll
    for (int i = 0; i < CM; ++i) {
      const int idx = lane + 32 * i;
      if (idx < m) s.kk[idx] = f.k.v[i];
    }
  };
  const int fx = lane < n ? lane : 0, fu = lane < m ? lane : 0;  // rows of the rounds
  // one forward stage from the set holding its data; the set is refilled
  // with stage k + 2 once committed
  // one forward stage from its operands in shared memory (row strides ldn
  // for n-wide rows, ldm for m-wide rows)
  auto frounds = [&](const float *sA, const float *sW, const float *sB, const float *sK,
                     const float *sc, const float *sp, const float *skk, int ldn, int ldm, int k) {
    // (every lane runs each round, lanes past its rows on row 0; only the
    // stores depend on the lane)
    // u_k = K_k x_k + k_k
    float2 xr[H2];
    lds_row2<n>(s.x, xr);
    {
      float2 kr[H2];
      lds_row2<n>(sK + fu * ldn, kr);
      const float t = dot2<n>(kr, xr) + skk[fu];
      if (lane < m) {
        s.u[lane] = t;
        I.u[(size_t)k * m + lane] = widen(t);
      }
    }
    __syncwarp();
    // v = A x + B u + c_{k+1} - delta p_{k+1}
    {
      float2 ar[H2], br[M2], ur[M2];
      lds_row2<n>(sA + fx * ldn, ar);
      lds_row2<m>(sB + fx * ldm, br);
      lds_row2<m>(s.u, ur);
      float2 acc = mul2(ar[0], xr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], xr[q], acc);
#pragma unroll
      for (int q = 0; q < M2; ++q) acc = fma2(br[q], ur[q], acc);
      const float vv = acc.x + acc.y + fmaf(-delta, sp[fx], sc[fx]);
      if (lane < n) s.v[lane] = vv;
    }
    __syncwarp();
    // x_{k+1} = v - delta W v, y_{k+1} = W v + p_{k+1}
    {
      float2 wr[H2], vr[H2];
      lds_row2<n>(sW + fx * ldn, wr);
      lds_row2<n>(s.v, vr);
      const float t = dot2<n>(wr, vr);
      const float xv = fmaf(-delta, t, s.v[fx]), yv = t + sp[fx];
      if (lane < n) {
        s.x[lane] = xv;
        I.x[(size_t)(k + 1) * n + lane] = widen(xv);
        I.y[(size_t)(k + 1) * n + lane] = widen(yv);
      }
    }
    __syncwarp();
  };
  __syncwarp();
  if constexpr (chunk16_size(NX, NU)) {
    // rows of a multiple of 16 bytes: every operand block of a stage is
    // contiguous in global memory, so a ring of kFwdSlots stages is filled
    // by 16-byte cp.async chunks, the lanes taking them in turn (the factor
    // and copies were written by this warp; the warp syncs above order those
    // stores before the copies, which read through L2)
    constexpr int SL = SM::kFwdSlot, D = SM::kFwdSlots;
    constexpr int oW = nn, oB = 2 * nn, oK = 2 * nn + nm, oc = 2 * nn + 2 * nm, op = oc + n,
                  ok = op + n;
    static_assert(SL % 4 == 0 && nn % 4 == 0 && nm % 4 == 0 && n % 4 == 0 && m % 4 == 0,
                  "16-byte blocks");
    auto cp = [](const float *p) { return reinterpret_cast<const char *>(p); };
    const Blk16 fb[7] = {{cp(gAf), nn * 4, 0, nn / 4},           {cp(gW + nn), nn * 4, oW * 4, nn / 4},
                         {cp(gBf), nm * 4, oB * 4, nm / 4},     {cp(gK), nm * 4, oK * 4, nm / 4},
                         {cp(gcf + n), n * 4, oc * 4, n / 4},    {cp(gpv + n), n * 4, op * 4, n / 4},
                         {cp(gkv), m * 4, ok * 4, m / 4}};
    ChunkPlan<7, (SL / 4 + 31) / 32> plan;
    plan.init(fb, lane);
    auto fissue = [&](int k) {
      if (k < N) plan.issue(reinterpret_cast<unsigned char *>(s.fring + (k % D) * SL), k);
      cp_async_commit();
    };
#pragma unroll 1
    for (int j = 0; j < D - 1; ++j) fissue(j);
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      fissue(k + D - 1);
      cp_async_wait<D - 1>();
      __syncwarp();
      const float *sl = s.fring + (k % D) * SL;
      frounds(sl, sl + oW, sl + oB, sl + oK, sl + oc, sl + op, sl + ok, n, m, k);
    }
    cp_async_wait<0>();
  } else {
    FwdSet f0, f1;
    fprefetch(f0, 0);
    if (N > 1) fprefetch(f1, 1);
    auto fstage = [&](FwdSet &f, int k) {
      fcommit(f);
      if (k + 2 < N) fprefetch(f, k + 2);
      __syncwarp();
      frounds(s.A, s.W, s.B, s.K, s.c, s.p, s.kk, N4, M4, k);
    };
    for (int k = 0; k < N; k += 2) {
      fstage(f0, k);
      if (k + 1 < N) fstage(f1, k + 1);
    }
  }
}

template <int NX, int NU, bool SOLVE>
__global__ void __launch_bounds__(32) k_sweep32(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  sweep32_body<NX, NU, SOLVE>(a, inst_of(a, slot), smem_raw, threadIdx.x);
}

}  // namespace rlqr

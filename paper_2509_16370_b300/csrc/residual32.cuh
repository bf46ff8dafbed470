// residual32.cuh -- the first residual of the mixed-precision path for the
// sizes of sweep32.cuh (Section "Residual Computation"): FP64-accurate
// float-float arithmetic on the FP32 pipes, plus the FP64 certificate of the
// control pivots G_i stored by the FP32 sweep.
//
// Sizes: n even, 2n + m <= 32 (one lane per row of a stage), m <= 8; an odd m
// runs its control segments padded to m + 1 with zero coefficients and zero
// z entries (the pad stays zero in shared memory).
//
// One CTA of RW warps per instance; warp w takes stages w, w + RW, ... and
// loads stage s + RW into registers while it computes stage s.  The rows of
// K z + b of stage s (same layout as k_residual in residual.cuh):
//   x rows  [Q_s  M_s  A_s^T] [x_s; u_s; y_{s+1}] + q_s - y_s
//   u rows  [M_s^T R_s B_s^T] [x_s; u_s; y_{s+1}] + r_s
//   c rows  [A_s  B_s  0    ] [x_s; u_s; y_{s+1}] + c_{s+1} - x_{s+1} - delta y_{s+1}
// Lane r < 2n+m walks three coefficient segments of its row through its own
// shared-memory pointers (the transposes A^T, B^T, M^T are staged next to A,
// B, M), so every coefficient read is a vector row load and the warp runs
// one instruction stream.  Each coefficient and each z entry is split into
// hi + lo FP32 parts (split_f64); two neighbouring terms are accumulated as
// a packed pair with the two-product of Dekker and the two-sum of Knuth
// (f32x2 instructions), and the pair is merged at the end.  Error per term
// about 2^-45 |K_ij z_j|, far below what the 1e-9 backward-error test needs.
#pragma once

#include "common.cuh"
#include "refine.cuh"
#include "sweep32.cuh"

namespace rlqr {

template <int NX, int NU>
struct Rs32Warp {
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4;
  alignas(16) float Ah[NX * N4];
  alignas(16) float Al[NX * N4];
  alignas(16) float Ath[NX * N4];
  alignas(16) float Atl[NX * N4];
  alignas(16) float Qh[NX * N4];
  alignas(16) float Ql[NX * N4];
  alignas(16) float Bh[NX * M4];
  alignas(16) float Bl[NX * M4];
  alignas(16) float Mh[NX * M4];
  alignas(16) float Ml[NX * M4];
  alignas(16) float Bth[NU * N4];
  alignas(16) float Btl[NU * N4];
  alignas(16) float Mth[NU * N4];
  alignas(16) float Mtl[NU * N4];
  alignas(16) float Rh[NU * M4];
  alignas(16) float Rl[NU * M4];
  alignas(16) float zero[N4];
  alignas(16) float xh[N4];
  alignas(16) float xl[N4];
  alignas(16) float uh[M4];
  alignas(16) float ul[M4];
  alignas(16) float yh[N4];
  alignas(16) float yl[N4];
};

constexpr int kResWarps = 4;

template <int NX, int NU>
constexpr bool res32_fits() {
  return NX % 2 == 0 && NX >= 2 && NU >= 1 && NU <= 8 && 2 * NX + NU <= 32;
}

// Packed float-float accumulation of two terms: (sh, sl) += (ah + al)(zh + zl)
// elementwise, zhn = -zh.  The product's rounding error comes from an FMA
// (exact), the sum's from the two-sum; the cross terms and al zl (dropped,
// below 2^-46 of the term) go to the low part.
__device__ __forceinline__ void ff2_fma(float2 &sh, float2 &sl, float2 ah, float2 al, float2 zh,
                                        float2 zhn, float2 zl) {
  const float2 pn = mul2(ah, zhn);                       // -fl(ah zh)
  const float2 e = fma2(ah, zh, pn);                     // ah zh - fl(ah zh), exact
  const float2 s = sub2(sh, pn);                         // sh + p
  const float2 bb = sub2(s, sh);
  const float2 err = sub2(sub2(sh, sub2(s, bb)), add2(pn, bb));  // (sh + p) - s, exact
  sh = s;
  sl = add2(sl, add2(err, fma2(ah, zl, fma2(al, zh, e))));
}

template <int CNT, int L, int LD, int LDT>
__device__ __forceinline__ void commit_split(const LaneSeg<double, CNT> &pf, int len, int lane,
                                             float *dh, float *dl, float *th, float *tl) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < len) {
      const int row = idx / L, col = idx - row * L;
      const float2 v = split_f64(pf.v[i]);
      dh[row * LD + col] = v.x;
      dl[row * LD + col] = v.y;
      if (th) {
        th[col * LDT + row] = v.x;
        tl[col * LDT + row] = v.y;
      }
    }
  }
}

template <int CNT, int L, int LD>
__device__ __forceinline__ void commit_split_sym(const LaneSeg<double, CNT> &pf, int lane, float *dh,
                                                 float *dl) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < L * L) {
      const int row = idx / L, col = idx - row * L;
      if (row <= col) {
        const float2 v = split_f64(pf.v[i]);
        dh[row * LD + col] = v.x;
        dl[row * LD + col] = v.y;
        dh[col * LD + row] = v.x;
        dl[col * LD + row] = v.y;
      }
    }
  }
}

template <int L>
__device__ __forceinline__ float2 abs_sum2(const float2 (&r)[L / 2], float2 acc) {
#pragma unroll
  for (int q = 0; q < L / 2; ++q)
    acc = add2(acc, make_float2(fabsf(r[q].x), fabsf(r[q].y)));
  return acc;
}

// The residual rows of one stage by one warp (lane r < 2n+m: row r of the
// stage, as in k_res32): prefetch() loads the stage's FP64 data and this
// lane's z and b entries into registers, commit() splits them into the FP32
// hi / lo parts in shared memory (the caller then syncs the warp), row()
// returns this lane's row of K z + b in FP64 accuracy and raises kmaxf to
// the row's |K| sum.  Used by k_res32 and by the fused first refinement pass.
template <int NX, int NU>
struct Res32Rows {
  static constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  static constexpr int ME = m + (m & 1), H2 = n / 2, M2 = ME / 2, RS = 2 * n + m;
  static constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  using SW = Rs32Warp<NX, NU>;
  static constexpr int N4 = SW::N4, M4 = SW::M4;
  LaneSeg<double, CP> pA, pQ;
  LaneSeg<double, CB> pB, pM;
  LaneSeg<double, CR> pR;
  double zv, b1, b2;  // this lane's z entry and row data
  const float *s1h, *s1l, *s2h, *s2l, *s3h, *s3l;
  float kconst, bh, bl;
  float2 dsp;

  // Row pointers of this lane; the pad column of odd m and s.zero cleared.
  __device__ __forceinline__ void init(SW &s, int lane, double delta) {
    if constexpr (ME != m) {
      float4 *z4 = reinterpret_cast<float4 *>(&s);
      for (int e = lane; e < (int)(sizeof(SW) / 16); e += 32) z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    zv = b1 = b2 = 0.0;
    s1h = s1l = s2h = s2l = s3h = s3l = s.zero;
    kconst = 0.f;
    if (lane < n) {
      s1h = s.Qh + lane * N4; s1l = s.Ql + lane * N4;
      s2h = s.Mh + lane * M4; s2l = s.Ml + lane * M4;
      s3h = s.Ath + lane * N4; s3l = s.Atl + lane * N4;
      kconst = 1.f;
    } else if (lane < n + m) {
      const int t = lane - n;
      s1h = s.Mth + t * N4; s1l = s.Mtl + t * N4;
      s2h = s.Rh + t * M4; s2l = s.Rl + t * M4;
      s3h = s.Bth + t * N4; s3l = s.Btl + t * N4;
    } else if (lane < RS) {
      const int i = lane - n - m;
      s1h = s.Ah + i * N4; s1l = s.Al + i * N4;
      s2h = s.Bh + i * M4; s2l = s.Bl + i * M4;
      kconst = 1.f + abs_f32_trunc(delta);
    }
    if (lane < N4) s.zero[lane] = 0.f;
    dsp = split_f64(-delta);
  }

  __device__ __forceinline__ void prefetch(const Inst &I, int st, int lane) {
    pA.load(I.A + (size_t)st * nn, nn, lane);
    pQ.load(I.Q + (size_t)st * nn, nn, lane);
    pB.load(I.B + (size_t)st * nm, nm, lane);
    pM.load(I.M + (size_t)st * nm, nm, lane);
    pR.load(I.R + (size_t)st * mmm, mmm, lane);
    // this lane's z entry and data terms, chosen by selects (lanes past RS
    // load entry 0 of the c rows and never use it): no divergent branch
    const bool xr = lane < n, ur = !xr && lane < n + m;
    const int i = xr ? lane : ur ? lane - n : (lane < RS ? lane - n - m : 0);
    const size_t ox = (size_t)st * n, ou = (size_t)st * m, oc = (size_t)(st + 1) * n;
    const double *zb = xr ? I.x + ox : ur ? I.u + ou : I.y + oc;
    const double *b1b = xr ? I.q + ox : ur ? I.r + ou : I.c + oc;
    const double *b2b = xr ? I.y + ox : I.x + oc;
    zv = __ldg(zb + i);
    b1 = __ldg(b1b + i);
    b2 = ur ? 0.0 : __ldg(b2b + i);
  }

  // Split the prefetched stage into shared memory (the caller syncs the warp
  // before and after: the previous stage's rows may still be reading it).
  __device__ __forceinline__ void commit(SW &s, int lane, unsigned long long &zbits,
                                         unsigned long long &bbits) {
    __syncwarp();
    commit_split<CP, n, N4, N4>(pA, nn, lane, s.Ah, s.Al, s.Ath, s.Atl);
    commit_split_sym<CP, n, N4>(pQ, lane, s.Qh, s.Ql);
    commit_split<CB, m, M4, N4>(pB, nm, lane, s.Bh, s.Bl, s.Bth, s.Btl);
    commit_split<CB, m, M4, N4>(pM, nm, lane, s.Mh, s.Ml, s.Mth, s.Mtl);
    commit_split_sym<CR, m, M4>(pR, lane, s.Rh, s.Rl);
    // z entry of this lane and the row's data terms (float-float)
    // x rows b = q - y_k, u rows r, c rows c - x_{k+1} - delta y_{k+1}, on
    // every lane (b2 is zero on the u rows, the delta term a zero product
    // off the c rows: both add exactly nothing); only the stores and the
    // maxima depend on the lane
    bh = 0.f;
    bl = 0.f;
    const bool xr = lane < n, ur = !xr && lane < n + m, cr = !xr && !ur && lane < RS;
    const float2 zs = split_f64(zv);
    ff_add(bh, bl, split_f64(b1));
    ff_add(bh, bl, ff_neg(split_f64(b2)));
    ff_fma(bh, bl, cr ? dsp : make_float2(0.f, 0.f), zs);
    if (lane < RS) {
      float *dh = xr ? s.xh + lane : ur ? s.uh + (lane - n) : s.yh + (lane - n - m);
      float *dl = xr ? s.xl + lane : ur ? s.ul + (lane - n) : s.yl + (lane - n - m);
      *dh = zs.x;
      *dl = zs.y;
    }
    const bool act = lane < RS;
    zbits = act ? max(zbits, abs_bits(zv)) : zbits;
    bbits = act ? max(bbits, abs_bits(b1)) : bbits;
  }

  // This lane's row (lane < RS) after commit() and a warp sync.
  __device__ __forceinline__ double row(const SW &s, int lane, float &kmaxf) const {
    float2 sh = make_float2(bh, 0.f), sl = make_float2(bl, 0.f), ka = make_float2(kconst, 0.f);
    {
      float2 ch[H2], cl[H2], zh[H2], zl[H2];
      lds_row2<n>(s1h, ch);
      lds_row2<n>(s1l, cl);
      lds_row2<n>(s.xh, zh);
      lds_row2<n>(s.xl, zl);
#pragma unroll
      for (int q = 0; q < H2; ++q)
        ff2_fma(sh, sl, ch[q], cl[q], zh[q], make_float2(-zh[q].x, -zh[q].y), zl[q]);
      ka = abs_sum2<n>(ch, ka);
    }
    {
      float2 ch[M2], cl[M2], zh[M2], zl[M2];
      lds_row2<ME>(s2h, ch);
      lds_row2<ME>(s2l, cl);
      lds_row2<ME>(s.uh, zh);
      lds_row2<ME>(s.ul, zl);
#pragma unroll
      for (int q = 0; q < M2; ++q)
        ff2_fma(sh, sl, ch[q], cl[q], zh[q], make_float2(-zh[q].x, -zh[q].y), zl[q]);
      ka = abs_sum2<ME>(ch, ka);
    }
    {
      float2 ch[H2], cl[H2], zh[H2], zl[H2];
      lds_row2<n>(s3h, ch);
      lds_row2<n>(s3l, cl);
      lds_row2<n>(s.yh, zh);
      lds_row2<n>(s.yl, zl);
#pragma unroll
      for (int q = 0; q < H2; ++q)
        ff2_fma(sh, sl, ch[q], cl[q], zh[q], make_float2(-zh[q].x, -zh[q].y), zl[q]);
      ka = abs_sum2<n>(ch, ka);
    }
    // merge the two accumulators of the pair
    float h0 = sh.x, l0 = sl.x;
    ff_add(h0, l0, make_float2(sh.y, sl.y));
    kmaxf = fmaxf(kmaxf, ka.x + ka.y);
    return widen(h0) + widen(l0);
  }
};

// Rows x_N (Q_N x_N + q_N - y_N) and c_0 (c_0 - delta y_0 - x_0) in FP64,
// row r < 2n of the pair; the maxima of the backward error are raised.
__device__ __forceinline__ double res_end_row(const Inst &I, int r, float &kmaxf,
                                              unsigned long long &zbits,
                                              unsigned long long &bbits) {
  const int N = I.N, n = I.n, nn = n * n;
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
    kmaxf = fmaxf(kmaxf, ra);
    bbits = max(bbits, abs_bits(qv));
  } else {
    const int i = r - n;
    const double xv = __ldg(I.x + i), yv = __ldg(I.y + i), cv = __ldg(I.c + i);
    v = cv - I.delta * yv - xv;
    zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
    kmaxf = fmaxf(kmaxf, 1.f + abs_f32_trunc(I.delta));
    bbits = max(bbits, abs_bits(cv));
  }
  return v;
}

// store: write res into the workspace for the refinement; cert_g: FP64
// certificate of the stored control pivots (bit1 of the flags).
template <int NX, int NU>
__device__ __forceinline__ void res32_instance(const BatchArgs &a, int slot, int store, int cert_g,
                                               unsigned char *smem_raw);

template <int NX, int NU>
__global__ void __launch_bounds__(32 * kResWarps) k_res32(BatchArgs a, int store, int cert_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one instance per block; recheck launches use fewer blocks than
  // instances and stride over the slots
  for (int slot = blockIdx.x; slot < a.count; slot += gridDim.x)
    res32_instance<NX, NU>(a, slot, store, cert_g, smem_raw);
}

template <int NX, int NU>
__device__ __forceinline__ void res32_instance(const BatchArgs &a, int slot, int store, int cert_g,
                                               unsigned char *smem_raw) {
  static_assert(res32_fits<NX, NU>(), "dimensions outside the warp residual");
  constexpr int n = NX, m = NU, mmm = m * m, RS = 2 * n + m;
  using SW = Rs32Warp<NX, NU>;
  __shared__ double s_red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  SW &s = reinterpret_cast<SW *>(smem_raw)[warp];
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  if (a.recheck && (I.st->converged || I.st->pivot_status == RLQR_ERR_SINGULAR)) return;
  const int N = I.N;
  const double delta = I.delta;
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;

  // ---- FP64 certificate of the control pivots with margin, one stage per
  // thread (pd_margin_f32); a decision without its margin escalates the
  // instance to the FP64 recursion
  if (cert_g) {
    const float *gG = reinterpret_cast<const float *>(I.ws + I.L.G);
    int bad = 0, esc = 0;
    for (int st = threadIdx.x; st < N; st += blockDim.x) {
      const int dec = pd_margin_f32<m>(gG + (size_t)st * mmm, m, (double)kMarginTau);
      const uint8_t old = I.flags[st];
      I.flags[st] = (uint8_t)((old & 1) | (dec == kPdYes ? 2 : 0));
      bad |= dec == kPdNo;
      esc |= dec == kPdAmbiguous;
    }
    const int any_bad = __syncthreads_or(bad);
    const int any_esc = __syncthreads_or(esc);
    if (threadIdx.x == 0) {
      if (any_bad && I.st->pivot_status == RLQR_OK) I.st->pivot_status = RLQR_NOT_PD;
      if (any_esc) I.st->escalated = 1;
    }
  }

  // ---- residual rows of the stages of this warp
  Res32Rows<NX, NU> R;
  R.init(s, lane, delta);
  float kmaxf = 0.f;
  unsigned long long rbits = 0, zbits = 0, bbits = 0;
  int st = warp;
  if (st < N) R.prefetch(I, st, lane);
  for (; st < N; st += kResWarps) {
    R.commit(s, lane, zbits, bbits);
    if (st + kResWarps < N) R.prefetch(I, st + kResWarps, lane);
    __syncwarp();
    if (lane < RS) {
      const double v = R.row(s, lane, kmaxf);
      rbits = max(rbits, abs_bits(v));
      if (store) {
        if (lane < n) rq[(size_t)st * n + lane] = v;
        else if (lane < n + m) rr[(size_t)st * m + lane - n] = v;
        else rc[(size_t)(st + 1) * n + lane - n - m] = v;
      }
    }
  }
  // ---- rows x_N (Q_N x_N + q_N - y_N) and c_0 (c_0 - delta y_0 - x_0), FP64
  for (int r = threadIdx.x; r < 2 * n; r += blockDim.x) {
    const double v = res_end_row(I, r, kmaxf, zbits, bbits);
    if (store) {
      if (r < n) rq[(size_t)N * n + r] = v;
      else rc[r - n] = v;
    }
    rbits = max(rbits, abs_bits(v));
  }
  const double rmax = block_max_dyn(bits_to_double(rbits), s_red);
  const double zmax = block_max_dyn(bits_to_double(zbits), s_red);
  const double kmax = block_max_dyn((double)kmaxf, s_red);
  const double bmax = block_max_dyn(bits_to_double(bbits), s_red);
  if (threadIdx.x == 0) {
    InstState *stp = I.st;
    stp->kmax = kmax;
    stp->bmax = bmax;
    const double den = kmax * zmax + bmax;
    const double rel = den > 0.0 ? rmax / den : rmax;
    stp->rmax = rmax;
    stp->zmax = zmax;
    stp->rel = rel;
    stp->upd = 0.0;  // a residual computed from scratch
    const int32_t conv = (rel <= a.tol) ? 1 : 0;
    stp->converged = conv;
    if (a.rel) a.rel[b] = rel;
    if (a.iters) a.iters[b] = stp->iters;
    write_status(a, b, stp, conv);
  }
}

}  // namespace rlqr

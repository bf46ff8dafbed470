// refine32.cuh -- refinement pass of the mixed-precision path for the sizes
// of sweep32.cuh: one warp per instance, FP32 factor and FP32 data copies
// written by the sweep, FP64 iterate and residual.
//
// One pass solves K dz = -res with the stored factor (Corollary p-recurrence
// backward, eq. recover-x0 / control-law / recover-x forward), adds dz to z
// in FP64 and updates the FP64 residual as res <- res + K dz, with K dz in
// FP32 (|dz| ~ u_32 |z|, so the update is accurate to ~u_32^2 |K||z|; see
// refine.cuh).  The rows of K dz for stage k (Section "Residual
// Computation"):
//   x rows  Q_k dx_k + M_k du_k + A_k^T dy_{k+1} - dy_k
//   u rows  M_k^T dx_k + R_k du_k + B_k^T dy_{k+1}
//   c rows  A_k dx_k + B_k du_k - dx_{k+1} - delta dy_{k+1}
// are computed by lanes 0 .. 2n+m-1 in one instruction stream: each lane
// walks three row segments (coefficients of dx_k, du_k, dy_{k+1}) through
// its own shared-memory pointers, which is why the transposes A^T, B^T, M^T
// and K^T are staged next to A, B, M and K.  The FP64 updates of z and res
// are one FP64 add per lane each (lanes r < n: x_{k+1}, n <= r < n+m: u_k,
// n+m <= r: y_{k+1}).
#pragma once

#include "common.cuh"
#include "sweep32.cuh"

namespace rlqr {

template <int NX, int NU>
struct Rf32 {
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4;
  alignas(16) float W[NX * N4];
  alignas(16) float A[NX * N4];
  alignas(16) float At[NX * N4];
  alignas(16) float B[NX * M4];
  alignas(16) float Bt[NU * N4];
  alignas(16) float K[NU * N4];
  alignas(16) float Kt[NX * M4];
  alignas(16) float Gi[NU * M4];
  alignas(16) float Q[NX * N4];
  alignas(16) float M[NX * M4];
  alignas(16) float Mt[NU * N4];
  alignas(16) float R[NU * M4];
  alignas(16) float zero[N4];
  alignas(16) float p[N4];
  alignas(16) float kk[M4];
  alignas(16) float cr[N4];  // c' (residual rows c) of the stage
  alignas(16) float qr[N4];
  alignas(16) float rr[M4];
  alignas(16) float g[N4];
  alignas(16) float h[M4];
  alignas(16) float w[N4];
  alignas(16) float d[4][N4];  // dx_k, dy_k, dx_{k+1}, dy_{k+1} (rotating)
  alignas(16) float du[M4];
};

// Commit a lane-strided FP32 segment of a row-major rows x L matrix to
// shared memory (row stride LD) and, optionally, its transpose (row stride LDT).
template <int CNT, int L, int LD, int LDT>
__device__ __forceinline__ void commit_f32(const LaneSeg<float, CNT> &pf, int len, int lane,
                                           float *dst, float *dstT) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < len) {
      const int row = idx / L, col = idx - row * L;
      dst[row * LD + col] = pf.v[i];
      if (dstT) dstT[col * LDT + row] = pf.v[i];
    }
  }
}

// Symmetric L x L matrix from its upper triangle.
template <int CNT, int L, int LD>
__device__ __forceinline__ void commit_f32_sym(const LaneSeg<float, CNT> &pf, int lane, float *dst) {
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int idx = lane + 32 * i;
    if (idx < L * L) {
      const int row = idx / L, col = idx - row * L;
      if (row <= col) {
        dst[row * LD + col] = pf.v[i];
        dst[col * LD + row] = pf.v[i];
      }
    }
  }
}

template <int NX, int NU>
__global__ void __launch_bounds__(32) k_refine32(BatchArgs a) {
  static_assert(sweep32_fits<NX, NU>(), "dimensions outside the FP32 warp kernels");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int H2 = n / 2, M2 = m / 2;
  using SM = Rf32<NX, NU>;
  constexpr int N4 = SM::N4, M4 = SM::M4;
  constexpr int RS = 2 * n + m;  // residual rows of a stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int lane = threadIdx.x;
  const int slot = blockIdx.x;
  if (slot >= a.count) return;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  InstState *stp = I.st;
  if (stp->converged || stp->pivot_status == RLQR_ERR_SINGULAR) return;
  const int N = I.N;
  const float delta = (float)I.delta;
  const double delta64 = I.delta;
  const float *gW = reinterpret_cast<const float *>(I.ws + I.L.W);
  const float *gK = reinterpret_cast<const float *>(I.ws + I.L.K);
  const float *gGi = reinterpret_cast<const float *>(I.ws + I.L.Gi);
  float *gkv = reinterpret_cast<float *>(I.ws + I.L.kv);
  float *gpv = reinterpret_cast<float *>(I.ws + I.L.pv);
  const float *gAf = reinterpret_cast<const float *>(I.ws + I.L.Af);
  const float *gBf = reinterpret_cast<const float *>(I.ws + I.L.Bf);
  const float *gQf = reinterpret_cast<const float *>(I.ws + I.L.Qf);
  const float *gMf = reinterpret_cast<const float *>(I.ws + I.L.Mf);
  const float *gRf = reinterpret_cast<const float *>(I.ws + I.L.Rf);
  double *rq = reinterpret_cast<double *>(I.ws + I.L.res);
  double *rr = rq + (size_t)(N + 1) * n;
  double *rc = rr + (size_t)N * m;
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  constexpr int CV = (n + 31) / 32, CM = (m + 31) / 32;
  if (lane < N4) s.zero[lane] = 0.f;

  // ---------------- backward: p-recurrence with the residual as right-hand side
  LaneSeg<float, CP> bW, bA;
  LaneSeg<float, CB> bB, bK;
  LaneSeg<float, CR> bG;
  LaneSeg<double, CV> bq, bc;
  LaneSeg<double, CM> br;
  auto bprefetch = [&](int k) {
    bW.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    bA.load_cg(gAf + (size_t)k * nn, nn, lane);
    bB.load_cg(gBf + (size_t)k * nm, nm, lane);
    bK.load_cg(gK + (size_t)k * nm, nm, lane);
    bG.load_cg(gGi + (size_t)k * mmm, mmm, lane);
    bq.load_cg(rq + (size_t)k * n, n, lane);
    bc.load_cg(rc + (size_t)(k + 1) * n, n, lane);
    br.load_cg(rr + (size_t)k * m, m, lane);
  };
  auto bcommit = [&]() {
    commit_f32<CP, n, N4, N4>(bW, nn, lane, s.W, nullptr);
    commit_f32<CP, n, N4, N4>(bA, nn, lane, s.A, s.At);
    commit_f32<CB, m, M4, N4>(bB, nm, lane, s.B, s.Bt);
    commit_f32<CB, n, N4, M4>(bK, nm, lane, s.K, s.Kt);
    commit_f32<CR, m, M4, M4>(bG, mmm, lane, s.Gi, nullptr);
#pragma unroll
    for (int i = 0; i < CV; ++i) {
      const int idx = lane + 32 * i;
      if (idx < n) {
        s.qr[idx] = f64_to_f32_rz(bq.v[i]);
        s.cr[idx] = f64_to_f32_rz(bc.v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < CM; ++i) {
      const int idx = lane + 32 * i;
      if (idx < m) s.rr[idx] = f64_to_f32_rz(br.v[i]);
    }
  };
  if (lane < n) {
    const float v = f64_to_f32_rz(__ldcg(rq + (size_t)N * n + lane));
    s.p[lane] = v;
    gpv[(size_t)N * n + lane] = v;
  }
  bprefetch(N - 1);
  for (int k = N - 1; k >= 0; --k) {
    __syncwarp();
    bcommit();
    if (k > 0) bprefetch(k - 1);
    __syncwarp();
    // g = p + W (c' - delta p)
    if (lane < n) {
      float2 wr[H2], cr[H2], pr[H2];
      lds_row2<n>(s.W + lane * N4, wr);
      lds_row2<n>(s.cr, cr);
      lds_row2<n>(s.p, pr);
#pragma unroll
      for (int q = 0; q < H2; ++q) cr[q] = fma2(bcast2(-delta), pr[q], cr[q]);
      s.g[lane] = s.p[lane] + dot2<n>(wr, cr);
    }
    __syncwarp();
    // h = r' + B^T g
    if (lane < m) {
      float2 br2[H2], gr[H2];
      lds_row2<n>(s.Bt + lane * N4, br2);
      lds_row2<n>(s.g, gr);
      s.h[lane] = s.rr[lane] + dot2<n>(br2, gr);
    }
    __syncwarp();
    // p_k = q' + A^T g + K^T h (lanes < n);  k_k = -G^{-1} h (lanes n .. n+m-1)
    if (lane < n) {
      float2 ar[H2], gr[H2], kr[M2], hr[M2];
      lds_row2<n>(s.At + lane * N4, ar);
      lds_row2<n>(s.g, gr);
      lds_row2<m>(s.Kt + lane * M4, kr);
      lds_row2<m>(s.h, hr);
      float2 acc = mul2(ar[0], gr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], gr[q], acc);
#pragma unroll
      for (int q = 0; q < M2; ++q) acc = fma2(kr[q], hr[q], acc);
      const float pv = s.qr[lane] + (acc.x + acc.y);
      s.p[lane] = pv;
      gpv[(size_t)k * n + lane] = pv;
    } else if (lane < n + m) {
      float2 gr2[M2], hr[M2];
      lds_row2<m>(s.Gi + (lane - n) * M4, gr2);
      lds_row2<m>(s.h, hr);
      gkv[(size_t)k * m + lane - n] = -dot2<m>(gr2, hr);
    }
  }

  // ---------------- forward rollout, FP64 update of z and of the residual
  unsigned long long rbits = 0, zbits = 0, dzbits = 0;
  // per-lane row segments of K dz (lane r < RS); see the header comment
  const float *seg1 = s.zero, *seg2 = s.zero, *seg3 = s.zero;
  double *zp = nullptr, *resp = nullptr;  // this lane's FP64 z and res element at stage 0
  size_t zstride = 0, rstride = 0;
  if (lane < n) {
    seg1 = s.Q + lane * N4; seg2 = s.M + lane * M4; seg3 = s.At + lane * N4;
    zp = I.x + n + lane; zstride = n; resp = rq + lane; rstride = n;
  } else if (lane < n + m) {
    const int t = lane - n;
    seg1 = s.Mt + t * N4; seg2 = s.R + t * M4; seg3 = s.Bt + t * N4;
    zp = I.u + t; zstride = m; resp = rr + t; rstride = m;
  } else if (lane < RS) {
    const int i = lane - n - m;
    seg1 = s.A + i * N4; seg2 = s.B + i * M4; seg3 = s.zero;
    zp = I.y + n + i; zstride = n; resp = rc + n + i; rstride = n;
  }
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c'_0 - delta p_0
  float *dx = s.d[0], *dy = s.d[1], *dxn = s.d[2], *dyn = s.d[3];
  __syncwarp();
  for (int e = lane; e < nn; e += 32) {
    const int row = e / n;
    s.W[row * N4 + e - row * n] = __ldcg(gW + e);
  }
  if (lane < n) s.w[lane] = fmaf(-delta, s.p[lane], f64_to_f32_rz(__ldcg(rc + lane)));
  __syncwarp();
  if (lane < n) {
    float2 wr[H2], vr[H2];
    lds_row2<n>(s.W + lane * N4, wr);
    lds_row2<n>(s.w, vr);
    const float t = dot2<n>(wr, vr);
    const float dxv = fmaf(-delta, t, s.w[lane]), dyv = t + s.p[lane];
    dx[lane] = dxv;
    dy[lane] = dyv;
    const double xv = I.x[lane] + widen(dxv), yv = I.y[lane] + widen(dyv);
    I.x[lane] = xv;
    I.y[lane] = yv;
    zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
    dzbits = max(dzbits, max(abs_bits(widen(dxv)), abs_bits(widen(dyv))));
    const double r0 = __ldcg(rc + lane) - widen(dxv) - delta64 * widen(dyv);
    rc[lane] = r0;
    rbits = max(rbits, abs_bits(r0));
  }
  LaneSeg<float, CP> fW, fA, fQ;
  LaneSeg<float, CB> fB, fK, fM;
  LaneSeg<float, CR> fR;
  LaneSeg<float, CM> fk;
  LaneSeg<float, CV> fp;
  LaneSeg<double, CV> fc;
  double zold = 0.0, rold = 0.0;
  auto fprefetch = [&](int k) {
    fW.load_cg(gW + (size_t)(k + 1) * nn, nn, lane);
    fA.load_cg(gAf + (size_t)k * nn, nn, lane);
    fB.load_cg(gBf + (size_t)k * nm, nm, lane);
    fK.load_cg(gK + (size_t)k * nm, nm, lane);
    fk.load_cg(gkv + (size_t)k * m, m, lane);
    fp.load_cg(gpv + (size_t)(k + 1) * n, n, lane);
    fc.load_cg(rc + (size_t)(k + 1) * n, n, lane);
    fQ.load_cg(gQf + (size_t)k * nn, nn, lane);
    fM.load_cg(gMf + (size_t)k * nm, nm, lane);
    fR.load_cg(gRf + (size_t)k * mmm, mmm, lane);
    if (lane < RS) {
      zold = __ldcg(zp + (size_t)k * zstride);
      rold = __ldcg(resp + (size_t)k * rstride);
    }
  };
  auto fcommit = [&]() {
    commit_f32<CP, n, N4, N4>(fW, nn, lane, s.W, nullptr);
    commit_f32<CP, n, N4, N4>(fA, nn, lane, s.A, s.At);
    commit_f32<CB, m, M4, N4>(fB, nm, lane, s.B, s.Bt);
    commit_f32<CB, n, N4, M4>(fK, nm, lane, s.K, nullptr);
    commit_f32_sym<CP, n, N4>(fQ, lane, s.Q);
    commit_f32<CB, m, M4, N4>(fM, nm, lane, s.M, s.Mt);
    commit_f32_sym<CR, m, M4>(fR, lane, s.R);
#pragma unroll
    for (int i = 0; i < CM; ++i) {
      const int idx = lane + 32 * i;
      if (idx < m) s.kk[idx] = fk.v[i];
    }
#pragma unroll
    for (int i = 0; i < CV; ++i) {
      const int idx = lane + 32 * i;
      if (idx < n) {
        s.p[idx] = fp.v[i];
        s.cr[idx] = f64_to_f32_rz(fc.v[i]);
      }
    }
  };
  fprefetch(0);
  for (int k = 0; k < N; ++k) {
    __syncwarp();
    fcommit();
    const double z0 = zold, r0 = rold;
    if (k + 1 < N) fprefetch(k + 1);
    __syncwarp();
    // du_k = K_k dx_k + k_k
    if (lane < m) {
      float2 kr[H2], xr[H2];
      lds_row2<n>(s.K + lane * N4, kr);
      lds_row2<n>(dx, xr);
      s.du[lane] = dot2<n>(kr, xr) + s.kk[lane];
    }
    __syncwarp();
    // w = A dx + B du + c'_{k+1} - delta p_{k+1}
    if (lane < n) {
      float2 ar[H2], xr[H2], br2[M2], ur[M2];
      lds_row2<n>(s.A + lane * N4, ar);
      lds_row2<n>(dx, xr);
      lds_row2<m>(s.B + lane * M4, br2);
      lds_row2<m>(s.du, ur);
      float2 acc = mul2(ar[0], xr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], xr[q], acc);
#pragma unroll
      for (int q = 0; q < M2; ++q) acc = fma2(br2[q], ur[q], acc);
      s.w[lane] = (acc.x + acc.y) + fmaf(-delta, s.p[lane], s.cr[lane]);
    }
    __syncwarp();
    // dx_{k+1} = w - delta W w, dy_{k+1} = W w + p_{k+1}
    if (lane < n) {
      float2 wr[H2], vr[H2];
      lds_row2<n>(s.W + lane * N4, wr);
      lds_row2<n>(s.w, vr);
      const float t = dot2<n>(wr, vr);
      dxn[lane] = fmaf(-delta, t, s.w[lane]);
      dyn[lane] = t + s.p[lane];
    }
    __syncwarp();
    // K dz rows of stage k and the FP64 updates (lanes < RS)
    if (lane < RS) {
      float2 c1[H2], x1[H2], c2[M2], u2[M2], c3[H2], y3[H2];
      lds_row2<n>(seg1, c1);
      lds_row2<n>(dx, x1);
      lds_row2<m>(seg2, c2);
      lds_row2<m>(s.du, u2);
      lds_row2<n>(seg3, c3);
      lds_row2<n>(dyn, y3);
      float2 acc = mul2(c1[0], x1[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(c1[q], x1[q], acc);
#pragma unroll
      for (int q = 0; q < M2; ++q) acc = fma2(c2[q], u2[q], acc);
#pragma unroll
      for (int q = 0; q < H2; ++q) acc = fma2(c3[q], y3[q], acc);
      float t = acc.x + acc.y, dz;
      if (lane < n) {
        t -= dy[lane];
        dz = dxn[lane];
      } else if (lane < n + m) {
        dz = s.du[lane - n];
      } else {
        const int i = lane - n - m;
        t -= fmaf(delta, dyn[i], dxn[i]);
        dz = dyn[i];
      }
      const double zv = z0 + widen(dz), rv = r0 + widen(t);
      zp[(size_t)k * zstride] = zv;
      resp[(size_t)k * rstride] = rv;
      zbits = max(zbits, abs_bits(zv));
      dzbits = max(dzbits, abs_bits(widen(dz)));
      rbits = max(rbits, abs_bits(rv));
    }
    float *t1 = dx; dx = dxn; dxn = t1;
    float *t2 = dy; dy = dyn; dyn = t2;
  }
  // terminal rows x_N: res += Q_N dx_N - dy_N
  __syncwarp();
  for (int e = lane; e < nn; e += 32) {
    const int i = e / n, j = e - i * n;
    if (i <= j) {
      const float v = f64_to_f32_rz(__ldg(I.Q + (size_t)N * nn + e));
      s.Q[i * N4 + j] = v;
      s.Q[j * N4 + i] = v;
    }
  }
  __syncwarp();
  if (lane < n) {
    float2 qr2[H2], xr[H2];
    lds_row2<n>(s.Q + lane * N4, qr2);
    lds_row2<n>(dx, xr);
    const float t = dot2<n>(qr2, xr) - dy[lane];
    double *dst = rq + (size_t)N * n + lane;
    const double nv = __ldcg(dst) + widen(t);
    *dst = nv;
    rbits = max(rbits, abs_bits(nv));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
    zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
    dzbits = max(dzbits, __shfl_xor_sync(0xffffffffu, dzbits, o));
  }
  if (lane == 0) {
    const double rmax = bits_to_double(rbits), zmax = bits_to_double(zbits);
    // rounding bound of this pass's FP32 residual update, accumulated over
    // passes and included in the reported backward error
    stp->upd += 2.0 * RS * 0x1p-24 * stp->kmax * bits_to_double(dzbits);
    const double den = stp->kmax * zmax + stp->bmax;
    const double rel = den > 0.0 ? (rmax + stp->upd) / den : rmax + stp->upd;
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

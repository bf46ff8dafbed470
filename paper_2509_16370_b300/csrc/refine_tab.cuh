// refine_tab.cuh -- refinement pass of the mixed-precision path for the sizes
// of the tableau sweep (tab32.cuh): one warp per instance, FP32 factor and
// FP32 data copies written by the sweep, FP64 iterate and residual.
//
// One pass solves K dz = -res with the stored factor (Corollary p-recurrence
// backward, eq. recover-x0 / control-law / recover-x forward), adds dz to z
// in FP64 and updates the FP64 residual as res <- res + K dz, with K dz in
// FP32 (|dz| ~ u_32 |z|, so the update is accurate to ~u_32^2 |K||z|;
// convergence is certified for rel plus the update's rounding bound).  The
// rows of K dz for stage k (Section "Residual Computation"):
//   x rows  Q_k dx_k + M_k du_k + A_k^T dy_{k+1} - dy_k
//   u rows  M_k^T dx_k + R_k du_k + B_k^T dy_{k+1}
//   c rows  A_k dx_k + B_k du_k - dx_{k+1} - delta dy_{k+1}
// Each lane r < 2n+m walks three coefficient rows of its K dz row.
//
// Every stage's operands (factor rows, transposed copies, FP64 residual and
// iterate entries) arrive by cp.async in a ring of shared-memory slots
// several stages ahead of the dependency chain, so the chain itself is the
// three (backward) and three (forward) broadcast rounds of its matrix-vector
// products.
#pragma once

#include <cstddef>

#include "common.cuh"
#include "residual32.cuh"
#include "tab32.cuh"

namespace rlqr {

template <int NX, int NU>
struct Rt32 {
  static constexpr int n = NX, m = NU;
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4;
  struct BSlot {  // backward stage k
    alignas(16) float W[NX * N4];   // rows of W_{k+1}
    alignas(16) float At[NX * N4];  // row i = column i of A_k
    alignas(16) float Kt[NX * M4];  // row i = column i of K_k
    alignas(16) float Bt[NU * N4];  // row t = column t of B_k
    alignas(16) float Gi[NU * M4];  // rows of G_k^{-1}
    double q[N4], r[M4], c[N4];     // residual rows q_k, r_k, c_{k+1}
  };
  struct FSlot {  // forward stage k
    alignas(16) float K[NU * N4];
    alignas(16) float A[NX * N4];
    alignas(16) float At[NX * N4];
    alignas(16) float B[NX * M4];
    alignas(16) float Bt[NU * N4];
    alignas(16) float W[NX * N4];   // W_{k+1}
    alignas(16) float Q[NX * N4];   // symmetric (upper triangle mirrored)
    alignas(16) float M[NX * M4];
    alignas(16) float Mt[NU * N4];
    alignas(16) float R[NU * M4];   // symmetric (upper triangle mirrored)
    alignas(16) float p[N4];        // p_{k+1} of the correction
    alignas(16) float kk[M4];       // k_k of the correction
    double c[N4];                   // residual rows c_{k+1} (right-hand side)
    double z[2 * NX + NU];          // iterate entries this lane updates (row layout below)
    double res[2 * NX + NU];        // residual entries this lane updates
  };
  static constexpr int DB = 8, DF = 5;
  static constexpr size_t kRing = DB * sizeof(BSlot) > DF * sizeof(FSlot) ? DB * sizeof(BSlot)
                                                                          : DF * sizeof(FSlot);
  alignas(16) unsigned char ring[kRing];
  alignas(16) float zero[N4 + M4];
  alignas(16) float p[N4];
  alignas(16) float g[N4];
  alignas(16) float h[M4];
  alignas(16) float cr[N4];
  alignas(16) float qr[N4];
  alignas(16) float rr[M4];
  alignas(16) float w[N4];
  alignas(16) float du[M4];
  alignas(16) float d[4][N4];  // dx_k, dy_k, dx_{k+1}, dy_{k+1} (rotating)
};

// FUSED (the first pass of the fused route): the residual of the solution
// is not read but computed here, stage by stage ahead of the backward chain
// that consumes it (Res32Rows, float-float as in k_res32, in a Rs32Warp
// after the Rt32 in shared memory), and written for the forward pass; the
// norms of the backward error come from the same rows.
template <int NX, int NU, bool FUSED>
__device__ __forceinline__ void refine_tab_instance(const BatchArgs &a, int slot,
                                                    unsigned char *smem_raw);

template <int NX, int NU, bool FUSED>
__host__ __device__ constexpr size_t refine_tab_smem() {
  return sizeof(Rt32<NX, NU>) + (FUSED ? sizeof(Rs32Warp<NX, NU>) : 0);
}

// One instance per block; passes after the first use fewer blocks than
// instances (most instances have converged) and stride over the slots.
template <int NX, int NU, bool FUSED>
__global__ void __launch_bounds__(32) k_refine_tab(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int slot = blockIdx.x; slot < a.count; slot += gridDim.x) {
    refine_tab_instance<NX, NU, FUSED>(a, slot, smem_raw);
    __syncwarp();
  }
}

template <int NX, int NU, bool FUSED>
__device__ __forceinline__ void refine_tab_instance(const BatchArgs &a, int slot,
                                                    unsigned char *smem_raw) {
  static_assert(tab32_fits<NX, NU>(), "dimensions outside the tableau kernels");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int H2 = n / 2, U2 = (m + 1) / 2;
  using SM = Rt32<NX, NU>;
  using BS = typename SM::BSlot;
  using FS = typename SM::FSlot;
  constexpr int N4 = SM::N4, M4 = SM::M4, DB = SM::DB, DF = SM::DF;
  constexpr int RS = 2 * n + m;  // residual rows of a stage
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  Rs32Warp<NX, NU> &rsw = *reinterpret_cast<Rs32Warp<NX, NU> *>(smem_raw + sizeof(SM));
  const int lane = threadIdx.x;
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

  // this lane's stage-independent element positions (lane-strided elements
  // of an n x n, n x m and m x m block; destination offsets of the row-major
  // and transposed copies)
  int oN[CP], oNt[CP], oB[CB], oBt[CB], oK[CB], oKt[CB], oR[CR], oRs[CR];
  bool upN[CP], upR[CR];
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    const int e = lane + 32 * i, r = e / n, c = e - r * n;
    oN[i] = r * N4 + c;
    oNt[i] = c * N4 + r;
    upN[i] = r <= c;
  }
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int e = lane + 32 * i, r = e / m, c = e - r * m;  // n x m (B, M)
    oB[i] = r * M4 + c;
    oBt[i] = c * N4 + r;
    const int t = e / n, j = e - t * n;                      // m x n (K)
    oK[i] = t * N4 + j;
    oKt[i] = j * M4 + t;
  }
#pragma unroll
  for (int i = 0; i < CR; ++i) {
    const int e = lane + 32 * i, r = e / m, c = e - r * m;
    oR[i] = r * M4 + c;
    oRs[i] = c * M4 + r;
    upR[i] = r <= c;
  }
  {  // zero the shared memory: padding entries of every slot read as zeros
    float4 *z4 = reinterpret_cast<float4 *>(smem_raw);
    for (int e = lane; e < (int)(sizeof(SM) / 16); e += 32) z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  // Sizes of chunk16_size (rows of a multiple of 16 bytes, so the slots have
  // no row padding): the per-stage blocks that are contiguous in global
  // memory (factor rows, row-major data copies, residual rows) are staged as
  // 16-byte chunks, the lanes taking them in turn; the transposed and the
  // mirrored copies element by element as for the other sizes.
  constexpr bool kC16 = chunk16_size(NX, NU);
  constexpr int NBB = FUSED ? 2 : 5, NBF = 8;
  constexpr int CB16 = (nn * 4 + mmm * 4 + (FUSED ? 0 : (2 * n + m) * 8)) / 16;
  constexpr int CF16 = (2 * nn * 4 + 3 * nm * 4 + n * 4 + m * 4 + n * 8) / 16;
  ChunkPlan<NBB, kC16 ? (CB16 + 31) / 32 : 1> bplan;
  ChunkPlan<NBF, kC16 ? (CF16 + 31) / 32 : 1> fplan;
  if constexpr (kC16) {
    static_assert(SM::N4 == NX && SM::M4 == NU, "unpadded slots");
    static_assert(sizeof(BS) % 16 == 0 && sizeof(FS) % 16 == 0, "16-byte slot strides");
    static_assert(offsetof(BS, W) % 16 == 0 && offsetof(BS, Gi) % 16 == 0 &&
                      offsetof(BS, q) % 16 == 0 && offsetof(BS, r) % 16 == 0 &&
                      offsetof(BS, c) % 16 == 0 && offsetof(FS, K) % 16 == 0 &&
                      offsetof(FS, A) % 16 == 0 && offsetof(FS, B) % 16 == 0 &&
                      offsetof(FS, W) % 16 == 0 && offsetof(FS, M) % 16 == 0 &&
                      offsetof(FS, c) % 16 == 0 && offsetof(FS, p) % 16 == 0 &&
                      offsetof(FS, kk) % 16 == 0,
                  "16-byte block offsets");
    auto cp = [](const void *p) { return reinterpret_cast<const char *>(p); };
    if constexpr (FUSED) {
      const Blk16 bb[NBB] = {{cp(gW + nn), nn * 4, offsetof(BS, W), nn / 4},
                             {cp(gGi), mmm * 4, offsetof(BS, Gi), mmm / 4}};
      bplan.init(bb, lane);
    } else {
      const Blk16 bb[NBB] = {{cp(gW + nn), nn * 4, offsetof(BS, W), nn / 4},
                             {cp(gGi), mmm * 4, offsetof(BS, Gi), mmm / 4},
                             {cp(rq), n * 8, offsetof(BS, q), n / 2},
                             {cp(rr), m * 8, offsetof(BS, r), m / 2},
                             {cp(rc + n), n * 8, offsetof(BS, c), n / 2}};
      bplan.init(bb, lane);
    }
    const Blk16 fb[NBF] = {
        {cp(gK), nm * 4, offsetof(FS, K), nm / 4},    {cp(gAf), nn * 4, offsetof(FS, A), nn / 4},
        {cp(gBf), nm * 4, offsetof(FS, B), nm / 4},   {cp(gW + nn), nn * 4, offsetof(FS, W), nn / 4},
        {cp(gMf), nm * 4, offsetof(FS, M), nm / 4},   {cp(gpv + n), n * 4, offsetof(FS, p), n / 4},
        {cp(gkv), m * 4, offsetof(FS, kk), m / 4},    {cp(rc + n), n * 8, offsetof(FS, c), n / 2}};
    fplan.init(fb, lane);
  }

  // rows of the backward rounds this lane works on: bi (a row < n), bt (a
  // row < m) and bk (row lane - n of G^{-1} on lanes n .. n+m-1); 0 elsewhere
  const int bi = lane < n ? lane : 0, bt = lane < m ? lane : 0;
  const int bk = (lane >= n && lane < n + m) ? lane - n : 0;

  // ---------------- backward: p-recurrence with the residual as right-hand side
  BS *bring = reinterpret_cast<BS *>(s.ring);
  auto bissue = [&](int k) {
    if constexpr (kC16) {
      if (k >= 0) {
        BS &d = bring[(N - 1 - k) % DB];
        bplan.issue(reinterpret_cast<unsigned char *>(&d), k);
        const float *A = gAf + (size_t)k * nn, *K = gK + (size_t)k * nm, *B = gBf + (size_t)k * nm;
#pragma unroll
        for (int i = 0; i < CP; ++i) {
          const int e = lane + 32 * i;
          if (e < nn) cp_async4(&d.At[oNt[i]], A + e);
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const int e = lane + 32 * i;
          if (e < nm) {
            cp_async4(&d.Kt[oKt[i]], K + e);
            cp_async4(&d.Bt[oBt[i]], B + e);
          }
        }
      }
      cp_async_commit();
      return;
    }
    if (k >= 0) {
      BS &d = bring[(N - 1 - k) % DB];
      const float *W = gW + (size_t)(k + 1) * nn, *A = gAf + (size_t)k * nn;
      const float *K = gK + (size_t)k * nm, *B = gBf + (size_t)k * nm, *G = gGi + (size_t)k * mmm;
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const int e = lane + 32 * i;
        if (e < nn) {
          cp_async4(&d.W[oN[i]], W + e);
          cp_async4(&d.At[oNt[i]], A + e);
        }
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int e = lane + 32 * i;
        if (e < nm) {
          cp_async4(&d.Kt[oKt[i]], K + e);
          cp_async4(&d.Bt[oBt[i]], B + e);
        }
      }
#pragma unroll
      for (int i = 0; i < CR; ++i) {
        const int e = lane + 32 * i;
        if (e < mmm) cp_async4(&d.Gi[oR[i]], G + e);
      }
      if constexpr (!FUSED) {
        if (lane < n) {
          cp_async8(&d.q[lane], rq + (size_t)k * n + lane);
          cp_async8(&d.c[lane], rc + (size_t)(k + 1) * n + lane);
        }
        if (lane < m) cp_async8(&d.r[lane], rr + (size_t)k * m + lane);
      }
    }
    cp_async_commit();
  };
  __syncwarp();
  // the residual rows computed here (FUSED): this lane's norms of the
  // backward error, and the stage pipeline of Res32Rows
  Res32Rows<NX, NU> R;
  float kmaxf = 0.f;
  unsigned long long fzbits = 0, fbbits = 0;
  if constexpr (FUSED) {
    R.init(rsw, lane, delta64);
    R.prefetch(I, N - 1, lane);
  }
  if (lane < n) {
    float v;
    if constexpr (FUSED) {
      const double v64 = res_end_row(I, lane, kmaxf, fzbits, fbbits);  // row x_N
      rq[(size_t)N * n + lane] = v64;
      v = f64_to_f32_rz(v64);
    } else {
      v = f64_to_f32_rz(__ldcg(rq + (size_t)N * n + lane));
    }
    s.p[lane] = v;
    gpv[(size_t)N * n + lane] = v;
  }
#pragma unroll 1
  for (int j = 0; j < DB - 1; ++j) bissue(N - 1 - j);
#pragma unroll 1
  for (int k = N - 1; k >= 0; --k) {
    if constexpr (FUSED) {
      // the residual rows of stage k (lane r: row r), kept in FP64 for the
      // forward pass and handed to the chain in FP32 (c rows through s.w)
      R.commit(rsw, lane, fzbits, fbbits);
      if (k > 0) R.prefetch(I, k - 1, lane);
      __syncwarp();
      if (lane < RS) {
        const double v = R.row(rsw, lane, kmaxf);
        const float vf = f64_to_f32_rz(v);
        if (lane < n) {
          rq[(size_t)k * n + lane] = v;
          s.qr[lane] = vf;
        } else if (lane < n + m) {
          rr[(size_t)k * m + lane - n] = v;
          s.rr[lane - n] = vf;
        } else {
          rc[(size_t)(k + 1) * n + lane - n - m] = v;
          s.w[lane - n - m] = vf;
        }
      }
    }
    bissue(k - (DB - 1));
    cp_async_wait<DB - 1>();
    const BS &d = bring[(N - 1 - k) % DB];
    if constexpr (FUSED) {
      __syncwarp();
      if (lane < n) s.cr[lane] = fmaf(-delta, s.p[lane], s.w[lane]);  // v = c' - delta p
    } else {
      // this lane's residual entries, truncated to FP32 (it copied them)
      const float qv = f64_to_f32_rz(d.q[bi]);
      const float cv = fmaf(-delta, s.p[bi], f64_to_f32_rz(d.c[bi]));  // v = c' - delta p
      const float rv = f64_to_f32_rz(d.r[bt]);
      if (lane < n) {
        s.qr[lane] = qv;
        s.cr[lane] = cv;
      }
      if (lane < m) s.rr[lane] = rv;
    }
    __syncwarp();
    // The rounds below run on every lane (lanes past a round's rows work on
    // row 0 and discard it): only the stores depend on the lane, so the warp
    // takes no divergent branch.
    // g = p + W v
    {
      float2 wr[H2], vr[H2];
      ld_seg<H2, 0, H2>(d.W + bi * N4, wr);
      ld_seg<H2, 0, H2>(s.cr, vr);
      const float gv = s.p[bi] + dot2<n>(wr, vr);
      if (lane < n) s.g[lane] = gv;
    }
    __syncwarp();
    // h = r' + B^T g
    float2 gr[H2];
    ld_seg<H2, 0, H2>(s.g, gr);
    {
      float2 br[H2];
      ld_seg<H2, 0, H2>(d.Bt + bt * N4, br);
      const float hv = s.rr[bt] + dot2<n>(br, gr);
      if (lane < m) s.h[lane] = hv;
    }
    __syncwarp();
    // p_k = q' + A^T g + K^T h (lanes < n);  k_k = -G^{-1} h (lanes n .. n+m-1)
    float2 hr[U2];
    ld_seg<U2, 0, U2>(s.h, hr);
    {
      float2 ar[H2], kr[U2], gi[U2];
      ld_seg<H2, 0, H2>(d.At + bi * N4, ar);
      ld_seg<U2, 0, U2>(d.Kt + bi * M4, kr);
      ld_seg<U2, 0, U2>(d.Gi + bk * M4, gi);
      float2 acc = mul2(ar[0], gr[0]), acck = mul2(gi[0], hr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], gr[q], acc);
#pragma unroll
      for (int q = 0; q < U2; ++q) acc = fma2(kr[q], hr[q], acc);
#pragma unroll
      for (int q = 1; q < U2; ++q) acck = fma2(gi[q], hr[q], acck);
      const float pv = s.qr[bi] + (acc.x + acc.y), kv = -(acck.x + acck.y);
      if (lane < n) {
        s.p[lane] = pv;
        gpv[(size_t)k * n + lane] = pv;
      } else if (lane < n + m) {
        gkv[(size_t)k * m + lane - n] = kv;
      }
    }
    __syncwarp();  // the slot may be refilled from here on
  }
  if constexpr (FUSED) {
    if (lane < n) rc[lane] = res_end_row(I, n + lane, kmaxf, fzbits, fbbits);  // row c_0
  }
  cp_async_wait<0>();
  __threadfence_block();  // p, k and the residual rows, read back by cp.async below
  __syncwarp();

  // ---------------- forward rollout, FP64 update of z and of the residual
  // sbits: max over the updated rows of sum |coefficient| |dz term| (FP32),
  // which bounds the rounding of this pass's FP32 residual update
  unsigned long long rbits = 0, zbits = 0, sbits = 0;
  // this lane's row of K dz: coefficient rows (offsets into a slot) of dx_k,
  // du_k, dy_{k+1}, and its FP64 iterate / residual entries
  const bool xr_ = lane < n, ur_ = lane >= n && lane < n + m, cr_ = lane >= n + m && lane < RS;
  double *zp = nullptr, *resp = nullptr;  // entry at stage 0; stride zs, rs per stage
  size_t zs = 0, rs = 0;
  if (xr_) {
    zp = I.x + n + lane; zs = n; resp = rq + lane; rs = n;
  } else if (ur_) {
    zp = I.u + (lane - n); zs = m; resp = rr + (lane - n); rs = m;
  } else if (cr_) {
    zp = I.y + n + (lane - n - m); zs = n; resp = rc + n + (lane - n - m); rs = n;
  }
  FS *fring = reinterpret_cast<FS *>(s.ring);
  auto fissue = [&](int k) {
    if constexpr (kC16) {
      if (k < N) {
        FS &f = fring[k % DF];
        fplan.issue(reinterpret_cast<unsigned char *>(&f), k);
        const float *A = gAf + (size_t)k * nn, *Q = gQf + (size_t)k * nn;
        const float *B = gBf + (size_t)k * nm, *M = gMf + (size_t)k * nm;
        const float *R = gRf + (size_t)k * mmm;
#pragma unroll
        for (int i = 0; i < CP; ++i) {
          const int e = lane + 32 * i;
          if (e < nn) {
            cp_async4(&f.At[oNt[i]], A + e);
            if (upN[i]) {
              cp_async4(&f.Q[oN[i]], Q + e);
              cp_async4(&f.Q[oNt[i]], Q + e);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const int e = lane + 32 * i;
          if (e < nm) {
            cp_async4(&f.Bt[oBt[i]], B + e);
            cp_async4(&f.Mt[oBt[i]], M + e);
          }
        }
#pragma unroll
        for (int i = 0; i < CR; ++i) {
          const int e = lane + 32 * i;
          if (e < mmm && upR[i]) {
            cp_async4(&f.R[oR[i]], R + e);
            cp_async4(&f.R[oRs[i]], R + e);
          }
        }
        if (zp) {
          cp_async8(&f.z[lane], zp + (size_t)k * zs);
          cp_async8(&f.res[lane], resp + (size_t)k * rs);
        }
      }
      cp_async_commit();
      return;
    }
    if (k < N) {
      FS &f = fring[k % DF];
      const float *W = gW + (size_t)(k + 1) * nn, *A = gAf + (size_t)k * nn, *Q = gQf + (size_t)k * nn;
      const float *K = gK + (size_t)k * nm, *B = gBf + (size_t)k * nm, *M = gMf + (size_t)k * nm;
      const float *R = gRf + (size_t)k * mmm;
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const int e = lane + 32 * i;
        if (e < nn) {
          cp_async4(&f.A[oN[i]], A + e);
          cp_async4(&f.At[oNt[i]], A + e);
          cp_async4(&f.W[oN[i]], W + e);
          if (upN[i]) {
            cp_async4(&f.Q[oN[i]], Q + e);
            cp_async4(&f.Q[oNt[i]], Q + e);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int e = lane + 32 * i;
        if (e < nm) {
          cp_async4(&f.K[oK[i]], K + e);
          cp_async4(&f.B[oB[i]], B + e);
          cp_async4(&f.Bt[oBt[i]], B + e);
          cp_async4(&f.M[oB[i]], M + e);
          cp_async4(&f.Mt[oBt[i]], M + e);
        }
      }
#pragma unroll
      for (int i = 0; i < CR; ++i) {
        const int e = lane + 32 * i;
        if (e < mmm && upR[i]) {
          cp_async4(&f.R[oR[i]], R + e);
          cp_async4(&f.R[oRs[i]], R + e);
        }
      }
      if (lane < n) {
        cp_async4(&f.p[lane], gpv + (size_t)(k + 1) * n + lane);
        cp_async8(&f.c[lane], rc + (size_t)(k + 1) * n + lane);
      }
      if (lane < m) cp_async4(&f.kk[lane], gkv + (size_t)k * m + lane);
      if (zp) {
        cp_async8(&f.z[lane], zp + (size_t)k * zs);
        cp_async8(&f.res[lane], resp + (size_t)k * rs);
      }
    }
    cp_async_commit();
  };
  // x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c'_0 - delta p_0
  float *dx = s.d[0], *dy = s.d[1], *dxn = s.d[2], *dyn = s.d[3];
  if (lane < n) s.w[lane] = fmaf(-delta, s.p[lane], f64_to_f32_rz(__ldcg(rc + lane)));
  __syncwarp();
  if (lane < n) {
    float2 wr[H2], vr[H2];
    const float *w0 = gW + lane * n;
#pragma unroll
    for (int q = 0; q < H2; ++q) wr[q] = __ldcg(reinterpret_cast<const float2 *>(w0) + q);
    ld_seg<H2, 0, H2>(s.w, vr);
    const float t = dot2<n>(wr, vr);
    const float dxv = fmaf(-delta, t, s.w[lane]), dyv = t + s.p[lane];
    dx[lane] = dxv;
    dy[lane] = dyv;
    const double xv = I.x[lane] + widen(dxv), yv = I.y[lane] + widen(dyv);
    I.x[lane] = xv;
    I.y[lane] = yv;
    zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
    const double r0 = __ldcg(rc + lane) - widen(dxv) - delta64 * widen(dyv);
    rc[lane] = r0;
    rbits = max(rbits, abs_bits(r0));
  }
  // the ring held the backward slots: clear it for the forward layout's padding
  __syncwarp();
  {
    float4 *z4 = reinterpret_cast<float4 *>(s.ring);
    for (int e = lane; e < (int)(SM::kRing / 16); e += 32) z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncwarp();
#pragma unroll 1
  for (int j = 0; j < DF - 1; ++j) fissue(j);
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    fissue(k + DF - 1);
    cp_async_wait<DF - 1>();
    __syncwarp();
    const FS &f = fring[k % DF];
    // (every lane runs each round, lanes past its rows on row 0; only the
    // stores depend on the lane)
    // du_k = K_k dx_k + k_k
    float2 xr[H2];
    ld_seg<H2, 0, H2>(dx, xr);
    {
      float2 kr[H2];
      ld_seg<H2, 0, H2>(f.K + bt * N4, kr);
      const float duv = dot2<n>(kr, xr) + f.kk[bt];
      if (lane < m) s.du[lane] = duv;
    }
    __syncwarp();
    // w = A dx + B du + c'_{k+1} - delta p_{k+1}
    float2 ur[U2];
    ld_seg<U2, 0, U2>(s.du, ur);
    float wv;
    {
      float2 ar[H2], br[U2];
      ld_seg<H2, 0, H2>(f.A + bi * N4, ar);
      ld_seg<U2, 0, U2>(f.B + bi * M4, br);
      float2 acc = mul2(ar[0], xr[0]);
#pragma unroll
      for (int q = 1; q < H2; ++q) acc = fma2(ar[q], xr[q], acc);
#pragma unroll
      for (int q = 0; q < U2; ++q) acc = fma2(br[q], ur[q], acc);
      wv = (acc.x + acc.y) + fmaf(-delta, f.p[bi], f64_to_f32_rz(f.c[bi]));
      if (lane < n) s.w[lane] = wv;
    }
    __syncwarp();
    // dx_{k+1} = w - delta W w, dy_{k+1} = W w + p_{k+1}
    float2 vr[H2];
    ld_seg<H2, 0, H2>(s.w, vr);
    {
      float2 wr[H2];
      ld_seg<H2, 0, H2>(f.W + bi * N4, wr);
      const float t = dot2<n>(wr, vr);
      const float dxv = fmaf(-delta, t, wv), dyv = t + f.p[bi];
      if (lane < n) {
        dxn[lane] = dxv;
        dyn[lane] = dyv;
      }
    }
    __syncwarp();
    // K dz rows of stage k and the FP64 updates (lanes < RS)
    if (lane < RS) {
      const float *c1 = xr_ ? f.Q + lane * N4 : ur_ ? f.Mt + (lane - n) * N4 : f.A + (lane - n - m) * N4;
      const float *c2 = xr_ ? f.M + lane * M4 : ur_ ? f.R + (lane - n) * M4 : f.B + (lane - n - m) * M4;
      const float *c3 = xr_ ? f.At + lane * N4 : ur_ ? f.Bt + (lane - n) * N4 : s.zero;
      float2 a1[H2], a2[U2], a3[H2], y3[H2];
      ld_seg<H2, 0, H2>(c1, a1);
      ld_seg<U2, 0, U2>(c2, a2);
      ld_seg<H2, 0, H2>(c3, a3);
      ld_seg<H2, 0, H2>(dyn, y3);
      float2 acc = mul2(a1[0], xr[0]), sab = mul2(abs2(a1[0]), abs2(xr[0]));
#pragma unroll
      for (int q = 1; q < H2; ++q) {
        acc = fma2(a1[q], xr[q], acc);
        sab = fma2(abs2(a1[q]), abs2(xr[q]), sab);
      }
#pragma unroll
      for (int q = 0; q < U2; ++q) {
        acc = fma2(a2[q], ur[q], acc);
        sab = fma2(abs2(a2[q]), abs2(ur[q]), sab);
      }
#pragma unroll
      for (int q = 0; q < H2; ++q) {
        acc = fma2(a3[q], y3[q], acc);
        sab = fma2(abs2(a3[q]), abs2(y3[q]), sab);
      }
      // the row's own terms, by selects rather than branches: x rows -dy_k
      // (dz = dx_{k+1}), u rows none (dz = du_k), c rows -dx_{k+1} - delta
      // dy_{k+1} (dz = dy_{k+1})
      const float dyx = dy[bi], dxx = dxn[bi], duu = s.du[bk];
      const int ic = cr_ ? lane - n - m : 0;
      const float dxc = dxn[ic], dyc = dyn[ic];
      float t = acc.x + acc.y, sa = sab.x + sab.y;
      t -= xr_ ? dyx : (cr_ ? fmaf(delta, dyc, dxc) : 0.f);
      sa += xr_ ? fabsf(dyx) : (cr_ ? fmaf(delta, fabsf(dyc), fabsf(dxc)) : 0.f);
      const float dz = xr_ ? dxx : (ur_ ? duu : dyc);
      const double zv = f.z[lane] + widen(dz), rv = f.res[lane] + widen(t);
      zp[(size_t)k * zs] = zv;
      resp[(size_t)k * rs] = rv;
      zbits = max(zbits, abs_bits(zv));
      rbits = max(rbits, abs_bits(rv));
      sbits = max(sbits, abs_bits(widen(sa)));
    }
    float *t1 = dx; dx = dxn; dxn = t1;
    float *t2 = dy; dy = dyn; dyn = t2;
    __syncwarp();  // the slot and the rotated vectors are free from here on
  }
  cp_async_wait<0>();
  // terminal rows x_N: res += Q_N dx_N - dy_N (Q_N upper triangle, FP64 data)
  if (lane < n) {
    float t = -dy[lane], sa = fabsf(dy[lane]);
    const double *QN = I.Q + (size_t)N * nn;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const float qv = f64_to_f32_rz(__ldg(QN + min(lane, j) * n + max(lane, j)));
      t = fmaf(qv, dx[j], t);
      sa = fmaf(fabsf(qv), fabsf(dx[j]), sa);
    }
    double *dst = rq + (size_t)N * n + lane;
    const double nv = __ldcg(dst) + widen(t);
    *dst = nv;
    rbits = max(rbits, abs_bits(nv));
    sbits = max(sbits, abs_bits(widen(sa)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
    zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
    sbits = max(sbits, __shfl_xor_sync(0xffffffffu, sbits, o));
  }
  if constexpr (FUSED) {
    // the norms of K and b from the rows computed in the backward pass; the
    // rounding bound starts from this freshly computed residual
    for (int o = 16; o > 0; o >>= 1) {
      kmaxf = fmaxf(kmaxf, __shfl_xor_sync(0xffffffffu, kmaxf, o));
      fbbits = max(fbbits, __shfl_xor_sync(0xffffffffu, fbbits, o));
    }
    if (lane == 0) {
      stp->kmax = (double)kmaxf;
      stp->bmax = bits_to_double(fbbits);
      stp->upd = 0.0;
    }
  }
  if (lane == 0) {
    const double rmax = bits_to_double(rbits), zmax = bits_to_double(zbits);
    // Rounding of this pass's FP32 residual update, row by row: at most
    // RS + 3 rounded operations and coefficients truncated to FP32 (relative
    // error below 2 u_32) give |error| <= (RS + 6) u_32 S_row (1 + O(u_32)),
    // S_row = sum |coefficient| |dz term|; S_row itself is computed in FP32
    // (relative error below (RS + 3) u_32).  (RS + 8) u_32 (1 + 2^-16)
    // max_row S_row therefore bounds the update's error in every entry.  The
    // bound accumulates over passes, and the backward error reported (and
    // tested against tol) includes it.
    stp->upd += (double)(RS + 8) * 0x1p-24 * (1.0 + 0x1p-16) * bits_to_double(sbits);
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

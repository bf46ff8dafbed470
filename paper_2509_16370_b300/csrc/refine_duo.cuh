// refine_duo.cuh -- refinement pass of the mixed-precision path with two
// warps per instance, for the sizes of the tableau sweep (tab32.cuh).
//
// The pass solves K dz = -res with the stored FP32 factor (Corollary
// p-recurrence backward, eq. recover-x0 / control-law / recover-x forward),
// adds dz to z in FP64 and updates the FP64 residual as res <- res + K dz
// (Section "Residual Computation"), exactly as k_refine_tab does.  Here the
// work is split by its place on the dependency chain:
//   warp 0 (the chain) runs only the recursion: per stage three dependent
//     broadcast matrix-vector products backward (g, h, p_k / k_k) and three
//     forward (du_k, w, dx_{k+1} / dy_{k+1});
//   warp 1 (the helper) issues every cp.async copy of the stage operands,
//     prepares the right-hand sides (FP64 -> FP32), and in the forward pass
//     computes the rows of K dz with their FP64 updates of z and res.  In the
//     fused variant (first pass of the fused residual route) it also computes
//     the residual of the solution itself, stage by stage ahead of the chain
//     (Res32Rows, float-float), so the residual's issue load runs beside the
//     chain instead of on it.
// Splitting the stage costs instructions (hand-over, vectors re-read by the
// helper: about 18 % more per stage) and the 9 named barriers a block uses
// cap an SM at 7 blocks.  So the split pays while the SMs hold few
// instances, each instance's chain being the bound, and loses at full
// occupancy, where the one-warp pass (refine_tab.cuh) keeps fewer
// instructions in flight; the batched driver chooses per launch.
//
// The warps hand stages over through named barriers (bar.arrive by the
// producing warp, bar.sync by the consuming one; hardware waits on barriers
// whose every arrival has a matching sync, so no wait can be left open):
//   backward  FULL[t % DB]   helper -> chain  stage t's slot is ready
//             EMPTY[t % NE]  chain -> helper  stage t's slot may be refilled
//   forward   FULL[k % NF]   helper -> chain  stage k's slot is ready
//             VEC[k % NV]    chain -> helper  dx_{k+1}, dy_{k+1}, du_k written
// (t = N - 1 - k counts the backward stages).  The helper runs up to
// DB - PB - 1 stages ahead of the chain backward; forward the chain runs up
// to LF stages ahead of the helper.  The counts NE = DB - PB, NF = NV = LF + 1
// and the vector ring depth LF + 2 are the smallest for which no barrier can
// receive a second arrival before the sync of its first and no ring entry
// is overwritten while it is read.
#pragma once

#include <cstddef>

#include "common.cuh"
#include "residual32.cuh"
#include "tab32.cuh"

namespace rlqr {

template <int ID>
__device__ __forceinline__ void duo_sync_id() {
  asm volatile("bar.sync %0, 64;" ::"n"(ID) : "memory");
}
template <int ID>
__device__ __forceinline__ void duo_arrive_id() {
  asm volatile("bar.arrive %0, 64;" ::"n"(ID) : "memory");
}
// Barrier id in [LO, HI] as an immediate (a register id would make the
// compiler reserve all 16 barriers of the CTA).
template <int LO, int HI>
__device__ __forceinline__ void duo_sync(int id) {
  if constexpr (LO == HI) {
    duo_sync_id<LO>();
  } else {
    if (id == LO) duo_sync_id<LO>();
    else duo_sync<LO + 1, HI>(id);
  }
}
template <int LO, int HI>
__device__ __forceinline__ void duo_arrive(int id) {
  if constexpr (LO == HI) {
    duo_arrive_id<LO>();
  } else {
    if (id == LO) duo_arrive_id<LO>();
    else duo_arrive<LO + 1, HI>(id);
  }
}

__host__ __device__ constexpr size_t duo_max(size_t x, size_t y) { return x > y ? x : y; }
__host__ __device__ constexpr size_t duo_up16(size_t x) { return (x + 15) / 16 * 16; }

template <int NX, int NU>
struct Rd32 {
  static constexpr int N4 = (NX + 3) / 4 * 4, M4 = (NU + 3) / 4 * 4, RS = 2 * NX + NU;
  static constexpr int DB = 5, PB = 2, NE = DB - PB;   // backward ring
  static constexpr int LF = 3, DF = 6, NF = LF + 1, NV = LF + 1, NVR = LF + 2;  // forward
  struct BSlot {  // backward stage k
    alignas(16) float W[NX * N4];   // rows of W_{k+1}
    alignas(16) float At[NX * N4];  // row i = column i of A_k
    alignas(16) float Kt[NX * M4];  // row i = column i of K_k
    alignas(16) float Bt[NU * N4];  // row t = column t of B_k
    alignas(16) float Gi[NU * M4];  // rows of G_k^{-1}
    alignas(16) float qf[N4];       // residual rows q_k, r_k, c_{k+1} in FP32 (helper)
    alignas(16) float rf[M4];
    alignas(16) float cf[N4];
    double q[N4], r[M4], c[N4];     // the same rows in FP64, copied (non-fused)
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
    alignas(16) float cv[N4];       // c'_{k+1} - delta p_{k+1} (helper)
    double c[N4];                   // residual rows c_{k+1}
    double z[RS];                   // iterate entries the helper lanes update
    double res[RS];                 // residual entries the helper lanes update
  };
  struct Vec {  // chain results of one stage: dx_k, dy_k, du_k
    alignas(16) float dx[N4];
    alignas(16) float dy[N4];
    alignas(16) float du[M4];
  };
  // the fused residual's split stage sits in the ring behind the backward slots
  static constexpr size_t kResOff = duo_up16(DB * sizeof(BSlot));
  static constexpr size_t kRing =
      duo_max(DF * sizeof(FSlot), kResOff + sizeof(Rs32Warp<NX, NU>));
  alignas(16) unsigned char ring[kRing];
  alignas(16) float zero[N4 + M4];
  alignas(16) float p[N4];   // chain: p_{k+1} backward, p_0 at the forward start
  alignas(16) float g[N4];
  alignas(16) float h[M4];
  alignas(16) float cr[N4];
  alignas(16) float w[N4];
  Vec vec[NVR];
  unsigned long long red[2][5];  // per warp: rbits, zbits, sbits, bbits, kmax (float bits)
};

template <int NX, int NU>
__host__ __device__ constexpr size_t refine_duo_smem() {
  return sizeof(Rd32<NX, NU>);
}

template <int NX, int NU, bool FUSED>
__device__ __forceinline__ void refine_duo_instance(const BatchArgs &a, int slot,
                                                    unsigned char *smem_raw);

// One instance per block of two warps; passes after the first use fewer
// blocks than instances (most instances have converged) and stride over the
// slots.  Seven blocks per SM hold a 1036-instance batch in one wave.
template <int NX, int NU, bool FUSED>
__global__ void __launch_bounds__(64, 7) k_refine_duo(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int slot = blockIdx.x; slot < a.count; slot += gridDim.x) {
    refine_duo_instance<NX, NU, FUSED>(a, slot, smem_raw);
    __syncthreads();
  }
}

template <int NX, int NU, bool FUSED>
__device__ __forceinline__ void refine_duo_instance(const BatchArgs &a, int slot,
                                                    unsigned char *smem_raw) {
  static_assert(tab32_fits<NX, NU>(), "dimensions outside the tableau kernels");
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int H2 = n / 2, U2 = (m + 1) / 2;
  using SM = Rd32<NX, NU>;
  using BS = typename SM::BSlot;
  using FS = typename SM::FSlot;
  using VC = typename SM::Vec;
  constexpr int N4 = SM::N4, M4 = SM::M4, RS = SM::RS;
  constexpr int DB = SM::DB, PB = SM::PB, NE = SM::NE;
  constexpr int LF = SM::LF, DF = SM::DF, NF = SM::NF, NV = SM::NV, NVR = SM::NVR;
  constexpr int CP = (nn + 31) / 32, CB = (nm + 31) / 32, CR = (mmm + 31) / 32;
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rows of the chain's rounds this lane works on: bi (< n), bt (< m), bk (row
  // lane - n of G^{-1} on lanes n .. n+m-1); 0 elsewhere
  const int bi = lane < n ? lane : 0, bt = lane < m ? lane : 0;
  const int bk = (lane >= n && lane < n + m) ? lane - n : 0;
  const int b = inst_of(a, slot);
  const Inst I = get_inst(a, b);
  InstState *stp = I.st;
  if (stp->converged || stp->pivot_status == RLQR_ERR_SINGULAR) return;  // both warps
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

  // this lane's stage-independent element positions (helper: lane-strided
  // elements of an n x n, n x m and m x m block; destination offsets of the
  // row-major and transposed copies)
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
    for (int e = threadIdx.x; e < (int)(sizeof(SM) / 16); e += 64)
      z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();

  // maxima of this lane: |res|, |z|, the update's rounding sums, and (fused)
  // |b| and the row sums of |K|
  unsigned long long rbits = 0, zbits = 0, sbits = 0, fzbits = 0, fbbits = 0;
  float kmaxf = 0.f;

  // ---------------- backward: p-recurrence with the residual as right-hand side
  BS *bring = reinterpret_cast<BS *>(s.ring);
  if (warp == 0) {
    // ----- chain
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
    __syncwarp();
#pragma unroll 1
    for (int t = 0; t < N; ++t) {
      const int k = N - 1 - t;
      duo_sync<1, DB>(1 + t % DB);  // FULL: stage k's slot is ready
      const BS &d = bring[t % DB];
      // (every lane runs each round on a clamped row; only the stores depend
      // on the lane, so the chain takes no divergent branch)
      {
        const float cv = fmaf(-delta, s.p[bi], d.cf[bi]);  // v = c' - delta p
        if (lane < n) s.cr[lane] = cv;
      }
      __syncwarp();
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
        const float hv = d.rf[bt] + dot2<n>(br, gr);
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
        const float pv = d.qf[bi] + (acc.x + acc.y), kv = -(acck.x + acck.y);
        if (lane < n) {
          s.p[lane] = pv;
          gpv[(size_t)k * n + lane] = pv;
        } else if (lane < n + m) {
          gkv[(size_t)k * m + lane - n] = kv;
        }
      }
      __syncwarp();
      if (t < N - DB) duo_arrive<DB + 1, DB + NE>(DB + 1 + t % NE);  // EMPTY: slot free
    }
  } else {
    // ----- helper: copies of stage k = N - 1 - t into slot t % DB.  Sizes of
    // chunk16_size: the blocks contiguous in global memory (W rows, G^{-1},
    // residual rows) as 16-byte chunks, the lanes taking them in turn.
    constexpr bool kC16 = chunk16_size(NX, NU);
    constexpr int NBB = FUSED ? 2 : 5;
    constexpr int CB16 = (nn * 4 + mmm * 4 + (FUSED ? 0 : (2 * n + m) * 8)) / 16;
    ChunkPlan<NBB, kC16 ? (CB16 + 31) / 32 : 1> bplan;
    if constexpr (kC16) {
      static_assert(SM::N4 == NX && SM::M4 == NU, "unpadded slots");
      static_assert(sizeof(BS) % 16 == 0 && offsetof(BS, W) % 16 == 0 &&
                        offsetof(BS, Gi) % 16 == 0 && offsetof(BS, q) % 16 == 0 &&
                        offsetof(BS, r) % 16 == 0 && offsetof(BS, c) % 16 == 0,
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
    }
    auto bissue = [&](int t) {
      if constexpr (kC16) {
        if (t < N) {
          const int k = N - 1 - t;
          BS &d = bring[t % DB];
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
      if (t < N) {
        const int k = N - 1 - t;
        BS &d = bring[t % DB];
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
    Rs32Warp<NX, NU> &rsw = *reinterpret_cast<Rs32Warp<NX, NU> *>(s.ring + SM::kResOff);
    Res32Rows<NX, NU> R;
    if constexpr (FUSED) {
      R.init(rsw, lane, delta64);
      R.prefetch(I, N - 1, lane);
    }
#pragma unroll 1
    for (int j = 0; j < PB; ++j) bissue(j);
#pragma unroll 1
    for (int t = 0; t < N; ++t) {
      const int k = N - 1 - t;
      // refill the slot of stage t + PB - DB once the chain is done with it
      if (t + PB < N && t + PB >= DB) duo_sync<DB + 1, DB + NE>(DB + 1 + (t + PB - DB) % NE);
      bissue(t + PB);
      BS &d = bring[t % DB];
      if constexpr (FUSED) {
        // the residual rows of stage k (lane r: row r), kept in FP64 for
        // the forward pass and handed to the chain in FP32
        R.commit(rsw, lane, fzbits, fbbits);
        if (k > 0) R.prefetch(I, k - 1, lane);
        __syncwarp();
        if (lane < RS) {
          const double v = R.row(rsw, lane, kmaxf);
          const float vf = f64_to_f32_rz(v);
          if (lane < n) {
            rq[(size_t)k * n + lane] = v;
            d.qf[lane] = vf;
          } else if (lane < n + m) {
            rr[(size_t)k * m + lane - n] = v;
            d.rf[lane - n] = vf;
          } else {
            rc[(size_t)(k + 1) * n + lane - n - m] = v;
            d.cf[lane - n - m] = vf;
          }
        }
        cp_async_wait<PB>();
      } else {
        cp_async_wait<PB>();
        // this lane's residual entries, truncated to FP32 (it copied them)
        if (lane < n) {
          d.qf[lane] = f64_to_f32_rz(d.q[lane]);
          d.cf[lane] = f64_to_f32_rz(d.c[lane]);
        }
        if (lane < m) d.rf[lane] = f64_to_f32_rz(d.r[lane]);
      }
      duo_arrive<1, DB>(1 + t % DB);  // FULL
    }
    if constexpr (FUSED) {
      if (lane < n) rc[lane] = res_end_row(I, n + lane, kmaxf, fzbits, fbbits);  // row c_0
    }
  }
  cp_async_wait<0>();
  __threadfence();  // p, k and the residual rows, read back by cp.async below
  __syncthreads();
  {  // the ring held the backward slots: clear it for the forward layout's padding
    float4 *z4 = reinterpret_cast<float4 *>(s.ring);
    for (int e = threadIdx.x; e < (int)(SM::kRing / 16); e += 64) z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  // ---------------- forward rollout, FP64 update of z and of the residual
  FS *fring = reinterpret_cast<FS *>(s.ring);
  if (warp == 0) {
    // ----- chain: x_0 = v0 - delta W_0 v0, y_0 = W_0 v0 + p_0 with v0 = c'_0 - delta p_0
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
      s.vec[0].dx[lane] = dxv;
      s.vec[0].dy[lane] = dyv;
      const double xv = I.x[lane] + widen(dxv), yv = I.y[lane] + widen(dyv);
      I.x[lane] = xv;
      I.y[lane] = yv;
      zbits = max(zbits, max(abs_bits(xv), abs_bits(yv)));
      const double r0 = __ldcg(rc + lane) - widen(dxv) - delta64 * widen(dyv);
      rc[lane] = r0;
      rbits = max(rbits, abs_bits(r0));
    }
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      duo_sync<1, NF>(1 + k % NF);  // FULL: stage k's slot is ready
      const FS &f = fring[k % DF];
      VC &vk = s.vec[k % NVR];
      VC &vn = s.vec[(k + 1) % NVR];
      // du_k = K_k dx_k + k_k
      float2 xr[H2];
      ld_seg<H2, 0, H2>(vk.dx, xr);
      {
        float2 kr[H2];
        ld_seg<H2, 0, H2>(f.K + bt * N4, kr);
        const float duv = dot2<n>(kr, xr) + f.kk[bt];
        if (lane < m) vk.du[lane] = duv;
      }
      __syncwarp();
      // w = A dx + B du + c'_{k+1} - delta p_{k+1}
      float2 ur[U2];
      ld_seg<U2, 0, U2>(vk.du, ur);
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
        wv = (acc.x + acc.y) + f.cv[bi];
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
          vn.dx[lane] = dxv;
          vn.dy[lane] = dyv;
        }
      }
      __syncwarp();
      duo_arrive<NF + 1, NF + NV>(NF + 1 + k % NV);  // VEC: stage k's vectors written
    }
  } else {
    // ----- helper: copies, right-hand sides and the rows of K dz.  Lane r <
    // RS owns row r of a stage; its FP64 iterate / residual entries (entry at
    // stage 0, stride per stage):
    const bool xr_ = lane < n, ur_ = lane >= n && lane < n + m, cr_ = lane >= n + m && lane < RS;
    double *zp = nullptr, *resp = nullptr;
    size_t zs = 0, rs = 0;
    if (xr_) {
      zp = I.x + n + lane; zs = n; resp = rq + lane; rs = n;
    } else if (ur_) {
      zp = I.u + (lane - n); zs = m; resp = rr + (lane - n); rs = m;
    } else if (cr_) {
      zp = I.y + n + (lane - n - m); zs = n; resp = rc + n + (lane - n - m); rs = n;
    }
    // sizes of chunk16_size: the blocks contiguous in global memory as
    // 16-byte chunks, the transposed and mirrored ones element by element
    constexpr bool kC16f = chunk16_size(NX, NU);
    constexpr int NBF = 8;
    constexpr int CF16 = (2 * nn * 4 + 3 * nm * 4 + n * 4 + m * 4 + n * 8) / 16;
    ChunkPlan<NBF, kC16f ? (CF16 + 31) / 32 : 1> fplan;
    if constexpr (kC16f) {
      static_assert(sizeof(FS) % 16 == 0 && offsetof(FS, K) % 16 == 0 &&
                        offsetof(FS, A) % 16 == 0 && offsetof(FS, B) % 16 == 0 &&
                        offsetof(FS, W) % 16 == 0 && offsetof(FS, M) % 16 == 0 &&
                        offsetof(FS, p) % 16 == 0 && offsetof(FS, kk) % 16 == 0 &&
                        offsetof(FS, c) % 16 == 0,
                    "16-byte block offsets");
      auto cp = [](const void *p) { return reinterpret_cast<const char *>(p); };
      const Blk16 fb[NBF] = {
          {cp(gK), nm * 4, offsetof(FS, K), nm / 4},    {cp(gAf), nn * 4, offsetof(FS, A), nn / 4},
          {cp(gBf), nm * 4, offsetof(FS, B), nm / 4},   {cp(gW + nn), nn * 4, offsetof(FS, W), nn / 4},
          {cp(gMf), nm * 4, offsetof(FS, M), nm / 4},   {cp(gpv + n), n * 4, offsetof(FS, p), n / 4},
          {cp(gkv), m * 4, offsetof(FS, kk), m / 4},    {cp(rc + n), n * 8, offsetof(FS, c), n / 2}};
      fplan.init(fb, lane);
    }
    auto fissue = [&](int k) {
      if constexpr (kC16f) {
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
    // the chain's right-hand side c'_{k+1} - delta p_{k+1} (this lane copied both)
    auto ready = [&](int k) {
      FS &f = fring[k % DF];
      if (lane < n) f.cv[lane] = fmaf(-delta, f.p[lane], f64_to_f32_rz(f.c[lane]));
    };
#pragma unroll 1
    for (int j = 0; j < DF; ++j) fissue(j);
    cp_async_wait<DF - LF>();  // stages 0 .. LF - 1
#pragma unroll 1
    for (int j = 0; j < LF && j < N; ++j) {
      ready(j);
      duo_arrive<1, NF>(1 + j % NF);
    }
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      if (k + LF < N) {  // hand stage k + LF to the chain
        cp_async_wait<DF - LF - 1>();
        ready(k + LF);
        duo_arrive<1, NF>(1 + (k + LF) % NF);
      }
      duo_sync<NF + 1, NF + NV>(NF + 1 + k % NV);  // VEC: the chain finished stage k
      const FS &f = fring[k % DF];
      const VC &vk = s.vec[k % NVR];
      const VC &vn = s.vec[(k + 1) % NVR];
      // K dz rows of stage k and the FP64 updates (lanes < RS)
      if (lane < RS) {
        const float *c1 = xr_ ? f.Q + lane * N4 : ur_ ? f.Mt + (lane - n) * N4 : f.A + (lane - n - m) * N4;
        const float *c2 = xr_ ? f.M + lane * M4 : ur_ ? f.R + (lane - n) * M4 : f.B + (lane - n - m) * M4;
        const float *c3 = xr_ ? f.At + lane * N4 : ur_ ? f.Bt + (lane - n) * N4 : s.zero;
        float2 a1[H2], a2[U2], a3[H2], x1[H2], u2[U2], y3[H2];
        ld_seg<H2, 0, H2>(c1, a1);
        ld_seg<U2, 0, U2>(c2, a2);
        ld_seg<H2, 0, H2>(c3, a3);
        ld_seg<H2, 0, H2>(vk.dx, x1);
        ld_seg<U2, 0, U2>(vk.du, u2);
        ld_seg<H2, 0, H2>(vn.dy, y3);
        float2 acc = mul2(a1[0], x1[0]), sab = mul2(abs2(a1[0]), abs2(x1[0]));
#pragma unroll
        for (int q = 1; q < H2; ++q) {
          acc = fma2(a1[q], x1[q], acc);
          sab = fma2(abs2(a1[q]), abs2(x1[q]), sab);
        }
#pragma unroll
        for (int q = 0; q < U2; ++q) {
          acc = fma2(a2[q], u2[q], acc);
          sab = fma2(abs2(a2[q]), abs2(u2[q]), sab);
        }
#pragma unroll
        for (int q = 0; q < H2; ++q) {
          acc = fma2(a3[q], y3[q], acc);
          sab = fma2(abs2(a3[q]), abs2(y3[q]), sab);
        }
        float t = acc.x + acc.y, sa = sab.x + sab.y, dz;
        if (xr_) {
          t -= vk.dy[lane];
          sa += fabsf(vk.dy[lane]);
          dz = vn.dx[lane];
        } else if (ur_) {
          dz = vk.du[lane - n];
        } else {
          const int i = lane - n - m;
          t -= fmaf(delta, vn.dy[i], vn.dx[i]);
          sa += fmaf(delta, fabsf(vn.dy[i]), fabsf(vn.dx[i]));
          dz = vn.dy[i];
        }
        const double zv = f.z[lane] + widen(dz), rv = f.res[lane] + widen(t);
        zp[(size_t)k * zs] = zv;
        resp[(size_t)k * rs] = rv;
        zbits = max(zbits, abs_bits(zv));
        rbits = max(rbits, abs_bits(rv));
        sbits = max(sbits, abs_bits(widen(sa)));
      }
      __syncwarp();  // every lane is done with the slot
      fissue(k + DF);
    }
    cp_async_wait<0>();
    // terminal rows x_N: res += Q_N dx_N - dy_N (Q_N upper triangle, FP64 data)
    if (lane < n) {
      const VC &vN = s.vec[N % NVR];
      float t = -vN.dy[lane], sa = fabsf(vN.dy[lane]);
      const double *QN = I.Q + (size_t)N * nn;
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const float qv = f64_to_f32_rz(__ldg(QN + min(lane, j) * n + max(lane, j)));
        t = fmaf(qv, vN.dx[j], t);
        sa = fmaf(fabsf(qv), fabsf(vN.dx[j]), sa);
      }
      double *dst = rq + (size_t)N * n + lane;
      const double nv = __ldcg(dst) + widen(t);
      *dst = nv;
      rbits = max(rbits, abs_bits(nv));
      sbits = max(sbits, abs_bits(widen(sa)));
    }
  }

  // ---------------- maxima over both warps, convergence
  for (int o = 16; o > 0; o >>= 1) {
    rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
    zbits = max(zbits, __shfl_xor_sync(0xffffffffu, zbits, o));
    sbits = max(sbits, __shfl_xor_sync(0xffffffffu, sbits, o));
    fbbits = max(fbbits, __shfl_xor_sync(0xffffffffu, fbbits, o));
    kmaxf = fmaxf(kmaxf, __shfl_xor_sync(0xffffffffu, kmaxf, o));
  }
  if (lane == 0) {
    s.red[warp][0] = rbits;
    s.red[warp][1] = zbits;
    s.red[warp][2] = sbits;
    s.red[warp][3] = fbbits;
    s.red[warp][4] = __float_as_uint(kmaxf);  // kmaxf >= 0: the bits order like the values
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    rbits = max(s.red[0][0], s.red[1][0]);
    zbits = max(s.red[0][1], s.red[1][1]);
    sbits = max(s.red[0][2], s.red[1][2]);
    if constexpr (FUSED) {
      // the norms of K and b from the rows computed in the backward pass;
      // the rounding bound starts from this freshly computed residual
      stp->kmax = (double)__uint_as_float((unsigned)max(s.red[0][4], s.red[1][4]));
      stp->bmax = bits_to_double(max(s.red[0][3], s.red[1][3]));
      stp->upd = 0.0;
    }
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

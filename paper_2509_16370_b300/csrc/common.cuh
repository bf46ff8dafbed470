// common.cuh -- shared definitions of the B300 dual-regularized LQR library.
//
// Data layout (see include/rlqr.h): every problem array is FP64, row-major,
// stage-major and contiguous.  Q_i and R_i are symmetric; the kernels read
// their upper triangle only (row <= column).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rlqr.h"

namespace rlqr {

constexpr size_t kAlign = 256;

__host__ __device__ inline size_t align_up(size_t v, size_t a = kAlign) {
  return (v + a - 1) / a * a;
}

// Per-instance state at the start of the instance's workspace.
struct InstState {
  double kmax;     // ||K_LQR||_inf (row sums of |K|)
  double bmax;     // ||[s; c]||_inf
  double rmax;     // ||K z + b||_inf of the current iterate
  double zmax;     // ||z||_inf of the current iterate
  double rel;      // rmax / (kmax * zmax + bmax)
  int32_t pivot_status;  // RLQR_OK / RLQR_NOT_PD / RLQR_ERR_SINGULAR from the sweep
  int32_t iters;         // refinement passes done
  int32_t converged;     // rel <= tol
  int32_t r_singular;    // scan path: some R_i had a zero or non-finite pivot
  int32_t escalated;     // mixed path: a pivot decision lacked its margin, so the
                         // flags were (or are to be) re-decided by the FP64 recursion
  double upd;      // mixed path: bound on the rounding errors that the residual
                   // updates of the refinement passes left in res (absolute)
  double dzmax;    // scan path: max |dz| of the current refinement pass
};

// Byte offsets of the arrays of one instance's workspace.  `tsize` is the
// size of the factor's element type (8 = FP64 path, 4 = mixed path).
struct WsLayout {
  size_t W;      // (N+1) n n   W_i = P_i (I + delta P_i)^{-1}
  size_t K;      // N m n       K_i = -G_i^{-1} H_i
  size_t Gi;     // N m m       G_i^{-1}
  size_t kv;     // N m         k_i of the last solve
  size_t pv;     // (N+1) n     p_i of the last solve
  size_t G;      // N m m       control pivots G_i (mixed path: certified in FP64 later)
  size_t res;    // FP64 residual res_q (N+1)n | res_r N m | res_c (N+1)n
  // mixed path: FP32 copies of the data written by the sweep (truncated),
  // read by the forward pass and the refinement instead of the FP64 arrays
  size_t Af;     // N n n
  size_t Bf;     // N n m
  size_t cf;     // (N+1) n
  size_t Qf;     // N n n (as given; readers take the upper triangle)
  size_t Mf;     // N n m
  size_t Rf;     // N m m (as given; readers take the upper triangle)
  // mixed path, compile-time CTA and tableau sweeps: state pivots whose FP32
  // Gershgorin proof failed are certified afterwards from the stored FP32 P_i
  size_t Pc;     // (N+1) n n FP32 P_i of the pending stages
  size_t pend;   // (N+1) bytes: 1 = bit0 of flags[i] still to decide
  size_t total;
};

// (n, m) of the compile-time CTA sweep (seqx.cuh)
__host__ __device__ constexpr bool seqx_size(int n, int m) {
  return (n == 24 && m == 8) || (n == 32 && m == 8) || (n == 48 && m == 16);
}

// (n, m) of the FP32 tableau warp sweep (tab32.cuh)
__host__ __device__ constexpr bool tab_size(int n, int m) {
  return ((n == 4 || n == 6) && (m == 1 || m == 2)) || (n == 12 && (m == 3 || m == 4));
}

// (n, m) whose refinement stages the contiguous per-stage blocks (rows of a
// multiple of 16 bytes: n, m multiples of 4, the tableau warp sizes) as
// 16-byte chunks.
__host__ __device__ constexpr bool chunk16_size(int n, int m) {
  return n % 4 == 0 && m % 4 == 0 && n >= 4 && m >= 4 && 2 * n <= 32 && 2 * m + n + 1 <= 32;
}

// Margin of the mixed path's pivot certificate: a decision taken from an
// FP32-computed pivot matrix X is kept only when X - tau D (PD claims) or
// X + tau D (indefinite claims) provably has the same inertia, D = |diag X|
// (relative to the Jacobi-scaled matrix); otherwise the FP64 recursion
// decides.  2^-15 ~ 3.1e-5, about 500 times the FP32 unit roundoff.
constexpr float kMarginTau = 0x1p-15f;

__host__ __device__ inline WsLayout ws_layout(int N, int n, int m, int tsize) {
  WsLayout L;
  size_t o = align_up(sizeof(InstState));
  L.W = o;
  o = align_up(o + (size_t)(N + 1) * n * n * tsize);
  L.K = o;
  o = align_up(o + (size_t)N * m * n * tsize);
  L.Gi = o;
  o = align_up(o + (size_t)N * m * m * tsize);
  L.kv = o;
  o = align_up(o + (size_t)N * m * tsize);
  L.pv = o;
  o = align_up(o + (size_t)(N + 1) * n * tsize);
  L.G = o;
  o = align_up(o + (size_t)N * m * m * tsize);
  L.res = o;
  o = align_up(o + ((size_t)(N + 1) * n * 2 + (size_t)N * m) * sizeof(double));
  const size_t ts = tsize == 4 ? 4 : 0;  // the FP32 copies exist in the mixed path only
  L.Af = o;
  o = align_up(o + (size_t)N * n * n * ts);
  L.Bf = o;
  o = align_up(o + (size_t)N * n * m * ts);
  L.cf = o;
  o = align_up(o + (size_t)(N + 1) * n * ts);
  L.Qf = o;
  o = align_up(o + (size_t)N * n * n * ts);
  L.Mf = o;
  o = align_up(o + (size_t)N * n * m * ts);
  L.Rf = o;
  o = align_up(o + (size_t)N * m * m * ts);
  const bool cta_sizes = ts != 0 && (seqx_size(n, m) || tab_size(n, m));
  L.Pc = o;
  o = align_up(o + (cta_sizes ? (size_t)(N + 1) * n * n * 4 : 0));
  L.pend = o;
  o = align_up(o + (cta_sizes ? (size_t)(N + 1) : 0));
  L.total = o;
  return L;
}

// Kernel-side view of a batch (or of one instance when `single` is set).
struct BatchArgs {
  int count;
  int single;
  // single instance
  int N, n, m;
  double delta;
  const double *Q, *M, *R, *q, *r, *A, *B, *c;
  double *x, *u, *y;
  uint8_t *flags;
  // batch (device arrays [count])
  const int32_t *dN, *dn, *dm;
  const double *ddelta;
  const int64_t *oQ, *oM, *oR, *oq, *or_, *oA, *oB, *oc, *ox, *ou, *oy, *of;
  const int64_t *ows;  // per-instance workspace byte offsets
  const int32_t *perm; // launch slot -> instance (grouped launches of a ragged batch), or null
  int goff;            // first slot of this launch's group in perm
  // shared
  char *ws;
  int tsize;
  int32_t *status;  // per-instance outputs, may be null
  double *rel;
  int32_t *iters;
  double tol;
  int max_refine;
  // residual launches: recompute the residual only for the instances that
  // have not converged (after a refinement pass whose rounding bound could
  // not certify convergence)
  int recheck;
  // refinement launches: index of the pass (0 = first)
  int rpass;
  // warp sizes of the mixed path: the first refinement pass computes the
  // residual itself (no separate first-residual launch)
  int fused_res;
  // warps per instance of the mixed refinement passes of the warp sizes:
  // 1 (k_refine_tab), 2 (k_refine_duo), 0 = 1
  int refine_warps;
};

// Instance of a launch slot: the identity, or the group's entry of perm.
__device__ __forceinline__ int inst_of(const BatchArgs &a, int slot) {
  return a.perm ? a.perm[a.goff + slot] : slot;
}

struct Inst {
  int N, n, m;
  double delta;
  const double *Q, *M, *R, *q, *r, *A, *B, *c;
  double *x, *u, *y;
  uint8_t *flags;
  char *ws;
  InstState *st;
  WsLayout L;
};

__device__ __forceinline__ Inst get_inst(const BatchArgs &a, int b) {
  Inst I;
  if (a.single) {
    I.N = a.N; I.n = a.n; I.m = a.m; I.delta = a.delta;
    I.Q = a.Q; I.M = a.M; I.R = a.R; I.q = a.q; I.r = a.r; I.A = a.A; I.B = a.B; I.c = a.c;
    I.x = a.x; I.u = a.u; I.y = a.y; I.flags = a.flags;
    I.ws = a.ws;
  } else {
    I.N = a.dN[b]; I.n = a.dn[b]; I.m = a.dm[b]; I.delta = a.ddelta[b];
    I.Q = a.Q + a.oQ[b]; I.M = a.M + a.oM[b]; I.R = a.R + a.oR[b];
    I.q = a.q + a.oq[b]; I.r = a.r + a.or_[b]; I.A = a.A + a.oA[b];
    I.B = a.B + a.oB[b]; I.c = a.c + a.oc[b];
    I.x = a.x + a.ox[b]; I.u = a.u + a.ou[b]; I.y = a.y + a.oy[b];
    I.flags = a.flags + a.of[b];
    I.ws = a.ws + a.ows[b];
  }
  I.st = reinterpret_cast<InstState *>(I.ws);
  I.L = ws_layout(I.N, I.n, I.m, a.tsize);
  return I;
}

// FP64 <-> FP32 conversions with integer operations only.  On B300 the
// conversion instructions share the FP64 pipe (2 results per clock per SM),
// so an FP32 sweep that converted its FP64 inputs element by element would
// spend more issue time converting than computing.
//   f64_to_f32_rz: truncation of the significand (round toward zero, relative
//   error < 2^-23); magnitudes below 2^-126 give signed zero, at or above
//   2^128 +-inf; NaN stays NaN.
//   f32_to_f64: exact for FP32 normals, zero, inf and NaN; FP32 subnormals
//   (below 2^-126) give signed zero.
__device__ __forceinline__ float f64_to_f32_rz(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned ahi = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  unsigned bits = ((ahi - 0x38000000u) << 3) | (lo >> 29);
  if (ahi < 0x38100000u) bits = 0u;
  if (ahi >= 0x47f00000u)
    bits = (ahi > 0x7ff00000u || (ahi == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(bits | sign);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f), sign = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = sign | ((a >> 3) + 0x38000000u), lo = a << 29;
  if (a < 0x00800000u) {
    hi = sign;
    lo = 0u;
  } else if (a >= 0x7f800000u) {
    hi = sign | 0x7ff00000u | ((a & 0x7fffffu) >> 3);
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Float-float (unevaluated sum hi + lo of two FP32 numbers) arithmetic, used
// to evaluate FP64-accurate residuals on the FP32 pipes: the two-product of
// Dekker (the FMA gives the exact rounding error of a product) and the
// two-sum of Knuth (the exact rounding error of a sum).  The __f*_rn
// intrinsics are never contracted into FMAs, which the error terms rely on.
//
// split_f64: v = hi + lo + e with hi = f64_to_f32_rz(v) and |e| < 2^-46 |v|
// (lo keeps the top 23 of the 29 significand bits that hi drops; lo is zero
// when |v| < 2^-80, where the absolute error stays below 2^-103).
__device__ __forceinline__ float2 split_f64(double v) {
  const unsigned hi_w = (unsigned)__double2hiint(v), lo_w = (unsigned)__double2loint(v);
  const unsigned ex = (hi_w >> 20) & 0x7ffu;  // biased FP64 exponent
  // the dropped bits (lo_w & 0x1fffffff) >> 6 as an exact FP32 integer
  const float rem = __fsub_rn(__uint_as_float(0x4b000000u | ((lo_w & 0x1fffffffu) >> 6)), 8388608.0f);
  // scale 2^(ex - 1023 - 52 + 6) as an FP32 power of two (ex - 942 = its field)
  const float scale = (ex >= 943u && ex <= 1196u) ? __uint_as_float((ex - 942u) << 23) : 0.0f;
  const float lo = __uint_as_float(__float_as_uint(__fmul_rn(rem, scale)) | (hi_w & 0x80000000u));
  return make_float2(f64_to_f32_rz(v), lo);
}

// (sh, sl) += (ah + al) (zh + zl), dropping al zl (below 2^-46 of the term)
__device__ __forceinline__ void ff_fma(float &sh, float &sl, float2 a, float2 z) {
  const float p = __fmul_rn(a.x, z.x);
  const float e = fmaf(a.x, z.x, -p);  // a.x z.x = p + e exactly
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // sh + p = s + err
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, fmaf(a.x, z.y, fmaf(a.y, z.x, e))));
}

// (sh, sl) += (bh + bl)
__device__ __forceinline__ void ff_add(float &sh, float &sl, float2 b) {
  const float s = __fadd_rn(sh, b.x);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, b.y));
}

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

// Packed FP32 pairs (fma/add/mul .f32x2, sm_100 and later): one instruction
// does two FP32 operations with the latency of one.  The operands are
// float2 register pairs.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

// Reciprocal of an elimination pivot.  FP32: the hardware approximation
// refined by one Newton step for 1/d, r <- r + r (1 - d r), which squares
// its relative error (within about one ulp of 1/d; d = 0, +-inf or an FP32
// subnormal gives inf or NaN).  It replaces the IEEE division on the
// critical path of each elimination step.  FP64: the IEEE quotient.
__device__ __forceinline__ float recip_pivot(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return fmaf(r, fmaf(-d, r, 1.0f), r);
}
__device__ __forceinline__ double recip_pivot(double d) { return 1.0 / d; }

// Gershgorin certificate for row i of S = I + delta P (P stored in FP32,
// delta the FP64 regularization):  1 + delta (P_ii - sum_{j != i} |P_ij|) > 0.
// `off_ru` is the off-diagonal sum accumulated with round-up additions and
// delta_up >= delta (FP64 delta rounded up); the difference is rounded down
// and the product up, so every rounding works against the claim and `true`
// proves that the row's Gershgorin disc lies in (0, inf).  All rows true
// proves S positive definite (S is symmetric).  NaN gives false.
__device__ __forceinline__ bool gershgorin_row_pd(float p_ii, float off_ru, float delta_up) {
  const float d = __fsub_rd(p_ii, off_ru);
  return d >= 0.0f || __fmul_ru(delta_up, -d) < 1.0f;
}

// Robust Gershgorin row test for S = I + delta P (P in FP32, delta the FP64
// regularization): with d = P_ii - sum_{j != i} |P_ij| (the sum rounded up),
// the row's disc of S - tau diag(S) lies in (0, inf) when
//   (1 + delta d) - tau (1 + delta P_ii) > 0,
// evaluated with every rounding against the claim (delta_dn <= delta <=
// delta_up, both FP32).  All rows true proves lambda_min(D^-1/2 S D^-1/2) >
// tau, D = diag(S).  NaN gives false.
__device__ __forceinline__ bool gershgorin_row_margin(float p_ii, float off_ru, float delta_dn,
                                                      float delta_up, float tau) {
  const float d = __fsub_rd(p_ii, off_ru);
  const float g = d >= 0.f ? __fadd_rd(1.f, __fmul_rd(delta_dn, d))
                           : __fsub_rd(1.f, __fmul_ru(delta_up, -d));
  const float sd = p_ii >= 0.f ? __fadd_ru(1.f, __fmul_ru(delta_up, p_ii))
                               : __fsub_ru(1.f, __fmul_rd(delta_dn, -p_ii));
  return __fsub_rd(g, __fmul_ru(tau, sd)) > 0.f;
}

// Asynchronous global -> shared copies (cp.async): each thread copies its
// own elements, commits them as a group and later waits until at most N of
// its groups are still in flight.  A hardware wait, no polling.  The copied
// bytes are visible to the copying thread after the wait; other threads see
// them after a barrier that follows that wait.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
// 16-byte copy, L2 only (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

// A per-stage block of 16-byte chunks: the chunk j of stage k sits at
// p + k * stride + 16 j (bytes) in global memory and goes to byte dst + 16 j
// of a shared-memory slot.
struct Blk16 {
  const char *p;
  uint32_t stride, dst;
  int n;
};

// This lane's chunks (lane, lane + 32, ...) of the blocks b[0..NB), numbered
// consecutively, as (source at stage 0, stride, slot offset); dst = ~0u past
// the last chunk.
template <int NB, int CH>
struct ChunkPlan {
  const char *src[CH];
  uint32_t stride[CH], dst[CH];
  __device__ __forceinline__ void init(const Blk16 (&b)[NB], int lane) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int c = lane + 32 * i;
      src[i] = b[0].p;
      stride[i] = 0u;
      dst[i] = ~0u;
      int start = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (c >= start && c < start + b[j].n) {
          src[i] = b[j].p + 16 * (c - start);
          stride[i] = b[j].stride;
          dst[i] = b[j].dst + 16u * (uint32_t)(c - start);
        }
        start += b[j].n;
      }
    }
  }
  // the copies of stage k into slot
  __device__ __forceinline__ void issue(unsigned char *slot, int k) const {
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (dst[i] != ~0u) cp_async16(slot + dst[i], src[i] + (size_t)k * stride[i]);
  }
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Working-precision conversion used by the staging helpers.
template <typename T, typename S>
__device__ __forceinline__ T to_work(S v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float to_work<float, double>(double v) {
  return f64_to_f32_rz(v);
}
// Widening of a working-precision value to FP64 (exact).
__device__ __forceinline__ double widen(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double widen(double v) { return v; }

// Thread-strided register staging of a contiguous global segment: element
// `threadIdx.x + i*THREADS` of the segment goes to v[i].  Used to prefetch the
// next stage's data while the current stage computes.
// Problem data is read through the read-only path (it is never written by
// the library); workspace arrays written earlier in the same kernel are read
// with load_cg (L2, coherent with the block's own earlier stores).
template <typename S, int THREADS, int CNT>
struct RegSeg {
  S v[CNT > 0 ? CNT : 1];
  __device__ __forceinline__ void load(const S *__restrict__ g, int len) {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      int idx = threadIdx.x + i * THREADS;
      if (idx < len) v[i] = __ldg(g + idx);
    }
  }
  __device__ __forceinline__ void load_cg(const S *g, int len) {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      int idx = threadIdx.x + i * THREADS;
      if (idx < len) v[i] = __ldcg(g + idx);
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(T *s, int len) const {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      int idx = threadIdx.x + i * THREADS;
      if (idx < len) s[idx] = to_work<T>(v[i]);
    }
  }
  // Store a row-major n x n symmetric matrix given by its upper triangle:
  // element (i, j), i <= j, goes to (i, j) and (j, i); the lower one is unused.
  template <typename T>
  __device__ __forceinline__ void store_sym(T *s, int n) const {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      int idx = threadIdx.x + i * THREADS;
      if (idx < n * n) {
        const int r = idx / n, c = idx - r * n;
        if (r <= c) {
          const T w = to_work<T>(v[i]);
          s[r * n + c] = w;
          s[c * n + r] = w;
        }
      }
    }
  }
};

// Lane-strided register staging for warp-per-instance kernels: element
// `lane + 32 i` of the segment goes to v[i].
template <typename S, int CNT>
struct LaneSeg {
  S v[CNT > 0 ? CNT : 1];
  __device__ __forceinline__ void load(const S *__restrict__ g, int len, int lane) {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const int idx = lane + 32 * i;
      if (idx < len) v[i] = __ldg(g + idx);
    }
  }
  __device__ __forceinline__ void load_cg(const S *g, int len, int lane) {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const int idx = lane + 32 * i;
      if (idx < len) v[i] = __ldcg(g + idx);
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(T *s, int len, int lane) const {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const int idx = lane + 32 * i;
      if (idx < len) s[idx] = to_work<T>(v[i]);
    }
  }
  // row-major n x n symmetric matrix given by its upper triangle
  template <typename T>
  __device__ __forceinline__ void store_sym(T *s, int n, int lane) const {
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const int idx = lane + 32 * i;
      if (idx < n * n) {
        const int r = idx / n, c = idx - r * n;
        if (r <= c) {
          const T w = to_work<T>(v[i]);
          s[r * n + c] = w;
          s[c * n + r] = w;
        }
      }
    }
  }
};

// Dimension policies: DynDims reads (n, m) at run time (bounded by NM, MM);
// FixDims makes them compile-time constants so that every loop bound and
// index division folds (the common sizes get their own instantiation).
template <int NMAX, int MMAX>
struct DynDims {
  static constexpr int NM = NMAX, MM = MMAX;
  int n, m;
  __device__ __forceinline__ DynDims(int n_, int m_) : n(n_), m(m_) {}
};

template <int NX, int NU>
struct FixDims {
  static constexpr int NM = NX, MM = NU;
  static constexpr int n = NX, m = NU;
  __device__ __forceinline__ FixDims(int, int) {}
};

// Row-major lower-triangle (diagonal included) decode: e -> (i, c), c <= i.
__device__ __forceinline__ void tri_decode(int e, int &i, int &c) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= e) ++r;
  if (r * (r + 1) / 2 > e) --r;
  i = r;
  c = e - r * (r + 1) / 2;
}

// |v| of a double as an order-preserving integer (max-reductions on the INT
// pipe: FP64 min/max would take FP64 issue slots, which are scarce on B300).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// |v| truncated to FP32 with integer operations only (relative error below
// 2^-23; 0 below the FP32 normal range, +inf above it or for inf / NaN).
// Used for norms that only scale a backward error: an FP64 -> FP32
// conversion instruction would take FP64 issue slots on B300.
__device__ __forceinline__ float abs_f32_trunc(double v) {
  const unsigned hi = (unsigned)__double2hiint(v) & 0x7fffffffu;
  const unsigned lo = (unsigned)__double2loint(v);
  const int e = (int)(hi >> 20);
  if (e < 897) return 0.f;
  if (e > 1150) return __uint_as_float(0x7f800000u);
  return __uint_as_float(((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

__device__ __forceinline__ bool finite_nonzero(double d) { return isfinite(d) && d != 0.0; }

// Certificate decision with margin for a symmetric m x m pivot matrix X
// computed in FP32 (row-major; the entries X[c][i], c <= i, are read), by one
// thread: unpivoted LDL^T in FP64 of X - tau D and, when that is not PD, of
// X + tau D, with D = diag(max(|X_jj|, 2^-24 max_j |X_jj|)).
//   kPdYes: every pivot of X - tau D is positive, so the Jacobi-scaled X has
//           lambda_min > tau: X and every X + E with E below tau (scaled) are PD;
//   kPdNo:  a pivot of X + tau D is <= 0, so lambda_min < -tau: robustly not PD;
//   kPdAmbiguous: neither (the decision is left to the FP64 recursion), also
//           for non-finite entries.
enum { kPdNo = 0, kPdYes = 1, kPdAmbiguous = 2 };
template <int MAXM>
__device__ __forceinline__ int pd_margin_f32(const float *X, int m, double tau) {
  double L[MAXM * (MAXM + 1) / 2];
  double dmax = 0.0;
  for (int j = 0; j < m; ++j) dmax = fmax(dmax, fabs(widen(__ldcg(X + j * m + j))));
  const double floor_d = 0x1p-24 * dmax;
  for (int pass = 0; pass < 2; ++pass) {
    const double sg = pass == 0 ? -tau : tau;
    for (int i = 0; i < m; ++i)
      for (int c = 0; c <= i; ++c) {
        double v = widen(__ldcg(X + c * m + i));
        if (c == i) v += sg * fmax(fabs(v), floor_d);
        L[i * (i + 1) / 2 + c] = v;
      }
    bool pos = true;
    for (int j = 0; j < m; ++j) {
      const double d = L[j * (j + 1) / 2 + j];
      if (!isfinite(d)) return kPdAmbiguous;
      if (!(d > 0.0)) {
        pos = false;
        break;
      }
      const double rd = 1.0 / d;
      for (int i = j + 1; i < m; ++i) {
        const double lij = L[i * (i + 1) / 2 + j] * rd;
        for (int c = j + 1; c <= i; ++c) L[i * (i + 1) / 2 + c] -= lij * L[c * (c + 1) / 2 + j];
      }
    }
    if (pass == 0 && pos) return kPdYes;
    if (pass == 1 && !pos) return kPdNo;
  }
  return kPdAmbiguous;
}

// Proof in FP32, by one warp, that I + delta P - tau D is positive definite
// (D = diag(I + delta P); delta > 0; P symmetric FP32, row-major NX x NX,
// NX <= 64; tau >= 0 the certificate's margin).  Method: the
// verification of positive definiteness of S. M. Rump (BIT 46, 2006) applied
// to A = P + I/delta, which is PD exactly when I + delta P is.  A is scaled
// as D A D with D the powers of two nearest diag(A)^(-1/2) (exact), its
// diagonal entries d_i are lowered by c + tau d_i (the margin: A - tau
// diag(A) is a positive multiple of I + delta P - tau D) and the result S is
// Cholesky-factored (S = R^T R,
// R upper) in FP32 with correctly rounded square roots and divisions.  If
// that run completes (every pivot finite and positive), the backward error
// of Cholesky (Demmel; Higham, "Accuracy and Stability of Numerical
// Algorithms", Thm 10.5: R^T R = S + dS, |dS| <= gamma_{n+1} |R^T| |R|)
// gives ||dS||_2 <= gamma_{n+1} / (1 - gamma_{n+1}) tr(S), so
// lambda_min(D A D) >= c - ||dS||_2 - (underflow terms) > 0 for
// c = gamma' tr + 2^-120, every bound rounded outward.  Returns 1 when the
// proof succeeds; 0 decides nothing.  Registers only: lane l holds the upper
// triangle's columns l and l + 32; row j of R reaches the other lanes by
// shuffles.
template <int NX>
__device__ __noinline__ int warp_pd_proof_f32(const float *P, double delta, float tau) {
  static_assert(NX >= 1 && NX <= 64, "one warp, two columns per lane");
  constexpr int R0 = NX < 32 ? NX : 32;  // rows held for column lane (<= lane)
  constexpr int R1 = NX > 32 ? NX : 1;   // rows held for column lane + 32
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int c0 = lane, c1 = lane + 32;
  const bool h0 = c0 < NX, h1 = c1 < NX;
  const float invd = __double2float_rd(__ddiv_rd(1.0, delta));  // <= 1/delta
  // diagonal of A (rounded down), power-of-two scales, trace bound
  auto scale_of = [](float a) {
    int ex = 0;
    frexpf(a, &ex);
    return __int_as_float((127 - (ex >> 1)) << 23);  // 2^-(ex/2), a normal number
  };
  const float a0 = h0 ? __fadd_rd(__ldcg(P + c0 * NX + c0), invd) : 1.f;
  const float a1 = h1 ? __fadd_rd(__ldcg(P + c1 * NX + c1), invd) : 1.f;
  int bad = !(a0 > 0.f && a0 <= 3.0e38f) || !(a1 > 0.f && a1 <= 3.0e38f);
  const float s0 = bad ? 1.f : scale_of(a0), s1 = bad ? 1.f : scale_of(a1);
  float tr = __fadd_ru(h0 ? a0 * s0 * s0 : 0.f, h1 ? a1 * s1 * s1 : 0.f);
  for (int o = 16; o > 0; o >>= 1) tr = __fadd_ru(tr, __shfl_xor_sync(FULL, tr, o));
  if (__any_sync(FULL, bad)) return 0;
  const float num = (float)(NX + 1) * 0x1p-24f;               // (n+1) u, exact
  const float den = __fsub_rd(1.0f, __fmul_ru(2.0f, num));    // 1 - 2 (n+1) u
  const float gam = __fmul_ru(__fdiv_ru(num, den), 1.01f);    // >= gamma/(1-gamma)
  const float c = __fadd_ru(__fmul_ru(gam, tr), 0x1p-120f);
  // this lane's columns of the upper triangle of S = D A D - c I
  float x0[R0], x1[R1];
#pragma unroll
  for (int i = 0; i < R0; ++i) {
    const float si = __shfl_sync(FULL, s0, i);
    float v = 0.f;
    if (h0 && i < c0) v = (si * __ldcg(P + i * NX + c0)) * s0;
    if (h0 && i == c0) {
      const float dg = a0 * s0 * s0;  // exact: scaling by powers of two
      v = __fsub_rd(__fsub_rd(dg, c), __fmul_ru(tau, dg));
    }
    x0[i] = v;
    bad |= !(fabsf(v) <= 3.0e38f);
  }
  if constexpr (NX > 32) {
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const float si = __shfl_sync(FULL, i < 32 ? s0 : s1, i & 31);
      float v = 0.f;
      if (h1 && i < c1) v = (si * __ldcg(P + i * NX + c1)) * s1;
      if (h1 && i == c1) {
        const float dg = a1 * s1 * s1;
        v = __fsub_rd(__fsub_rd(dg, c), __fmul_ru(tau, dg));
      }
      x1[i] = v;
      bad |= !(fabsf(v) <= 3.0e38f);
    }
  }
  if (__any_sync(FULL, bad)) return 0;
  // right-looking Cholesky
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    float d;
    if (j < 32) d = __shfl_sync(FULL, x0[j < R0 ? j : 0], j);
    else d = __shfl_sync(FULL, x1[j < R1 ? j : 0], j & 31);
    if (!(d > 0.f && d <= 3.0e38f)) return 0;  // uniform over the warp
    const float rj = __fsqrt_rn(d);
    if (j < R0 && h0 && c0 > j) x0[j] = __fdiv_rn(x0[j], rj);
    if constexpr (NX > 32) {
      if (h1 && c1 > j) x1[j] = __fdiv_rn(x1[j], rj);
    }
#pragma unroll
    for (int i = j + 1; i < NX; ++i) {
      float uji;  // R_ji, held by the owner of column i
      if (i < 32) uji = __shfl_sync(FULL, x0[j < R0 ? j : 0], i);
      else uji = __shfl_sync(FULL, x1[j < R1 ? j : 0], i & 31);
      if (i < R0 && c0 >= i) x0[i < R0 ? i : 0] = fmaf(-uji, x0[j < R0 ? j : 0], x0[i < R0 ? i : 0]);
      if constexpr (NX > 32) {
        if (c1 >= i && h1) x1[i] = fmaf(-uji, x1[j], x1[i]);
      }
    }
  }
  return 1;
}

// Block-wide max of non-negative doubles (all threads return the result).
template <int THREADS>
__device__ __forceinline__ double block_max(double v, double *scratch /* >= THREADS/32 */) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < THREADS / 32; ++i) r = fmax(r, scratch[i]);
  __syncthreads();
  return r;
}

}  // namespace rlqr

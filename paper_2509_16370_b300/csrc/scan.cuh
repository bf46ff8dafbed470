// scan.cuh -- the associative-scan form of the dual-regularized Riccati
// recursion (Section "Parallel Algorithm") for one long-horizon instance.
//
// The N stages are cut into C chunks of L stages (chunk c: stages
// [cL, min(cL + L, N))).  With the interval elements (P, A, C)_{i->i+1} of eq.
// lqr-gpu-init-running (the controls eliminated through R_i^{-1}) and the
// combination rule of eq. lqr-gpu-combo, written with the single inverse
// T = (I + C_ij P_jk)^{-1}:
//   A_ik = A_jk T A_ij,  C_ik = A_jk T C_ij A_jk^T + C_jk,
//   P_ik = A_ij^T P_jk T A_ij + P_ij          (Corollary inverse-helper-corollary)
// the path is
//   k_scan_reduce    one CTA per chunk: the chunk's element, folded from the
//                    right (acc <- e_i (+) acc); block C writes the terminal
//                    element (Q_N, 0, 0) of eq. lqr-gpu-init-terminal;
//   k_scan_level     one level of a Hillis-Steele suffix scan over the C + 1
//                    elements: after ceil(log2(C+1)) levels element c holds the
//                    composition of chunks c..C-1 and the terminal, whose P is
//                    P_{cL} (the value function at the chunk's first stage);
//   k_scan_finalize  one CTA per chunk: from P at the chunk's end, the
//                    sequential step of Theorem main-seq-theorem for every
//                    stage of the chunk (W, G, H, K, P, the pivot certificate),
//                    and the product Phi_c = F_s ... F_{e-1} of the maps of
//                    Corollary p-recurrence, F_i = (A_i + B_i K_i)^T (I - delta W_{i+1}).
// Accuracy of the FP32 scan: composing a chunk's elements in FP32 loses about
// three digits (I + C_ij P_jk of a chunk interval has condition ~1e4-1e5 on
// the test problems), while the sequential recursion contracts an error in
// its starting P strongly (1e-3 -> 3e-6 over 8 stages there).  The mixed path
// therefore runs the finalize twice: a P-only pass gives every chunk's P at
// its first stage, and the full pass of chunk c starts from chunk c+1's value,
// so that each boundary error has been contracted by the sequential
// recursion.  The contraction needs only a few stages (1e-3 -> 3e-6 in 8
// stages on the n = 32 test), so a chunk longer than kInnerK stages also gets
// the element of its stages [s + kInnerK, e) from the fold (SI), composed with
// the next chunk's suffix element by k_scan_inner into P at s + kInnerK (PI),
// and its P-only pass runs the kInnerK stages from there to s only.  The FP64
// scan is accurate to ~1e-11 and finalizes directly.
// The vector passes (scan_vec.cuh) use Phi_c for p (p_s = Phi_c p_e + phi_c)
// and Phi_c^T for x (x_e = Phi_c^T x_s + psi_c, since the x map of a stage,
// (I - delta W_{i+1})(A_i + B_i K_i), is F_i^T for symmetric W).
//
// The factor is written in the workspace layout of the sequential path
// (W, K, G^{-1}, G, the FP32 data copies in the mixed path) so that the
// residual and the refinement see the same arrays.
#pragma once

#include "common.cuh"

namespace rlqr {

// Scan-specific arrays after the common workspace of the instance.
struct ScanLayout {
  int C, L;        // chunks, stages per chunk
  size_t S0, S1;   // (C+1) x 3 n^2 elements (P, A, C), ping-pong
  size_t Phi;      // C x n^2
  size_t phi;      // C x n      p offsets of the chunks
  size_t psi;      // C x n      x offsets of the chunks
  size_t pb;       // (C+1) x n  p at the chunk starts (index C: p_N)
  size_t xb;       // (C+1) x n  x at the chunk starts (index C: x_N)
  size_t PstA;     // C x n^2    P at the chunk starts from the P-only pass (mixed path)
  size_t PstB;     // C x n^2    P at the chunk starts from the final pass
  size_t SI;       // C x 3 n^2  elements of stages [s + kInnerK, e) (mixed path)
  size_t PI;       // C x n^2    P at s + kInnerK (mixed path)
  size_t total;    // bytes after `base`
};

// Stages of the P-only pass of a chunk longer than this (see above).
constexpr int kInnerK = 16;
__host__ __device__ inline bool chunk_has_inner(int len) { return len > kInnerK; }

__host__ __device__ inline ScanLayout scan_layout(int N, int n, int L, int tsize) {
  ScanLayout S;
  S.L = L;
  S.C = (N + L - 1) / L;
  const size_t C = (size_t)S.C, nn = (size_t)n * n;
  size_t o = 0;
  S.S0 = o;
  o = align_up(o + (C + 1) * 3 * nn * tsize);
  S.S1 = o;
  o = align_up(o + (C + 1) * 3 * nn * tsize);
  S.Phi = o;
  o = align_up(o + C * nn * tsize);
  S.phi = o;
  o = align_up(o + C * n * tsize);
  S.psi = o;
  o = align_up(o + C * n * tsize);
  S.pb = o;
  o = align_up(o + (C + 1) * n * tsize);
  S.xb = o;
  o = align_up(o + (C + 1) * n * tsize);
  S.PstA = o;
  o = align_up(o + C * nn * tsize);
  S.PstB = o;
  o = align_up(o + C * nn * tsize);
  // (sized for every chunking of the mixed path, so that the layout grows
  // with the chunk count and the largest count bounds every other)
  const bool inner = tsize == 4;
  S.SI = o;
  o = align_up(o + (inner ? C * 3 * nn * tsize : 0));
  S.PI = o;
  o = align_up(o + (inner ? C * nn * tsize : 0));
  S.total = o;
  return S;
}

// Chunk length: enough chunks for one wave of CTAs on a 148-SM part (a few
// CTAs per SM), at least 8 stages per chunk.
__host__ __device__ inline int scan_chunk_len(int N) {
  int L = (N + 443) / 444;
  return L < 8 ? 8 : L;
}

namespace scan {

constexpr int kTH = 256;  // threads of the scan CTAs

// Compile-time-size product with 2x2 register tiles: D (R x C) = alpha *
// op(A) op(B) (+ Add), K inner; R, C even; leading dimensions even so that
// pairs load as one 8-byte access.  FP32 pairs use fma.rn.f32x2.  D must not
// alias A or B (it may alias Add).  No barrier.
template <typename T, int R, int C, int K, bool TA, bool TB>
__device__ __forceinline__ void mmt(T *D, int ldd, const T *A, int lda, const T *B, int ldb,
                                    const T *Add, int ldadd, T alpha) {
  static_assert(R % 2 == 0 && C % 2 == 0, "even tile dimensions");
  constexpr int TC = C / 2, NT = (R / 2) * TC;
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    const int tr = t / TC, tc = t - tr * TC, r0 = 2 * tr, c0 = 2 * tc;
    if constexpr (sizeof(T) == 4) {
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int k = 0; k < K; ++k) {
        float x0, x1;
        float2 y;
        if (TA) {
          const float2 xa = *reinterpret_cast<const float2 *>(A + k * lda + r0);
          x0 = xa.x;
          x1 = xa.y;
        } else {
          x0 = A[r0 * lda + k];
          x1 = A[(r0 + 1) * lda + k];
        }
        if (TB) {
          y = make_float2(B[c0 * ldb + k], B[(c0 + 1) * ldb + k]);
        } else {
          y = *reinterpret_cast<const float2 *>(B + k * ldb + c0);
        }
        s0 = fma2(bcast2(x0), y, s0);
        s1 = fma2(bcast2(x1), y, s1);
      }
      const float al = (float)alpha;
      float2 o0 = make_float2(s0.x * al, s0.y * al), o1 = make_float2(s1.x * al, s1.y * al);
      if (Add) {
        o0.x += Add[r0 * ldadd + c0];
        o0.y += Add[r0 * ldadd + c0 + 1];
        o1.x += Add[(r0 + 1) * ldadd + c0];
        o1.y += Add[(r0 + 1) * ldadd + c0 + 1];
      }
      *reinterpret_cast<float2 *>(D + r0 * ldd + c0) = o0;
      *reinterpret_cast<float2 *>(D + (r0 + 1) * ldd + c0) = o1;
    } else {
      T a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll 8
      for (int k = 0; k < K; ++k) {
        const T x0 = TA ? A[k * lda + r0] : A[r0 * lda + k];
        const T x1 = TA ? A[k * lda + r0 + 1] : A[(r0 + 1) * lda + k];
        const T y0 = TB ? B[c0 * ldb + k] : B[k * ldb + c0];
        const T y1 = TB ? B[(c0 + 1) * ldb + k] : B[k * ldb + c0 + 1];
        a00 = fma(x0, y0, a00);
        a01 = fma(x0, y1, a01);
        a10 = fma(x1, y0, a10);
        a11 = fma(x1, y1, a11);
      }
      T o00 = a00 * alpha, o01 = a01 * alpha, o10 = a10 * alpha, o11 = a11 * alpha;
      if (Add) {
        o00 += Add[r0 * ldadd + c0];
        o01 += Add[r0 * ldadd + c0 + 1];
        o10 += Add[(r0 + 1) * ldadd + c0];
        o11 += Add[(r0 + 1) * ldadd + c0 + 1];
      }
      D[r0 * ldd + c0] = o00;
      D[r0 * ldd + c0 + 1] = o01;
      D[(r0 + 1) * ldd + c0] = o10;
      D[(r0 + 1) * ldd + c0 + 1] = o11;
    }
  }
}

// ---- 3xTF32 tensor-core products (FP32 data, sm_80+ mma.sync on the tensor
// pipe).  Each FP32 operand x is split as x = hi + lo with hi = tf32(x)
// (round to nearest) and lo = tf32(x - hi); the product is accumulated in
// FP32 as lo_a hi_b + hi_a lo_b + hi_a hi_b (the lo_a lo_b term, below
// 2^-22 of the product, is dropped).  Fragment layouts of
// mma.m16n8k8.row.col.f32.tf32.tf32.f32 (PTX ISA): with g = lane / 4 and
// t = lane % 4,
//   A (16 x 8): a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (8 x 8):  b0 (t, g), b1 (t + 4, g)
//   C (16 x 8): c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
__device__ __forceinline__ uint32_t tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_rn(x);
  lo = tf32_rn(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// D (R x C) = alpha op(A) op(B) (+ Add) with 3xTF32 tensor-core products,
// R % 16 == 0, C % 8 == 0, K % 8 == 0; one warp per 16 x 8 output tile.  The
// same contract as mmt (D must not alias A or B; no barrier).
template <int R, int C, int K, bool TA, bool TB>
__device__ __forceinline__ void mmt_tc(float *D, int ldd, const float *A, int lda, const float *B,
                                       int ldb, const float *Add, int ldadd, float alpha) {
  static_assert(R % 16 == 0 && C % 8 == 0 && K % 8 == 0, "tensor-core tile multiples");
  constexpr int TR = R / 16, TCn = C / 8, NT = TR * TCn;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  auto ea = [&](int r, int k) { return TA ? A[k * lda + r] : A[r * lda + k]; };
  auto eb = [&](int k, int c) { return TB ? B[c * ldb + k] : B[k * ldb + c]; };
  for (int tile = warp; tile < NT; tile += nw) {
    const int r0 = (tile / TCn) * 16, c0 = (tile % TCn) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 8) {
      uint32_t ah[4], al[4], bh[2], bl[2];
      tf32_split(ea(r0 + g, k0 + t), ah[0], al[0]);
      tf32_split(ea(r0 + g + 8, k0 + t), ah[1], al[1]);
      tf32_split(ea(r0 + g, k0 + t + 4), ah[2], al[2]);
      tf32_split(ea(r0 + g + 8, k0 + t + 4), ah[3], al[3]);
      tf32_split(eb(k0 + t, c0 + g), bh[0], bl[0]);
      tf32_split(eb(k0 + t + 4, c0 + g), bh[1], bl[1]);
      mma_tf32(acc, al, bh);
      mma_tf32(acc, ah, bl);
      mma_tf32(acc, ah, bh);
    }
    const int ra = r0 + g, rb = r0 + g + 8, ca = c0 + 2 * t;
    float o0 = acc[0] * alpha, o1 = acc[1] * alpha, o2 = acc[2] * alpha, o3 = acc[3] * alpha;
    if (Add) {
      o0 += Add[ra * ldadd + ca];
      o1 += Add[ra * ldadd + ca + 1];
      o2 += Add[rb * ldadd + ca];
      o3 += Add[rb * ldadd + ca + 1];
    }
    *reinterpret_cast<float2 *>(D + ra * ldd + ca) = make_float2(o0, o1);
    *reinterpret_cast<float2 *>(D + rb * ldd + ca) = make_float2(o2, o3);
  }
}

// The scan's products: 3xTF32 tensor cores where the tile shapes allow (FP32,
// R % 16 == 0, C % 8 == 0, K % 8 == 0), the FP32 / FP64 CUDA-core tiles
// otherwise.
template <typename T, int R, int C, int K, bool TA, bool TB>
__device__ __forceinline__ void mmp(T *D, int ldd, const T *A, int lda, const T *B, int ldb,
                                    const T *Add, int ldadd, T alpha) {
  if constexpr (sizeof(T) == 4 && R % 16 == 0 && C % 8 == 0 && K % 8 == 0)
    mmt_tc<R, C, K, TA, TB>(D, ldd, A, lda, B, ldb, Add, ldadd, alpha);
  else
    mmt<T, R, C, K, TA, TB>(D, ldd, A, lda, B, ldb, Add, ldadd, alpha);
}

// Threads per row of gjr: a power of two <= 32 (a row's threads share a warp).
template <int R, int TH>
constexpr int gj_tpr() {
  int t = 1;
  while (t * 2 <= 32 && t * 2 * R <= TH) t *= 2;
  return t;
}

// Gauss-Jordan without pivoting on the R x W matrix M (left block R x R),
// register-resident: thread (i, g) holds columns g, g + TPR, ... of row i.
// Step j: the threads of row j publish it in `rowbuf` (2 W entries,
// double-buffered), one barrier, and every row takes its own entry of column
// j from the thread holding it by a shuffle.  Afterwards the right block of M
// holds (left)^{-1} (right).  Pivot decisions into *bit / *sing (thread 0)
// when given.  The caller puts a barrier before (M written by others).
template <typename T, int R, int W, int TH>
__device__ __forceinline__ void gjr(T *M, int ld, T *rowbuf, int *bit, int *sing) {
  constexpr int TPR = gj_tpr<R, TH>(), CPT = (W + TPR - 1) / TPR;
  const int tid = threadIdx.x, i = tid / TPR, g = tid - (tid / TPR) * TPR;
  const bool act = i < R;
  const int lane = tid & 31, base = lane & ~(TPR - 1);
  T v[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = g + k * TPR;
    v[k] = (act && c < W) ? M[i * ld + c] : (T)0;
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    T *rb = rowbuf + (j & 1) * W;
    if (act && i == j) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = g + k * TPR;
        if (c < W) rb[c] = v[k];
      }
    }
    __syncthreads();
    const T d = rb[j];
    if (tid == 0 && bit) {
      if (!((double)d > 0.0)) *bit = 0;
      if (!finite_nonzero((double)d)) *sing = 1;
    }
    const T f = __shfl_sync(0xffffffffu, v[j / TPR], base | (j % TPR)) * recip_pivot(d);
    if (act && i != j) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = g + k * TPR;
        if (c > j && c < W) v[k] = fma(-f, rb[c], v[k]);
      }
    }
  }
  // scale the right block by 1 / d_i and store it
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = g + k * TPR;
    if (act && c < W) M[i * ld + c] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = g + k * TPR;
    if (act && c >= R && c < W) M[i * ld + c] = v[k] * recip_pivot(M[i * ld + i]);
  }
  __syncthreads();
}

// Lower triangle mirrored onto the upper one (exact symmetry).  No barrier.
template <typename T>
__device__ __forceinline__ void mirror_lower(int n, T *M, int ld) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    if (i < j) M[i * ld + j] = M[j * ld + i];
  }
}

template <typename T>
__device__ __forceinline__ T to_T(double v) {
  return to_work<T>(v);
}

// Shared memory of the reduce / level kernels (row stride n + 1).
template <typename T, int NX, int NU>
struct CombSmem {
  static constexpr int LD = NX + 2, LD3 = 3 * NX + 2, LDR = NU + 2 * NX + 2;  // even strides
  T P1[NX * LD], A1[NX * LD], C1[NX * LD];   // earlier element
  T P2[NX * LD], A2[NX * LD], C2[NX * LD];   // later element (the accumulator)
  T Pn[NX * LD], An[NX * LD], Cn[NX * LD];   // result
  T G3[NX * LD3];                            // [I + C1 P2 | A1 | C1]
  T T1[NX * LD], T2[NX * LD];
  T Q[NX * LD], A[NX * LD], B[NX * NU], M[NX * NU];
  T RX[NU * LDR];                            // [R | M^T | B^T]
  T rowbuf[2 * (3 * NX + 2)];                // pivot rows of the eliminations
  int rbit, rsing;                           // pivot decisions of the R_i elimination
};

// The stage element (P, A, C)_{i->i+1} into (P1, A1, C1); eq. lqr-gpu-init-running.
template <typename T, int NX, int NU>
__device__ void stage_element(const Inst &I, int i, CombSmem<T, NX, NU> &s) {
  constexpr int n = NX, m = NU, LD = CombSmem<T, NX, NU>::LD, LDR = CombSmem<T, NX, NU>::LDR;
  const int tid = threadIdx.x;
  const double *Q = I.Q + (size_t)i * n * n, *A = I.A + (size_t)i * n * n;
  const double *B = I.B + (size_t)i * n * m, *M = I.M + (size_t)i * n * m;
  const double *R = I.R + (size_t)i * m * m;
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    s.Q[r * LD + c] = to_T<T>(__ldg(Q + (r <= c ? e : c * n + r)));
    s.A[r * LD + c] = to_T<T>(__ldg(A + e));
  }
  for (int e = tid; e < n * m; e += blockDim.x) {
    const int r = e / m, c = e - r * m;
    const T bv = to_T<T>(__ldg(B + e)), mv = to_T<T>(__ldg(M + e));
    s.B[e] = bv;
    s.M[e] = mv;
    s.RX[c * LDR + m + r] = mv;       // M^T
    s.RX[c * LDR + m + n + r] = bv;   // B^T
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e - r * m;
    s.RX[r * LDR + c] = to_T<T>(__ldg(R + (r <= c ? e : c * m + r)));
  }
  __syncthreads();
  // R^{-1} [M^T | B^T]; a zero or non-finite pivot of R_i is recorded in the
  // instance state (the scan needs every R_i invertible)
  gjr<T, NU, NU + 2 * NX, kTH>(s.RX, LDR, s.rowbuf, &s.rbit, &s.rsing);
  if (tid == 0 && s.rsing) atomicOr(&I.st->r_singular, 1);
  // P = Q - M (R^{-1} M^T), A = A - B (R^{-1} M^T), C = delta I + B (R^{-1} B^T)
  mmp<T, NX, NX, NU, false, false>(s.P1, LD, s.M, m, s.RX + m, LDR, s.Q, LD, (T)-1);
  mmp<T, NX, NX, NU, false, false>(s.A1, LD, s.B, m, s.RX + m, LDR, s.A, LD, (T)-1);
  mmp<T, NX, NX, NU, false, false>(s.C1, LD, s.B, m, s.RX + m + n, LDR, nullptr, 0, (T)1);
  __syncthreads();
  const T delta = (T)I.delta;
  for (int r = tid; r < n; r += blockDim.x) s.C1[r * LD + r] += delta;
  mirror_lower<T>(n, s.P1, LD);
  mirror_lower<T>(n, s.C1, LD);
  __syncthreads();
}

// (Pn, An, Cn) = (P1, A1, C1) (+) (P2, A2, C2); eq. lqr-gpu-combo with one
// elimination of I + C1 P2 on [A1 | C1].  The six n x n products run on the
// tensor cores in 3xTF32 (mmp) for n a multiple of 16 in FP32.
template <typename T, int NX, int NU>
__device__ void combine(CombSmem<T, NX, NU> &s) {
  constexpr int n = NX, LD = CombSmem<T, NX, NU>::LD, LD3 = CombSmem<T, NX, NU>::LD3;
  const int tid = threadIdx.x;
  __syncthreads();
  mmp<T, NX, NX, NX, false, false>(s.G3, LD3, s.C1, LD, s.P2, LD, nullptr, 0, (T)1);  // C1 P2
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    s.G3[r * LD3 + n + c] = s.A1[r * LD + c];
    s.G3[r * LD3 + 2 * n + c] = s.C1[r * LD + c];
  }
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) s.G3[r * LD3 + r] += (T)1;
  __syncthreads();
  gjr<T, NX, 3 * NX, kTH>(s.G3, LD3, s.rowbuf, nullptr, nullptr);   // XA = T A1, XC = T C1
  const T *XA = s.G3 + n, *XC = s.G3 + 2 * n;
  mmp<T, NX, NX, NX, false, false>(s.An, LD, s.A2, LD, XA, LD3, nullptr, 0, (T)1);   // A2 XA
  mmp<T, NX, NX, NX, false, false>(s.T1, LD, s.A2, LD, XC, LD3, nullptr, 0, (T)1);   // A2 XC
  mmp<T, NX, NX, NX, false, false>(s.T2, LD, s.P2, LD, XA, LD3, nullptr, 0, (T)1);   // P2 XA
  __syncthreads();
  mmp<T, NX, NX, NX, false, true>(s.Cn, LD, s.T1, LD, s.A2, LD, s.C2, LD, (T)1);     // (A2 XC) A2^T + C2
  mmp<T, NX, NX, NX, true, false>(s.Pn, LD, s.A1, LD, s.T2, LD, s.P1, LD, (T)1);     // A1^T (P2 XA) + P1
  __syncthreads();
  mirror_lower<T>(n, s.Pn, LD);
  mirror_lower<T>(n, s.Cn, LD);
  __syncthreads();
}

template <typename T, int NX>
__device__ __forceinline__ void load_elem(const T *g, T *P, T *A, T *C, int LD) {
  constexpr int n = NX, nn = n * n;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    P[r * LD + c] = g[e];
    A[r * LD + c] = g[nn + e];
    C[r * LD + c] = g[2 * nn + e];
  }
}

template <typename T, int NX>
__device__ __forceinline__ void store_elem(T *g, const T *P, const T *A, const T *C, int LD) {
  constexpr int n = NX, nn = n * n;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    g[e] = P[r * LD + c];
    g[nn + e] = A[r * LD + c];
    g[2 * nn + e] = C[r * LD + c];
  }
}

}  // namespace scan

// Chunk elements into S0 (blocks 0..C-1) and the terminal element (block C).
// ident_terminal: block C writes the identity element (0, I, 0) instead, so
// that the suffix scan's first entry is the interval element of stages
// 0..N-1 alone (a horizon shard's summary).  inner: a chunk longer than
// kInnerK also stores the element of its stages [s + kInnerK, e) into SI.
// Three CTAs per SM in FP32 (the chunk count is sized for one wave of them):
// the register cap keeps the compiler from trading occupancy for ILP.
template <typename T, int NX, int NU>
__global__ void __launch_bounds__(scan::kTH, sizeof(T) == 4 ? 3 : 1)
    k_scan_reduce(BatchArgs a, ScanLayout SL, size_t sbase, int ident_terminal, int inner) {
  using SM = scan::CombSmem<T, NX, NU>;
  constexpr int n = NX, nn = n * n, LD = SM::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const Inst I = get_inst(a, 0);
  const int N = I.N, c = blockIdx.x;
  T *S0 = reinterpret_cast<T *>(I.ws + sbase + SL.S0);
  T *out = S0 + (size_t)c * 3 * nn;
  if (threadIdx.x == 0) {
    s.rbit = 1;
    s.rsing = 0;
  }
  if (c == SL.C) {  // terminal element (Q_N, 0, 0); instance state reset
    if (threadIdx.x == 0) {
      I.st->pivot_status = RLQR_OK;
      I.st->escalated = 0;
      I.st->iters = 0;
      I.st->converged = 0;
      I.st->rel = 0.0;
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      out[e] = ident_terminal
                   ? (T)0
                   : scan::to_T<T>(__ldg(I.Q + (size_t)N * nn + (r <= col ? e : col * n + r)));
      out[nn + e] = (ident_terminal && r == col) ? (T)1 : (T)0;
      out[2 * nn + e] = (T)0;
    }
    return;
  }
  const int s0 = c * SL.L, e0 = min(s0 + SL.L, N);
  // the inner element [s0 + kInnerK, e0): the accumulator once it reaches ik
  const int ik = (inner && chunk_has_inner(e0 - s0)) ? s0 + kInnerK : -1;
  T *sin = reinterpret_cast<T *>(I.ws + sbase + SL.SI) + (size_t)c * 3 * nn;
  // acc (P2, A2, C2) = e_{e0-1}
  scan::stage_element<T, NX, NU>(I, e0 - 1, s);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, col = e - r * n, o = r * LD + col;
    s.P2[o] = s.P1[o];
    s.A2[o] = s.A1[o];
    s.C2[o] = s.C1[o];
  }
  if (e0 - 1 == ik) {
    __syncthreads();
    scan::store_elem<T, NX>(sin, s.P2, s.A2, s.C2, LD);
  }
  for (int i = e0 - 2; i >= s0; --i) {
    scan::stage_element<T, NX, NU>(I, i, s);
    scan::combine<T, NX, NU>(s);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n, o = r * LD + col;
      s.P2[o] = s.Pn[o];
      s.A2[o] = s.An[o];
      s.C2[o] = s.Cn[o];
    }
    if (i == ik) {
      __syncthreads();
      scan::store_elem<T, NX>(sin, s.P2, s.A2, s.C2, LD);
    }
  }
  __syncthreads();
  scan::store_elem<T, NX>(out, s.P2, s.A2, s.C2, LD);
}

// One level of the suffix scan: dst[c] = src[c] (+) src[c + d] (c + d <= C),
// otherwise src[c].
template <typename T, int NX, int NU>
__global__ void __launch_bounds__(scan::kTH) k_scan_level(BatchArgs a, ScanLayout SL, size_t sbase,
                                                          int d, int from1) {
  using SM = scan::CombSmem<T, NX, NU>;
  constexpr int nn = NX * NX, LD = SM::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const Inst I = get_inst(a, 0);
  const int c = blockIdx.x;
  const T *src = reinterpret_cast<const T *>(I.ws + sbase + (from1 ? SL.S1 : SL.S0));
  T *dst = reinterpret_cast<T *>(I.ws + sbase + (from1 ? SL.S0 : SL.S1));
  if (c + d > SL.C) {
    for (int e = threadIdx.x; e < 3 * nn; e += blockDim.x)
      dst[(size_t)c * 3 * nn + e] = src[(size_t)c * 3 * nn + e];
    return;
  }
  scan::load_elem<T, NX>(src + (size_t)c * 3 * nn, s.P1, s.A1, s.C1, LD);
  scan::load_elem<T, NX>(src + (size_t)(c + d) * 3 * nn, s.P2, s.A2, s.C2, LD);
  scan::combine<T, NX, NU>(s);
  scan::store_elem<T, NX>(dst + (size_t)c * 3 * nn, s.Pn, s.An, s.Cn, LD);
}

// P at stage s + kInnerK of every chunk with an inner element: (SI[c] (+)
// suffix element c + 1).P, the value the chunk's P-only pass starts from.
template <typename T, int NX, int NU>
__global__ void __launch_bounds__(scan::kTH) k_scan_inner(BatchArgs a, ScanLayout SL, size_t sbase,
                                                          int from1) {
  using SM = scan::CombSmem<T, NX, NU>;
  constexpr int n = NX, nn = n * n, LD = SM::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const Inst I = get_inst(a, 0);
  const int c = blockIdx.x, s0 = c * SL.L, e0 = min(s0 + SL.L, I.N);
  if (!chunk_has_inner(e0 - s0)) return;
  const T *Sfin = reinterpret_cast<const T *>(I.ws + sbase + (from1 ? SL.S1 : SL.S0));
  const T *sin = reinterpret_cast<const T *>(I.ws + sbase + SL.SI) + (size_t)c * 3 * nn;
  T *pin = reinterpret_cast<T *>(I.ws + sbase + SL.PI) + (size_t)c * nn;
  scan::load_elem<T, NX>(sin, s.P1, s.A1, s.C1, LD);
  scan::load_elem<T, NX>(Sfin + (size_t)(c + 1) * 3 * nn, s.P2, s.A2, s.C2, LD);
  scan::combine<T, NX, NU>(s);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, col = e - r * n;
    pin[e] = s.Pn[r * LD + col];
  }
}

// Shared memory of the finalize kernel (row stride n + 1).
template <typename T, int NX, int NU>
struct FinSmem {
  static constexpr int LD = NX + 2, LD2 = 2 * NX + 2, LDG = 2 * NU + NX + 2;  // even strides
  T P[NX * LD], W[NX * LD], Q[NX * LD], A[NX * LD], WA[NX * LD], ABK[NX * LD], Ft[NX * LD];
  T T1[NX * LD], PhiA[NX * LD], PhiB[NX * LD];
  T S2[NX * LD2];                  // [I + delta P | P]
  T B[NX * NU], M[NX * NU], WB[NX * NU], K[NU * NX], H[NU * NX];
  T GH[NU * LDG];                  // [G | H | I]
  T rowbuf[2 * (2 * NX + 2 * NU + 2)];
  double S64[NX * NX];             // FP64 LDL^T of I + delta P (FP32 certificate fallback)
  int bit, sing, pass;
};

// PASS 1: P-only pass from the scanned boundaries, writes PstA[c] = P at the
// chunk's first stage.  PASS 0 (from the scanned boundaries) / PASS 2 (from
// PstA[c+1]; the terminal Q_N for the last chunk): the full pass below, which
// also writes PstB[c].
// From P at the chunk's end: the sequential step (Theorem main-seq-theorem,
// eq. value-fn-formulas) for every stage i of the chunk, writing W_{i+1},
// K_i, G_i^{-1}, flags[i+1] (bit0; bit1 set at N), G_i (mixed path: for the
// FP64 certificate; plain FP64 path: the pivot decision of G_i, merged by
// k_scan_flags) and the FP32 data copies (mixed path); P_i and Phi_c.  Chunk 0
// also pivots P_0 (W_0, flags[0]).  The instance's pivot status is the worst
// over the chunks (atomicMax).
template <typename T, int NX, int NU, int PASS>
__global__ void __launch_bounds__(scan::kTH, sizeof(T) == 4 ? 3 : 1)
    k_scan_finalize(BatchArgs a, ScanLayout SL, size_t sbase, int from1) {
  constexpr bool FULL = PASS != 1;
  using SM = FinSmem<T, NX, NU>;
  constexpr bool FP32 = sizeof(T) == 4;
  constexpr int n = NX, m = NU, nn = n * n, nm = n * m, mmm = m * m;
  constexpr int LD = SM::LD, LD2 = SM::LD2, LDG = SM::LDG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const int tid = threadIdx.x;
  const Inst I = get_inst(a, 0);
  const int N = I.N, c = blockIdx.x;
  const int s0 = c * SL.L, e0 = min(s0 + SL.L, N);
  const T delta = (T)I.delta;
  const float delta_up = __double2float_ru(I.delta), delta_dn = __double2float_rd(I.delta);
  const T *Sfin = reinterpret_cast<const T *>(I.ws + sbase + (from1 ? SL.S1 : SL.S0));
  T *gPhi = reinterpret_cast<T *>(I.ws + sbase + SL.Phi) + (size_t)c * nn;
  T *gW = reinterpret_cast<T *>(I.ws + I.L.W);
  T *gK = reinterpret_cast<T *>(I.ws + I.L.K);
  T *gGi = reinterpret_cast<T *>(I.ws + I.L.Gi);
  T *gG = reinterpret_cast<T *>(I.ws + I.L.G);
  uint8_t *gpd = reinterpret_cast<uint8_t *>(I.ws + I.L.G);  // plain FP64: G_i decisions
  float *gAf = reinterpret_cast<float *>(I.ws + I.L.Af);
  float *gBf = reinterpret_cast<float *>(I.ws + I.L.Bf);
  float *gQf = reinterpret_cast<float *>(I.ws + I.L.Qf);
  float *gMf = reinterpret_cast<float *>(I.ws + I.L.Mf);
  float *gRf = reinterpret_cast<float *>(I.ws + I.L.Rf);
  float *gcf = reinterpret_cast<float *>(I.ws + I.L.cf);
  T *Phi = s.PhiA, *Phi2 = s.PhiB;
  T *PstA = reinterpret_cast<T *>(I.ws + sbase + SL.PstA);
  T *PstB = reinterpret_cast<T *>(I.ws + sbase + SL.PstB);

  // P at the chunk's end: the P of suffix element c + 1 (for the last chunk
  // the terminal element's Q_N), or in PASS 2 chunk c+1's P-only result.
  // PASS 1 of a chunk with an inner element starts at s0 + kInnerK instead.
  const bool from_inner = PASS == 1 && chunk_has_inner(e0 - s0);
  const T *Pend = from_inner ? reinterpret_cast<const T *>(I.ws + sbase + SL.PI) + (size_t)c * nn
                  : (PASS == 2 && c + 1 < SL.C) ? PstA + (size_t)(c + 1) * nn
                                                : Sfin + (size_t)(c + 1) * 3 * nn;
  const int i_first = from_inner ? s0 + kInnerK - 1 : e0 - 1;
  for (int e = tid; e < nn; e += blockDim.x) {
    const int r = e / n, col = e - r * n;
    s.P[r * LD + col] = Pend[e];
    Phi[r * LD + col] = (r == col) ? (T)1 : (T)0;
  }
  int notpd = 0, singular = 0;

  // state pivot of the P in s.P: W into s.W and gWk; returns bit0
  auto state_pivot = [&](T *gWk) -> int {
    __syncthreads();
    if (tid == 0) {
      s.bit = 1;
      s.sing = 0;
      s.pass = 1;
    }
    for (int e = tid; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const T pv = s.P[r * LD + col];
      s.S2[r * LD2 + col] = (r == col ? (T)1 : (T)0) + delta * pv;
      s.S2[r * LD2 + n + col] = pv;
    }
    __syncthreads();
    if constexpr (!FULL) {
      scan::gjr<T, NX, 2 * NX, scan::kTH>(s.S2, LD2, s.rowbuf, nullptr, nullptr);
    } else if constexpr (FP32) {
      // Gershgorin proof with the certificate's margin in FP32 with directed
      // rounding; otherwise the FP64 LDL^T of I + delta P - tau D (D its
      // diagonal) proves it or the instance is escalated to the FP64
      // recursion (bit0 then stays 1 until that decides)
      if (tid < n) {
        float off = 0.f;
        for (int j = 0; j < n; ++j)
          if (j != tid) off = __fadd_ru(off, fabsf((float)s.P[tid * LD + j]));
        if (!gershgorin_row_margin((float)s.P[tid * LD + tid], off, delta_dn, delta_up, kMarginTau))
          atomicAnd(&s.pass, 0);
      }
      __syncthreads();
      if (!s.pass) {
        for (int e = tid; e < nn; e += blockDim.x) {
          const int r = e / n, col = e - r * n;
          double v = (r == col ? 1.0 : 0.0) + I.delta * widen((float)s.P[r * LD + col]);
          if (r == col) v -= (double)kMarginTau * fabs(v);
          s.S64[e] = v;
        }
        for (int j = 0; j < n; ++j) {
          __syncthreads();
          const double d = s.S64[j * n + j];
          if (tid == 0) {
            if (!(d > 0.0)) s.bit = 0;
            if (!finite_nonzero(d)) s.sing = 1;
          }
          const double rd = 1.0 / d;
          const int r = n - j - 1;
          __syncthreads();
          for (int idx = tid; idx < r * (r + 1) / 2; idx += blockDim.x) {
            int i, cc;
            tri_decode(idx, i, cc);
            i += j + 1;
            cc += j + 1;
            s.S64[i * n + cc] -= s.S64[i * n + j] * (s.S64[cc * n + j] * rd);
          }
        }
        __syncthreads();
      }
      scan::gjr<T, NX, 2 * NX, scan::kTH>(s.S2, LD2, s.rowbuf, nullptr, nullptr);
    } else {
      scan::gjr<T, NX, 2 * NX, scan::kTH>(s.S2, LD2, s.rowbuf, &s.bit, &s.sing);
    }
    // W = right block, exactly symmetric (lower triangle mirrored)
    for (int e = tid; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const int lo = r >= col ? r : col, hi = r >= col ? col : r;
      const T w = s.S2[lo * LD2 + n + hi];
      s.W[r * LD + col] = w;
      if (FULL) gWk[e] = w;
    }
    __syncthreads();
    if (FP32 && FULL) {
      // no decision with margin: the FP64 recursion decides this instance
      if ((!s.bit || s.sing) && tid == 0) I.st->escalated = 1;
      return 1;
    }
    if (s.sing) singular = 1;
    return s.bit;
  };

  for (int i = i_first; i >= s0; --i) {
    const int bit0 = state_pivot(gW + (size_t)(i + 1) * nn);
    // the stage's data (and its FP32 copies in the mixed path)
    const double *Q = I.Q + (size_t)i * nn, *A = I.A + (size_t)i * nn;
    const double *B = I.B + (size_t)i * nm, *M = I.M + (size_t)i * nm;
    const double *R = I.R + (size_t)i * mmm;
    for (int e = tid; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const T av = scan::to_T<T>(__ldg(A + e));
      s.Q[r * LD + col] = scan::to_T<T>(__ldg(Q + (r <= col ? e : col * n + r)));
      s.A[r * LD + col] = av;
      if (FP32 && FULL) {
        gAf[(size_t)i * nn + e] = (float)av;
        gQf[(size_t)i * nn + e] = f64_to_f32_rz(__ldg(Q + e));
      }
    }
    for (int e = tid; e < nm; e += blockDim.x) {
      const T bv = scan::to_T<T>(__ldg(B + e)), mv = scan::to_T<T>(__ldg(M + e));
      s.B[e] = bv;
      s.M[e] = mv;
      if (FP32 && FULL) {
        gBf[(size_t)i * nm + e] = (float)bv;
        gMf[(size_t)i * nm + e] = (float)mv;
      }
    }
    for (int e = tid; e < mmm; e += blockDim.x) {
      const int r = e / m, col = e - r * m;
      s.GH[r * LDG + col] = scan::to_T<T>(__ldg(R + (r <= col ? e : col * m + r)));
      s.GH[r * LDG + m + n + col] = (r == col) ? (T)1 : (T)0;
      if (FP32 && FULL) gRf[(size_t)i * mmm + e] = f64_to_f32_rz(__ldg(R + e));
    }
    if (FP32 && FULL && tid < n)
      gcf[(size_t)(i + 1) * n + tid] = f64_to_f32_rz(__ldg(I.c + (size_t)(i + 1) * n + tid));
    __syncthreads();
    // WA = W A, WB = W B
    scan::mmt<T, NX, NX, NX, false, false>(s.WA, LD, s.W, LD, s.A, LD, nullptr, 0, (T)1);
    scan::mmt<T, NX, NU, NX, false, false>(s.WB, m, s.W, LD, s.B, m, nullptr, 0, (T)1);
    __syncthreads();
    // G = R + B^T WB, H = M^T + B^T WA
    scan::mmt<T, NU, NU, NX, true, false>(s.GH, LDG, s.B, m, s.WB, m, s.GH, LDG, (T)1);
    scan::mmt<T, NU, NX, NX, true, false>(s.H, n, s.B, m, s.WA, LD, nullptr, 0, (T)1);
    __syncthreads();
    for (int e = tid; e < m * n; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const T h = s.H[e] + s.M[col * m + r];
      s.H[e] = h;
      s.GH[r * LDG + m + col] = h;
    }
    __syncthreads();
    if (FP32 && FULL)
      for (int e = tid; e < mmm; e += blockDim.x) {
        const int r = e / m, col = e - r * m;
        gG[(size_t)i * mmm + e] = s.GH[r * LDG + col];
      }
    if (tid == 0) {
      s.bit = 1;
      s.sing = 0;
    }
    __syncthreads();
    scan::gjr<T, NU, 2 * NU + NX, scan::kTH>(s.GH, LDG, s.rowbuf,
                                             (FP32 || !FULL) ? nullptr : &s.bit,
                                             (FP32 || !FULL) ? nullptr : &s.sing);
    const int bit1 = s.bit;
    if (!FP32 && s.sing) singular = 1;
    // K = -G^{-1} H, G^{-1}
    for (int e = tid; e < m * n; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const T kv = -s.GH[r * LDG + m + col];
      s.K[e] = kv;
      if (FULL) gK[(size_t)i * nm + e] = kv;
    }
    if (FULL)
      for (int e = tid; e < mmm; e += blockDim.x) {
        const int r = e / m, col = e - r * m;
        gGi[(size_t)i * mmm + e] = s.GH[r * LDG + m + n + col];
      }
    __syncthreads();
    // P_i = Q + A^T WA + H^T K (exactly symmetric), A + B K
    scan::mmt<T, NX, NX, NX, true, false>(s.T1, LD, s.A, LD, s.WA, LD, s.Q, LD, (T)1);
    scan::mmt<T, NX, NX, NU, false, false>(s.ABK, LD, s.B, m, s.K, n, s.A, LD, (T)1);
    __syncthreads();
    scan::mmt<T, NX, NX, NU, true, false>(s.Ft, LD, s.H, n, s.K, n, s.T1, LD, (T)1);
    __syncthreads();
    for (int e = tid; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      const int lo = r >= col ? r : col, hi = r >= col ? col : r;
      s.P[r * LD + col] = s.Ft[lo * LD + hi];
    }
    __syncthreads();
    if constexpr (FULL) {
      // Ft = (I - delta W)(A + B K) = F_i^T;  Phi <- F_i Phi = Ft^T Phi
      scan::mmt<T, NX, NX, NX, false, false>(s.Ft, LD, s.W, LD, s.ABK, LD, s.ABK, LD, -delta);
      __syncthreads();
      scan::mmt<T, NX, NX, NX, true, false>(Phi2, LD, s.Ft, LD, Phi, LD, nullptr, 0, (T)1);
      T *tmp = Phi;
      Phi = Phi2;
      Phi2 = tmp;
    }
    if (FULL && tid == 0) {
      I.flags[i + 1] = (uint8_t)(bit0 | (i + 1 == N ? 2 : 0));
      if (!FP32) gpd[i] = (uint8_t)bit1;
      if (!bit0 || (!FP32 && !bit1)) notpd = 1;
    }
    __syncthreads();
  }
  if constexpr (!FULL) {
    for (int e = tid; e < nn; e += blockDim.x) {
      const int r = e / n, col = e - r * n;
      PstA[(size_t)c * nn + e] = s.P[r * LD + col];
    }
    return;
  }
  for (int e = tid; e < nn; e += blockDim.x) {
    const int r = e / n, col = e - r * n;
    gPhi[e] = Phi[r * LD + col];
    PstB[(size_t)c * nn + e] = s.P[r * LD + col];
  }
  if (c == 0) {
    const int bit0 = state_pivot(gW);
    if (FP32 && tid < n) gcf[tid] = f64_to_f32_rz(__ldg(I.c + tid));
    if (tid == 0) {
      I.flags[0] = (uint8_t)bit0;
      if (!bit0) notpd = 1;
    }
  }
  if (tid == 0) {
    if (__ldcg(&I.st->r_singular)) singular = 1;  // set by k_scan_reduce
    const int st = singular ? RLQR_ERR_SINGULAR : (notpd ? RLQR_NOT_PD : RLQR_OK);
    atomicMax(&I.st->pivot_status, st);
  }
}

// Plain FP64 path: bit1 of flags[i] from the stored decisions of the G_i.
static __global__ void k_scan_flags(BatchArgs a) {
  const Inst I = get_inst(a, 0);
  const uint8_t *gpd = reinterpret_cast<const uint8_t *>(I.ws + I.L.G);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.N; i += gridDim.x * blockDim.x)
    I.flags[i] = (uint8_t)(I.flags[i] | (gpd[i] << 1));
}

}  // namespace rlqr

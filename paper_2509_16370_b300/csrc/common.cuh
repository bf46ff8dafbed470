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
  int32_t pad;
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
  size_t total;
};

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
  // shared
  char *ws;
  int tsize;
  int32_t *status;  // per-instance outputs, may be null
  double *rel;
  int32_t *iters;
  double tol;
  int max_refine;
};

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
      if (idx < len) s[idx] = (T)v[i];
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
          s[r * n + c] = (T)v[i];
          s[c * n + r] = (T)v[i];
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
      if (idx < len) s[idx] = (T)v[i];
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
          s[r * n + c] = (T)v[i];
          s[c * n + r] = (T)v[i];
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

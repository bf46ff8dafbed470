// scan_launch.cuh -- launch sequences of the associative-scan path, included
// by the translation units scan_fp32.cu / scan_fp64.cu.
#pragma once

#include "launch.cuh"
#include "scan.cuh"
#include "scan_vec.cuh"

namespace rlqr {

// Levels of the suffix scan over C + 1 elements; the result lands in S1 when
// their number is odd.
inline int scan_levels(int C) {
  int l = 0;
  for (int d = 1; d <= C; d <<= 1) ++l;
  return l;
}

template <typename T, int NX, int NU>
static cudaError_t scan_factor_sz(const BatchArgs &a, const ScanLayout &SL, size_t sbase,
                                  cudaStream_t s) {
  cudaError_t e;
  // the R_i pivot record of this factorization starts clear
  if ((e = cudaMemsetAsync(&reinterpret_cast<InstState *>(a.ws)->r_singular, 0, sizeof(int32_t),
                           s)) != cudaSuccess)
    return e;
  {
    auto k = k_scan_reduce<T, NX, NU>;
    const size_t b = sizeof(scan::CombSmem<T, NX, NU>);
    if ((e = set_smem(k, b)) != cudaSuccess) return e;
    LaunchScope ls("k_scan_reduce", s);
    k<<<SL.C + 1, scan::kTH, b, s>>>(a, SL, sbase, 0, sizeof(T) == 4 ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int from1 = 0;
  {
    auto k = k_scan_level<T, NX, NU>;
    const size_t b = sizeof(scan::CombSmem<T, NX, NU>);
    if ((e = set_smem(k, b)) != cudaSuccess) return e;
    for (int d = 1; d <= SL.C; d <<= 1) {
      LaunchScope ls("k_scan_level", s);
      k<<<SL.C + 1, scan::kTH, b, s>>>(a, SL, sbase, d, from1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      from1 ^= 1;
    }
  }
  {
    const size_t b = sizeof(FinSmem<T, NX, NU>);
    if constexpr (sizeof(T) == 4) {
      // P at s + kInnerK of the long chunks, the P-only pass, then the full
      // pass from the contracted boundaries
      auto ki = k_scan_inner<T, NX, NU>;
      auto k1 = k_scan_finalize<T, NX, NU, 1>;
      auto k2 = k_scan_finalize<T, NX, NU, 2>;
      const size_t bc = sizeof(scan::CombSmem<T, NX, NU>);
      if ((e = set_smem(ki, bc)) != cudaSuccess) return e;
      if ((e = set_smem(k1, b)) != cudaSuccess) return e;
      if ((e = set_smem(k2, b)) != cudaSuccess) return e;
      if (chunk_has_inner(SL.L)) {
        LaunchScope ls("k_scan_level", s);
        ki<<<SL.C, scan::kTH, bc, s>>>(a, SL, sbase, from1);
      }
      LaunchScope ls("k_scan_finalize", s);
      k1<<<SL.C, scan::kTH, b, s>>>(a, SL, sbase, from1);
      k2<<<SL.C, scan::kTH, b, s>>>(a, SL, sbase, from1);
    } else {
      auto k = k_scan_finalize<T, NX, NU, 0>;
      if ((e = set_smem(k, b)) != cudaSuccess) return e;
      LaunchScope ls("k_scan_finalize", s);
      k<<<SL.C, scan::kTH, b, s>>>(a, SL, sbase, from1);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (sizeof(T) == 8) {
    LaunchScope ls("k_scan_flags", s);
    k_scan_flags<<<(a.N + 255) / 256, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int NX, int NU, bool FROM_RES>
static cudaError_t scan_solve_sz(const BatchArgs &a, const ScanLayout &SL, size_t sbase,
                                 cudaStream_t s) {
  cudaError_t e;
  const int sfin1 = scan_levels(SL.C) & 1;
  const size_t vb = sizeof(scan::VecSmem<T, NX, NU>);
  auto p0 = k_scan_pvec<T, NX, NU, 0, FROM_RES>;
  auto p1 = k_scan_pvec<T, NX, NU, 1, FROM_RES>;
  auto x0 = k_scan_xvec<T, NX, NU, 0, FROM_RES>;
  auto x1 = k_scan_xvec<T, NX, NU, 1, FROM_RES>;
  if ((e = set_smem(p0, vb)) != cudaSuccess) return e;
  if ((e = set_smem(p1, vb)) != cudaSuccess) return e;
  if ((e = set_smem(x0, vb)) != cudaSuccess) return e;
  if ((e = set_smem(x1, vb)) != cudaSuccess) return e;
  const char *tag = FROM_RES ? "k_scan_refine" : "k_scan_solve";
  {
    LaunchScope ls(tag, s);
    p0<<<SL.C, 32, vb, s>>>(a, SL, sbase);
    k_scan_pbound<T, NX, FROM_RES><<<1, 32, 0, s>>>(a, SL, sbase);
    p1<<<SL.C, 32, vb, s>>>(a, SL, sbase);
    x0<<<SL.C, 32, vb, s>>>(a, SL, sbase, sfin1);
    k_scan_xbound<T, NX, FROM_RES><<<1, 32, 0, s>>>(a, SL, sbase);
    x1<<<SL.C, 32, vb, s>>>(a, SL, sbase, sfin1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int NX, int NU>
static cudaError_t scan_residual_sz(const BatchArgs &a, int cert_g, int do_res, cudaStream_t s) {
  LaunchScope ls(do_res ? "k_res_grid" : "k_cert_grid", s);
  if (do_res) k_norms_reset<<<1, 1, 0, s>>>(a, 1);
  const int blocks = 148 * 8;
  k_res_grid<NX, NU><<<blocks, 128, 0, s>>>(a, cert_g, do_res);
  if (do_res) k_res_final<<<1, 1, 0, s>>>(a, 0);
  else k_scan_status<<<1, 1, 0, s>>>(a);
  return cudaGetLastError();
}

#define RLQR_SCAN_SIZES(X) \
  X(4, 2)                  \
  X(6, 2)                  \
  X(12, 4)                 \
  X(32, 8)

template <typename T>
cudaError_t launch_scan_factor(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                               size_t sbase, cudaStream_t s) {
#define RLQR_SCAN_F(NX, NU) \
  if (n == NX && m == NU) return scan_factor_sz<T, NX, NU>(a, SL, sbase, s);
  RLQR_SCAN_SIZES(RLQR_SCAN_F)
#undef RLQR_SCAN_F
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_scan_solve(int n, int m, bool from_res, const BatchArgs &a,
                              const ScanLayout &SL, size_t sbase, cudaStream_t s) {
#define RLQR_SCAN_S(NX, NU)                                                        \
  if (n == NX && m == NU)                                                          \
    return from_res ? scan_solve_sz<T, NX, NU, true>(a, SL, sbase, s)              \
                    : scan_solve_sz<T, NX, NU, false>(a, SL, sbase, s);
  RLQR_SCAN_SIZES(RLQR_SCAN_S)
#undef RLQR_SCAN_S
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_scan_residual(int n, int m, const BatchArgs &a, int cert_g, int do_res,
                                 cudaStream_t s) {
#define RLQR_SCAN_R(NX, NU) \
  if (n == NX && m == NU) return scan_residual_sz<NX, NU>(a, cert_g, do_res, s);
  RLQR_SCAN_SIZES(RLQR_SCAN_R)
#undef RLQR_SCAN_R
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_scan_norms(const BatchArgs &a, cudaStream_t s) {
  LaunchScope ls("k_norms_grid", s);
  k_norms_reset<<<1, 1, 0, s>>>(a, 0);
  k_norms_grid<<<148 * 4, 256, 0, s>>>(a);
  k_res_final<<<1, 1, 0, s>>>(a, 1);
  return cudaGetLastError();
}

}  // namespace rlqr

// launch_impl.cuh -- kernel selection, included by launch_fp32.cu and
// launch_fp64.cu (one translation unit per precision).
#pragma once

#include <algorithm>

#include "launch.cuh"
#include "refine.cuh"
#include "seq.cuh"
#include "seq_warp.cuh"
#include "sweep32.cuh"
#include "residual32.cuh"
#include "seqx.cuh"
#include "tab32.cuh"
#include "refine_duo.cuh"
#include "refine_tab.cuh"

namespace rlqr {

// Kernel selection.  Sizes that the workloads use get compile-time
// dimensions (FixDims); everything else runs the bucket kernel whose maxima
// (NM, MM) cover it (DynDims).
template <typename T, class D, int TH, bool SOLVE>
static cudaError_t launch_seq_impl(const BatchArgs &a, cudaStream_t s) {
  auto kern = k_seq<T, D, TH, SOLVE>;
  const size_t bytes = SeqSmem<T, D::NM, D::MM>::bytes(sizeof(T) == 4);
  cudaError_t e = set_smem(kern, bytes);
  if (e != cudaSuccess) return e;
  LaunchScope ls(sizeof(T) == 4 ? (SOLVE ? "k_seq_fp32_solve" : "k_seq_fp32_factor")
                                : (SOLVE ? "k_seq_fp64_solve" : "k_seq_fp64_factor"), s);
  kern<<<a.count, TH, bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T, class D, int TH, bool FROM_RES>
static cudaError_t launch_solve_impl(const BatchArgs &a, cudaStream_t s) {
  auto kern = k_solve<T, D, TH, FROM_RES>;
  const size_t bytes = SolveSmem<T, D::NM, D::MM>::bytes();
  cudaError_t e = set_smem(kern, bytes);
  if (e != cudaSuccess) return e;
  LaunchScope ls(FROM_RES ? "k_solve_refine" : (sizeof(T) == 4 ? "k_solve_fp32" : "k_solve_fp64"),
                 s);
  kern<<<a.count, TH, bytes, s>>>(a);
  return cudaGetLastError();
}

// Fixed-size instantiations: (n, m, threads).
#define RLQR_FIXED_SIZES(X) \
  X(4, 2, 64)               \
  X(6, 1, 64)               \
  X(6, 2, 64)               \
  X(12, 4, 128)             \
  X(24, 8, 256)             \
  X(32, 8, 256)             \
  X(48, 16, 256)

// Certificate of the state pivots the FP32 CTA sweep left undecided: the
// FP32 proof, then the FP64 decision for what it did not prove.  4 warps per
// block, about 32 warps per SM over the grid and at least 16 warps per
// instance (its stages spread over them).
template <int NX>
cudaError_t launch_seqx_cert(const BatchArgs &a, cudaStream_t s) {
  const int gy = std::max(4, std::min(65535, (148 * 8 + a.count - 1) / a.count));
  auto k64 = k_seqx_cert64<NX>;
  const size_t bytes = (size_t)4 * NX * NX * sizeof(double);
  cudaError_t e = set_smem(k64, bytes);
  if (e != cudaSuccess) return e;
  LaunchScope ls("k_cert_state", s);
  k_seqx_cert<NX><<<dim3(a.count, gy), 128, 0, s>>>(a);
  k64<<<dim3(a.count, gy), 128, bytes, s>>>(a);
  return cudaGetLastError();
}

// One warp per instance for the small sizes (2 n <= 32, 2 m + n + 1 <= 32);
// the FP32 sweep of even n and m runs the block-pivot kernel of sweep32.cuh,
// that of even n and odd m the tableau kernel of tab32.cuh.
template <typename T, int NX, int NU, bool SOLVE>
static cudaError_t launch_seq_warp(const BatchArgs &a, cudaStream_t s) {
  const char *name = sizeof(T) == 4 ? (SOLVE ? "k_seq_fp32_solve" : "k_seq_fp32_factor")
                                    : (SOLVE ? "k_seq_fp64_solve" : "k_seq_fp64_factor");
  if constexpr (sizeof(T) == 4 && sweep32_fits<NX, NU>()) {
    // even n and m: the block-pivot warp sweep of sweep32.cuh (its certificate
    // is decided in the kernel, with the margin; escalation marks the rest)
    auto kern = k_sweep32<NX, NU, SOLVE>;
    const size_t bytes = sizeof(Sw32<NX, NU>);
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    LaunchScope ls(name, s);
    kern<<<a.count, 32, bytes, s>>>(a);
    return cudaGetLastError();
  } else if constexpr (sizeof(T) == 4 && tab32_fits<NX, NU>()) {
    // even n, odd m: tableau sweep (two warps per instance), then the
    // deferred certificate of the state pivots its Gershgorin test left open
    auto kern = k_tab32<NX, NU, SOLVE>;
    const size_t bytes = sizeof(Tb32<NX, NU>);
    cudaError_t e = set_smem_carveout(kern, bytes);  // 7 CTAs of ~21 KB per SM
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(name, s);
      kern<<<a.count, 64, bytes, s>>>(a);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    return launch_seqx_cert<NX>(a, s);
  } else {
    constexpr int WPC = 1;  // one instance per CTA: spreads the warps evenly over the SMs
    auto kern = k_seq_warp<T, NX, NU, WPC, SOLVE>;
    const size_t bytes = sizeof(WarpSmem<T, NX, NU>) * WPC;
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    LaunchScope ls(name, s);
    kern<<<(a.count + WPC - 1) / WPC, 32 * WPC, bytes, s>>>(a);
    return cudaGetLastError();
  }
}

template <typename T, int NX, int NU, bool FROM_RES>
static cudaError_t launch_solve_warp(const BatchArgs &a, cudaStream_t s) {
  const char *name =
      FROM_RES ? "k_solve_refine" : (sizeof(T) == 4 ? "k_solve_fp32" : "k_solve_fp64");
  if constexpr (sizeof(T) == 4 && FROM_RES && tab32_fits<NX, NU>()) {
    // the factor and the FP32 data copies come from k_sweep32 or k_tab32;
    // the fused route's first pass computes the residual itself
    const bool fused = a.fused_res && a.rpass == 0;
    // later passes find most instances converged: fewer, striding blocks
    const int grid = a.rpass == 0 ? a.count : std::min(a.count, 148 * 4);
    // two warps per instance (routes 6 and 7 of the tuner) split each
    // stage's work between a chain warp and a copy / row warp; with the
    // branch-free one-warp rounds the single warp is faster at every batch
    // size measured (1 to 1024 instances), so it is the default
    const bool duo = a.refine_warps == 2;
    if (duo) {
      auto kern = fused ? k_refine_duo<NX, NU, true> : k_refine_duo<NX, NU, false>;
      const size_t bytes = refine_duo_smem<NX, NU>();
      cudaError_t e = set_smem_carveout(kern, bytes);
      if (e != cudaSuccess) return e;
      LaunchScope ls(name, s);
      kern<<<grid, 64, bytes, s>>>(a);
      return cudaGetLastError();
    }
    auto kern = fused ? k_refine_tab<NX, NU, true> : k_refine_tab<NX, NU, false>;
    const size_t bytes = fused ? refine_tab_smem<NX, NU, true>() : refine_tab_smem<NX, NU, false>();
    cudaError_t e = set_smem_carveout(kern, bytes);
    if (e != cudaSuccess) return e;
    LaunchScope ls(name, s);
    kern<<<grid, 32, bytes, s>>>(a);
    return cudaGetLastError();
  } else {
    constexpr int WPC = 1;  // one instance per CTA: spreads the warps evenly over the SMs
    auto kern = k_solve_warp<T, NX, NU, WPC, FROM_RES>;
    const size_t bytes = sizeof(WarpSmem<T, NX, NU>) * WPC;
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    LaunchScope ls(name, s);
    kern<<<(a.count + WPC - 1) / WPC, 32 * WPC, bytes, s>>>(a);
    return cudaGetLastError();
  }
}

#define RLQR_WARP_SIZES(X) \
  X(4, 1)                  \
  X(4, 2)                  \
  X(6, 1)                  \
  X(6, 2)                  \
  X(12, 3)                 \
  X(12, 4)

template <typename T, bool SOLVE>
cudaError_t launch_seq(int n, int m, bool uniform, const BatchArgs &a, cudaStream_t s) {
  if (uniform) {
#define RLQR_SEQ_WARP(NX, NU) \
    if (n == NX && m == NU) return launch_seq_warp<T, NX, NU, SOLVE>(a, s);
    RLQR_WARP_SIZES(RLQR_SEQ_WARP)
#undef RLQR_SEQ_WARP
  }
  if (uniform) {
    // the larger compile-time sizes: register-tiled CTA sweep
#define RLQR_SEQ_X(NX, NU)                                             \
    if (n == NX && m == NU) {                                          \
      auto kern = k_seqx<T, NX, NU, SOLVE>;                            \
      const size_t bytes = sizeof(SxSmem<T, NX, NU>);                  \
      cudaError_t e = set_smem(kern, bytes);                           \
      if (e != cudaSuccess) return e;                                  \
      LaunchScope ls(sizeof(T) == 4 ? (SOLVE ? "k_seq_fp32_solve" : "k_seq_fp32_factor") \
                                    : (SOLVE ? "k_seq_fp64_solve" : "k_seq_fp64_factor"), s); \
      kern<<<a.count, scan::kTH, bytes, s>>>(a);                       \
      e = cudaGetLastError();                                          \
      if (e != cudaSuccess || sizeof(T) != 4) return e;                \
      return launch_seqx_cert<NX>(a, s);                               \
    }
    RLQR_SEQ_X(24, 8)
    RLQR_SEQ_X(32, 8)
    RLQR_SEQ_X(48, 16)
#undef RLQR_SEQ_X
  }
  if (uniform && SOLVE) {
#define RLQR_SEQ_FIXED(NX, NU, TH) \
    if (n == NX && m == NU) return launch_seq_impl<T, FixDims<NX, NU>, TH, SOLVE>(a, s);
    RLQR_FIXED_SIZES(RLQR_SEQ_FIXED)
#undef RLQR_SEQ_FIXED
  }
  switch (bucket_of(n, m)) {
    case 0: return launch_seq_impl<T, DynDims<8, 4>, 128, SOLVE>(a, s);
    case 1: return launch_seq_impl<T, DynDims<16, 8>, 128, SOLVE>(a, s);
    case 2: return launch_seq_impl<T, DynDims<32, 16>, 256, SOLVE>(a, s);
    case 3: return launch_seq_impl<T, DynDims<48, 16>, 256, SOLVE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, bool FROM_RES>
cudaError_t launch_solve(int n, int m, bool uniform, const BatchArgs &a, cudaStream_t s) {
  if (uniform) {
#define RLQR_SOLVE_WARP(NX, NU) \
    if (n == NX && m == NU) return launch_solve_warp<T, NX, NU, FROM_RES>(a, s);
    RLQR_WARP_SIZES(RLQR_SOLVE_WARP)
#undef RLQR_SOLVE_WARP
  }
  if (uniform && FROM_RES) {
#define RLQR_SOLVE_FIXED(NX, NU, TH) \
    if (n == NX && m == NU) return launch_solve_impl<T, FixDims<NX, NU>, TH, FROM_RES>(a, s);
    RLQR_FIXED_SIZES(RLQR_SOLVE_FIXED)
#undef RLQR_SOLVE_FIXED
  }
  switch (bucket_of(n, m)) {
    case 0: return launch_solve_impl<T, DynDims<8, 4>, 128, FROM_RES>(a, s);
    case 1: return launch_solve_impl<T, DynDims<16, 8>, 128, FROM_RES>(a, s);
    case 2: return launch_solve_impl<T, DynDims<32, 16>, 256, FROM_RES>(a, s);
    case 3: return launch_solve_impl<T, DynDims<48, 16>, 256, FROM_RES>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_residual32(int n, int m, bool uniform, const BatchArgs &a, int cert_g,
                              cudaStream_t s) {
  if (uniform) {
#define RLQR_RES32(NX, NU)                                                   \
    if constexpr (res32_fits<NX, NU>()) {                                    \
      if (n == NX && m == NU) {                                              \
        auto kern = k_res32<NX, NU>;                                         \
        const size_t bytes = sizeof(Rs32Warp<NX, NU>) * kResWarps;           \
        cudaError_t e = set_smem(kern, bytes);                               \
        if (e != cudaSuccess) return e;                                      \
        LaunchScope ls("k_residual_ff", s);                                  \
        const int grid = a.recheck ? std::min(a.count, 148 * 4) : a.count;  \
        kern<<<grid, 32 * kResWarps, bytes, s>>>(a, 1, cert_g);             \
        return cudaGetLastError();                                           \
      }                                                                      \
    }
    RLQR_WARP_SIZES(RLQR_RES32)
#undef RLQR_RES32
  }
  return cudaErrorNotSupported;
}

}  // namespace rlqr

// launch.cuh -- kernel selection shared by the translation units of the
// library (the FP32 and FP64 kernel instantiations compile separately).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace rlqr {

// ---- optional per-kernel timing (rlqr_instrument)
struct Instr {
  bool on = false;
  int n = 0;                     // launches recorded (timed ones: min(n, kMax))
  static constexpr int kMax = 8192;
  cudaEvent_t ev[2 * kMax];
  const char *name[kMax];
  int created = 0;               // events created so far
};
extern Instr g_instr;

struct LaunchScope {             // brackets one kernel launch
  int slot = -1;
  cudaStream_t s;
  LaunchScope(const char *name, cudaStream_t st) : s(st) {
    if (!g_instr.on) return;
    int i = g_instr.n++;
    if (i >= Instr::kMax) return;
    while (g_instr.created < 2 * (i + 1)) {
      if (cudaEventCreate(&g_instr.ev[g_instr.created]) != cudaSuccess) return;
      ++g_instr.created;
    }
    g_instr.name[i] = name;
    slot = i;
    cudaEventRecord(g_instr.ev[2 * i], s);
  }
  ~LaunchScope() {
    if (slot >= 0) cudaEventRecord(g_instr.ev[2 * slot + 1], s);
  }
};

// Dimension buckets: the smallest (NM, MM) >= (n, m) selects the kernel
// instantiation.  Sizes above the last bucket are rejected.
constexpr int kMaxN = 48, kMaxM = 16;

inline int bucket_of(int n, int m) {
  if (n <= 8 && m <= 4) return 0;
  if (n <= 16 && m <= 8) return 1;
  if (n <= 32 && m <= 16) return 2;
  if (n <= 48 && m <= 16) return 3;
  return -1;
}

template <typename F>
inline cudaError_t set_smem(F *kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Same, and the largest shared-memory carveout of the unified L1 / shared
// storage, for kernels whose occupancy is set by their shared memory.
template <typename F>
inline cudaError_t set_smem_carveout(F *kernel, size_t bytes) {
  cudaError_t e = set_smem(kernel, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// Defined in launch_fp32.cu / launch_fp64.cu (explicit instantiations).
template <typename T, bool SOLVE>
cudaError_t launch_seq(int n, int m, bool uniform, const BatchArgs &a, cudaStream_t s);

// ---- persistent sweep of a ragged batch (ragged.cuh, mixed precision)
constexpr int kRaggedClasses = 7;  // the exact size classes of the batched driver

// A size class's place in the persistent sweep: 1 = warp sweep, 2 = CTA
// sweep, 0 = not covered.  Class indices as size_class() numbers them:
// (4,2), (6,1), (6,2), (12,4), (24,8), (32,8), (48,16).
__host__ __device__ inline int ragged_kind(int cls) {
  switch (cls) {
    case 0: case 2: case 3: return 1;
    case 4: case 5: case 6: return 2;
    default: return 0;
  }
}

struct RaggedPlan {
  int off[kRaggedClasses];  // class c occupies perm[off[c] .. off[c] + cnt[c])
  int cnt[kRaggedClasses];
};

// The work items (int4 per item, at most one per instance) and the two-int
// counter block (meta) live in the batch header.  The FP32 sweeps of every
// instance of the classes in P, in one launch on s; the deferred state-pivot
// certificates of the CTA-sweep classes follow (launch_seq_cert).
cudaError_t launch_ragged_sweep(const BatchArgs &a, const RaggedPlan &P, const int32_t *perm,
                                int4 *items, int32_t *meta, cudaStream_t s);
// The deferred certificate of the FP32 CTA sweep for a group of size (n, m)
// (cudaSuccess and nothing launched for sizes without one).
cudaError_t launch_seq_cert(int n, int m, const BatchArgs &a, cudaStream_t s);
template <typename T, bool FROM_RES>
cudaError_t launch_solve(int n, int m, bool uniform, const BatchArgs &a, cudaStream_t s);
// First residual of the mixed path (stored for the refinement) with the
// compile-time-size kernel; cudaErrorNotSupported when the sizes have none.
template <typename T>
cudaError_t launch_residual32(int n, int m, bool uniform, const BatchArgs &a, int cert_g,
                              cudaStream_t s);

// Associative-scan path of one long-horizon instance (scan_fp32.cu /
// scan_fp64.cu); cudaErrorNotSupported for sizes without an instantiation.
struct ScanLayout;
template <typename T>
cudaError_t launch_scan_factor(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                               size_t sbase, cudaStream_t s);
template <typename T>
cudaError_t launch_scan_solve(int n, int m, bool from_res, const BatchArgs &a,
                              const ScanLayout &SL, size_t sbase, cudaStream_t s);
template <typename T>
cudaError_t launch_scan_residual(int n, int m, const BatchArgs &a, int cert_g, int do_res,
                                 cudaStream_t s);
template <typename T>
cudaError_t launch_scan_norms(const BatchArgs &a, cudaStream_t s);

// Horizon shards of one long instance, FP64 (shard.cu); cudaErrorNotSupported
// for sizes without scan kernels.
cudaError_t launch_shard_element(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                                 size_t sbase, double *elem, cudaStream_t s);
cudaError_t launch_shard_boundary(int n, int m, int G, int g, const double *elems,
                                  const double *QN, double *P_end, double *P_start,
                                  cudaStream_t s);
cudaError_t launch_shard_pmap(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                              size_t sbase, double *Phi, double *phi, cudaStream_t s);
cudaError_t launch_shard_p_end(int G, int g, int n, const double *Phis, const double *phis,
                               const double *qN, double *p_end, cudaStream_t s);
cudaError_t launch_shard_x_start(int g, int n, const double *Phis, const double *psis,
                                 double *x_start, cudaStream_t s);
cudaError_t launch_shard_x_offset(int n, const double *Phi, const double *x_first,
                                  const double *x_last, double *psi, cudaStream_t s);
cudaError_t launch_shard_entry(int n, double delta, const double *P_start,
                               const double *x_start, const double *x_first, double *c0,
                               cudaStream_t s);

}  // namespace rlqr

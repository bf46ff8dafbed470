// launch_fp32.cu -- FP32 (mixed-precision) kernel instantiations.
#include "launch_impl.cuh"
#include "ragged.cuh"

namespace rlqr {

cudaError_t launch_ragged_sweep(const BatchArgs &a, const RaggedPlan &P, const int32_t *perm,
                                int4 *items, int32_t *meta, cudaStream_t s) {
  cudaError_t e;
  {
    LaunchScope ls("k_plan", s);
    k_ragged_items<<<1, 1024, 0, s>>>(P, perm, a.dN, items, meta);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = set_smem(k_ragged_sweep, kRaggedSmem)) != cudaSuccess) return e;
  // one wave of resident CTAs: every SM keeps taking items until none is left
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ragged_sweep, scan::kTH,
                                                         kRaggedSmem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  LaunchScope ls("k_seq_fp32_solve", s);
  k_ragged_sweep<<<sms * per_sm, scan::kTH, kRaggedSmem, s>>>(a, perm, items, meta);
  return cudaGetLastError();
}

cudaError_t launch_seq_cert(int n, int m, const BatchArgs &a, cudaStream_t s) {
  if (n == 24 && m == 8) return launch_seqx_cert<24>(a, s);
  if (n == 32 && m == 8) return launch_seqx_cert<32>(a, s);
  if (n == 48 && m == 16) return launch_seqx_cert<48>(a, s);
  return cudaSuccess;
}

template cudaError_t launch_seq<float, true>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_seq<float, false>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_solve<float, true>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_solve<float, false>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_residual32<float>(int, int, bool, const BatchArgs &, int, cudaStream_t);

}  // namespace rlqr

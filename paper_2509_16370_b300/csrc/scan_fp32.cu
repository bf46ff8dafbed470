// scan_fp32.cu -- FP32 (mixed-precision) instantiations of the scan path.
#include "scan_launch.cuh"

namespace rlqr {

template cudaError_t launch_scan_factor<float>(int, int, const BatchArgs &, const ScanLayout &,
                                               size_t, cudaStream_t);
template cudaError_t launch_scan_solve<float>(int, int, bool, const BatchArgs &,
                                              const ScanLayout &, size_t, cudaStream_t);
template cudaError_t launch_scan_residual<float>(int, int, const BatchArgs &, int, int,
                                                 cudaStream_t);
template cudaError_t launch_scan_norms<float>(const BatchArgs &, cudaStream_t);

}  // namespace rlqr

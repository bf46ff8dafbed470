// scan_fp64.cu -- FP64 (plain) instantiations of the scan path.
#include "scan_launch.cuh"

namespace rlqr {

template cudaError_t launch_scan_factor<double>(int, int, const BatchArgs &, const ScanLayout &,
                                               size_t, cudaStream_t);
template cudaError_t launch_scan_solve<double>(int, int, bool, const BatchArgs &,
                                              const ScanLayout &, size_t, cudaStream_t);
template cudaError_t launch_scan_residual<double>(int, int, const BatchArgs &, int, int,
                                                 cudaStream_t);
template cudaError_t launch_scan_norms<double>(const BatchArgs &, cudaStream_t);

}  // namespace rlqr

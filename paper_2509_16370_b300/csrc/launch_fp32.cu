// launch_fp32.cu -- FP32 (mixed-precision) kernel instantiations.
#include "launch_impl.cuh"

namespace rlqr {

template cudaError_t launch_seq<float, true>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_seq<float, false>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_solve<float, true>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_solve<float, false>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_residual32<float>(int, int, bool, const BatchArgs &, int, cudaStream_t);

}  // namespace rlqr

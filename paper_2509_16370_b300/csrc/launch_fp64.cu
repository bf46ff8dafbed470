// launch_fp64.cu -- FP64 kernel instantiations.
#include "launch_impl.cuh"

namespace rlqr {

template cudaError_t launch_seq<double, true>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_seq<double, false>(int, int, bool, const BatchArgs &, cudaStream_t);
template cudaError_t launch_solve<double, false>(int, int, bool, const BatchArgs &, cudaStream_t);

}  // namespace rlqr

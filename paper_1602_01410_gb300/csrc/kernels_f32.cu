// FP32 instantiations of the iteration kernels.
#include "iter_launch.cuh"

namespace dcv {
template cudaError_t launch_row<float>(const RowArgs<float> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_col<float>(const ColArgs<float> &, int, int, size_t, cudaStream_t);
template cudaError_t prepare_kernels<float>(int, int, size_t, size_t);
}  // namespace dcv

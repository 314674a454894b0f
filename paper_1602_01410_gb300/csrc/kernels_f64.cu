// FP64 instantiations of the iteration kernels.
#include "iter_launch.cuh"

namespace dcv {
template cudaError_t launch_row<double>(const RowArgs<double> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_col<double>(const ColArgs<double> &, int, int, size_t, cudaStream_t);
template cudaError_t prepare_kernels<double>(int, int, size_t, size_t);
}  // namespace dcv

// FP32 instantiations of the iteration kernels.
#include "iter_launch.cuh"

namespace dcv {
template cudaError_t launch_row<float>(const RowArgs<float> &, const LaunchCfg &, cudaStream_t);
template cudaError_t launch_col<float>(const ColArgs<float> &, const LaunchCfg &, cudaStream_t);
template cudaError_t prepare_row<float>(const LaunchCfg &);
template cudaError_t prepare_col<float>(const LaunchCfg &);
template cudaError_t launch_row_half<float>(const RowArgs<float> &, const LaunchCfg &, int, cudaStream_t);
}  // namespace dcv
